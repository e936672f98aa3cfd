"""Tile-width tuner table and the batch API's argument checks, without a GPU."""
from __future__ import annotations

import ctypes

import pytest

from paper_2411_19702_gb300 import autotune
from paper_2411_19702_gb300 import build as gbuild
from paper_2411_19702_gb300 import gbmi


@pytest.fixture(scope="module", autouse=True)
def lib():
    gbmi.load(gbuild.build())
    yield
    gbmi.tuner_clear()


def test_cost_model_prefers_wide_tiles_for_large_n_and_narrow_for_tiny_n():
    gbmi.tuner_clear()
    assert gbmi.tile_n(100_000, 10_000) == 256
    assert gbmi.tile_n(5_000, 64) == 64


def test_tuner_entries_cover_their_bucket_only():
    gbmi.tuner_clear()
    before = gbmi.tile_n(100_000, 10_000)
    gbmi.tuner_set(100_000, 10_000, 128)
    # same bucket: floor(log2 m) = 16, floor(2 log2 n) = 26
    assert gbmi.tile_n(70_000, 10_500) == 128
    assert gbmi.tile_n(100_000, 10_000) == 128
    # other buckets keep the model's choice
    assert gbmi.tile_n(300_000, 10_000) == before
    assert gbmi.tile_n(100_000, 20_000) == gbmi.tile_n(100_000, 20_000)
    gbmi.tuner_clear()
    assert gbmi.tile_n(100_000, 10_000) == before


def test_tuner_rejects_bad_widths():
    with pytest.raises(gbmi.GbmiError):
        gbmi.tuner_set(1000, 100, 96)
    with pytest.raises(gbmi.GbmiError):
        gbmi.set_option(gbmi.OPT_TILE_N, 100)


def test_tail_options_range():
    for bad in (5, -1):
        with pytest.raises(gbmi.GbmiError):
            gbmi.set_option(gbmi.OPT_TAIL_COLS, bad)
    with pytest.raises(gbmi.GbmiError):
        gbmi.set_option(gbmi.OPT_TAIL_SPLIT, 16)
    for ok in (0, 2, 3, 4, 1):
        gbmi.set_option(gbmi.OPT_TAIL_COLS, ok)


def test_autotune_table_round_trip(tmp_path):
    table = {"16,26": {"m": 100_000, "n": 10_000, "tile_n": 128, "pair": 1,
                       "ms": {"single64": 3.0, "single128": 2.0, "single256": 2.5,
                              "pair": 1.5}},
             "12,12": {"m": 5000, "n": 64, "tile_n": 64, "pair": 0, "split": 8,
                       "ms": {"single64": 0.1, "single128": 0.2, "single256": 0.3,
                              "pair": 0.4},
                       "ms_split": {"0": 0.05, "1": 0.1, "8": 0.04}}}
    path = str(tmp_path / "tune.json")
    autotune.save(table, path)
    gbmi.tuner_clear()
    got = autotune.load(path)
    assert got == table
    assert gbmi.tile_n(100_000, 10_000) == 128
    assert gbmi.tuner_pair(100_000, 10_000) == 1
    assert gbmi.tuner_pair(5000, 64) == 0
    assert gbmi.tuner_pair(5000, 5000) == -1          # untuned bucket: the built-in rule
    assert gbmi.tuner_split(5000, 64) == 8
    assert gbmi.tuner_split(100_000, 10_000) == 0     # no split entry: the cost model
    assert autotune.bucket(100_000, 10_000) == (16, 26)
    gbmi.tuner_clear()
    assert gbmi.tuner_pair(100_000, 10_000) == -1


def test_tuner_split_argument_checks():
    for bad in (-1, 129):
        with pytest.raises(gbmi.GbmiError):
            gbmi.tuner_set_split(1000, 100, bad)
    with pytest.raises(gbmi.GbmiError):
        gbmi.tuner_set_split(0, 100, 2)
    gbmi.tuner_set_split(1000, 100, 4)
    assert gbmi.tuner_split(1000, 100) == 4
    assert gbmi.tuner_split(1000, 100_000) == 0
    gbmi.tuner_clear()
    assert gbmi.tuner_split(1000, 100) == 0


def test_tuner_pair_argument_checks():
    with pytest.raises(gbmi.GbmiError):
        gbmi.tuner_set_pair(1000, 100, 2)
    with pytest.raises(gbmi.GbmiError):
        gbmi.tuner_set_pair(0, 100, 1)
    gbmi.tuner_set_pair(1000, 100, 1)
    assert gbmi.tuner_pair(1000, 100) == 1
    gbmi.tuner_set_pair(1000, 100, -1)
    assert gbmi.tuner_pair(1000, 100) == -1
    gbmi.tuner_clear()


def test_batch_argument_errors_need_no_gpu():
    lib = gbmi.load()
    plan = ctypes.c_void_p()
    assert lib.gbmi_batch_create(None, 0, ctypes.byref(plan)) == gbmi.ERR_ARG
    jobs = (gbmi._Job * 1)()
    jobs[0] = gbmi._Job(0, 0, 10, 4, 0, 0)          # null X and out
    assert lib.gbmi_batch_create(jobs, 1, ctypes.byref(plan)) == gbmi.ERR_ARG
    jobs[0] = gbmi._Job(16, 0, (1 << 24) + 1, 4, 0, 32)   # m beyond the fused limit
    assert lib.gbmi_batch_create(jobs, 1, ctypes.byref(plan)) == gbmi.ERR_ARG
    assert b"2^24" in lib.gbmi_last_error_string()


def test_server_argument_errors_need_no_gpu():
    lib = gbmi.load()
    srv = ctypes.c_void_p()
    assert lib.gbmi_server_create(1024, 4, ctypes.byref(srv)) == gbmi.ERR_ARG   # budget < 1 MiB
    assert not srv.value
    assert lib.gbmi_server_create(1 << 30, 0, ctypes.byref(srv)) == gbmi.ERR_ARG
    assert b"max_batch" in lib.gbmi_last_error_string()
    i = ctypes.c_int64()
    assert lib.gbmi_server_add_dataset(None, 16, 10, 4, ctypes.byref(i)) == gbmi.ERR_ARG
    assert lib.gbmi_server_submit(None, 0, -1, ctypes.byref(i)) == gbmi.ERR_ARG
    assert lib.gbmi_server_wait(None, 0, 0, None, None) == gbmi.ERR_ARG
    assert lib.gbmi_server_release(None, 0) == gbmi.ERR_ARG
    assert lib.gbmi_server_remove_dataset(None, 0) == gbmi.ERR_ARG
    assert lib.gbmi_server_stats(None, None) == gbmi.ERR_ARG
    assert lib.gbmi_server_destroy(None) == gbmi.OK


def test_out_of_core_argument_errors_need_no_gpu():
    lib = gbmi.load()
    assert lib.gbmi_mi_all_pairs_to_host(None, 10, 4, 16, 0) == gbmi.ERR_ARG
    assert lib.gbmi_mi_all_pairs_to_host(16, 10, 4, None, 0) == gbmi.ERR_ARG
    assert lib.gbmi_mi_all_pairs_to_host(16, 10, 4, 16, -1) == gbmi.ERR_ARG
    assert b"panel_rows" in lib.gbmi_last_error_string()
    assert lib.gbmi_mi_all_pairs_to_host(16, (1 << 24) + 1, 4, 16, 0) == gbmi.ERR_ARG
    assert lib.gbmi_mi_cross_to_host(16, None, 10, 4, 4, 16, 0) == gbmi.ERR_ARG


def test_csr_argument_errors_need_no_gpu():
    lib = gbmi.load()
    assert lib.gbmi_mi_all_pairs_csr(None, 16, 10, 4, 3, 16) == gbmi.ERR_ARG
    assert lib.gbmi_mi_all_pairs_csr(16, None, 10, 4, 3, 16) == gbmi.ERR_ARG   # nnz > 0, no col
    assert lib.gbmi_mi_all_pairs_csr(16, 16, 10, 4, -1, 16) == gbmi.ERR_ARG
    assert lib.gbmi_mi_all_pairs_csr(16, 16, 10, 4, 41, 16) == gbmi.ERR_ARG   # nnz > m * n
    assert lib.gbmi_counts_all_pairs_csr(16, 16, 0, 4, 0, 16) == gbmi.ERR_ARG  # m = 0
    assert lib.gbmi_counts_all_pairs_csr(16, 16, 10, 4, 3, None) == gbmi.ERR_ARG


def test_environment_sets_option_defaults_and_logging():
    import os
    import subprocess
    import sys
    code = ("from paper_2411_19702_gb300 import gbmi; lib = gbmi.load(); "
            "print(lib.gbmi_tile_n(100000, 10000)); "
            "lib.gbmi_mi_all_pairs_to_host(None, 10, 4, None, 0)")
    env = dict(os.environ, GBMI_TILE_N="64", GBMI_LOG="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))), timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "64"
    assert "gbmi: null pointer" in r.stderr
    env = dict(os.environ, GBMI_TILE_N="100")          # not a tile width: ignored
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))), timeout=120)
    assert r.stdout.strip() != "100" and r.returncode == 0


def test_tail_cols_plan():
    # automatic: the last partial wave (tiles mod units) in the 2-4 shares that
    # fill the fewest share-length waves; nothing when no plan ends sooner
    gbmi.set_option(gbmi.OPT_TAIL_COLS, 1)
    assert gbmi.tail_cols_plan(865, 76) == (29, 2)    # 10^4 variables on 76 CTA pairs
    assert gbmi.tail_cols_plan(100, 76) == (24, 3)    # 72 thirds: one third-length wave
    assert gbmi.tail_cols_plan(152, 76) == (0, 0)     # no partial wave
    assert gbmi.tail_cols_plan(50, 76) == (0, 0)      # fewer tiles than slots
    assert gbmi.tail_cols_plan(140, 76) == (0, 0)     # 64 left: every plan takes a whole wave
    assert gbmi.tail_cols_plan(0, 76) == (0, 0)
    gbmi.set_option(gbmi.OPT_TAIL_COLS, 3)            # forced: every tile in 3 shares
    assert gbmi.tail_cols_plan(865, 76) == (865, 3)
    gbmi.set_option(gbmi.OPT_TAIL_COLS, 0)            # off
    assert gbmi.tail_cols_plan(865, 76) == (0, 0)
    gbmi.set_option(gbmi.OPT_TAIL_COLS, 1)
