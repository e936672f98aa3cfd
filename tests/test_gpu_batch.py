"""Batched grouped runs: one persistent Gram launch over many datasets.

Each job's output must be bit-identical to the same problem run alone (the
counts are exact and the per-pair arithmetic is the same), and match the
FP64 oracle within 1e-6.  The plan's CUDA graph is replayed, and pointed at
new buffers of the same shapes.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import autotune, gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


def _rand(m, n, seed, dev="cuda"):
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    p = torch.rand(n, generator=g, device=dev) * 0.4 + 0.02
    return (torch.rand((m, n), generator=g, device=dev) < p).to(torch.uint8)


SHAPES = [(1000, 200, None), (129, 127, None), (3000, 520, 77), (257, 64, None), (5000, 33, 300),
          (2048, 1000, None), (1, 5, None), (777, 300, 130), (40000, 700, None), (513, 257, 257)]


def _problems(seed0=0):
    Xs, Ys = [], []
    for k, (m, n, n2) in enumerate(SHAPES):
        Xs.append(_rand(m, n, seed0 + 2 * k))
        Ys.append(None if n2 is None else _rand(m, n2, seed0 + 2 * k + 1))
    return Xs, Ys


def _alone(X, Y):
    return gbmi.mi_all_pairs(X, path="fused") if Y is None else gbmi.mi_cross(X, Y, path="fused")


def test_batch_matches_single_calls_and_oracle():
    Xs, Ys = _problems()
    b = gbmi.Batch(Xs, Ys)
    assert b.tiles > 0
    outs = b.run()
    gbmi.sync()
    for X, Y, got in zip(Xs, Ys, outs):
        want = _alone(X, Y)
        gbmi.sync()
        assert torch.equal(got, want)
        if X.shape[0] * X.shape[1] <= 2_000_000:
            ref, _ = oracle.mi_matrix(X.cpu().numpy(), None if Y is None else Y.cpu().numpy())
            assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - ref)) <= 1e-6
    b.close()


def test_batch_graph_replay_and_new_buffers():
    Xs, Ys = _problems(100)
    b = gbmi.Batch(Xs, Ys)
    first = [o.clone() for o in b.run()]
    second = b.run()
    gbmi.sync()
    for a, c in zip(first, second):
        assert torch.equal(a, c)
    Xs2, Ys2 = _problems(200)
    outs2 = b.set_io(Xs2, Ys2)
    b.run()
    gbmi.sync()
    for X, Y, got in zip(Xs2, Ys2, outs2):
        assert torch.equal(got, _alone(X, Y))
    b.close()


def test_one_shot_batch_and_fp64_combine():
    Xs, Ys = _problems(300)
    gbmi.set_option(gbmi.OPT_FIXUP, 1)
    try:
        outs = gbmi.mi_batch(Xs, Ys)
        alone = [_alone(X, Y) for X, Y in zip(Xs, Ys)]
        gbmi.sync()
    finally:
        gbmi.set_option(gbmi.OPT_FIXUP, 0)
    for got, want in zip(outs, alone):
        assert torch.equal(got, want)


def test_autotuner_installs_choices_and_keeps_results():
    shapes = [(4000, 96), (20000, 900)]
    table = autotune.tune(shapes, reps=2)
    assert len(table) == 2
    for entry in table.values():
        assert entry["tile_n"] in (64, 128, 256)
        assert entry["pair"] in (0, 1)
        assert set(entry["ms"]) == {"single64", "single128", "single256", "pair"}
        assert gbmi.tile_n(entry["m"], entry["n"]) == entry["tile_n"]
        assert gbmi.tuner_pair(entry["m"], entry["n"]) == entry["pair"]
        # both buckets are narrow enough for the sample split to be timed
        assert set(entry["ms_split"]) == {str(p) for p in autotune.SPLITS}
        assert entry["split"] in autotune.SPLITS
        assert gbmi.tuner_split(entry["m"], entry["n"]) == entry["split"]
    X = _rand(4000, 96, 7)
    Y = _rand(20000, 900, 8)
    got, goty = gbmi.mi_all_pairs(X, path="fused"), gbmi.mi_all_pairs(Y, path="fused")
    b = gbmi.Batch([X, Y])
    bx, by = b.run()
    gbmi.set_option(gbmi.OPT_TILE_N, 256)
    try:
        ref = gbmi.mi_all_pairs(X, path="fused")
    finally:
        gbmi.set_option(gbmi.OPT_TILE_N, 0)
    gbmi.tuner_clear()
    refy = gbmi.mi_all_pairs(Y, path="fused")
    gbmi.sync()
    assert torch.equal(got, ref)
    assert torch.equal(goty, refy)
    assert torch.equal(bx, ref) and torch.equal(by, refy)
    b.close()


@pytest.mark.parametrize("parts", [1, 2, 5, 16])
def test_tuned_sample_split_keeps_results(parts):
    # few variables, many samples: a call the cost model may split; a tuned
    # part count must give the same bits as no split at all
    X = _rand(200_000, 200, 3)
    gbmi.set_option(gbmi.OPT_SPLIT_K, 1)
    try:
        ref = gbmi.mi_all_pairs(X, path="fused")
        refc = gbmi.counts_all_pairs(X, path="plain")
    finally:
        gbmi.set_option(gbmi.OPT_SPLIT_K, 0)
    gbmi.tuner_set_split(200_000, 200, parts)
    try:
        gbmi.profile(enable=True, reset=True)
        got = gbmi.mi_all_pairs(X, path="fused")
        gotc = gbmi.counts_all_pairs(X, path="plain")
        prof = gbmi.profile(enable=False)
    finally:
        gbmi.tuner_clear()
    gbmi.sync()
    assert torch.equal(got, ref) and torch.equal(gotc, refc)
    split = prof.get("gram_tc_split_counts", {}).get("launches", 0) > 0
    assert split == (parts > 1), prof


def test_batch_on_cta_pairs_matches_single_calls():
    """Every job's Gram on CTA pairs (forced); the default rule puts the large jobs there."""
    Xs, Ys = _problems(400)
    gbmi.set_option(gbmi.OPT_PAIR, 2)
    try:
        b = gbmi.Batch(Xs, Ys)
        outs = b.run()
        gbmi.sync()
        for X, Y, got in zip(Xs, Ys, outs):
            assert torch.equal(got, _alone(X, Y))
        b.close()
    finally:
        gbmi.set_option(gbmi.OPT_PAIR, 1)
