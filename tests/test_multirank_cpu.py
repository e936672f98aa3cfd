"""The N > 1 host path of the benchmark on CPU ranks (gloo, world size 2).

With several GPUs every rank runs an independent replica (its own seed, no
collective on the data path), or, with --scaling strong, its shard of one
problem (the same input on every rank); the only cross-rank steps are the
barrier and the maximum of the per-rank times, from which rank 0 reports the
whole-job rate.  The reference arm runs on rank 0 alone.
"""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import simdata
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_s = 0.010 * (rank + 1)          # rank 1 is the slow one
        dist.barrier()
        slowest = bench.max_over_ranks(local_s, dist, "cpu")
        rate = bench.whole_job_rate(1000, world, slowest)
        srate = bench.strong_rate(1000, slowest)
        X, _ = simdata.make(64, 16, bench.replica_seed(2, rank), "beta", 0.0, 0.0, device="cpu")
        Xs, _ = simdata.make(64, 16, bench.workload_seed(2, rank, True), "beta", 0.0, 0.0,
                             device="cpu")
        q.put((rank, slowest, rate, np.asarray(X)[:8].tobytes(), srate,
               np.asarray(Xs)[:8].tobytes()))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, slowest, rate, _, srate, _ in out:
        assert slowest == pytest.approx(0.020)        # every rank sees the slowest time
        assert rate == pytest.approx(2 * 1000 / 0.020)  # all ranks' units / slowest time
        assert srate == pytest.approx(1000 / 0.020)     # one split problem's units
    assert out[0][3] != out[1][3]                      # replicas draw independent inputs
    assert out[0][5] == out[1][5]                      # a split problem has one input


def test_helpers_without_process_group():
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
    assert bench.replica_seed(2, 3) == 5
    assert bench.workload_seed(2, 3, True) == 2 and bench.workload_seed(2, 3, False) == 5
    assert bench.strong_rate(10, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--m", "2000", "--n", "50", "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
