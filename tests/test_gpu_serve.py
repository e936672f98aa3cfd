"""Serving: continuous batching over resident datasets.

Every served result must be bit-identical to the same problem run alone
through the single-call path (exact counts, same per-pair arithmetic),
whatever the requests it was batched with, and match the FP64 oracle within
1e-6.  Memory admission must hold requests back until outputs are released,
not fail them; a request that could never fit fails at submit.
"""
from __future__ import annotations

import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


def _rand(m, n, seed, dev="cuda"):
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    p = torch.rand(n, generator=g, device=dev) * 0.4 + 0.02
    return (torch.rand((m, n), generator=g, device=dev) < p).to(torch.uint8)


def _alone(X, Y):
    out = gbmi.mi_all_pairs(X, path="fused") if Y is None else gbmi.mi_cross(X, Y, path="fused")
    gbmi.sync()
    return out


# (m, n) of the datasets; requests pair datasets of equal m for cross MI
DATASETS = [(1000, 200), (1000, 77), (129, 127), (3000, 520), (3000, 300), (257, 64), (1, 5),
            (40000, 700), (40000, 33), (777, 300)]
REQUESTS = [(0, None), (0, 1), (2, None), (3, None), (3, 4), (4, None), (5, None), (6, None),
            (7, None), (7, 8), (8, 7), (9, None), (1, 0), (0, None), (4, 3)]


def _datasets(seed0):
    return [_rand(m, n, seed0 + k) for k, (m, n) in enumerate(DATASETS)]


def test_served_results_equal_single_calls_and_oracle():
    Xs = _datasets(0)
    with gbmi.Server(1 << 30, max_batch=8) as srv:
        ids = [srv.add_dataset(X) for X in Xs]
        tickets = [srv.submit(ids[a], None if b is None else ids[b]) for a, b in REQUESTS]
        for (a, b), t in zip(REQUESTS, tickets):
            got, lat = srv.wait(t)
            assert lat >= 0
            X, Y = Xs[a], None if b is None else Xs[b]
            assert got.shape == (X.shape[1], X.shape[1] if Y is None else Y.shape[1])
            assert torch.equal(got, _alone(X, Y))
            if X.shape[0] * X.shape[1] <= 2_000_000:
                ref, _ = oracle.mi_matrix(X.cpu().numpy(), None if Y is None else Y.cpu().numpy())
                assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - ref)) <= 1e-6
            srv.release(t)
        st = srv.stats()
        assert st["completed"] == len(REQUESTS)
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        assert st["batches"] >= 1 and st["requests_per_batch"] >= 1
        assert st["pairs_per_s"] > 0


def test_requests_from_several_threads():
    Xs = _datasets(50)
    with gbmi.Server(1 << 30, max_batch=4) as srv:
        ids = [srv.add_dataset(X) for X in Xs]
        results, errors = {}, []

        def client(c):
            try:
                for k in range(c, len(REQUESTS), 3):
                    a, b = REQUESTS[k]
                    t = srv.submit(ids[a], None if b is None else ids[b])
                    got, _ = srv.wait(t, timeout_ms=60_000)
                    results[k] = got.clone()
                    srv.release(t)
            except Exception as e:  # surfaced below
                errors.append(e)

        th = [threading.Thread(target=client, args=(c,)) for c in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors
        for k, (a, b) in enumerate(REQUESTS):
            assert torch.equal(results[k], _alone(Xs[a], None if b is None else Xs[b]))


def test_memory_admission_waits_for_released_outputs():
    X = _rand(5000, 1000, 7)
    want = _alone(X, None)
    out_bytes = 1000 * 1000 * 4
    # room for the resident dataset and about two outputs: later requests
    # wait in the queue until earlier outputs are released
    budget = 5120 * 1024 + 1000 * 32 + 2 * out_bytes + (2 << 20)
    with gbmi.Server(budget, max_batch=8) as srv:
        ds = srv.add_dataset(X)
        tickets = [srv.submit(ds) for _ in range(6)]
        for t in tickets:
            got, _ = srv.wait(t, timeout_ms=60_000)
            assert torch.equal(got, want)
            srv.release(t)
        assert srv.stats()["completed"] == 6
        big = srv.add_dataset(_rand(100, 20000, 8))     # 1.6 GB of output: never fits
        with pytest.raises(gbmi.GbmiError) as e:
            srv.submit(big)
        assert e.value.status == gbmi.ERR_OOM


def test_remove_dataset_after_its_requests():
    Xs = _datasets(90)
    with gbmi.Server(1 << 30) as srv:
        a, b = srv.add_dataset(Xs[3]), srv.add_dataset(Xs[4])
        t1, t2 = srv.submit(a), srv.submit(a, b)
        srv.remove_dataset(a)                 # still read by t1, t2: dropped when they finish
        with pytest.raises(gbmi.GbmiError):
            srv.submit(a)
        g1, _ = srv.wait(t1)
        g2, _ = srv.wait(t2)
        assert torch.equal(g1, _alone(Xs[3], None))
        assert torch.equal(g2, _alone(Xs[3], Xs[4]))
        srv.release(t1)
        srv.release(t2)
        with pytest.raises(gbmi.GbmiError):
            srv.remove_dataset(a)
        t3 = srv.submit(b)                    # b is resident: no repack
        g3, _ = srv.wait(t3)
        assert torch.equal(g3, _alone(Xs[4], None))
        srv.release(t3)
        with pytest.raises(gbmi.GbmiError):
            srv.submit(a, b)


def test_requests_on_cta_pairs_match_single_calls():
    """Every request's Gram on CTA pairs (forced), then large ones only (default rule)."""
    Xs = _datasets(70) + [_rand(2000, 1000, 71), _rand(2000, 800, 72)]
    reqs = REQUESTS + [(10, None), (10, 11), (11, None)]
    for mode in (2, 1):
        gbmi.set_option(gbmi.OPT_PAIR, mode)
        try:
            with gbmi.Server(1 << 30, max_batch=8) as srv:
                ids = [srv.add_dataset(X) for X in Xs]
                tickets = [srv.submit(ids[a], None if b is None else ids[b]) for a, b in reqs]
                for (a, b), t in zip(reqs, tickets):
                    got, _ = srv.wait(t, timeout_ms=60_000)
                    assert torch.equal(got, _alone(Xs[a], None if b is None else Xs[b]))
                    srv.release(t)
        finally:
            gbmi.set_option(gbmi.OPT_PAIR, 1)


def test_cancel_queued_request_and_state():
    X = _rand(5000, 1000, 90)
    want = _alone(X, None)
    out_bytes = 1000 * 1000 * 4
    budget = 5120 * 1024 + 1000 * 32 + out_bytes + (3 << 20)   # one output at a time
    with gbmi.Server(budget, max_batch=4) as srv:
        ds = srv.add_dataset(X)
        tickets = [srv.submit(ds) for _ in range(4)]
        st = srv.state()
        assert st["datasets"] == 1 and st["queued"] + st["running"] >= 3
        srv.cancel(tickets[3])                   # outputs are held: it cannot have started
        with pytest.raises(gbmi.GbmiError) as e:
            srv.wait(tickets[3], timeout_ms=1000)
        assert e.value.status == gbmi.ERR_ARG
        for t in tickets[:3]:
            got, _ = srv.wait(t, timeout_ms=60_000)
            assert torch.equal(got, want)
            with pytest.raises(gbmi.GbmiError):
                srv.cancel(t)                    # done: not cancellable
            srv.release(t)
        srv.release(tickets[3])
        st = srv.state()
        assert st["queued"] == 0 and st["running"] == 0
        assert st["bytes_in_use"] > 0            # the dataset stays resident until removed
        srv.remove_dataset(ds)
        assert srv.state()["datasets"] == 0
