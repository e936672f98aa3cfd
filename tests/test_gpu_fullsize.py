"""Parity at the full benchmark sizes, on sampled outputs the oracle computes
one by one, plus whole-matrix properties that hold at any size.

paper scale (m=100,000, n=10,000, Beta(0.5,5) densities, 1% planted noisy
copies): the fused all-pairs call in the benchmark's launch configuration;
every count of the tensor-core Gram equals the popcount Gram's; 20,000
seeded pairs, all planted pairs and 500 diagonal entries against the FP64
oracle (MI within 1e-6, counts exact); symmetry of the whole matrix.

precision (m=2^20, n=2^14): full tensor-core vs popcount count equality with
FP4 and with FP8 operands; MI on every pair among 448 seeded columns (100,576
pairs) against the oracle, and the two operand forms' MI matrices bit-identical.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import simdata  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _check_sampled(X_host_T, out, n11_dev, pi, pj):
    counts, want = oracle.mi_pairs_t(X_host_T, X_host_T, pi, pj)
    ti = torch.from_numpy(pi).cuda()
    tj = torch.from_numpy(pj).cuda()
    got = out[ti, tj].double().cpu().numpy()
    err = np.abs(got - want)
    assert err.max() <= 1e-6, f"max |MI - oracle| = {err.max()} at pair {np.argmax(err)}"
    if n11_dev is not None:
        c = n11_dev[ti, tj].cpu().numpy().astype(np.int64)
        assert np.array_equal(c, counts[:, 0])
    return float(err.max())


def test_paper_scale_sampled_parity():
    r = simdata.PAPER
    X, info = simdata.from_recipe(r, device="cuda")
    out = gbmi.mi_all_pairs(X)                       # AUTO -> fused at this size
    tc = gbmi.counts_all_pairs(X, path="plain")
    pc = gbmi.counts_all_pairs(X, path="popcount")
    gbmi.sync()
    assert torch.equal(tc, pc), "tensor-core and popcount counts differ"
    del pc
    assert torch.equal(torch.diagonal(tc), X.sum(dim=0, dtype=torch.int32))
    assert torch.equal(out, out.T), "MI matrix not symmetric"
    assert bool(torch.all(out >= 0))

    XT = oracle.transpose(X.cpu().numpy())
    pi, pj = simdata.sample_pairs(r.n, r.n, 20_000, seed=r.seed)
    tg, sr = info["planted_targets"], info["planted_sources"]
    d = np.random.default_rng(5).choice(r.n, 500, replace=False).astype(np.int64)
    pi = np.concatenate([pi, np.minimum(tg, sr), d])
    pj = np.concatenate([pj, np.maximum(tg, sr), d])
    err = _check_sampled(XT, out, tc, pi, pj)
    # planted noisy copies carry far more MI than unrelated pairs (a copy of a
    # very sparse column is mostly flip noise, so only the medians are compared)
    planted = out[torch.from_numpy(tg).cuda(), torch.from_numpy(sr).cuda()]
    unrelated = out[torch.from_numpy(pi[:20_000]).cuda(), torch.from_numpy(pj[:20_000]).cuda()]
    assert float(planted.median()) > 100 * float(unrelated.median())
    print(f"paper scale: max |MI - oracle| over {len(pi)} pairs = {err:.3e}")


@pytest.fixture
def _fp4_restored():
    yield
    gbmi.set_option(gbmi.OPT_FP4, 1)


def test_precision_config_counts_and_sampled_mi(_fp4_restored):
    r = simdata.PRECISION
    X, _ = simdata.from_recipe(r, device="cuda")
    pc = gbmi.counts_all_pairs(X, path="popcount")
    outs = {}
    for fp4 in (1, 0):
        gbmi.set_option(gbmi.OPT_FP4, fp4)
        tc = gbmi.counts_all_pairs(X, path="plain")
        gbmi.sync()
        assert torch.equal(tc, pc), f"tensor-core (fp4={fp4}) and popcount counts differ at m=2^20"
        del tc
        outs[fp4] = gbmi.mi_all_pairs(X)
        gbmi.sync()
    gbmi.set_option(gbmi.OPT_FP4, 1)
    assert torch.equal(outs[1], outs[0]), "FP4 and FP8 operands give different MI"
    out = outs[1]
    del outs
    cols = np.sort(np.random.default_rng(7).choice(r.n, 448, replace=False)).astype(np.int64)
    sub = X[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    XT = oracle.transpose(sub)
    iu, ju = np.triu_indices(len(cols))
    assert len(iu) >= 100_000
    counts, want = oracle.mi_pairs_t(XT, XT, iu.astype(np.int64), ju.astype(np.int64))
    ti = torch.from_numpy(cols[iu]).cuda()
    tj = torch.from_numpy(cols[ju]).cuda()
    got = out[ti, tj].double().cpu().numpy()
    assert np.abs(got - want).max() <= 1e-6
    assert np.array_equal(pc[ti, tj].cpu().numpy().astype(np.int64), counts[:, 0])
    print(f"precision config: max |MI - oracle| over {len(iu)} pairs = "
          f"{np.abs(got - want).max():.3e}")
