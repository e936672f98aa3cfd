"""CTA-pair Gram: clusters of two SMs sharing one tcgen05 cta_group::2 MMA.

The pair kernel computes 256 x 256 tiles (256 x 240 with FP4 operands; each
SM stages half of A and half
of B; CTA 0 loads both halves and issues the MMAs, both CTAs run the
epilogue on their half of the accumulator).  Counts must be bit-exact
(against the oracle and the popcount path, up to 2^24 samples per launch and
in chunks beyond), MI bit-identical to the single-CTA kernel and within 1e-6
of the oracle, and a bounded wait that runs out must unwind both CTAs.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [(1000, 200), (1, 1), (1, 5), (129, 127), (300, 257), (1031, 300), (2000, 520),
          (5000, 1024), (40000, 700)]


def _data(m, n, seed, lo=0.02, hi=0.5):
    rng = np.random.default_rng(seed)
    p = rng.uniform(lo, hi, size=n)
    return (rng.random((m, n)) < p).astype(np.uint8)


def _single(fn, *a, **k):
    gbmi.set_option(gbmi.OPT_PAIR, 0)
    try:
        out = fn(*a, **k)
        gbmi.sync()
        return out
    finally:
        gbmi.set_option(gbmi.OPT_PAIR, 2)


@pytest.fixture(autouse=True, params=[1, 0], ids=["fp4", "fp8"])
def _operand_form(request):
    """Both operand forms: FP4 (256 x 240 pair tiles) and FP8 (256 x 256)."""
    gbmi.set_option(gbmi.OPT_FP4, request.param)
    yield request.param
    gbmi.set_option(gbmi.OPT_FP4, 1)


@pytest.fixture(scope="module", autouse=True)
def _pair():
    gbmi.load()
    gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 0)
    gbmi.set_option(gbmi.OPT_PAIR, 2)        # every shape on CTA pairs
    yield
    gbmi.set_option(gbmi.OPT_PAIR, 1)


@pytest.mark.parametrize("m,n", SHAPES)
def test_counts_exact(m, n):
    X = _data(m, n, 21)
    Xd = torch.from_numpy(X).cuda()
    got = gbmi.counts_all_pairs(Xd, path="plain")
    gbmi.sync()
    if m * n <= 4_000_000:
        _, want = oracle.mi_matrix(X)
    else:
        want = gbmi.counts_all_pairs(Xd, path="popcount").cpu().numpy()
    assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("m,n", SHAPES)
def test_mi_matches_oracle_and_single_cta(m, n):
    X = _data(m, n, 22)
    Xd = torch.from_numpy(X).cuda()
    for path in ("fused", "plain"):
        got = gbmi.mi_all_pairs(Xd, path=path)
        gbmi.sync()
        assert torch.equal(got, _single(gbmi.mi_all_pairs, Xd, path=path))
        assert torch.equal(got, got.t())
    if m * n <= 4_000_000:
        want, _ = oracle.mi_matrix(X)
        assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - want)) <= 1e-6


def test_cross():
    X, Y = _data(777, 300, 23), _data(777, 130, 24)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    want, n11 = oracle.mi_matrix(X, Y)
    got = gbmi.counts_cross(Xd, Yd, path="plain")
    gbmi.sync()
    assert np.array_equal(got.cpu().numpy(), n11)
    mi = gbmi.mi_cross(Xd, Yd, path="fused")
    gbmi.sync()
    assert np.max(np.abs(mi.cpu().numpy().astype(np.float64) - want)) <= 1e-6
    assert torch.equal(mi, _single(gbmi.mi_cross, Xd, Yd, path="fused"))


@pytest.mark.parametrize("m", [2 ** 20 + 3, 2 ** 24, 2 ** 24 + 129])
def test_all_ones_reach_every_count(m):
    Xd = torch.ones((m, 16), dtype=torch.uint8, device="cuda")
    Xd[::2, 1] = 0
    got = gbmi.counts_all_pairs(Xd, path="plain").cpu().numpy()
    gbmi.sync()
    assert got[0, 0] == m and got[2, 15] == m
    assert got[1, 1] == m // 2 and got[0, 1] == m // 2 and got[1, 0] == m // 2


def test_fp64_combine_on_pairs():
    X = _data(3000, 520, 25)
    Xd = torch.from_numpy(X).cuda()
    want, _ = oracle.mi_matrix(X)
    gbmi.set_option(gbmi.OPT_FIXUP, 1)
    try:
        got = gbmi.mi_all_pairs(Xd, path="fused")
        gbmi.sync()
        assert torch.equal(got, _single(gbmi.mi_all_pairs, Xd, path="fused"))
    finally:
        gbmi.set_option(gbmi.OPT_FIXUP, 0)
    assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - want)) <= 1e-6


def test_out_of_core_panels_on_pairs():
    Xd = torch.from_numpy(_data(3000, 1100, 26)).cuda()
    want = gbmi.mi_all_pairs(Xd, path="fused").cpu()
    for panel in (0, 300, 512):
        assert torch.equal(gbmi.mi_all_pairs_to_host(Xd, panel_rows=panel), want)
    Yd = torch.from_numpy(_data(3000, 333, 27)).cuda()
    assert torch.equal(gbmi.mi_cross_to_host(Xd, Yd, panel_rows=256),
                       gbmi.mi_cross(Xd, Yd, path="fused").cpu())


def test_bounded_wait_unwinds_both_ctas():
    """CTA 0's loader issues no copies (test hook): its MMA thread's wait runs
    out, the abort reaches the partner CTA, both unwind, free the pair's
    tensor memory and leave the context usable."""
    X = torch.from_numpy(_data(512, 300, 28)).cuda()
    gbmi.set_option(gbmi.OPT_TIMEOUT_NS, 50_000_000)
    gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 1)
    try:
        gbmi.mi_all_pairs(X, path="fused")
        with pytest.raises(gbmi.GbmiError) as e:
            gbmi.sync()
        assert e.value.status == gbmi.ERR_TIMEOUT
    finally:
        gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 0)
        gbmi.set_option(gbmi.OPT_TIMEOUT_NS, 2_000_000_000)
    out = gbmi.mi_all_pairs(X, path="fused")
    gbmi.sync()
    want, _ = oracle.mi_matrix(X.cpu().numpy())
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - want)) <= 1e-6
