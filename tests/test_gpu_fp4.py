"""FP4 operands: 0/1 packed as E2M1 nibbles, Gram on the block-scaled FP4 MMA.

With GBMI_OPT_FP4 (the default) the pack writes two samples per byte (E2M1
0x0 / 0x2 = 1.0) in blocks of 256 samples, and the Gram runs tcgen05
kind::mxf4 with every scale factor 1.0; tiles are at most 240 wide (the scale
factors take 16 columns of each accumulator buffer).  0 and 1 are exact in
E2M1, so counts must equal the oracle's and the FP8 path's bit for bit, and
MI must be bit-identical to the FP8 path (the epilogue sees the same
integers).  Shapes straddle the 240-column tile edge, the 256-sample K block
and the 128/256-row blocks of both kernels.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (255, 239), (256, 240), (257, 241), (513, 480), (700, 481), (1000, 719),
          (2049, 960), (5000, 1201)]


def _data(m, n, seed, lo=0.02, hi=0.5):
    rng = np.random.default_rng(seed)
    p = rng.uniform(lo, hi, size=n)
    return (rng.random((m, n)) < p).astype(np.uint8)


_COUNTS = {}


def _oracle_counts(m, n, seed):
    """The oracle's N11 of _data(m, n, seed), computed once per shape."""
    key = (m, n, seed)
    if key not in _COUNTS:
        _COUNTS[key] = oracle.mi_matrix(_data(m, n, seed))[1]
    return _COUNTS[key]


@pytest.fixture(autouse=True)
def _options():
    gbmi.load()
    gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 0)
    gbmi.set_option(gbmi.OPT_FP4, 1)
    yield
    gbmi.set_option(gbmi.OPT_FP4, 1)
    gbmi.set_option(gbmi.OPT_PAIR, 1)
    gbmi.set_option(gbmi.OPT_TILE_N, 0)
    gbmi.set_option(gbmi.OPT_SPLIT_K, 0)


def _with(fp4, fn, *a, **k):
    gbmi.set_option(gbmi.OPT_FP4, fp4)
    try:
        out = fn(*a, **k)
        gbmi.sync()
        return out
    finally:
        gbmi.set_option(gbmi.OPT_FP4, 1)


# single-CTA tiles of every width (256 runs as 240 with FP4) and CTA pairs
KERNELS = [(0, 64), (0, 128), (0, 256), (2, 0)]


@pytest.mark.parametrize("pair,tile", KERNELS, ids=["single64", "single128", "single240", "pair"])
@pytest.mark.parametrize("m,n", SHAPES)
def test_counts_exact(m, n, pair, tile):
    X = _data(m, n, 31)
    Xd = torch.from_numpy(X).cuda()
    gbmi.set_option(gbmi.OPT_PAIR, pair)
    gbmi.set_option(gbmi.OPT_TILE_N, tile)
    got = gbmi.counts_all_pairs(Xd, path="plain")
    gbmi.sync()
    assert np.array_equal(got.cpu().numpy(), _oracle_counts(m, n, 31))


@pytest.mark.parametrize("pair", [0, 2], ids=["single", "pair"])
@pytest.mark.parametrize("m,n", [(300, 241), (2049, 960), (40000, 1500)])
def test_mi_bit_identical_to_fp8_and_oracle(m, n, pair):
    X = _data(m, n, 32)
    Xd = torch.from_numpy(X).cuda()
    gbmi.set_option(gbmi.OPT_PAIR, pair)
    for path in ("fused", "plain"):
        a = _with(1, gbmi.mi_all_pairs, Xd, path=path)
        b = _with(0, gbmi.mi_all_pairs, Xd, path=path)
        assert torch.equal(a, b), path
    rng = np.random.default_rng(5)
    pi = rng.integers(0, n, 300)
    pj = rng.integers(0, n, 300)
    _, want = oracle.mi_pairs(X, pi, pj)
    got = a[torch.from_numpy(pi).cuda(), torch.from_numpy(pj).cuda()].double().cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-6


def test_cross_exact_and_identical():
    X, Y = _data(1031, 300, 33), _data(1031, 517, 34)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    want, n11 = oracle.mi_matrix(X, Y)
    for pair in (0, 2):
        gbmi.set_option(gbmi.OPT_PAIR, pair)
        got = gbmi.counts_cross(Xd, Yd, path="plain")
        gbmi.sync()
        assert np.array_equal(got.cpu().numpy(), n11)
        a = _with(1, gbmi.mi_cross, Xd, Yd, path="fused")
        b = _with(0, gbmi.mi_cross, Xd, Yd, path="fused")
        assert torch.equal(a, b)
        assert np.max(np.abs(a.cpu().numpy().astype(np.float64) - want)) <= 1e-6


@pytest.mark.parametrize("m", [4096, 65536 + 77, 300001])
def test_sample_split_exact(m):
    """Sample split (parts of whole 256-sample K blocks) with FP4 operands."""
    n = 96
    X = _data(m, n, 35)
    Xd = torch.from_numpy(X).cuda()
    gbmi.set_option(gbmi.OPT_SPLIT_K, 2)
    got = gbmi.counts_all_pairs(Xd, path="plain")
    mi = gbmi.mi_all_pairs(Xd, path="fused")
    gbmi.sync()
    gbmi.set_option(gbmi.OPT_SPLIT_K, 1)
    ref = gbmi.counts_all_pairs(Xd, path="popcount")
    mi1 = _with(0, gbmi.mi_all_pairs, Xd, path="fused")
    assert torch.equal(got, ref)
    assert torch.equal(mi, mi1)


def test_padding_samples_do_not_count():
    """m = 1 .. 257 around the 256-sample K block: the pack zeroes the
    padding half-bytes of the last block, so all-ones columns count m."""
    for m in (1, 2, 127, 128, 129, 255, 256, 257):
        X = torch.ones((m, 5), dtype=torch.uint8, device="cuda")
        c = gbmi.counts_all_pairs(X, path="plain")
        gbmi.sync()
        assert torch.all(c == m).item(), m


def test_batch_and_host_call_both_forms_match_single_calls():
    """Grouped batches (pair and single-CTA jobs, aligned and unaligned rows)
    and the host-buffer pipeline, planned with either operand form, give the
    single calls' MI bit for bit."""
    shapes = [(300, 100), (5000, 800), (1031, 241), (70000, 900), (257, 1000)]
    Xs = [torch.from_numpy(_data(m, n, 40 + k)).cuda() for k, (m, n) in enumerate(shapes)]
    want = [_with(1, gbmi.mi_all_pairs, X) for X in Xs]
    for fp4 in (1, 0):
        gbmi.set_option(gbmi.OPT_FP4, fp4)
        try:
            outs = gbmi.mi_batch(Xs)
            gbmi.sync()
            host = gbmi.mi_all_pairs_host(Xs[3].cpu())
        finally:
            gbmi.set_option(gbmi.OPT_FP4, 1)
        for k, (o, w) in enumerate(zip(outs, want)):
            assert torch.equal(o, w), (fp4, k)
        assert np.array_equal(np.asarray(host), want[3].cpu().numpy()), fp4
