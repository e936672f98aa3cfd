"""Direct operand path: the tensor cores read X itself (MN-major E4M3, no pack).

A byte 1 is the E4M3 subnormal 2^-9, so the accumulator holds count * 2^-18;
counts must still be bit-exact (against the oracle and the popcount path, up
to m = 2^24 per launch and beyond in chunks), MI bit-identical to the packed
path (same counts, same epilogue) and within 1e-6 of the oracle.  Shapes the
direct path cannot take (n not a multiple of 16, unaligned X) must fall back
to the packed path; a byte other than 0 / 1 must be reported, not hidden.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [(1000, 208), (1, 16), (129, 128), (300, 256), (1031, 304), (2000, 528),
          (5000, 1024), (40000, 96)]


def _data(m, n, seed, lo=0.02, hi=0.5):
    rng = np.random.default_rng(seed)
    p = rng.uniform(lo, hi, size=n)
    return (rng.random((m, n)) < p).astype(np.uint8)


def _packed(fn, *a, **k):
    gbmi.set_option(gbmi.OPT_DIRECT, 0)
    try:
        out = fn(*a, **k)
        gbmi.sync()
        return out
    finally:
        gbmi.set_option(gbmi.OPT_DIRECT, 1)


@pytest.fixture(scope="module", autouse=True)
def _direct():
    gbmi.load()
    gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 0)
    gbmi.set_option(gbmi.OPT_DIRECT, 1)
    yield
    gbmi.set_option(gbmi.OPT_DIRECT, 0)


@pytest.mark.parametrize("m,n", SHAPES)
def test_counts_exact(m, n):
    X = _data(m, n, 11)
    _, n11 = oracle.mi_matrix(X) if m * n <= 4_000_000 else (None, None)
    Xd = torch.from_numpy(X).cuda()
    got = gbmi.counts_all_pairs(Xd, path="plain")
    gbmi.sync()
    want = n11 if n11 is not None else gbmi.counts_all_pairs(Xd, path="popcount").cpu().numpy()
    assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("m,n", SHAPES)
def test_mi_matches_oracle_and_packed_path(m, n):
    X = _data(m, n, 12)
    Xd = torch.from_numpy(X).cuda()
    got = gbmi.mi_all_pairs(Xd, path="fused")
    gbmi.sync()
    assert torch.equal(got, _packed(gbmi.mi_all_pairs, Xd, path="fused"))
    assert torch.equal(got, got.t())
    if m * n <= 4_000_000:
        want, _ = oracle.mi_matrix(X)
        assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - want)) <= 1e-6


@pytest.mark.parametrize("tile_n", [64, 128, 256])
def test_tile_widths(tile_n):
    X = _data(3000, 400, 13)
    Xd = torch.from_numpy(X).cuda()
    gbmi.set_option(gbmi.OPT_TILE_N, tile_n)
    try:
        got = gbmi.mi_all_pairs(Xd, path="fused")
        gbmi.sync()
    finally:
        gbmi.set_option(gbmi.OPT_TILE_N, 0)
    assert torch.equal(got, _packed(gbmi.mi_all_pairs, Xd, path="fused"))


def test_cross_and_plain_path():
    X, Y = _data(777, 304, 14), _data(777, 144, 15)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    want, n11 = oracle.mi_matrix(X, Y)
    got = gbmi.counts_cross(Xd, Yd, path="plain")
    gbmi.sync()
    assert np.array_equal(got.cpu().numpy(), n11)
    for path in ("fused", "plain"):
        mi = gbmi.mi_cross(Xd, Yd, path=path)
        gbmi.sync()
        assert np.max(np.abs(mi.cpu().numpy().astype(np.float64) - want)) <= 1e-6
        assert torch.equal(mi, _packed(gbmi.mi_cross, Xd, Yd, path=path))


@pytest.mark.parametrize("m", [2 ** 20 + 3, 2 ** 24, 2 ** 24 + 129])
def test_all_ones_reach_every_count(m):
    Xd = torch.ones((m, 16), dtype=torch.uint8, device="cuda")
    Xd[::2, 1] = 0                                   # column 1: ceil(m / 2) ... zeros on even rows
    got = gbmi.counts_all_pairs(Xd, path="plain").cpu().numpy()
    gbmi.sync()
    odd = m // 2
    assert got[0, 0] == m and got[2, 15] == m
    assert got[1, 1] == odd and got[0, 1] == odd and got[1, 0] == odd


def test_fallback_shapes_use_the_packed_path():
    X = _data(1000, 200, 16)                         # n % 16 != 0
    want, _ = oracle.mi_matrix(X)
    got = gbmi.mi_all_pairs(torch.from_numpy(X).cuda(), path="fused")
    gbmi.sync()
    assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - want)) <= 1e-6
    X = _data(1000, 64, 17)                          # unaligned base: 1 byte in
    buf = torch.zeros(1000 * 64 + 16, dtype=torch.uint8, device="cuda")
    view = buf[1:1 + 1000 * 64].view(1000, 64)
    view.copy_(torch.from_numpy(X).cuda())
    got = gbmi.mi_all_pairs(view, path="fused")
    gbmi.sync()
    want, _ = oracle.mi_matrix(X)
    assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - want)) <= 1e-6


def test_non_binary_byte_is_reported():
    X = torch.from_numpy(_data(500, 64, 18)).cuda()
    X[7, 9] = 2
    gbmi.mi_all_pairs(X, path="fused")
    with pytest.raises(gbmi.GbmiError) as e:
        gbmi.sync()
    assert e.value.status == gbmi.ERR_NOT_BINARY
    X[7, 9] = 1                                      # the context is still usable
    got = gbmi.mi_all_pairs(X, path="fused")
    gbmi.sync()
    want, _ = oracle.mi_matrix(X.cpu().numpy())
    assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - want)) <= 1e-6


def test_out_of_core_panels():
    X = torch.from_numpy(_data(3000, 1024, 19)).cuda()
    want = gbmi.mi_all_pairs(X, path="fused").cpu()
    got = gbmi.mi_all_pairs_to_host(X, panel_rows=300)
    assert torch.equal(got, want)
    Y = torch.from_numpy(_data(3000, 160, 20)).cuda()
    got = gbmi.mi_cross_to_host(X, Y, panel_rows=128)
    assert torch.equal(got, gbmi.mi_cross(X, Y, path="fused").cpu())
