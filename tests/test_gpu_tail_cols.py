"""Column shares of the tail of a tensor-core launch (GBMI_OPT_TAIL_COLS).

The tiles of the persistent Gram launch's last partial wave run as 2 to 4
column shares each: every share is an MMA as wide as its columns (cut at
multiples of 32 after the tile's first needed column) over all samples, with
the epilogue's warps dividing the share's columns.  The counts are the same
integers, so MI and counts must be bit-identical to the unsplit launch, on the
single-CTA and the CTA-pair kernels, for all-pairs and cross problems, FP4 and
FP8 operands, the fused and the plain path, forced shares of every tile into
2, 3 and 4, and within 1e-6 of the FP64 oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


def _data(m, n, seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.02, 0.5, size=n)
    X = (rng.random((m, n)) < p).astype(np.uint8)
    if n > 3:
        X[:, 3] = X[:, 0]
    return torch.from_numpy(X).cuda()


@pytest.fixture(autouse=True)
def _restore():
    yield
    gbmi.set_option(gbmi.OPT_TAIL_COLS, 1)
    gbmi.set_option(gbmi.OPT_PAIR, 1)
    gbmi.set_option(gbmi.OPT_FP4, 1)
    gbmi.set_option(gbmi.OPT_SPLIT_K, 0)


def _mi(X, cols, Y=None, path="fused"):
    gbmi.set_option(gbmi.OPT_TAIL_COLS, cols)
    n = X.shape[1]
    shape = (n, n) if Y is None else (n, Y.shape[1])
    out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    if Y is None:
        gbmi.mi_all_pairs(X, out=out, path=path)
    else:
        gbmi.mi_cross(X, Y, out=out, path=path)
    gbmi.sync()
    return out


def _counts(X, cols, Y=None):
    gbmi.set_option(gbmi.OPT_TAIL_COLS, cols)
    if Y is None:
        c = gbmi.counts_all_pairs(X, path="plain")
    else:
        c = gbmi.counts_cross(X, Y, path="plain")
    gbmi.sync()
    return c


@pytest.mark.parametrize("pair", [0, 2])
@pytest.mark.parametrize("fp4", [1, 0])
@pytest.mark.parametrize("m,n", [(3000, 700), (1031, 300), (20000, 1300), (700, 2500),
                                 (900, 40)])
def test_forced_shares_are_bit_identical(m, n, pair, fp4):
    gbmi.set_option(gbmi.OPT_PAIR, pair)
    gbmi.set_option(gbmi.OPT_FP4, fp4)
    gbmi.set_option(gbmi.OPT_SPLIT_K, 1)
    X = _data(m, n, m + n)
    ref = _mi(X, 0)
    assert not torch.isnan(ref).any()
    for parts in (2, 3, 4):
        assert torch.equal(_mi(X, parts), ref), parts
    assert torch.equal(_mi(X, 1), ref)


@pytest.mark.parametrize("pair", [0, 2])
def test_forced_shares_counts_and_plain_path(pair):
    gbmi.set_option(gbmi.OPT_PAIR, pair)
    gbmi.set_option(gbmi.OPT_SPLIT_K, 1)
    X = _data(5000, 1100, 3)
    ref_c = _counts(X, 0)
    pop = gbmi.counts_all_pairs(X, path="popcount")
    gbmi.sync()
    assert torch.equal(ref_c, pop)
    ref_mi = _mi(X, 0, path="plain")
    for parts in (2, 3, 4):
        assert torch.equal(_counts(X, parts), ref_c), parts
        assert torch.equal(_mi(X, parts, path="plain"), ref_mi), parts


@pytest.mark.parametrize("pair", [0, 2])
def test_forced_shares_cross(pair):
    gbmi.set_option(gbmi.OPT_PAIR, pair)
    gbmi.set_option(gbmi.OPT_SPLIT_K, 1)
    X, Y = _data(4000, 600, 5), _data(4000, 900, 6)
    ref = _mi(X, 0, Y)
    ref_c = _counts(X, 0, Y)
    for parts in (2, 4):
        assert torch.equal(_mi(X, parts, Y), ref)
        assert torch.equal(_counts(X, parts, Y), ref_c)


def test_shares_match_oracle():
    gbmi.set_option(gbmi.OPT_PAIR, 2)
    X = _data(2000, 520, 9)
    got = _mi(X, 3).cpu().numpy().astype(np.float64)
    want, _ = oracle.mi_matrix(X.cpu().numpy())
    assert float(np.max(np.abs(got - want))) <= 1e-6
    assert np.array_equal(got, got.T)


def test_automatic_shares_at_paper_width():
    # 10,000 variables on CTA pairs: 865 tiles of 256 x 240 on 76 pairs, so
    # the automatic rule runs the last 29 tiles as two column shares each
    X = _data(3000, 10000, 11)
    ref = _mi(X, 0)
    assert not torch.isnan(ref).any()
    assert torch.equal(_mi(X, 1), ref)

