"""Tail split of the fused MI launch (GBMI_OPT_TAIL_SPLIT).

The last tiles of the persistent Gram launch run as units that each add up a
share of the samples; every unit stores its exact int32 counts, and the unit
that arrives last adds the others' counts to its own before the MI epilogue.
Counts are integers either way, so the MI must be bit-identical to the
unsplit launch, on the single-CTA and the CTA-pair kernels, for all pairs and
cross problems, FP4 and FP8 operands, forced splits of every tile into 2 to 5
parts, and within 1e-6 of the FP64 oracle.
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
    gbmi.set_option(gbmi.OPT_TAIL_SPLIT, 0)
    gbmi.set_option(gbmi.OPT_PAIR, 1)
    gbmi.set_option(gbmi.OPT_FP4, 1)
    gbmi.set_option(gbmi.OPT_SPLIT_K, 0)


def _run(X, split, Y=None):
    gbmi.set_option(gbmi.OPT_TAIL_SPLIT, split)
    n = X.shape[1]
    shape = (n, n) if Y is None else (n, Y.shape[1])
    out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    if Y is None:
        gbmi.mi_all_pairs(X, out=out, path="fused")
    else:
        gbmi.mi_cross(X, Y, out=out, path="fused")
    gbmi.sync()
    return out


@pytest.mark.parametrize("pair", [0, 2])
@pytest.mark.parametrize("fp4", [1, 0])
@pytest.mark.parametrize("m,n", [(3000, 700), (1031, 300), (20000, 1300), (700, 2500)])
def test_forced_split_is_bit_identical(m, n, pair, fp4):
    gbmi.set_option(gbmi.OPT_PAIR, pair)
    gbmi.set_option(gbmi.OPT_FP4, fp4)
    gbmi.set_option(gbmi.OPT_SPLIT_K, 1)
    X = _data(m, n, m + n)
    ref = _run(X, 0)
    assert not torch.isnan(ref).any()
    for parts in (2, 3, 5):
        got = _run(X, parts)
        assert torch.equal(got, ref), parts
    assert torch.equal(_run(X, 1), ref)


@pytest.mark.parametrize("pair", [0, 2])
def test_split_cross_is_bit_identical(pair):
    gbmi.set_option(gbmi.OPT_PAIR, pair)
    gbmi.set_option(gbmi.OPT_SPLIT_K, 1)
    X, Y = _data(4000, 600, 5), _data(4000, 900, 6)
    ref = _run(X, 0, Y)
    for parts in (2, 4):
        assert torch.equal(_run(X, parts, Y), ref)


def test_split_matches_oracle():
    gbmi.set_option(gbmi.OPT_PAIR, 2)
    X = _data(2000, 520, 9)
    got = _run(X, 3).cpu().numpy().astype(np.float64)
    want, _ = oracle.mi_matrix(X.cpu().numpy())
    assert float(np.max(np.abs(got - want))) <= 1e-6
    assert np.array_equal(got, got.T)


def test_automatic_split_at_paper_width():
    # 10,000 variables on CTA pairs: 865 tiles of 256 x 240 on 76 pairs, so
    # the automatic rule splits the last 29 + 76 tiles; results must not move
    X = _data(3000, 10000, 11)
    ref = _run(X, 0)
    assert torch.equal(_run(X, 1), ref)
    assert not torch.isnan(ref).any()
