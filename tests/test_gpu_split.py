"""Tensor-core Grams with fewer tiles than SMs, split over sample ranges.

Each part writes its exact int32 counts into its own slice; the MI (or
counts) kernel adds the slices.  Results must be bit-identical with the split
off (one launch over all samples), on the fused, plain and counts calls, all
pairs and cross, including parts that end inside a K block and sample counts
beyond 2^24, and MI within 1e-6 of the oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


def _rand(m, n, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    p = torch.rand(n, generator=g, device="cuda") * 0.45 + 0.01
    return (torch.rand((m, n), generator=g, device="cuda") < p).to(torch.uint8)


@pytest.fixture
def split_modes():
    yield
    gbmi.set_option(gbmi.OPT_SPLIT_K, 0)


def _run(fn, mode):
    gbmi.set_option(gbmi.OPT_SPLIT_K, mode)
    out = fn()
    gbmi.sync()
    return out


@pytest.mark.parametrize("m,n", [(200_000, 100), (100_000, 1000), (65_537, 300), (40_000, 16)])
def test_split_equals_unsplit(split_modes, m, n):
    X = _rand(m, n, m + n)
    for path in ("fused", "plain"):
        split = _run(lambda: gbmi.mi_all_pairs(X, path=path), 0)
        whole = _run(lambda: gbmi.mi_all_pairs(X, path=path), 1)
        assert torch.equal(split, whole), path
    cs = _run(lambda: gbmi.counts_all_pairs(X, path="plain"), 0)
    cw = _run(lambda: gbmi.counts_all_pairs(X, path="popcount"), 0)
    assert torch.equal(cs, cw)
    Y = _rand(m, n // 2 + 3, 7 * m + n)
    xs = _run(lambda: gbmi.mi_cross(X, Y, path="fused"), 0)
    xw = _run(lambda: gbmi.mi_cross(X, Y, path="fused"), 1)
    assert torch.equal(xs, xw)


def test_split_matches_oracle_and_is_taken(split_modes):
    X = _rand(120_000, 200, 3)
    gbmi.set_option(gbmi.OPT_SPLIT_K, 0)
    gbmi.profile(enable=True, reset=True)
    got = gbmi.mi_all_pairs(X, path="fused")
    gbmi.sync()
    prof = gbmi.profile(enable=False)
    assert "gram_tc_split_counts" in prof and "mi_from_counts" in prof
    cols = np.arange(0, 200, 9)
    sub = X[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    want, _ = oracle.mi_matrix(sub)
    g = got[torch.from_numpy(cols).cuda()][:, torch.from_numpy(cols).cuda()]
    assert np.max(np.abs(g.double().cpu().numpy() - want)) <= 1e-6


def test_forced_split_on_a_small_case_and_fp64_combine(split_modes):
    X = _rand(9000, 70, 4)
    for fix in (0, 1):
        gbmi.set_option(gbmi.OPT_FIXUP, fix)
        try:
            a = _run(lambda: gbmi.mi_all_pairs(X, path="fused"), 2)
            b = _run(lambda: gbmi.mi_all_pairs(X, path="fused"), 1)
        finally:
            gbmi.set_option(gbmi.OPT_FIXUP, 0)
        assert torch.equal(a, b)
        want, _ = oracle.mi_matrix(X.cpu().numpy())
        assert np.max(np.abs(a.cpu().numpy().astype(np.float64) - want)) <= 1e-6


def test_split_beyond_one_exact_chunk(split_modes):
    m, n = (1 << 24) + 129, 40
    X = _rand(m, n, 5)
    a = _run(lambda: gbmi.counts_all_pairs(X, path="plain"), 0)
    b = _run(lambda: gbmi.counts_all_pairs(X, path="popcount"), 0)
    assert torch.equal(a, b)
    f0 = _run(lambda: gbmi.mi_all_pairs(X, path="fused"), 0)
    f1 = _run(lambda: gbmi.mi_all_pairs(X, path="fused"), 1)
    assert torch.equal(f0, f1)
