"""Exact counts at the accumulation limits, and the bounded device-side waits.

FP32 accumulation of 0/1 FP4 or FP8 products is exact while a count stays at
most 2^24; one Gram launch therefore accumulates at most 2^24 samples, the
plain path adds launch results in int32, and the fused path adds the earlier
chunks' int32 counts to its last launch's accumulator.  All-ones columns
make every accumulator reach m, the largest value it can hold for that m.
Every test runs with both operand forms (FP4: 256 samples per K block; FP8:
128).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, params=[1, 0], ids=["fp4", "fp8"])
def _operand_form(request):
    gbmi.set_option(gbmi.OPT_FP4, request.param)
    yield request.param
    gbmi.set_option(gbmi.OPT_FP4, 1)


@pytest.fixture(autouse=True)
def _reset_options():
    gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 0)
    gbmi.set_option(gbmi.OPT_TIMEOUT_NS, 2_000_000_000)
    yield
    gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 0)
    gbmi.set_option(gbmi.OPT_TIMEOUT_NS, 2_000_000_000)


@pytest.mark.parametrize("m", [1 << 10, 1 << 14, (1 << 20) + 3, (1 << 24) - 1, 1 << 24,
                               (1 << 24) + 1])
def test_all_ones_counts_reach_m(m):
    n = 8
    X = torch.ones((m, n), dtype=torch.uint8, device="cuda")
    for path in ("plain", "popcount"):
        c = gbmi.counts_all_pairs(X, path=path)
        gbmi.sync()
        assert torch.all(c == m).item(), f"{path}: counts differ from m={m}"
    # fused MI (one or two sample chunks): constant columns carry no information
    out = gbmi.mi_all_pairs(X, path="fused")
    gbmi.sync()
    assert torch.all(out == 0).item()


def test_counts_beyond_one_exact_chunk():
    """m = 2^24 + 129: two Gram launches whose int32 results are added."""
    m, n = (1 << 24) + 129, 8
    X = torch.ones((m, n), dtype=torch.uint8, device="cuda")
    X[5:, 3] = 0          # column 3 has 5 ones
    X[::2, 4] = 0         # column 4 has ceil(m/2) ones at odd rows
    c = gbmi.counts_all_pairs(X, path="plain")
    p = gbmi.counts_all_pairs(X, path="popcount")
    gbmi.sync()
    assert torch.equal(c, p)
    assert c[0, 0].item() == m and c[3, 3].item() == 5 and c[4, 4].item() == m // 2
    # AUTO takes the fused path in two sample chunks; MI of the constant
    # columns is 0 and MI(col 3; col 4) matches the oracle's counts
    out = gbmi.mi_all_pairs(X, path="auto")
    plain = gbmi.mi_all_pairs(X, path="plain")
    gbmi.sync()
    assert torch.equal(out, plain)
    cnt = c.cpu().numpy().astype(np.int64)
    n11 = cnt[3, 4]
    v3, v4 = cnt[3, 3], cnt[4, 4]
    want = oracle.mi_from_counts(n11, v3 - n11, v4 - n11, m - v3 - v4 + n11)
    assert abs(float(out[3, 4]) - want) <= 1e-6
    assert float(out[0, 1]) == 0.0


@pytest.mark.parametrize("fixup", [0, 1], ids=["fp32", "fp64_combine"])
def test_fused_mi_over_two_sample_chunks(fixup):
    """Random columns at m = 2^24 + 129: the fused path's two launches (int32
    counts of the first chunk added in the second one's MI epilogue) give the
    plain path's values bit for bit, and the oracle's within 1e-6 on sampled
    pairs (the sampled columns alone are copied to the host)."""
    m, n = (1 << 24) + 129, 200
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    p = torch.rand(n, generator=g, device="cuda") * 0.45 + 0.01
    X = (torch.rand((m, n), generator=g, device="cuda") < p).to(torch.uint8)
    X[:, 7] = X[:, 3] ^ (torch.rand(m, generator=g, device="cuda") < 0.05).to(torch.uint8)
    gbmi.set_option(gbmi.OPT_FIXUP, fixup)
    try:
        fused = gbmi.mi_all_pairs(X, path="fused")
        plain = gbmi.mi_all_pairs(X, path="plain")
        gbmi.sync()
    finally:
        gbmi.set_option(gbmi.OPT_FIXUP, 0)
    assert torch.equal(fused, plain)
    cols = np.array([0, 3, 7, 50, 101, 199])
    sub = X[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    pi, pj = np.triu_indices(len(cols))
    _, want = oracle.mi_pairs(sub, pi, pj)
    got = fused[torch.from_numpy(cols[pi]).cuda(), torch.from_numpy(cols[pj]).cuda()]
    assert np.max(np.abs(got.double().cpu().numpy() - want)) <= 1e-6
    assert float(fused[3, 7]) > 1e-3    # the planted noisy copy


def test_random_counts_at_precision_m_match_popcount():
    m, n = 1 << 20, 384
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    p = torch.rand(n, generator=g, device="cuda") * 0.48 + 0.02
    X = (torch.rand((m, n), generator=g, device="cuda") < p).to(torch.uint8)
    a = gbmi.counts_all_pairs(X, path="plain")
    b = gbmi.counts_all_pairs(X, path="popcount")
    gbmi.sync()
    assert torch.equal(a, b)
    assert torch.equal(torch.diagonal(a), X.sum(dim=0, dtype=torch.int32))


@pytest.mark.parametrize("pair", [0, 2], ids=["single", "pair"])
def test_bounded_wait_times_out_and_context_survives(pair):
    """The fused kernel's loader issues no copies (test hook), so its MMA
    thread's wait on the first stage can never complete: it must give up after
    the timeout, report GBMI_ERR_TIMEOUT, free its tensor memory and leave the
    context usable (single-CTA and CTA-pair kernels)."""
    X = torch.from_numpy((np.random.default_rng(1).random((512, 300)) < 0.3)
                         .astype(np.uint8)).cuda()
    gbmi.set_option(gbmi.OPT_PAIR, pair)
    gbmi.set_option(gbmi.OPT_TIMEOUT_NS, 50_000_000)
    gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 1)
    gbmi.mi_all_pairs(X, path="fused")
    with pytest.raises(gbmi.GbmiError) as e:
        gbmi.sync()
    assert e.value.status == gbmi.ERR_TIMEOUT
    gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 0)
    gbmi.set_option(gbmi.OPT_TIMEOUT_NS, 2_000_000_000)
    out = gbmi.mi_all_pairs(X, path="fused")
    gbmi.sync()
    gbmi.set_option(gbmi.OPT_PAIR, 1)
    want, _ = oracle.mi_matrix(X.cpu().numpy())
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - want)) <= 1e-6
