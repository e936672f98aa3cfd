"""Sparse input (CSR by samples): pair counts from each sample's ones, or the
dense 0/1 matrix written from the CSR arrays and the tensor-core path.

Every test runs with both forms forced.  Counts must be bit-exact against the
oracle's direct cell counts; MI within 1e-6 of the oracle and bit-identical to
the dense plain path (same counts, same per-pair arithmetic).  Edge cases:
empty samples, no ones at all, a sample with every variable set, m = 1,
n = 1.  Malformed CSR (indices out of range or not increasing, row bounds
outside the index array) is skipped by the kernels' own checks and reported,
and the context stays usable.  The cost model picks each form where it is
the cheaper one.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, params=[1, 2], ids=["enumerate", "densify"])
def csr_path(request):
    gbmi.set_option(gbmi.OPT_CSR_PATH, request.param)
    yield request.param
    gbmi.set_option(gbmi.OPT_CSR_PATH, 0)


def _data(m, n, seed, lo, hi):
    rng = np.random.default_rng(seed)
    p = rng.uniform(lo, hi, size=n)
    return (rng.random((m, n)) < p).astype(np.uint8)


def _csr(X):
    """CSR by samples, built on the host with numpy (independent of the library)."""
    rows, cols = np.nonzero(X)
    row_ptr = np.zeros(X.shape[0] + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return (torch.from_numpy(row_ptr).cuda(),
            torch.from_numpy(cols.astype(np.int32)).cuda())


CASES = [(1000, 200, 0.001, 0.05), (129, 127, 0.01, 0.3), (1031, 300, 0.0, 0.02),
         (2000, 520, 0.002, 0.01), (1, 5, 0.2, 0.8), (37, 1, 0.1, 0.9), (5000, 64, 0.05, 0.5)]


@pytest.mark.parametrize("m,n,lo,hi", CASES)
def test_counts_exact(m, n, lo, hi):
    X = _data(m, n, m + n, lo, hi)
    rp, ci = _csr(X)
    got = gbmi.counts_all_pairs_csr(rp, ci, n)
    gbmi.sync()
    _, n11 = oracle.mi_matrix(X)
    assert np.array_equal(got.cpu().numpy(), n11)


@pytest.mark.parametrize("m,n,lo,hi", CASES)
def test_mi_matches_oracle_and_dense_path(m, n, lo, hi):
    X = _data(m, n, 7 * m + n, lo, hi)
    rp, ci = _csr(X)
    got = gbmi.mi_all_pairs_csr(rp, ci, n)
    gbmi.sync()
    want, _ = oracle.mi_matrix(X)
    assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - want)) <= 1e-6
    dense = gbmi.mi_all_pairs(torch.from_numpy(X).cuda(), path="plain")
    gbmi.sync()
    assert torch.equal(got, dense)


def test_edge_rows_and_empty_matrix():
    X = _data(300, 70, 3, 0.01, 0.1)
    X[5] = 0                      # empty sample
    X[6] = 1                      # every variable set
    X[:, 9] = 0                   # a variable that is never 1
    rp, ci = _csr(X)
    got = gbmi.mi_all_pairs_csr(rp, ci, 70)
    gbmi.sync()
    want, _ = oracle.mi_matrix(X)
    assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - want)) <= 1e-6
    Z = np.zeros((50, 20), dtype=np.uint8)
    rp, ci = _csr(Z)
    got = gbmi.mi_all_pairs_csr(rp, ci, 20)
    gbmi.sync()
    assert torch.count_nonzero(got) == 0


def test_helper_matches_host_csr():
    X = _data(777, 130, 4, 0.01, 0.2)
    rp, ci = gbmi.csr_from_dense(torch.from_numpy(X).cuda())
    hrp, hci = _csr(X)
    assert torch.equal(rp, hrp) and torch.equal(ci, hci)


def test_larger_case_against_dense_tensor_core_path():
    X = torch.from_numpy(_data(100_000, 2000, 5, 0.0005, 0.01)).cuda()
    rp, ci = gbmi.csr_from_dense(X)
    got = gbmi.counts_all_pairs_csr(rp, ci, 2000)
    want = gbmi.counts_all_pairs(X, path="plain")
    gbmi.sync()
    assert torch.equal(got, want)
    mi = gbmi.mi_all_pairs_csr(rp, ci, 2000)
    gbmi.sync()
    assert torch.equal(mi, gbmi.mi_all_pairs(X, path="plain"))


@pytest.mark.parametrize("bad", ["unsorted", "duplicate", "out_of_range", "negative",
                                 "row_past_end"])
def test_malformed_csr_is_reported(bad):
    X = _data(200, 40, 6, 0.05, 0.3)
    rows, cols = np.nonzero(X)
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=200))]).astype(np.int64)
    cols = cols.astype(np.int32)
    r = int(np.argmax(np.diff(row_ptr) >= 3))   # a row with at least 3 ones
    b = int(row_ptr[r])
    if bad == "unsorted":
        cols[b], cols[b + 1] = cols[b + 1], cols[b]
    elif bad == "duplicate":
        cols[b + 1] = cols[b]
    elif bad == "out_of_range":
        cols[b] = 40
    elif bad == "negative":
        cols[b] = -1
    else:
        row_ptr[-1] = row_ptr[-1] + 5               # last row reaches past col_idx
    gbmi.mi_all_pairs_csr(torch.from_numpy(row_ptr).cuda(), torch.from_numpy(cols).cuda(), 40)
    with pytest.raises(gbmi.GbmiError) as e:
        gbmi.sync()
    assert e.value.status == gbmi.ERR_ARG
    rp, ci = _csr(X)                                  # the context still computes
    got = gbmi.mi_all_pairs_csr(rp, ci, 40)
    gbmi.sync()
    want, _ = oracle.mi_matrix(X)
    assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - want)) <= 1e-6


def test_cost_model_choice_and_agreement(csr_path):
    """Both forms give the same bits; with the model on, a sparse case takes the
    enumeration and a moderately sparse one the dense path (seen in the launch
    profile), with the same results."""
    if csr_path != 1:
        pytest.skip("runs once")
    cases = {"sparse": _data(20_000, 3000, 8, 0.0, 0.0004),
             "moderate": _data(20_000, 3000, 9, 0.005, 0.03)}
    for name, Xn in cases.items():
        X = torch.from_numpy(Xn).cuda()
        rp, ci = gbmi.csr_from_dense(X)
        outs = {}
        for mode in (1, 2, 0):
            gbmi.set_option(gbmi.OPT_CSR_PATH, mode)
            gbmi.profile(enable=True, reset=True)
            outs[mode] = gbmi.mi_all_pairs_csr(rp, ci, 3000)
            gbmi.sync()
            prof = gbmi.profile(enable=False)
            if mode == 0:
                took_dense = "csr_densify" in prof
                assert took_dense == (name == "moderate"), (name, sorted(prof))
        assert torch.equal(outs[1], outs[2]) and torch.equal(outs[0], outs[1])
