"""The paper's algebra and the per-pair formulas of the CUDA epilogue, on the CPU.

These tests involve neither the CUDA library nor its code: they check, in
exact integers or FP64 numpy, the identities the CUDA path relies on, so a
misreading of the paper shows up here first.

* Sec. 3.1, Eq. 6 and Eq. 7: with v = X^T 1 (the column counts) and C_ij = v_j,
  G00 = N - C - C^T + G11, G01 = C - G11, G10 = G01^T, where G_ab counts
  samples with (X_i, X_j) = (a, b).  (The paper's own text describes C three
  ways; only C_ij = v_j makes G01 the "0 then 1" count, which these checks fix.)
* Sec. 2 step 3: diag(G11) = v and diag(G00) = m - v.
* Epilogue form: with det = n11*n00 - n10*n01, every cell satisfies
  n_c*m - a_c*b_c = s_c*det (s = +1 for 11/00, -1 for 10/01), so
  MI = (1/m) sum_c n_c log2(1 + s_c det / (a_c b_c)).
* Fix-up form (n log n): m*MI = sum_c T(n_c) - T(v_i) - T(m - v_i) - T(v_j)
  - T(m - v_j) + T(m) with T(k) = k log2 k, which follows from Eq. 1.
"""
from __future__ import annotations

import numpy as np

import oracle


def _data(seed=21, m=389, n=23):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.02, 0.6, size=n)
    X = (rng.random((m, n)) < p).astype(np.int64)
    X[:, 4] = 0
    X[:, 9] = 1
    X[:, 11] = X[:, 2]
    X[:, 12] = 1 - X[:, 2]
    return X


def test_eq6_eq7_gram_identities():
    X = _data()
    m, n = X.shape
    nX = 1 - X
    G11 = X.T @ X
    G00 = nX.T @ nX           # common zeros
    G01 = nX.T @ X            # (X_i, X_j) = (0, 1)
    G10 = X.T @ nX            # (X_i, X_j) = (1, 0)
    v = X.sum(axis=0)
    N = np.full((n, n), m)
    C = np.tile(v, (n, 1))    # C_ij = v_j: every row is v^T
    assert np.array_equal(G00, N - C - C.T + G11)          # Eq. 6
    assert np.array_equal(G01, C - G11)                    # Eq. 7
    assert np.array_equal(G10, G01.T)
    assert np.array_equal(np.diag(G11), v)                 # marginals from the diagonal
    assert np.array_equal(np.diag(G00), m - v)
    # the other reading of C (every column is v) gives the transposed count
    assert not np.array_equal(G01, C.T - G11)


def test_counts_from_gram_match_oracle_cells():
    X = _data(22)
    m, n = X.shape
    G11 = X.T @ X
    v = X.sum(axis=0)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    n11 = G11[i, j]
    n10 = v[i] - n11
    n01 = v[j] - n11
    n00 = m - v[i] - v[j] + n11
    counts, _ = oracle.mi_pairs(X.astype(np.uint8), i, j)
    assert np.array_equal(counts, np.stack([n11, n10, n01, n00], axis=1))


def _cells(X):
    m, n = X.shape
    G11 = X.T @ X
    v = X.sum(axis=0)
    vi, vj = v[:, None], v[None, :]
    n11 = G11
    n10 = vi - n11
    n01 = vj - n11
    n00 = m - vi - vj + n11
    return m, v, n11, n10, n01, n00


def test_determinant_form_matches_oracle():
    X = _data(23)
    m, v, n11, n10, n01, n00 = _cells(X)
    vi, vj = v[:, None].astype(np.int64), v[None, :].astype(np.int64)
    det = n11 * n00 - n10 * n01
    cells = [(n11, vi, vj, 1), (n10, vi, m - vj, -1), (n01, m - vi, vj, -1),
             (n00, m - vi, m - vj, 1)]
    total = np.zeros(n11.shape)
    for nc, a, b, s in cells:
        # the identity n_c*m - a*b = s*det, exactly in integers
        assert np.array_equal(nc * m - a * b, s * det)
        with np.errstate(divide="ignore", invalid="ignore"):
            term = nc * np.log1p(s * det / (a * b).astype(np.float64)) / np.log(2.0)
        total += np.where(nc > 0, term, 0.0)
    mi = total / m
    want, _ = oracle.mi_matrix(X.astype(np.uint8))
    assert np.max(np.abs(mi - want)) < 1e-14
    assert np.all((det == 0) <= (np.abs(want) < 1e-15))


def test_nlogn_form_matches_oracle():
    X = _data(24)
    m, v, n11, n10, n01, n00 = _cells(X)

    def T(k):
        k = np.asarray(k, dtype=np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(k > 0, k * np.log2(np.where(k > 0, k, 1.0)), 0.0)

    vi, vj = v[:, None], v[None, :]
    s = (T(n11) + T(n00)) + (T(n10) + T(n01))
    mi = (s + (T(m) - ((T(vi) + T(m - vi)) + (T(vj) + T(m - vj))))) / m
    want, _ = oracle.mi_matrix(X.astype(np.uint8))
    assert np.max(np.abs(mi - want)) < 1e-13
