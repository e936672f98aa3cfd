"""Pins of the FP64 CPU oracle to facts fixed by the paper and by mathematics.

None of these checks re-types the oracle's formula.  They compare it with
  * hand-worked cases (tests/golden/hand_cases.txt, derived from Eq. 1/Eq. 2),
  * closed forms: MI(X;X) = MI(X;not X) = H(X), MI = 0 for a constant column and
    for a product (exactly independent) design,
  * numpy's integer Gram X^T X for the co-occurrence counts (Sec. 2 step 2),
  * the entropy decomposition MI = H(X) + H(Y) - H(X,Y) counted by brute force
    over sample tuples,
  * scikit-learn's ``mutual_info_score`` (the paper's pairwise baseline, Table 1),
    converted from nats to bits,
  * invariants: symmetry, 0 <= MI <= min(H(X), H(Y)), invariance under
    complementing a column, permuting samples and duplicating the dataset.
``test_planted_mistakes_are_caught`` compiles copies of the C source with one
plausible mistake each (a dropped term, a wrong sign, a wrong marginal, a
transposed operand, the wrong log base, a skipped sample, swapped cell labels)
and checks that at least one pin fails for every copy.
"""
from __future__ import annotations

import math
import os
from collections import Counter

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.txt")


def _closed_form(expr: str) -> float:
    return float(eval(expr, {"__builtins__": {}}, {"log2": math.log2}))


def load_hand_cases():
    cases = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            xs, ys, cnt, expr = line.split("|")
            x = np.array([int(c) for c in xs], dtype=np.uint8)
            y = np.array([int(c) for c in ys], dtype=np.uint8)
            cases.append((x, y, [int(t) for t in cnt.split()], expr.strip()))
    return cases


def entropy_bits(k: int, m: int) -> float:
    """H of a binary variable with k ones in m samples."""
    out = 0.0
    for c in (k, m - k):
        if c:
            p = c / m
            out -= p * math.log2(p)
    return out


def brute_force_mi(x: np.ndarray, y: np.ndarray) -> float:
    """MI = H(X) + H(Y) - H(X,Y), each entropy counted over sample tuples."""
    m = len(x)

    def H(seq):
        cnt = Counter(seq)
        return -math.fsum((c / m) * math.log2(c / m) for c in cnt.values())

    return H(x.tolist()) + H(y.tolist()) - H(list(zip(x.tolist(), y.tolist())))


def _rand_binary(rng, m, n, lo=0.05, hi=0.6):
    p = rng.uniform(lo, hi, size=n)
    return (rng.random((m, n)) < p).astype(np.uint8)


# ----------------------------------------------------------------------------
# pins: each takes an oracle.Oracle and returns a list of failure messages
# ----------------------------------------------------------------------------

def pin_hand_cases(o):
    bad = []
    for x, y, cnt, expr in load_hand_cases():
        X = np.stack([x, y], axis=1)
        counts, mi = o.mi_pairs(X, [0], [1])
        if counts[0].tolist() != cnt:
            bad.append(f"hand case {expr}: counts {counts[0].tolist()} != {cnt}")
        want = _closed_form(expr)
        if not abs(mi[0] - want) <= 1e-14:
            bad.append(f"hand case {expr}: MI {mi[0]!r} != {want!r}")
    return bad


def pin_closed_forms(o):
    bad = []
    rng = np.random.default_rng(11)
    m, n = 777, 12
    X = _rand_binary(rng, m, n)
    X[:, 3] = 0          # constant zero column
    X[:, 7] = 1          # constant one column
    notX = (1 - X).astype(np.uint8)
    both = np.concatenate([X, notX], axis=1)
    M, _ = o.mi_matrix(both)
    v = X.sum(axis=0)
    for j in range(n):
        h = entropy_bits(int(v[j]), m)
        if abs(M[j, j] - h) > 1e-13:
            bad.append(f"MI(X;X) != H(X) at column {j}: {M[j, j]} vs {h}")
        if abs(M[j, n + j] - h) > 1e-13:
            bad.append(f"MI(X;not X) != H(X) at column {j}: {M[j, n + j]} vs {h}")
    for c in (3, 7):
        if np.max(np.abs(M[c, :])) > 1e-15 or np.max(np.abs(M[:, c])) > 1e-15:
            bad.append(f"constant column {c} has non-zero MI")
    # exact product design: every (x, y) combination with multiplicity a_x * b_y
    a = {0: 3, 1: 5}
    b = {0: 7, 1: 2}
    xs, ys = [], []
    for xv in (0, 1):
        for yv in (0, 1):
            xs += [xv] * (a[xv] * b[yv])
            ys += [yv] * (a[xv] * b[yv])
    Xi = np.stack([np.array(xs, np.uint8), np.array(ys, np.uint8)], axis=1)
    _, mi = o.mi_pairs(Xi, [0], [1])
    if abs(mi[0]) > 1e-15:
        bad.append(f"independent product design has MI {mi[0]}")
    return bad


def pin_numpy_gram(o):
    bad = []
    rng = np.random.default_rng(12)
    X = _rand_binary(rng, 301, 19)
    _, n11 = o.mi_matrix(X)
    G = X.astype(np.int64).T @ X.astype(np.int64)
    if not np.array_equal(n11, G):
        bad.append("N11 differs from numpy X^T X")
    if not np.array_equal(o.column_counts(X), X.sum(axis=0).astype(np.int64)):
        bad.append("column counts differ from numpy sums")
    if not np.array_equal(np.diag(n11), X.sum(axis=0)):
        bad.append("diag(N11) != column sums")
    return bad


def pin_cell_counts(o):
    bad = []
    rng = np.random.default_rng(13)
    X = _rand_binary(rng, 257, 9)
    Y = _rand_binary(rng, 257, 9)
    i = np.repeat(np.arange(9), 9)
    j = np.tile(np.arange(9), 9)
    counts, _ = o.mi_pairs(X, i, j, Y=Y)
    vx, vy = X.sum(axis=0), Y.sum(axis=0)
    n11, n10, n01, n00 = counts.T
    direct11 = (X[:, i] & Y[:, j]).sum(axis=0)
    if not np.array_equal(n11, direct11):
        bad.append("n11 differs from a direct AND count")
    if not np.all(counts.sum(axis=1) == 257):
        bad.append("cells do not sum to m")
    if not np.array_equal(n11 + n10, vx[i]):
        bad.append("n11 + n10 != ones of the first variable")
    if not np.array_equal(n11 + n01, vy[j]):
        bad.append("n11 + n01 != ones of the second variable")
    if not np.array_equal(n00, ((1 - X[:, i]) & (1 - Y[:, j])).sum(axis=0)):
        bad.append("n00 differs from a direct count of common zeros")
    return bad


def pin_brute_force(o):
    bad = []
    rng = np.random.default_rng(14)
    for trial in range(40):
        m = int(rng.integers(1, 40))
        X = (rng.random((m, 2)) < rng.uniform(0.1, 0.9, 2)).astype(np.uint8)
        Y = (rng.random((m, 3)) < rng.uniform(0.1, 0.9, 3)).astype(np.uint8)
        M, _ = o.mi_matrix(X, Y)
        for a in range(2):
            for b in range(3):
                want = brute_force_mi(X[:, a], Y[:, b])
                if abs(M[a, b] - want) > 1e-13:
                    bad.append(f"brute force m={m} ({a},{b}): {M[a, b]} vs {want}")
        counts, mi = o.mi_pairs(X, [0, 1, 1], [2, 0, 1], Y=Y)
        for k, (a, b) in enumerate([(0, 2), (1, 0), (1, 1)]):
            want = brute_force_mi(X[:, a], Y[:, b])
            if abs(mi[k] - want) > 1e-13:
                bad.append(f"brute force pairs m={m} ({a},{b}): {mi[k]} vs {want}")
    return bad


def pin_sklearn(o):
    skm = pytest.importorskip("sklearn.metrics")
    bad = []
    rng = np.random.default_rng(15)
    X = _rand_binary(rng, 500, 7)
    Y = _rand_binary(rng, 500, 5)
    Y[:, 0] = X[:, 2] ^ (rng.random(500) < 0.1)   # one strongly dependent pair
    M, _ = o.mi_matrix(X, Y)
    pi = np.array([0, 2, 6, 3, 1], np.int64)
    pj = np.array([4, 0, 1, 3, 2], np.int64)
    _, mip = o.mi_pairs(X, pi, pj, Y=Y)
    for a in range(7):
        for b in range(5):
            want = skm.mutual_info_score(X[:, a], Y[:, b]) / math.log(2)
            if abs(M[a, b] - want) > 1e-12:
                bad.append(f"sklearn ({a},{b}): {M[a, b]} vs {want}")
    for k in range(len(pi)):
        want = skm.mutual_info_score(X[:, pi[k]], Y[:, pj[k]]) / math.log(2)
        if abs(mip[k] - want) > 1e-12:
            bad.append(f"sklearn pair ({pi[k]},{pj[k]}): {mip[k]} vs {want}")
    return bad


def pin_invariants(o):
    bad = []
    rng = np.random.default_rng(16)
    m, n = 613, 10
    X = _rand_binary(rng, m, n, 0.02, 0.5)
    X[:, 5] = X[:, 1] ^ (rng.random(m) < 0.05)
    M, _ = o.mi_matrix(X)
    v = X.sum(axis=0)
    H = np.array([entropy_bits(int(k), m) for k in v])
    if np.max(np.abs(M - M.T)) > 1e-15:
        bad.append("MI matrix not symmetric")
    if np.min(M) < -1e-15:
        bad.append(f"negative MI {np.min(M)}")
    if np.any(M > np.minimum.outer(H, H) + 1e-12):
        bad.append("MI exceeds min(H(X), H(Y))")
    Xc = X.copy()
    Xc[:, 1] = 1 - Xc[:, 1]
    Mc, _ = o.mi_matrix(Xc)
    if np.max(np.abs(Mc - M)) > 1e-13:
        bad.append("MI changes when a column is complemented")
    perm = rng.permutation(m)
    Mp, _ = o.mi_matrix(X[perm])
    if not np.array_equal(Mp, M):
        bad.append("MI changes when samples are permuted")
    Md, _ = o.mi_matrix(np.concatenate([X, X], axis=0))
    if np.max(np.abs(Md - M)) > 1e-13:
        bad.append("MI changes when the dataset is duplicated")
    return bad


PINS = [pin_hand_cases, pin_closed_forms, pin_numpy_gram, pin_cell_counts, pin_brute_force,
        pin_sklearn, pin_invariants]


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    bad = pin(orc)
    assert not bad, "\n".join(bad[:10])


def test_mi_from_counts_special_values(orc):
    assert orc.mi_from_counts(0, 0, 0, 0) == 0.0
    assert orc.mi_from_counts(5, 0, 0, 0) == 0.0        # one occupied cell: no information
    assert orc.mi_from_counts(3, 0, 0, 3) == pytest.approx(1.0, abs=1e-15)
    assert orc.mi_from_counts(0, 3, 3, 0) == pytest.approx(1.0, abs=1e-15)


def test_pair_index_checked(orc):
    X = np.zeros((4, 3), np.uint8)
    with pytest.raises(IndexError):
        orc.mi_pairs(X, [0], [3])


# (old text, new text) edits, one plausible mistake each
MUTANTS = {
    "drop_00_term": ("if (n00 > 0) mi += p00", "if (0) mi += p00"),
    "wrong_sign_10": ("if (n10 > 0) mi += p10", "if (n10 > 0) mi -= p10"),
    "wrong_marginal": ("const double py1 = p11 + p01", "const double py1 = p11 + p10"),
    "transposed_pair": ("oracle_cell_counts(AT + pi[k] * m, BT + pj[k] * m",
                        "oracle_cell_counts(AT + pj[k] * m, BT + pi[k] * m"),
    "natural_log": ("p11 * log2(p11", "p11 * log(p11"),
    "skip_last_sample": ("for (int64_t r = 0; r < m; ++r) {\n        int a",
                         "for (int64_t r = 0; r + 1 < m; ++r) {\n        int a"),
    "swapped_cell_labels": ("cnt[1] = c[1][0];\n    cnt[2] = c[0][1];",
                            "cnt[1] = c[0][1];\n    cnt[2] = c[1][0];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_are_caught(name, tmp_path):
    pytest.importorskip("sklearn.metrics")
    old, new = MUTANTS[name]
    with open(oracle.SOURCE) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    path = tmp_path / f"mutant_{name}.c"
    path.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(path), str(tmp_path / f"libmutant_{name}.so"))
    mutant = oracle.Oracle(lib)
    failures = []
    for pin in PINS:
        failures += pin(mutant)
    assert failures, f"no pin caught the planted mistake {name}"
