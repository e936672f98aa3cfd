"""Plain CPU oracle for all-pairs binary mutual information (FP64).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports, links or executes anything in this folder, and this folder imports
nothing from the product package.

The arithmetic lives in ``mi_oracle.c`` (plain C, OpenMP over pairs): for each
requested pair it walks all m samples, counts the four cells of the 2x2
contingency table and sums Eq. 1 / Eq. 2 of arXiv 2411.19702 in FP64 with
``log2``.  This module only compiles that file with gcc and marshals numpy
arrays into it.

Parity status: counts and MI are pinned (closed forms, hand-worked 4x2 and 6x2
cases, invariants, scikit-learn's ``mutual_info_score``, numpy's integer Gram
and exact high-precision brute force on tiny inputs; see
``tests/test_oracle_pins.py``, which also checks that planted mistakes in a
copy of the C source are caught).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "mi_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_default = None


def compile_source(src: str, out: str) -> str:
    """Compile an oracle C source file into a shared library (gcc, OpenMP when available)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``mi_oracle.c`` into ``_build/liboracle.so`` if it is missing or stale."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(SOURCE)):
        return _LIB_PATH
    return compile_source(SOURCE, _LIB_PATH)


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Oracle:
    """numpy front end of one compiled copy of the oracle's C source."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        f64p = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.oracle_transpose_u8.argtypes = [u8p, i64, i64, i64, u8p, ctypes.c_int]
        lib.oracle_transpose_u8.restype = None
        lib.oracle_mi_from_counts.argtypes = [i64, i64, i64, i64]
        lib.oracle_mi_from_counts.restype = ctypes.c_double
        lib.oracle_mi_pairs.argtypes = [u8p, i64, u8p, i64, i64, i64p, i64p, i64, i64p, f64p,
                                        ctypes.c_int]
        lib.oracle_mi_pairs.restype = ctypes.c_int
        lib.oracle_mi_matrix.argtypes = [u8p, i64, u8p, i64, i64, f64p, i64p, ctypes.c_int]
        lib.oracle_mi_matrix.restype = None
        lib.oracle_column_counts.argtypes = [u8p, i64, i64, i64p, ctypes.c_int]
        lib.oracle_column_counts.restype = None
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        self.lib = lib

    def max_threads(self) -> int:
        """Threads the OpenMP loops use by default (1 without OpenMP)."""
        return int(self.lib.oracle_max_threads())

    def transpose(self, X: np.ndarray, nthreads: int = 0) -> np.ndarray:
        """Samples x variables (m x n, uint8) -> variables x samples (n x m), contiguous."""
        X = np.ascontiguousarray(X, dtype=np.uint8)
        m, n = X.shape
        XT = np.empty((n, m), dtype=np.uint8)
        if m and n:
            self.lib.oracle_transpose_u8(_ptr(X, ctypes.c_uint8), m, n, n,
                                         _ptr(XT, ctypes.c_uint8), int(nthreads))
        return XT

    def mi_from_counts(self, n11: int, n10: int, n01: int, n00: int) -> float:
        """MI in bits of one 2x2 contingency table (Eq. 1 / Eq. 2)."""
        return float(self.lib.oracle_mi_from_counts(int(n11), int(n10), int(n01), int(n00)))

    def mi_pairs_t(self, AT: np.ndarray, BT: np.ndarray, pi, pj, nthreads: int = 0):
        """MI and cell counts for pairs (AT[pi[k]], BT[pj[k]]) of transposed data.

        Returns (counts int64[npairs, 4] as n11, n10, n01, n00; mi float64[npairs]).
        """
        AT = np.ascontiguousarray(AT, dtype=np.uint8)
        BT = np.ascontiguousarray(BT, dtype=np.uint8)
        if AT.shape[1] != BT.shape[1]:
            raise ValueError("AT and BT must have the same number of samples")
        m = AT.shape[1]
        pi = np.ascontiguousarray(pi, dtype=np.int64)
        pj = np.ascontiguousarray(pj, dtype=np.int64)
        if pi.shape != pj.shape or pi.ndim != 1:
            raise ValueError("pi and pj must be 1-D and of equal length")
        k = pi.shape[0]
        counts = np.zeros((k, 4), dtype=np.int64)
        mi = np.zeros(k, dtype=np.float64)
        if k == 0:
            return counts, mi
        rc = self.lib.oracle_mi_pairs(_ptr(AT, ctypes.c_uint8), AT.shape[0],
                                      _ptr(BT, ctypes.c_uint8), BT.shape[0], m,
                                      _ptr(pi, ctypes.c_int64), _ptr(pj, ctypes.c_int64), k,
                                      _ptr(counts, ctypes.c_int64), _ptr(mi, ctypes.c_double),
                                      int(nthreads))
        if rc != 0:
            raise IndexError("pair index out of range")
        return counts, mi

    def mi_pairs(self, X: np.ndarray, pi, pj, Y: np.ndarray | None = None, nthreads: int = 0):
        """MI and counts for pairs (column pi[k] of X, column pj[k] of Y, or of X)."""
        XT = self.transpose(X, nthreads)
        YT = XT if Y is None else self.transpose(Y, nthreads)
        return self.mi_pairs_t(XT, YT, pi, pj, nthreads)

    def mi_matrix(self, X: np.ndarray, Y: np.ndarray | None = None, nthreads: int = 0):
        """Full MI matrix (FP64, bits) and N11 counts between the columns of X and Y.

        Y=None gives the n x n all-pairs matrix of X (diagonal = entropy of each
        column); otherwise the n1 x n2 cross matrix.
        """
        XT = self.transpose(X, nthreads)
        YT = XT if Y is None else self.transpose(Y, nthreads)
        if XT.shape[1] != YT.shape[1]:
            raise ValueError("X and Y must have the same number of samples")
        na, nb, m = XT.shape[0], YT.shape[0], XT.shape[1]
        out = np.zeros((na, nb), dtype=np.float64)
        n11 = np.zeros((na, nb), dtype=np.int64)
        if na and nb:
            self.lib.oracle_mi_matrix(_ptr(XT, ctypes.c_uint8), na, _ptr(YT, ctypes.c_uint8), nb,
                                      m, _ptr(out, ctypes.c_double), _ptr(n11, ctypes.c_int64),
                                      int(nthreads))
        return out, n11

    def column_counts(self, X: np.ndarray, nthreads: int = 0) -> np.ndarray:
        """v_j = number of ones in column j of X (int64)."""
        XT = self.transpose(X, nthreads)
        v = np.zeros(XT.shape[0], dtype=np.int64)
        if XT.size:
            self.lib.oracle_column_counts(_ptr(XT, ctypes.c_uint8), XT.shape[0], XT.shape[1],
                                          _ptr(v, ctypes.c_int64), int(nthreads))
        return v


def default() -> Oracle:
    """The oracle compiled from ``mi_oracle.c`` (built on first use)."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
        return _default


def max_threads() -> int:
    return default().max_threads()


def transpose(X, nthreads: int = 0):
    return default().transpose(X, nthreads)


def mi_from_counts(n11, n10, n01, n00) -> float:
    return default().mi_from_counts(n11, n10, n01, n00)


def mi_pairs_t(AT, BT, pi, pj, nthreads: int = 0):
    return default().mi_pairs_t(AT, BT, pi, pj, nthreads)


def mi_pairs(X, pi, pj, Y=None, nthreads: int = 0):
    return default().mi_pairs(X, pi, pj, Y, nthreads)


def mi_matrix(X, Y=None, nthreads: int = 0):
    return default().mi_matrix(X, Y, nthreads)


def column_counts(X, nthreads: int = 0):
    return default().column_counts(X, nthreads)
