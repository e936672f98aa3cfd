"""The no-allocation entry point (mi_all_pairs_noalloc) against mi_all_pairs.

Some callers cannot let a library allocate device memory (their framework
owns the whole device through its own pool, or cudaFree's device-wide wait is
not acceptable in their loop).  mi_all_pairs_noalloc serves them from one
fixed 64 MiB scratch array inside the library.  These tests call it through
the C ABI twice in a row on different inputs (the scratch keeps the previous
call's contents, so the second call also checks that what must start at zero
is cleared) and compare with the regular entry point, within the MI tolerance
of the other GPU tests.  The file is named so that pytest collects it last.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu

MI_TOL = 1e-6


def _data(m, n, seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.02, 0.5, size=n)
    X = (rng.random((m, n)) < p).astype(np.uint8)
    X[:, 1] = X[:, 0]
    return torch.from_numpy(X).cuda()


def _noalloc(lib, X):
    m, n = X.shape
    out = torch.full((n, n), float("nan"), dtype=torch.float32, device=X.device)
    lib.gbmi_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    st = lib.mi_all_pairs_noalloc(ctypes.c_void_p(X.data_ptr()), m, n,
                                  ctypes.c_void_p(out.data_ptr()))
    assert st == gbmi.OK, gbmi.last_error()
    return out


def test_noalloc_matches_mi_all_pairs_on_two_calls_in_a_row():
    lib = gbmi.load()
    gbmi.set_option(gbmi.OPT_FIXUP, 0)
    for (m, n, seed) in [(3000, 300, 1), (1500, 517, 2)]:
        X = _data(m, n, seed)
        got = _noalloc(lib, X)
        want = gbmi.mi_all_pairs(X, path="fused")
        torch.cuda.synchronize()
        assert not torch.isnan(got).any()
        assert float((got - want).abs().max()) <= MI_TOL
        assert torch.equal(got, got.T)


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = gbmi.load()
    X = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    out = torch.empty((4, 4), dtype=torch.float32, device="cuda")
    # 2^24 samples x 1000 variables needs about 8 GiB of packed FP4 operand
    st = lib.mi_all_pairs_noalloc(ctypes.c_void_p(X.data_ptr()), 1 << 24, 1000,
                                  ctypes.c_void_p(out.data_ptr()))
    assert st == gbmi.ERR_ARG
    assert "64 MiB" in gbmi.last_error()
