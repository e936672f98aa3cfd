"""The tensor-core throughput probe (gbmi_mma_peak) that sets the Gram's roofline.

The probe issues back-to-back MMAs of the Gram kernel's forms on operands held
in shared memory.  These tests check that it runs every form, that its rates
are in a physically sensible range for a GB300 (between 1 and 25 PFLOP/s for
FP4, the block-scaled FP4 forms about twice FP8 E4M3 per MMA), and that
arguments outside the documented range are refused before any launch.
"""
from __future__ import annotations

import ctypes

import pytest

torch = pytest.importorskip("torch")

from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form,pair,n", [(1, 1, 240), (1, 0, 256), (2, 1, 256), (0, 1, 256),
                                         (0, 0, 128)])
def test_probe_runs_every_form(form, pair, n):
    r = gbmi.mma_peak(form, pair, n, 1 << 13)
    lo, hi = (1.0e15, 2.5e16) if form else (0.5e15, 1.25e16)
    assert lo < r["flops_per_s"] < hi, r
    assert r["ms"] > 0


def test_fp4_is_faster_than_fp8_per_mma():
    f4 = max(gbmi.mma_peak(1, 1, 256, 1 << 14)["flops_per_s"] for _ in range(2))
    f8 = max(gbmi.mma_peak(0, 1, 256, 1 << 14)["flops_per_s"] for _ in range(2))
    assert 1.5 < f4 / f8 < 4.0, (f4, f8)


def test_probe_argument_errors():
    lib = gbmi.load()
    f, t = ctypes.c_double(), ctypes.c_double()
    for form, pair, n, mmas in [(3, 1, 256, 16), (1, 1, 8, 16), (1, 1, 250, 16),
                                (1, 1, 512, 16), (1, 1, 256, 0)]:
        assert lib.gbmi_mma_peak(form, pair, n, mmas, ctypes.byref(f), ctypes.byref(t)) == \
            gbmi.ERR_ARG
    assert lib.gbmi_mma_peak(1, 1, 256, 16, None, None) == gbmi.ERR_ARG
