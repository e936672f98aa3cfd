"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every function include/gbmi.h declares, and the Python binding refuses to run
without a CUDA device (no CPU fallback)."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2411_19702_gb300 import build as gbuild
from paper_2411_19702_gb300 import gbmi


@pytest.fixture(scope="module")
def lib():
    path = gbuild.build()
    return gbmi.load(path)


def test_header_declares_the_boundary():
    names = gbmi.header_functions()
    for required in ("mi_all_pairs", "mi_cross", "gbmi_counts_all_pairs", "gbmi_set_stream",
                     "gbmi_sync", "gbmi_last_error_string", "mi_all_pairs_host"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in gbmi.header_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_no_torch_types_in_header():
    with open(gbmi.HEADER) as f:
        text = f.read()
    assert "torch" not in text.lower().replace("torch.", "")
    assert "extern \"C\"" in text


def test_version_and_counter_need_no_gpu(lib):
    assert gbmi.version() >= 100
    assert gbmi.launch_count() >= 0


def test_argument_errors_are_reported_without_a_gpu(lib):
    # null pointer and bad sizes are rejected before any CUDA call
    assert lib.mi_all_pairs(None, 10, 10, None) == gbmi.ERR_ARG
    assert b"null" in lib.gbmi_last_error_string()
    buf = (ctypes.c_uint8 * 16)()
    out = (ctypes.c_float * 16)()
    assert lib.mi_all_pairs(ctypes.addressof(buf), 0, 4, ctypes.addressof(out)) == gbmi.ERR_ARG
    assert lib.mi_all_pairs(ctypes.addressof(buf), 4, 0, ctypes.addressof(out)) == gbmi.ERR_ARG
    assert lib.gbmi_set_option(999, 1) == gbmi.ERR_ARG
    assert lib.gbmi_set_option(gbmi.OPT_TIMEOUT_NS, 0) == gbmi.ERR_ARG


def test_binding_rejects_cpu_tensors():
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        gbmi.mi_all_pairs(torch.zeros((4, 4), dtype=torch.uint8))


def test_product_path_does_not_reach_the_oracle():
    import os
    pkg = os.path.dirname(gbmi.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(root, f)) as fh:
                    text = fh.read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "mi_oracle" not in text, f


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="needs a machine without GPU")
def test_host_call_fails_loudly_without_gpu(lib):
    X = np.zeros((8, 4), np.uint8)
    with pytest.raises(gbmi.GbmiError):
        gbmi.mi_all_pairs_host(X)


def test_binding_option_numbers_match_the_header(lib):
    """Every GBMI_OPT_* value of the header has the same number in the binding,
    and every option, the operand form included, is accepted without a GPU."""
    import re
    text = open(gbmi.HEADER).read()
    opts = dict((k, int(v)) for k, v in re.findall(r"GBMI_OPT_(\w+)\s*=\s*(\d+)", text))
    assert "FP4" in opts and len(opts) >= 12
    for name, value in opts.items():
        assert getattr(gbmi, "OPT_" + name) == value, name
    assert lib.gbmi_set_option(gbmi.OPT_FP4, 0) == gbmi.OK
    assert lib.gbmi_set_option(gbmi.OPT_FP4, 1) == gbmi.OK
