"""Out-of-core output: the MI matrix in row panels straight into host memory.

Every panel split (one row per panel, ragged panels, automatic panels) must
give the same bits as the in-core fused call, for all pairs (panel plus its
mirror) and for cross MI, and match the FP64 oracle within 1e-6.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


def _rand(m, n, seed, dev="cuda"):
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    p = torch.rand(n, generator=g, device=dev) * 0.4 + 0.02
    return (torch.rand((m, n), generator=g, device=dev) < p).to(torch.uint8)


@pytest.mark.parametrize("m,n,panel", [(1000, 700, 128), (3000, 1000, 0), (5000, 777, 300),
                                       (129, 130, 7), (2048, 256, 256), (40000, 1500, 0)])
def test_all_pairs_to_host_equals_in_core(m, n, panel):
    X = _rand(m, n, m + n + panel)
    want = gbmi.mi_all_pairs(X, path="fused").cpu()
    got = gbmi.mi_all_pairs_to_host(X, panel_rows=panel)
    assert torch.equal(got, want)
    if m * n <= 3_000_000:
        ref, _ = oracle.mi_matrix(X.cpu().numpy())
        assert np.max(np.abs(got.numpy().astype(np.float64) - ref)) <= 1e-6


@pytest.mark.parametrize("m,n1,n2,panel", [(2000, 300, 500, 128), (1000, 1000, 77, 0),
                                           (777, 45, 3000, 16)])
def test_cross_to_host_equals_in_core(m, n1, n2, panel):
    X, Y = _rand(m, n1, 5 + m), _rand(m, n2, 6 + m)
    want = gbmi.mi_cross(X, Y, path="fused").cpu()
    got = gbmi.mi_cross_to_host(X, Y, panel_rows=panel)
    assert torch.equal(got, want)
    ref, _ = oracle.mi_matrix(X.cpu().numpy(), Y.cpu().numpy())
    assert np.max(np.abs(got.numpy().astype(np.float64) - ref)) <= 1e-6


def test_large_n_in_panels_into_pageable_and_pinned_memory():
    X = _rand(30000, 12000, 77)
    want = gbmi.mi_all_pairs(X, path="fused").cpu()
    got = gbmi.mi_all_pairs_to_host(X)                               # pinned, automatic panels
    assert torch.equal(got, want)
    pageable = torch.empty((12000, 12000), dtype=torch.float32)
    gbmi.mi_all_pairs_to_host(X, out=pageable, panel_rows=2048)
    assert torch.equal(pageable, want)


def test_to_host_argument_errors():
    X = _rand(100, 10, 1)
    with pytest.raises(ValueError):
        gbmi.mi_all_pairs_to_host(X, out=torch.empty((10, 9)))
    lib = gbmi.load()
    assert lib.gbmi_mi_all_pairs_to_host(X.data_ptr(), 100, 10, None, 0) == gbmi.ERR_ARG
    out = torch.empty((10, 10))
    assert lib.gbmi_mi_all_pairs_to_host(X.data_ptr(), 100, 10, out.data_ptr(), -1) == gbmi.ERR_ARG
    assert lib.gbmi_mi_all_pairs_to_host(X.data_ptr(), (1 << 24) + 1, 10, out.data_ptr(),
                                         0) == gbmi.ERR_ARG
