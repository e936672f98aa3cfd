"""Host-buffer entry points on the fused path: chunked upload + pack, one Gram
launch in panel-major order, and panel-by-panel download signalled by the
kernel through mapped host memory.

The result must be bit-identical to the device-pointer call on the same
input (same counts, same epilogue), for all pairs and cross MI, with the
upload split into several chunks (ragged last chunk) or one, on CTA pairs
and on single-CTA tiles, and into pageable as well as page-locked memory.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


def _data(m, n, seed, lo=0.02, hi=0.4):
    rng = np.random.default_rng(seed)
    p = rng.uniform(lo, hi, size=n)
    return (rng.random((m, n)) < p).astype(np.uint8)


@pytest.fixture(params=[1, 0], ids=["auto", "single_cta"])
def pair(request):
    gbmi.set_option(gbmi.OPT_PAIR, request.param)
    yield request.param
    gbmi.set_option(gbmi.OPT_PAIR, 1)


@pytest.mark.parametrize("m,n", [(5000, 1000), (70_001, 600), (200_000, 1500), (8192, 4100)])
def test_all_pairs_host_equals_device_call(m, n, pair):
    X = _data(m, n, m + n)
    want = gbmi.mi_all_pairs(torch.from_numpy(X).cuda(), path="fused").cpu()
    gbmi.sync()
    Xh = torch.from_numpy(X).pin_memory()
    out = torch.empty((n, n), dtype=torch.float32).pin_memory()
    gbmi.mi_all_pairs_host(Xh, out)
    assert torch.equal(out, want)
    out2 = torch.empty((n, n), dtype=torch.float32)            # pageable output
    gbmi.mi_all_pairs_host(torch.from_numpy(X), out2)
    assert torch.equal(out2, want)


def test_cross_host_equals_device_call_and_oracle(pair):
    X, Y = _data(30_000, 700, 1), _data(30_000, 450, 2)
    want = gbmi.mi_cross(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(),
                         path="fused").cpu()
    gbmi.sync()
    out = torch.empty((700, 450), dtype=torch.float32).pin_memory()
    gbmi.mi_cross_host(torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory(), out)
    assert torch.equal(out, want)
    ref, _ = oracle.mi_matrix(X[:3000], Y[:3000])
    small = torch.empty((700, 450), dtype=torch.float32)
    gbmi.mi_cross_host(torch.from_numpy(np.ascontiguousarray(X[:3000])),
                       torch.from_numpy(np.ascontiguousarray(Y[:3000])), small)
    assert np.max(np.abs(small.numpy().astype(np.float64) - ref)) <= 1e-6


def test_repeated_calls_reuse_the_pipeline():
    X = _data(40_000, 900, 3)
    Xh = torch.from_numpy(X).pin_memory()
    outs = []
    for _ in range(3):
        o = torch.empty((900, 900), dtype=torch.float32).pin_memory()
        gbmi.mi_all_pairs_host(Xh, o)
        outs.append(o)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])
    want = gbmi.mi_all_pairs(torch.from_numpy(X).cuda(), path="fused").cpu()
    gbmi.sync()
    assert torch.equal(outs[0], want)


def test_host_call_with_fp64_combine_runs_one_gram_chunk():
    X = _data(70_001, 600, 4)
    gbmi.set_option(gbmi.OPT_FIXUP, 1)
    try:
        want = gbmi.mi_all_pairs(torch.from_numpy(X).cuda(), path="fused").cpu()
        gbmi.sync()
        out = torch.empty((600, 600), dtype=torch.float32).pin_memory()
        gbmi.mi_all_pairs_host(torch.from_numpy(X).pin_memory(), out)
    finally:
        gbmi.set_option(gbmi.OPT_FIXUP, 0)
    assert torch.equal(out, want)
    default = torch.empty((600, 600), dtype=torch.float32)
    gbmi.mi_all_pairs_host(torch.from_numpy(X), default)          # four Gram chunks
    assert float((default - out).abs().max()) <= 1e-6
