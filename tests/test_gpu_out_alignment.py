"""Output buffers at any float offset.

The fused epilogue stores whole rows as 16- or 32-byte vectors only where the
output pointer and row width allow it (interior chunks of 4 or 8 columns),
and element by element elsewhere.  Outputs that start 1, 2, 4 or 8 floats
past a 32-byte boundary, with widths that are multiples of 8, of 4 only, or
odd, must give the same bits as an aligned output, and nothing outside the
n x n block may be written.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


def _data(m, n, seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.02, 0.5, size=n)
    X = (rng.random((m, n)) < p).astype(np.uint8)
    X[:, 1] = X[:, 0]
    return torch.from_numpy(X).cuda()


@pytest.fixture(autouse=True)
def _restore():
    yield
    gbmi.set_option(gbmi.OPT_PAIR, 1)


@pytest.mark.parametrize("pair", [1, 0])
@pytest.mark.parametrize("n", [1024, 1004, 1001])
@pytest.mark.parametrize("path", ["fused", "plain"])
def test_output_offsets_are_bit_identical(n, pair, path):
    gbmi.set_option(gbmi.OPT_PAIR, 2 if pair else 0)
    X = _data(3000, n, n)
    ref = torch.empty((n, n), dtype=torch.float32, device="cuda")
    gbmi.mi_all_pairs(X, out=ref, path=path)
    gbmi.sync()
    assert ref.data_ptr() % 32 == 0
    for off in (1, 2, 4, 8):
        buf = torch.full((n * n + 32,), -7.0, dtype=torch.float32, device="cuda")
        assert buf.data_ptr() % 32 == 0
        out = buf[off:off + n * n].view(n, n)
        gbmi.mi_all_pairs(X, out=out, path=path)
        gbmi.sync()
        assert torch.equal(out, ref), off
        assert bool((buf[:off] == -7.0).all()) and bool((buf[off + n * n:] == -7.0).all()), off


def test_cross_output_offset():
    gbmi.set_option(gbmi.OPT_PAIR, 2)
    X, Y = _data(2000, 512, 1), _data(2000, 776, 2)
    ref = torch.empty((512, 776), dtype=torch.float32, device="cuda")
    gbmi.mi_cross(X, Y, out=ref, path="fused")
    gbmi.sync()
    buf = torch.full((512 * 776 + 8,), -7.0, dtype=torch.float32, device="cuda")
    out = buf[4:4 + 512 * 776].view(512, 776)
    gbmi.mi_cross(X, Y, out=out, path="fused")
    gbmi.sync()
    assert torch.equal(out, ref)
    assert bool((buf[:4] == -7.0).all()) and bool((buf[4 + 512 * 776:] == -7.0).all())
