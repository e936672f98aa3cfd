"""One all-pairs problem split into shards of the Gram's tile list.

Every shard writes only the pairs of its share of the tiles; together the
shards must give mi_all_pairs's output bit for bit (no element left unwritten,
none written differently), on CTA pairs and on single-CTA tiles, and with
more shards than tiles (the extra shards write nothing).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu


def _rand(m, n, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    p = torch.rand(n, generator=g, device="cuda") * 0.45 + 0.01
    return (torch.rand((m, n), generator=g, device="cuda") < p).to(torch.uint8)


@pytest.fixture(params=[1, 0], ids=["auto_pair", "single_cta"])
def pair(request):
    gbmi.set_option(gbmi.OPT_PAIR, request.param)
    yield request.param
    gbmi.set_option(gbmi.OPT_PAIR, 1)


@pytest.mark.parametrize("m,n,shards", [(3000, 1500, 2), (5000, 2600, 4), (700, 300, 3),
                                        (129, 77, 1000)])
def test_shards_together_equal_the_whole(pair, m, n, shards):
    X = _rand(m, n, m + n + shards)
    want = gbmi.mi_all_pairs(X, path="fused")
    out = torch.full((n, n), float("nan"), device="cuda")
    for s in range(shards):
        gbmi.mi_all_pairs_shard(X, s, shards, out=out)
    gbmi.sync()
    assert torch.equal(out, want)


def test_one_shard_writes_only_its_tiles():
    X = _rand(4000, 2000, 5)
    want = gbmi.mi_all_pairs(X, path="fused")
    out = torch.full((2000, 2000), float("nan"), device="cuda")
    gbmi.mi_all_pairs_shard(X, 0, 2, out=out)
    gbmi.sync()
    done = ~torch.isnan(out)
    frac = float(done.float().mean())
    assert 0.2 < frac < 0.8                         # about half of the tiles
    assert torch.equal(out[done], want[done])
    assert torch.equal(done, done.t())              # both (i, j) and (j, i) of its pairs
    ref, _ = oracle.mi_matrix(X[:500, :300].cpu().numpy())
    part = gbmi.mi_all_pairs(X[:500, :300].contiguous(), path="fused")
    gbmi.sync()
    assert np.max(np.abs(part.cpu().numpy().astype(np.float64) - ref)) <= 1e-6


def test_shard_argument_errors():
    X = _rand(100, 40, 6)
    out = torch.empty((40, 40), device="cuda")
    lib = gbmi.load()
    for s, k in ((2, 2), (-1, 2), (0, 0)):
        assert lib.gbmi_mi_all_pairs_shard(X.data_ptr(), 100, 40, out.data_ptr(), s, k) \
            == gbmi.ERR_ARG
