"""GPU parity: the CUDA paths against the FP64 oracle, through the C ABI.

Bar (from the method and the hardware):
  * counts (N11 and the column counts) are integers: bit-exact;
  * MI: within 1e-6 absolute of the FP64 oracle (FP32 epilogue; the FP64
    combine takes pairs below 1e-4);
  * the all-pairs matrix is symmetric to the last bit;
  * every path (fused tensor core, plain tensor core, popcount) agrees.
Sizes span several 128 x 256 tiles and ragged tails in both m and n.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import simdata  # noqa: E402
from paper_2411_19702_gb300 import gbmi  # noqa: E402

pytestmark = pytest.mark.gpu

MI_TOL = 1e-6
PATHS = ["fused", "plain", "popcount"]
SHAPES = [(1000, 200), (1, 1), (1, 5), (37, 1), (500, 2), (129, 127), (700, 128), (700, 129),
          (300, 257), (1031, 300), (2000, 520)]


def _data(m, n, seed, lo=0.02, hi=0.5):
    rng = np.random.default_rng(seed)
    p = rng.uniform(lo, hi, size=n)
    return (rng.random((m, n)) < p).astype(np.uint8)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gbmi.load()
    gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 0)
    yield


@pytest.mark.parametrize("m,n", SHAPES)
def test_column_counts_exact(m, n):
    X = _data(m, n, 1)
    v = gbmi.column_counts(torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.array_equal(v, oracle.column_counts(X))


@pytest.mark.parametrize("path", ["popcount", "plain"])
@pytest.mark.parametrize("m,n", SHAPES)
def test_counts_all_pairs_exact(path, m, n):
    X = _data(m, n, 2)
    _, n11 = oracle.mi_matrix(X)
    got = gbmi.counts_all_pairs(torch.from_numpy(X).cuda(), path=path)
    gbmi.sync()
    assert np.array_equal(got.cpu().numpy(), n11)


@pytest.mark.parametrize("path", ["popcount", "plain"])
def test_counts_cross_exact(path):
    X, Y = _data(777, 300, 3), _data(777, 130, 4)
    _, n11 = oracle.mi_matrix(X, Y)
    got = gbmi.counts_cross(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), path=path)
    gbmi.sync()
    assert np.array_equal(got.cpu().numpy(), n11)


@pytest.fixture(params=[0, 1], ids=["fp32", "fp64combine"])
def fixup(request):
    gbmi.set_option(gbmi.OPT_FIXUP, request.param)
    yield request.param
    gbmi.set_option(gbmi.OPT_FIXUP, 0)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("m,n", SHAPES)
def test_mi_all_pairs_matches_oracle(path, m, n, fixup):
    X = _data(m, n, 5)
    want, _ = oracle.mi_matrix(X)
    out = gbmi.mi_all_pairs(torch.from_numpy(X).cuda(), path=path)
    gbmi.sync()
    got = out.cpu().numpy()
    assert np.max(np.abs(got.astype(np.float64) - want)) <= MI_TOL
    assert np.array_equal(got, got.T)
    assert np.all(got >= 0)


@pytest.mark.parametrize("tile_n", [64, 128, 256])
@pytest.mark.parametrize("m,n", [(1000, 200), (129, 127), (1031, 300), (700, 520), (300, 65)])
def test_tile_widths(tile_n, m, n):
    """Every tile width of the tensor-core Gram: exact counts, MI vs oracle,
    all-pairs and cross."""
    X = _data(m, n, 16)
    Y = _data(m, n // 2 + 3, 17)
    want, n11 = oracle.mi_matrix(X)
    wantc, n11c = oracle.mi_matrix(X, Y)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    gbmi.set_option(gbmi.OPT_TILE_N, tile_n)
    try:
        c = gbmi.counts_all_pairs(Xd, path="plain").cpu().numpy()
        cc = gbmi.counts_cross(Xd, Yd, path="plain").cpu().numpy()
        mi = gbmi.mi_all_pairs(Xd, path="fused").cpu().numpy()
        mic = gbmi.mi_cross(Xd, Yd, path="fused").cpu().numpy()
        gbmi.sync()
    finally:
        gbmi.set_option(gbmi.OPT_TILE_N, 0)
    assert np.array_equal(c, n11) and np.array_equal(cc, n11c)
    assert np.max(np.abs(mi.astype(np.float64) - want)) <= MI_TOL
    assert np.array_equal(mi, mi.T)
    assert np.max(np.abs(mic.astype(np.float64) - wantc)) <= MI_TOL


@pytest.mark.parametrize("path", PATHS)
def test_small_mi_relative_accuracy(path, fixup):
    """Near independence (most pairs of sparse data) the FP32 form has no
    cancellation: small MI values keep their relative accuracy too."""
    X = _data(20000, 300, 15, 0.01, 0.1)
    want, _ = oracle.mi_matrix(X)
    got = gbmi.mi_all_pairs(torch.from_numpy(X).cuda(), path=path).cpu().numpy()
    sel = (want > 1e-7) & (want < 1e-4)
    assert sel.sum() > 1000
    rel = np.abs(got[sel].astype(np.float64) - want[sel]) / want[sel]
    assert rel.max() <= 1e-4, rel.max()


@pytest.mark.parametrize("offset", [1, 3, 8, 13])
@pytest.mark.parametrize("m,n", [(300, 200), (257, 131), (1000, 64)])
def test_unaligned_input_base(offset, m, n):
    """X starting at any byte address (a view into a larger buffer)."""
    X = _data(m, n, 18)
    buf = torch.zeros(m * n + 64, dtype=torch.uint8, device="cuda")
    buf[offset:offset + m * n] = torch.from_numpy(X.reshape(-1)).cuda()
    Xv = buf[offset:offset + m * n].view(m, n)
    assert Xv.data_ptr() % 16 == offset % 16
    want, n11 = oracle.mi_matrix(X)
    v = gbmi.column_counts(Xv).cpu().numpy()
    c = gbmi.counts_all_pairs(Xv, path="plain").cpu().numpy()
    mi = gbmi.mi_all_pairs(Xv, path="fused").cpu().numpy()
    gbmi.sync()
    assert np.array_equal(v, X.sum(axis=0)) and np.array_equal(c, n11)
    assert np.max(np.abs(mi.astype(np.float64) - want)) <= MI_TOL


@pytest.mark.parametrize("path", PATHS)
def test_mi_cross_matches_oracle(path, fixup):
    X, Y = _data(1500, 290, 6), _data(1500, 77, 7)
    Y[:, 3] = X[:, 10]
    Y[:, 4] = 1 - X[:, 11]
    want, _ = oracle.mi_matrix(X, Y)
    out = gbmi.mi_cross(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), path=path)
    gbmi.sync()
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - want)) <= MI_TOL


@pytest.mark.parametrize("path", PATHS)
def test_degenerate_columns(path, fixup):
    m, n = 999, 260
    X = _data(m, n, 8)
    X[:, 0] = 0                      # constant zero
    X[:, 1] = 1                      # constant one
    X[:, 2] = X[:, 3]                # identical pair
    X[:, 4] = 1 - X[:, 5]            # complement pair
    X[:, 255] = X[:, 256]            # identical pair across the 256-column tile edge
    X[:, 6] = 0
    X[0, 6] = 1                      # a single one
    want, _ = oracle.mi_matrix(X)
    out = gbmi.mi_all_pairs(torch.from_numpy(X).cuda(), path=path)
    gbmi.sync()
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - want)) <= MI_TOL
    assert np.all(got[0] == 0) and np.all(got[1] == 0)
    assert abs(got[2, 3] - got[3, 3]) <= MI_TOL
    assert abs(got[4, 5] - got[5, 5]) <= MI_TOL


def test_paths_agree_with_and_without_fp64_combine():
    X = _data(5000, 300, 9, 0.01, 0.2)
    Xd = torch.from_numpy(X).cuda()
    want, _ = oracle.mi_matrix(X)
    outs = {}
    for fx in (0, 1):
        gbmi.set_option(gbmi.OPT_FIXUP, fx)
        try:
            for p in PATHS:
                outs[(p, fx)] = gbmi.mi_all_pairs(Xd, path=p).cpu().numpy()
        finally:
            gbmi.set_option(gbmi.OPT_FIXUP, 0)
    for key, got in outs.items():
        assert np.max(np.abs(got.astype(np.float64) - want)) <= MI_TOL, key
    for fx in (0, 1):
        for p in PATHS[1:]:
            assert np.max(np.abs(outs[(p, fx)] - outs[("fused", fx)])) <= 2 * MI_TOL


def test_mi_from_counts_matches_oracle():
    X = _data(700, 90, 10)
    want, n11 = oracle.mi_matrix(X)
    v = oracle.column_counts(X)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()  # noqa: E731
    out = gbmi.mi_from_counts(dev(n11), dev(v), dev(v), 700)
    gbmi.sync()
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - want)) <= MI_TOL


def test_host_entry_point():
    X = _data(1234, 150, 11)
    want, _ = oracle.mi_matrix(X)
    got = gbmi.mi_all_pairs_host(X)
    assert np.max(np.abs(got.astype(np.float64) - want)) <= MI_TOL
    Y = _data(1234, 40, 12)
    wantc, _ = oracle.mi_matrix(X, Y)
    gotc = gbmi.mi_cross_host(X, Y)
    assert np.max(np.abs(gotc.astype(np.float64) - wantc)) <= MI_TOL


def test_validate_binary():
    X = torch.zeros((100, 50), dtype=torch.uint8, device="cuda")
    X[3, 4] = 1
    assert gbmi.validate_binary(X)
    X[7, 9] = 2
    assert not gbmi.validate_binary(X)


def test_results_are_deterministic():
    X = torch.from_numpy(_data(3000, 600, 13)).cuda()
    a = gbmi.mi_all_pairs(X, path="fused").cpu().numpy()
    b = gbmi.mi_all_pairs(X, path="fused").cpu().numpy()
    assert np.array_equal(a, b)


def test_argument_errors():
    X = torch.zeros((10, 4), dtype=torch.uint8, device="cuda")
    out = torch.empty((4, 4), dtype=torch.float32, device="cuda")
    lib = gbmi.load()
    assert lib.mi_all_pairs(X.data_ptr(), 10, 4, None) == gbmi.ERR_ARG
    # output overlapping the input
    assert lib.mi_all_pairs(X.data_ptr(), 10, 4, X.data_ptr()) == gbmi.ERR_ARG
    assert lib.gbmi_mi_all_pairs_path(X.data_ptr(), 10, 4, out.data_ptr(), 9) == gbmi.ERR_ARG
    # empty shapes are refused before anything is launched
    assert lib.gbmi_mi_all_pairs_path(X.data_ptr(), 0, 4, out.data_ptr(),
                                      gbmi.PATH_FUSED) == gbmi.ERR_ARG
    assert lib.gbmi_mi_all_pairs_path(X.data_ptr(), 10, 0, out.data_ptr(),
                                      gbmi.PATH_FUSED) == gbmi.ERR_ARG


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("m,n", [(1000, 200), (129, 127), (3000, 1100), (777, 33)])
def test_every_output_element_is_written(path, m, n):
    """The output starts as NaN; a tile or a mirror store that is skipped shows up."""
    X = torch.from_numpy(_data(m, n, 31)).cuda()
    out = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda")
    gbmi.mi_all_pairs(X, out=out, path=path)
    gbmi.sync()
    assert not torch.isnan(out).any()
    Y = torch.from_numpy(_data(m, 45, 32)).cuda()
    outc = torch.full((n, 45), float("nan"), dtype=torch.float32, device="cuda")
    gbmi.mi_cross(X, Y, out=outc, path=path)
    gbmi.sync()
    assert not torch.isnan(outc).any()


def test_injected_allocation_failure_is_reported_and_recovers():
    X = torch.from_numpy(_data(2000, 300, 33)).cuda()
    gbmi.shutdown()                               # workspace released: the next call allocates
    gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 2)
    try:
        with pytest.raises(gbmi.GbmiError) as e:
            gbmi.mi_all_pairs(X, path="fused")
        assert e.value.status == gbmi.ERR_OOM
        assert "injected" in gbmi.last_error()
    finally:
        gbmi.set_option(gbmi.OPT_DEBUG_FLAGS, 0)
    got = gbmi.mi_all_pairs(X, path="fused")
    gbmi.sync()
    want, _ = oracle.mi_matrix(X.cpu().numpy())
    assert np.max(np.abs(got.cpu().numpy().astype(np.float64) - want)) <= MI_TOL
