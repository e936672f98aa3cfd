"""Python binding of libgbmi.so (ctypes): argument marshalling only.

Every function takes torch CUDA tensors (or numpy arrays for the ``*_host``
calls), checks dtypes and shapes, points the library at the tensor's current
stream and calls the C ABI of ``include/gbmi.h`` with raw pointers.  All
computation happens in the library's CUDA kernels.  There is no fallback: if
the library is missing or the GPU is not sm_103a, the call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgbmi.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gbmi.h")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_BINARY, ERR_UNSUPPORTED = range(7)
PATH_AUTO, PATH_FUSED, PATH_PLAIN, PATH_POPCOUNT = range(4)
(OPT_FIXUP, OPT_TIMEOUT_NS, OPT_DEBUG_FLAGS, OPT_GROUP_COLS, OPT_MAX_CTAS, OPT_PROFILE,
 OPT_TILE_N, OPT_DIRECT, OPT_PAIR, OPT_CSR_PATH, OPT_SPLIT_K, OPT_FP4,
 OPT_TAIL_SPLIT, OPT_TAIL_COLS) = range(1, 15)
_PATHS = {"auto": PATH_AUTO, "fused": PATH_FUSED, "plain": PATH_PLAIN, "popcount": PATH_POPCOUNT}
STATUS_NAMES = {OK: "OK", ERR_ARG: "ERR_ARG", ERR_OOM: "ERR_OOM", ERR_CUDA: "ERR_CUDA",
                ERR_TIMEOUT: "ERR_TIMEOUT", ERR_NOT_BINARY: "ERR_NOT_BINARY",
                ERR_UNSUPPORTED: "ERR_UNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class GbmiError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def header_functions() -> list[str]:
    """Names of the functions declared in include/gbmi.h."""
    with open(HEADER) as f:
        text = f.read()
    return re.findall(
        r"^\s*(?:gbmi_status|void\*|const char\*|uint64_t|int64_t|double|int)\s+(\w+)\s*\(",
        text, flags=re.M)


def load(path: str | None = None):
    """Load libgbmi.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libgbmi.so not found at {p}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        sig = {
            "mi_all_pairs": [vp, i64, i64, vp],
            "mi_cross": [vp, vp, i64, i64, i64, vp],
            "gbmi_mi_all_pairs_path": [vp, i64, i64, vp, i32],
            "gbmi_mi_all_pairs_shard": [vp, i64, i64, vp, i32, i32],
            "gbmi_mi_cross_path": [vp, vp, i64, i64, i64, vp, i32],
            "mi_all_pairs_host": [vp, i64, i64, vp],
            "mi_cross_host": [vp, vp, i64, i64, i64, vp],
            "gbmi_counts_all_pairs": [vp, i64, i64, vp, i32],
            "gbmi_counts_cross": [vp, vp, i64, i64, i64, vp, i32],
            "gbmi_column_counts": [vp, i64, i64, vp],
            "gbmi_mi_from_counts": [vp, vp, vp, i64, i64, i64, vp],
            "gbmi_validate_binary": [vp, i64, i64],
            "gbmi_set_stream": [vp],
            "gbmi_set_option": [i32, i64],
            "gbmi_sync": [],
            "gbmi_shutdown": [],
            "gbmi_profile_reset": [],
            "mi_all_pairs_noalloc": [vp, i64, i64, vp],
            "gbmi_mma_peak": [i32, i32, i32, i64, vp, vp],
            "gbmi_tuner_set": [i64, i64, i32],
            "gbmi_tuner_set_pair": [i64, i64, i32],
            "gbmi_tuner_pair": [i64, i64],
            "gbmi_tuner_set_split": [i64, i64, i32],
            "gbmi_tuner_split": [i64, i64],
            "gbmi_tail_cols_plan": [i32, i32, vp],
            "gbmi_tuner_clear": [],
            "gbmi_tile_n": [i64, i64],
            "gbmi_batch_create": [vp, i32, vp],
            "gbmi_batch_run": [vp],
            "gbmi_batch_set_io": [vp, vp, i32],
            "gbmi_batch_destroy": [vp],
            "gbmi_mi_batch": [vp, i32],
            "gbmi_mi_all_pairs_to_host": [vp, i64, i64, vp, i64],
            "gbmi_mi_cross_to_host": [vp, vp, i64, i64, i64, vp, i64],
            "gbmi_mi_all_pairs_csr": [vp, vp, i64, i64, i64, vp],
            "gbmi_counts_all_pairs_csr": [vp, vp, i64, i64, i64, vp],
            "gbmi_server_create": [i64, i32, vp],
            "gbmi_server_add_dataset": [vp, vp, i64, i64, vp],
            "gbmi_server_remove_dataset": [vp, i64],
            "gbmi_server_submit": [vp, i64, i64, vp],
            "gbmi_server_wait": [vp, i64, i64, vp, vp],
            "gbmi_server_release": [vp, i64],
            "gbmi_server_stats": [vp, vp],
            "gbmi_server_cancel": [vp, i64],
            "gbmi_server_state": [vp, vp, vp, vp, vp],
            "gbmi_server_destroy": [vp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.gbmi_get_stream.argtypes = []
        lib.gbmi_get_stream.restype = ctypes.c_void_p
        lib.gbmi_last_error_string.argtypes = []
        lib.gbmi_last_error_string.restype = ctypes.c_char_p
        lib.gbmi_launch_count.argtypes = []
        lib.gbmi_launch_count.restype = ctypes.c_uint64
        lib.gbmi_version.argtypes = []
        lib.gbmi_version.restype = ctypes.c_int
        lib.gbmi_profile_entries.argtypes = []
        lib.gbmi_profile_entries.restype = ctypes.c_int
        lib.gbmi_profile_name.argtypes = [ctypes.c_int]
        lib.gbmi_profile_name.restype = ctypes.c_char_p
        lib.gbmi_profile_ms.argtypes = [ctypes.c_int]
        lib.gbmi_profile_ms.restype = ctypes.c_double
        lib.gbmi_profile_launches.argtypes = [ctypes.c_int]
        lib.gbmi_profile_launches.restype = ctypes.c_int64
        lib.gbmi_batch_tiles.argtypes = [vp]
        lib.gbmi_batch_tiles.restype = ctypes.c_int64
        _lib = lib
        return lib


def _check(status: int):
    if status != OK:
        msg = load().gbmi_last_error_string()
        raise GbmiError(status, msg.decode() if msg else "")


def _path(path) -> int:
    return _PATHS[path] if isinstance(path, str) else int(path)


def _prep(X, name="X"):
    import torch
    if not isinstance(X, torch.Tensor) or not X.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if X.dtype not in (torch.uint8, torch.bool):
        raise TypeError(f"{name} must be uint8 (0/1) or bool")
    if X.dim() != 2:
        raise ValueError(f"{name} must be 2-D (samples x variables)")
    if X.dtype == torch.bool:
        X = X.view(torch.uint8)
    return X.contiguous()


def _bind_stream(dev):
    import torch
    lib = load()
    _check(lib.gbmi_set_stream(ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)))
    return lib


def mi_all_pairs(X, out=None, path="auto"):
    """n x n MI matrix (bits, float32) of the columns of X (m x n, uint8 0/1)."""
    import torch
    X = _prep(X)
    m, n = X.shape
    with torch.cuda.device(X.device):
        if out is None:
            out = torch.empty((n, n), dtype=torch.float32, device=X.device)
        assert out.shape == (n, n) and out.dtype == torch.float32 and out.is_contiguous()
        lib = _bind_stream(X.device)
        _check(lib.gbmi_mi_all_pairs_path(X.data_ptr(), m, n, out.data_ptr(), _path(path)))
    return out


def mi_all_pairs_shard(X, shard, num_shards, out=None):
    """Shard `shard` of `num_shards` of the fused all-pairs call: only the pairs of
    that contiguous share of the Gram's tile list are written into out (n x n);
    the shards' writes together are mi_all_pairs(X)'s output."""
    import torch
    X = _prep(X)
    m, n = X.shape
    with torch.cuda.device(X.device):
        if out is None:
            out = torch.empty((n, n), dtype=torch.float32, device=X.device)
        assert out.shape == (n, n) and out.dtype == torch.float32 and out.is_contiguous()
        lib = _bind_stream(X.device)
        _check(lib.gbmi_mi_all_pairs_shard(X.data_ptr(), m, n, out.data_ptr(), int(shard),
                                           int(num_shards)))
    return out


def mi_all_pairs_noalloc(X, out):
    """All-pairs MI through the entry point that allocates no device memory.

    For callers that cannot let the library allocate (their framework owns
    the device memory, or a cudaFree's device-wide wait is not acceptable):
    ``out`` (n x n float32, on X's device) must be provided; the library's
    own scratch is a fixed 64 MiB array.  Returns when the result is written.
    """
    import torch
    X = _prep(X)
    m, n = X.shape
    if out.shape != (n, n) or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 (n, n) tensor")
    if out.device != X.device:
        raise ValueError("out must be on X's device")
    with torch.cuda.device(X.device):
        lib = _bind_stream(X.device)
        _check(lib.mi_all_pairs_noalloc(X.data_ptr(), m, n, out.data_ptr()))
    return out


def mi_cross(X, Y, out=None, path="auto"):
    """n1 x n2 MI matrix between the columns of X (m x n1) and Y (m x n2)."""
    import torch
    X, Y = _prep(X), _prep(Y, "Y")
    if X.shape[0] != Y.shape[0]:
        raise ValueError("X and Y must have the same number of samples")
    m, n1 = X.shape
    n2 = Y.shape[1]
    with torch.cuda.device(X.device):
        if out is None:
            out = torch.empty((n1, n2), dtype=torch.float32, device=X.device)
        assert out.shape == (n1, n2) and out.dtype == torch.float32 and out.is_contiguous()
        lib = _bind_stream(X.device)
        _check(lib.gbmi_mi_cross_path(X.data_ptr(), Y.data_ptr(), m, n1, n2, out.data_ptr(),
                                      _path(path)))
    return out


def counts_all_pairs(X, path="plain", out=None):
    """N11 = X^T X as int32 (n x n) via the tensor cores ("plain") or popcount."""
    import torch
    X = _prep(X)
    m, n = X.shape
    with torch.cuda.device(X.device):
        if out is None:
            out = torch.empty((n, n), dtype=torch.int32, device=X.device)
        lib = _bind_stream(X.device)
        _check(lib.gbmi_counts_all_pairs(X.data_ptr(), m, n, out.data_ptr(), _path(path)))
    return out


def counts_cross(X, Y, path="plain", out=None):
    """N11 = X^T Y as int32 (n1 x n2)."""
    import torch
    X, Y = _prep(X), _prep(Y, "Y")
    m, n1 = X.shape
    n2 = Y.shape[1]
    with torch.cuda.device(X.device):
        if out is None:
            out = torch.empty((n1, n2), dtype=torch.int32, device=X.device)
        lib = _bind_stream(X.device)
        _check(lib.gbmi_counts_cross(X.data_ptr(), Y.data_ptr(), m, n1, n2, out.data_ptr(),
                                     _path(path)))
    return out


def column_counts(X):
    """v_j = number of ones in column j (int32)."""
    import torch
    X = _prep(X)
    m, n = X.shape
    with torch.cuda.device(X.device):
        v = torch.empty(n, dtype=torch.int32, device=X.device)
        lib = _bind_stream(X.device)
        _check(lib.gbmi_column_counts(X.data_ptr(), m, n, v.data_ptr()))
    return v


def mi_from_counts(N11, va, vb, m, out=None):
    """Elementwise MI (bits) from an int32 count matrix and the column counts."""
    import torch
    n1, n2 = N11.shape
    N11, va, vb = N11.contiguous(), va.contiguous(), vb.contiguous()
    with torch.cuda.device(N11.device):
        if out is None:
            out = torch.empty((n1, n2), dtype=torch.float32, device=N11.device)
        lib = _bind_stream(N11.device)
        _check(lib.gbmi_mi_from_counts(N11.data_ptr(), va.data_ptr(), vb.data_ptr(), int(m), n1,
                                       n2, out.data_ptr()))
    return out


def validate_binary(X) -> bool:
    """True if every entry of X is 0 or 1 (synchronous)."""
    import torch
    X = _prep(X)
    with torch.cuda.device(X.device):
        lib = _bind_stream(X.device)
        st = lib.gbmi_validate_binary(X.data_ptr(), X.shape[0], X.shape[1])
    if st == ERR_NOT_BINARY:
        return False
    _check(st)
    return True


def _host_array(A, dtype, name):
    """(object, pointer) of a contiguous host array: numpy, or a torch CPU tensor."""
    import numpy as np
    if hasattr(A, "data_ptr"):
        if A.is_cuda:
            raise TypeError(f"{name} must be in host memory")
        A = A.contiguous()
        return A, A.data_ptr()
    A = np.ascontiguousarray(A, dtype=dtype)
    return A, A.ctypes.data


def mi_all_pairs_host(X, out=None):
    """Host-buffer call: X is a numpy array or torch CPU tensor (uint8, m x n); out
    (n x n float32, page-locked for the fastest copies) is allocated if None."""
    import numpy as np
    X, xp = _host_array(X, np.uint8, "X")
    m, n = X.shape
    if out is None:
        out = np.empty((n, n), dtype=np.float32)
    if tuple(out.shape) != (n, n):
        raise ValueError(f"out must be {n} x {n}")
    out, op = _host_array(out, np.float32, "out")
    _check(load().mi_all_pairs_host(xp, m, n, op))
    return out


def mi_cross_host(X, Y, out=None):
    """Host-buffer cross MI between the columns of X (m x n1) and Y (m x n2)."""
    import numpy as np
    X, xp = _host_array(X, np.uint8, "X")
    Y, yp = _host_array(Y, np.uint8, "Y")
    m, n1 = X.shape
    if Y.shape[0] != m:
        raise ValueError("X and Y must have the same number of samples")
    n2 = Y.shape[1]
    if out is None:
        out = np.empty((n1, n2), dtype=np.float32)
    if tuple(out.shape) != (n1, n2):
        raise ValueError(f"out must be {n1} x {n2}")
    out, op = _host_array(out, np.float32, "out")
    _check(load().mi_cross_host(xp, yp, m, n1, n2, op))
    return out


def _host_out(shape, out):
    import torch
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    if (out.is_cuda or tuple(out.shape) != tuple(shape) or out.dtype != torch.float32
            or not out.is_contiguous()):
        raise ValueError(f"out must be a contiguous float32 host tensor of shape {shape}")
    return out


def mi_all_pairs_to_host(X, out=None, panel_rows=0):
    """n x n MI matrix of X (device) computed in row panels straight into host memory.

    ``out`` defaults to a page-locked host tensor; panel_rows = 0 picks the
    panel height automatically.  Returns ``out`` when complete.
    """
    import torch
    X = _prep(X)
    m, n = X.shape
    out = _host_out((n, n), out)
    with torch.cuda.device(X.device):
        lib = _bind_stream(X.device)
        _check(lib.gbmi_mi_all_pairs_to_host(X.data_ptr(), m, n, out.data_ptr(), int(panel_rows)))
    return out


def mi_cross_to_host(X, Y, out=None, panel_rows=0):
    """n1 x n2 MI matrix between the columns of X and Y, in row panels into host memory."""
    import torch
    X, Y = _prep(X), _prep(Y, "Y")
    m, n1 = X.shape
    if Y.shape[0] != m:
        raise ValueError("X and Y must have the same number of samples")
    n2 = Y.shape[1]
    out = _host_out((n1, n2), out)
    with torch.cuda.device(X.device):
        lib = _bind_stream(X.device)
        _check(lib.gbmi_mi_cross_to_host(X.data_ptr(), Y.data_ptr(), m, n1, n2, out.data_ptr(),
                                         int(panel_rows)))
    return out


def _csr(row_ptr, col_idx, n):
    import torch
    if not (isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda and row_ptr.dtype == torch.int64
            and row_ptr.dim() == 1 and row_ptr.numel() >= 2):
        raise TypeError("row_ptr must be a 1-D int64 CUDA tensor of m + 1 entries")
    if not (isinstance(col_idx, torch.Tensor) and col_idx.is_cuda and col_idx.dtype == torch.int32
            and col_idx.dim() == 1):
        raise TypeError("col_idx must be a 1-D int32 CUDA tensor")
    return row_ptr.contiguous(), col_idx.contiguous(), row_ptr.numel() - 1, int(n)


def mi_all_pairs_csr(row_ptr, col_idx, n, out=None):
    """n x n MI matrix of X given in CSR by samples (int64 row_ptr, int32 col_idx)."""
    import torch
    row_ptr, col_idx, m, n = _csr(row_ptr, col_idx, n)
    with torch.cuda.device(row_ptr.device):
        if out is None:
            out = torch.empty((n, n), dtype=torch.float32, device=row_ptr.device)
        lib = _bind_stream(row_ptr.device)
        _check(lib.gbmi_mi_all_pairs_csr(row_ptr.data_ptr(), col_idx.data_ptr() if col_idx.numel()
                                         else None, m, n, col_idx.numel(), out.data_ptr()))
    return out


def counts_all_pairs_csr(row_ptr, col_idx, n, out=None):
    """n x n int32 co-occurrence counts of X given in CSR by samples."""
    import torch
    row_ptr, col_idx, m, n = _csr(row_ptr, col_idx, n)
    with torch.cuda.device(row_ptr.device):
        if out is None:
            out = torch.empty((n, n), dtype=torch.int32, device=row_ptr.device)
        lib = _bind_stream(row_ptr.device)
        _check(lib.gbmi_counts_all_pairs_csr(row_ptr.data_ptr(), col_idx.data_ptr()
                                             if col_idx.numel() else None, m, n, col_idx.numel(),
                                             out.data_ptr()))
    return out


def csr_from_dense(X):
    """CSR by samples of a device uint8 0/1 matrix (torch ops; input preparation)."""
    import torch
    X = _prep(X)
    nz = torch.nonzero(X)                       # row-major order: rows, then increasing columns
    counts = torch.bincount(nz[:, 0], minlength=X.shape[0])
    row_ptr = torch.zeros(X.shape[0] + 1, dtype=torch.int64, device=X.device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return row_ptr, nz[:, 1].to(torch.int32).contiguous()


class _Job(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("n2", ctypes.c_int64), ("out", ctypes.c_void_p)]


def _jobs(Xs, Ys, outs):
    import torch
    Ys = list(Ys) if Ys is not None else [None] * len(Xs)
    if len(Ys) != len(Xs):
        raise ValueError("Ys must match Xs")
    arr = (_Job * len(Xs))()
    keep, out_list = [], []
    for k, X in enumerate(Xs):
        X = _prep(X)
        Y = None if Ys[k] is None else _prep(Ys[k], "Y")
        m, n = X.shape
        n2 = n if Y is None else Y.shape[1]
        if Y is not None and Y.shape[0] != m:
            raise ValueError(f"job {k}: X and Y must have the same number of samples")
        o = None if outs is None else outs[k]
        if o is None:
            o = torch.empty((n, n2), dtype=torch.float32, device=X.device)
        if o.shape != (n, n2) or o.dtype != torch.float32 or not o.is_contiguous():
            raise ValueError(f"job {k}: out must be a contiguous float32 ({n}, {n2}) tensor")
        arr[k] = _Job(X.data_ptr(), 0 if Y is None else Y.data_ptr(), m, n, n2 if Y is not None
                      else 0, o.data_ptr())
        keep += [X, Y]
        out_list.append(o)
    return arr, keep, out_list


class Batch:
    """A plan for many all-pairs (Y=None) or cross problems in one grouped run.

    ``run()`` launches the plan's CUDA graph (one grouped pack, one grouped
    per-variable pass and one persistent tensor-core Gram launch over the tiles
    of every job) on the current stream; ``outs`` are the output tensors.
    """

    def __init__(self, Xs, Ys=None, outs=None):
        import torch
        self._dev = _prep(Xs[0]).device
        arr, self._keep, self.outs = _jobs(Xs, Ys, outs)
        self._plan = ctypes.c_void_p()
        with torch.cuda.device(self._dev):
            lib = _bind_stream(self._dev)
            _check(lib.gbmi_batch_create(arr, len(Xs), ctypes.byref(self._plan)))

    @property
    def tiles(self) -> int:
        return int(load().gbmi_batch_tiles(self._plan))

    def run(self):
        import torch
        with torch.cuda.device(self._dev):
            lib = _bind_stream(self._dev)
            _check(lib.gbmi_batch_run(self._plan))
        return self.outs

    def set_io(self, Xs, Ys=None, outs=None):
        import torch
        arr, keep, out_list = _jobs(Xs, Ys, outs)
        with torch.cuda.device(self._dev):
            lib = _bind_stream(self._dev)
            _check(lib.gbmi_batch_set_io(self._plan, arr, len(Xs)))
        self._keep, self.outs = keep, out_list
        return self.outs

    def close(self):
        if self._plan:
            _check(load().gbmi_batch_destroy(self._plan))
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mi_batch(Xs, Ys=None, outs=None):
    """One-shot grouped run (create, run, wait, destroy); returns the outputs."""
    import torch
    arr, keep, out_list = _jobs(Xs, Ys, outs)
    dev = out_list[0].device
    with torch.cuda.device(dev):
        lib = _bind_stream(dev)
        _check(lib.gbmi_mi_batch(arr, len(Xs)))
    del keep
    return out_list


def tuner_set(m: int, n: int, tile_n: int):
    """Record the tile width for problems in the (m, n) bucket."""
    _check(load().gbmi_tuner_set(int(m), int(n), int(tile_n)))


def tuner_clear():
    _check(load().gbmi_tuner_clear())


def tuner_set_pair(m: int, n: int, pair: int):
    """Kernel choice for the (m, n) bucket: 1 CTA pairs, 0 single-CTA tiles, -1 the rule."""
    _check(load().gbmi_tuner_set_pair(int(m), int(n), int(pair)))


def tuner_pair(m: int, n: int) -> int:
    return int(load().gbmi_tuner_pair(int(m), int(n)))


def tuner_set_split(m: int, n: int, parts: int):
    """Sample split for the (m, n) bucket: 0 the cost model, 1 none, S >= 2 ranges."""
    _check(load().gbmi_tuner_set_split(int(m), int(n), int(parts)))


def tuner_split(m: int, n: int) -> int:
    return int(load().gbmi_tuner_split(int(m), int(n)))


def tail_cols_plan(tiles: int, units: int) -> tuple[int, int]:
    """(tiles split into column shares, shares per tile) for a launch of `tiles` on `units` slots."""
    parts = ctypes.c_int(0)
    S = int(load().gbmi_tail_cols_plan(int(tiles), int(units), ctypes.byref(parts)))
    return S, int(parts.value)


def tile_n(m: int, n: int) -> int:
    """Tile width an all-pairs call of shape (m, n) would use."""
    return int(load().gbmi_tile_n(int(m), int(n)))


def set_option(option: int, value: int):
    _check(load().gbmi_set_option(int(option), int(value)))


def sync():
    """Wait for the library's stream and raise on a device-side timeout."""
    _check(load().gbmi_sync())


def launch_count() -> int:
    return int(load().gbmi_launch_count())


def last_error() -> str:
    s = load().gbmi_last_error_string()
    return s.decode() if s else ""


def shutdown():
    _check(load().gbmi_shutdown())


def version() -> int:
    return int(load().gbmi_version())


def mma_peak(fp4: bool = True, pair: bool = True, n: int = 256, mmas: int = 1 << 16) -> dict:
    """Tensor-core throughput of one MMA form with shared-memory operands.

    Marshals gbmi_mma_peak: every SM (or CTA pair) issues ``mmas`` MMAs of
    M x n x K; returns ``{"flops_per_s": F, "ms": T}``.
    """
    import torch
    f, t = ctypes.c_double(), ctypes.c_double()
    lib = _bind_stream(torch.device("cuda", torch.cuda.current_device()))
    _check(lib.gbmi_mma_peak(int(bool(fp4)), int(bool(pair)), int(n), int(mmas),
                             ctypes.byref(f), ctypes.byref(t)))
    return {"flops_per_s": f.value, "ms": t.value}


def profile(enable: bool | None = None, reset: bool = False) -> dict:
    """Per-kernel device time from the library's event profiler.

    enable=True/False switches recording on/off; the return value maps each
    kernel name to {"ms": total ms, "launches": count} (waits for the work).
    """
    lib = load()
    if reset:
        _check(lib.gbmi_profile_reset())
    if enable is not None:
        set_option(OPT_PROFILE, 1 if enable else 0)
    out = {}
    for k in range(lib.gbmi_profile_entries()):
        out[lib.gbmi_profile_name(k).decode()] = {"ms": float(lib.gbmi_profile_ms(k)),
                                                  "launches": int(lib.gbmi_profile_launches(k))}
    return out


class _DeviceView:
    """A device buffer the server owns, exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4",
                                         "data": (ptr, False), "version": 3, "strides": None}


class Server:
    """Request loop with continuous batching over resident datasets.

    ``add_dataset(X)`` registers a device uint8 0/1 matrix (kept referenced
    until ``remove_dataset``); ``submit(a)`` / ``submit(a, b)`` queue the
    all-pairs or cross MI problem and return a ticket; ``wait(ticket)``
    returns ``(mi, latency_ms)`` where ``mi`` is a zero-copy float32 view of
    the server's output buffer, valid until ``release(ticket)``.
    """

    def __init__(self, budget_bytes: int, max_batch: int = 64, device=None):
        import torch
        self._dev = torch.device("cuda", torch.cuda.current_device() if device is None
                                 else torch.device(device).index or 0)
        self._srv = ctypes.c_void_p()
        self._data: dict[int, object] = {}
        self._shape: dict[int, tuple] = {}
        self._tshape: dict[int, tuple] = {}
        with torch.cuda.device(self._dev):
            _check(load().gbmi_server_create(int(budget_bytes), int(max_batch),
                                             ctypes.byref(self._srv)))

    def add_dataset(self, X) -> int:
        import torch
        X = _prep(X)
        if X.device != self._dev:
            raise ValueError(f"X is on {X.device}, the server on {self._dev}")
        torch.cuda.current_stream(X.device).synchronize()
        i = ctypes.c_int64()
        _check(load().gbmi_server_add_dataset(self._srv, X.data_ptr(), X.shape[0], X.shape[1],
                                              ctypes.byref(i)))
        self._data[i.value] = X
        self._shape[i.value] = tuple(X.shape)
        return i.value

    def remove_dataset(self, ds: int):
        _check(load().gbmi_server_remove_dataset(self._srv, int(ds)))
        self._data.pop(ds, None)

    def submit(self, a: int, b: int | None = None) -> int:
        t = ctypes.c_int64()
        _check(load().gbmi_server_submit(self._srv, int(a), -1 if b is None else int(b),
                                         ctypes.byref(t)))
        na = self._shape[a][1]
        self._tshape[t.value] = (na, na if b is None else self._shape[b][1])
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 0):
        import torch
        p, lat = ctypes.c_void_p(), ctypes.c_double()
        _check(load().gbmi_server_wait(self._srv, int(ticket), int(timeout_ms), ctypes.byref(p),
                                       ctypes.byref(lat)))
        view = torch.as_tensor(_DeviceView(p.value, self._tshape[ticket]), device=self._dev)
        return view, lat.value

    def release(self, ticket: int):
        _check(load().gbmi_server_release(self._srv, int(ticket)))
        self._tshape.pop(ticket, None)

    def cancel(self, ticket: int):
        """Cancel a still-queued request (raises if it is running or done)."""
        _check(load().gbmi_server_cancel(self._srv, int(ticket)))

    def state(self) -> dict:
        q, r, d, b = (ctypes.c_int64() for _ in range(4))
        _check(load().gbmi_server_state(self._srv, ctypes.byref(q), ctypes.byref(r),
                                        ctypes.byref(d), ctypes.byref(b)))
        return {"queued": q.value, "running": r.value, "datasets": d.value,
                "bytes_in_use": b.value}

    def stats(self) -> dict:
        st = (ctypes.c_double * 8)()
        _check(load().gbmi_server_stats(self._srv, st))
        keys = ("completed", "p50_ms", "p99_ms", "mean_ms", "max_ms", "pairs_per_s", "batches",
                "requests_per_batch")
        return dict(zip(keys, list(st)))

    def close(self):
        if self._srv:
            _check(load().gbmi_server_destroy(self._srv))
            self._srv = ctypes.c_void_p()
            self._data.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
