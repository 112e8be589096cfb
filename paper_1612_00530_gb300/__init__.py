"""Python binding of the compressed-SpMV library (include/spmvc.h).

Argument marshalling only: every step of the SpMV, compression and CG path
runs in libspmvc.so (CUDA C++ for sm_103a).  There is no CPU fallback: if
the library has not been built, loading it raises.  PyTorch supplies device
memory and streams; functions take CUDA tensors and pass their pointers and
the current stream through the C ABI.

The functions keep the C names: spmv_build, spmv_build_csr, spmv_compress,
spmv_set_order, spmv_info, spmv_decompress, spmv_export, spmv_import,
spmv_apply, spmv_apply_host, spmv_apply_f32, spmm_apply, spmv_batch_create,
spmv_batch_launch, spmv_batch_autotune, spmv_batch_free, spmv_apply_batched, cg_solve,
spmv_device_error, spmv_autotune, spmv_set_variant, spmv_set_tile,
spmv_set_spmm_kernel, spmv_set_f32_kernel, spmv_permutation, spmm_apply_noalloc, spmv_version.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libspmvc.so")

SPMV_OK, SPMV_EINVAL, SPMV_ENOMEM, SPMV_ECUDA, SPMV_ECORRUPT = 0, 1, 2, 3, 4
SPMV_EUNSUPPORTED, SPMV_ENOTCONVERGED, SPMV_ETIMEOUT, SPMV_EDEVICE = 5, 6, 7, 8
FORMATS = {"auto": 0, "ell": 1, "pattern": 2, "delta": 3, "dit": 4, "data_table": 5}
FORMAT_NAMES = {v: k for k, v in FORMATS.items()}
ORDERS = {"column": 0, "fast": 1}
CG_MODES = {"fp64": 0, "ir_fp32": 1}

_i32, _i64, _u64, _dbl, _p, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t


class spmv_gen_desc(ctypes.Structure):
    _fields_ = [("kind", _i32), ("nx", _i32), ("ny", _i32), ("nz", _i32), ("seed", _u64),
                ("drop_prob", _dbl), ("special_frac", _dbl), ("diag_rule", _i32), ("permute", _i32)]


class spmv_opts(ctypes.Structure):
    _fields_ = [("format", _i32), ("order", _i32), ("max_dict", _i32), ("min_count", _i32), ("reorder", _i32)]


class spmv_info_t(ctypes.Structure):
    _fields_ = [("n", _i64), ("nnz", _i64), ("format", _i32), ("order", _i32), ("dict_size", _i32),
                ("n_patterns", _i32), ("union_size", _i32), ("record_bytes", _i32), ("max_row_nnz", _i32),
                ("fast_eligible", _i32), ("n_slices", _i64), ("slices_value_raw", _i64), ("slices_col_raw", _i64),
                ("device_bytes", _i64), ("format_bytes", _i64), ("padding_bytes", _i64), ("checksum", _u64),
                ("fast_tile_rows", _i32), ("fast_variant", _i32), ("fast_block_threads", _i32),
                ("row_types", _i32), ("reordered", _i32), ("slices_col24", _i32), ("bandwidth", _i64)]


class spmv_cg_opts(ctypes.Structure):
    _fields_ = [("tol", _dbl), ("max_iter", _i32), ("mode", _i32), ("check_every", _i32),
                ("inner_max_iter", _i32), ("inner_tol", _dbl), ("nrhs", _i32), ("use_graph", _i32)]


class spmv_cg_result(ctypes.Structure):
    _fields_ = [("status", _i32), ("iterations", _i32), ("outer_iterations", _i32), ("history_len", _i32),
                ("rel_residual", _dbl), ("seconds", _dbl), ("history", ctypes.POINTER(_dbl))]


class SpmvError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None


def library() -> ctypes.CDLL:
    """The loaded libspmvc.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libspmvc.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        sig = {
            "spmv_build": [ctypes.POINTER(spmv_gen_desc), ctypes.POINTER(_p)],
            "spmv_build_csr": [_i64, _p, _p, _p, ctypes.POINTER(_p)],
            "spmv_compress": [_p, ctypes.POINTER(spmv_opts), ctypes.POINTER(_p)],
            "spmv_permutation": [_p, _p],
            "spmv_set_order": [_p, _i32],
            "spmv_info": [_p, ctypes.POINTER(spmv_info_t)],
            "spmv_decompress": [_p, _p, _p, _p],
            "spmv_export": [_p, _p, ctypes.POINTER(_sz)],
            "spmv_import": [_p, _sz, ctypes.POINTER(_p)],
            "spmv_apply": [_p, _p, _p, _p],
            "spmv_apply_host": [_p, _p, _p],
            "spmv_apply_f32": [_p, _p, _p, _p],
            "spmm_apply": [_p, _i32, _p, _i64, _p, _i64, _p],
            "spmv_batch_create": [_i32, _p, _p, _p, ctypes.POINTER(_p)],
            "spmv_batch_launch": [_p, _p],
            "spmv_batch_autotune": [_p, _i32, ctypes.POINTER(_i32)],
            "spmv_batch_free": [_p],
            "spmv_apply_batched": [_i32, _p, _p, _p, _p],
            "cg_solve": [_p, _p, _p, ctypes.POINTER(spmv_cg_opts), ctypes.POINTER(spmv_cg_result)],
            "spmv_cg_result_free": [ctypes.POINTER(spmv_cg_result)],
            "spmv_free": [_p],
            "spmv_device_error": [_p, ctypes.POINTER(_i32)],
            "spmv_autotune": [_p, _p, _p, _i32, ctypes.POINTER(_i32)],
            "spmv_set_variant": [_p, _i32, _i32],
            "spmv_set_tile": [_p, _i32, _i32, _i32],
            "spmv_set_spmm_kernel": [_p, _i32],
            "spmv_set_f32_kernel": [_p, _i32],
            "spmm_apply_noalloc": [_p, _i32, _p, _i64, _p, _i64, _p],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        for name in ("spmv_strerror",):
            getattr(lib, name).argtypes = [ctypes.c_int]
            getattr(lib, name).restype = ctypes.c_char_p
        for name in ("spmv_last_error", "spmv_version"):
            getattr(lib, name).argtypes = []
            getattr(lib, name).restype = ctypes.c_char_p
        _lib = lib
    return _lib


def _check(status: int, allow=()):
    if status != SPMV_OK and status not in allow:
        lib = library()
        raise SpmvError(status, f"{lib.spmv_strerror(status).decode()}: {lib.spmv_last_error().decode()}")
    return status


def spmv_version() -> str:
    return library().spmv_version().decode()


class SpmvMatrix:
    """Owns one spmv_mat_t; freed with spmv_free when garbage-collected."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.spmv_free(self.handle)
            self.handle = None

    @property
    def _as_parameter_(self):
        return _p(self.handle)

    def info(self) -> dict:
        return spmv_info(self)


def _new(fn, *args) -> SpmvMatrix:
    h = _p()
    _check(fn(*args, ctypes.byref(h)))
    return SpmvMatrix(h.value)


def spmv_build(kind: str = "hpcg", nx: int = 16, ny: int | None = None, nz: int | None = None, seed: int = 0,
               drop_prob: float = 0.10, special_frac: float = 0.05, diag_rule: int = 0,
               permute: bool = True) -> SpmvMatrix:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    d = spmv_gen_desc({"hpcg": 0, "irregular": 1}[kind], nx, ny, nz, seed, drop_prob, special_frac,
                      diag_rule, 1 if permute else 0)
    return _new(library().spmv_build, ctypes.byref(d))


def spmv_build_csr(rowptr, col, val) -> SpmvMatrix:
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    return _new(library().spmv_build_csr, len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data)


def spmv_compress(A: SpmvMatrix, format: str = "auto", order: str = "column", max_dict: int = 254,
                  min_count: int = 64, reorder: bool = False) -> SpmvMatrix:
    o = spmv_opts(FORMATS[format], ORDERS[order], max_dict, min_count, 1 if reorder else 0)
    return _new(library().spmv_compress, A, ctypes.byref(o))


def spmv_permutation(A: SpmvMatrix) -> np.ndarray:
    """perm[new] = old of a handle compressed with reorder=True."""
    perm = np.zeros(max(spmv_info(A)["n"], 1), np.int32)
    _check(library().spmv_permutation(A, perm.ctypes.data))
    return perm[: spmv_info(A)["n"]]


def spmv_set_order(A: SpmvMatrix, order: str) -> None:
    _check(library().spmv_set_order(A, ORDERS[order]))


def spmv_info(A: SpmvMatrix) -> dict:
    i = spmv_info_t()
    _check(library().spmv_info(A, ctypes.byref(i)))
    out = {name: getattr(i, name) for name, _ in spmv_info_t._fields_}
    out["format_name"] = FORMAT_NAMES[out["format"]]
    return out


def spmv_decompress(A: SpmvMatrix):
    info = spmv_info(A)
    rowptr = np.zeros(info["n"] + 1, np.int64)
    col = np.zeros(max(info["nnz"], 1), np.int32)
    val = np.zeros(max(info["nnz"], 1), np.float64)
    _check(library().spmv_decompress(A, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data))
    return rowptr, col[: info["nnz"]], val[: info["nnz"]]


def spmv_export(A: SpmvMatrix) -> bytes:
    n = _sz(0)
    _check(library().spmv_export(A, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(library().spmv_export(A, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def spmv_import(data: bytes) -> SpmvMatrix:
    buf = ctypes.create_string_buffer(data, len(data))
    return _new(library().spmv_import, buf, len(data))


# ----------------------------------------------------------------- device --
def _stream(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dptr(t, dtype_name: str) -> int:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise ValueError(f"expected {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _dptr_rows(t, dtype_name: str) -> int:
    """A row-major block whose rows may be padded (stride(1) == 1, the
    leading dimension stride(0) passed beside it)."""
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise ValueError(f"expected {dtype_name}, got {t.dtype}")
    if t.dim() != 2 or (t.shape[1] > 1 and t.stride(1) != 1) or t.stride(0) < t.shape[1]:
        raise ValueError("expected a 2-D row-major block (unit column stride)")
    return t.data_ptr()


def spmv_apply(A: SpmvMatrix, x, y, stream=None) -> None:
    _check(library().spmv_apply(A, _dptr(x, "float64"), _dptr(y, "float64"), _stream(stream)))


def spmv_apply_host(A: SpmvMatrix, x, y) -> None:
    """x, y: host float64 buffers (numpy arrays or CPU tensors, pinned or not)."""
    px = x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr()
    py = y.ctypes.data if isinstance(y, np.ndarray) else y.data_ptr()
    _check(library().spmv_apply_host(A, px, py))


def spmv_apply_f32(A: SpmvMatrix, x, y, stream=None) -> None:
    _check(library().spmv_apply_f32(A, _dptr(x, "float32"), _dptr(y, "float32"), _stream(stream)))


def spmm_apply(A: SpmvMatrix, X, Y, stream=None) -> None:
    k = X.shape[1]
    _check(library().spmm_apply(A, k, _dptr_rows(X, "float64"), X.stride(0), _dptr_rows(Y, "float64"),
                                Y.stride(0), _stream(stream)))


def spmm_apply_noalloc(A: SpmvMatrix, X, Y, stream=None) -> None:
    """Y = A X without any device allocation (pattern format, FAST order, A
    already on the device, at most 32 columns); see include/spmvc.h."""
    k = X.shape[1]
    _check(library().spmm_apply_noalloc(A, k, _dptr_rows(X, "float64"), X.stride(0), _dptr_rows(Y, "float64"),
                                        Y.stride(0), _stream(stream)))


class SpmvBatch:
    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.spmv_batch_free(self.handle)
            self.handle = None


def _ptr_arrays(mats, xs, ys):
    n = len(mats)
    hm = (_p * n)(*[m.handle for m in mats])
    hx = (_p * n)(*[_dptr(x, "float64") for x in xs])
    hy = (_p * n)(*[_dptr(y, "float64") for y in ys])
    return n, hm, hx, hy


def spmv_batch_create(mats, xs, ys) -> SpmvBatch:
    n, hm, hx, hy = _ptr_arrays(mats, xs, ys)
    h = _p()
    _check(library().spmv_batch_create(n, hm, hx, hy, ctypes.byref(h)))
    return SpmvBatch(h.value, (list(mats), list(xs), list(ys)))


def spmv_batch_launch(plan: SpmvBatch, stream=None) -> None:
    _check(library().spmv_batch_launch(plan.handle, _stream(stream)))


def spmv_batch_autotune(plan: SpmvBatch, reps: int = 10) -> int:
    """Times work items of 64..1024 rows (writes the plan's ys), keeps the
    fastest; returns its rows an item."""
    r = _i32(0)
    _check(library().spmv_batch_autotune(plan.handle, reps, ctypes.byref(r)))
    return r.value


def spmv_batch_free(plan: SpmvBatch) -> None:
    if plan.handle:
        _check(library().spmv_batch_free(plan.handle))
        plan.handle = None


def spmv_apply_batched(mats, xs, ys, stream=None) -> None:
    n, hm, hx, hy = _ptr_arrays(mats, xs, ys)
    _check(library().spmv_apply_batched(n, hm, hx, hy, _stream(stream)))


def cg_solve(A: SpmvMatrix, b, x, tol: float = 1e-10, max_iter: int = 10000, mode: str = "fp64",
             check_every: int = 16, inner_max_iter: int = 300, inner_tol: float = 1e-6,
             use_graph: bool = True) -> dict:
    """Solves A x = b; b and x are CUDA float64 of shape (n,) or (n, nrhs)."""
    nrhs = 1 if b.dim() == 1 else b.shape[1]
    if tuple(x.shape) != tuple(b.shape):
        raise ValueError("x and b must have the same shape")
    o = spmv_cg_opts(tol, max_iter, CG_MODES[mode], check_every, inner_max_iter, inner_tol, nrhs,
                     1 if use_graph else 0)
    r = spmv_cg_result()
    lib = library()
    st = _check(lib.cg_solve(A, _dptr(b, "float64"), _dptr(x, "float64"), ctypes.byref(o), ctypes.byref(r)),
                allow=(SPMV_ENOTCONVERGED,))
    hist = [r.history[i] for i in range(r.history_len)] if r.history else []
    out = dict(status=st, iterations=r.iterations, outer_iterations=r.outer_iterations,
               rel_residual=r.rel_residual, seconds=r.seconds, history=hist)
    lib.spmv_cg_result_free(ctypes.byref(r))
    return out


def spmv_autotune(A: SpmvMatrix, x, y, reps: int = 10) -> int:
    """Times A's kernel configurations on x, y (CUDA float64), each first
    checked against the COLUMN-order product; returns the chosen tile rows
    (z-block kernel: rows a CTA computes; TMA kernel: rows of its column
    block), 1 for the pre-converted kernel, 4 or 5 for the persistent ones,
    0 if nothing to tune."""
    c = _i32(0)
    _check(library().spmv_autotune(A, _dptr(x, "float64"), _dptr(y, "float64"), reps, ctypes.byref(c)))
    return c.value


def spmv_set_variant(A: SpmvMatrix, variant: int, tile_rows: int = 0) -> None:
    """FAST kernel by hand: 0 direct, 1 staged tiles (tile_rows), 2 pre-converted x,
    3 staged tiles of that copy, 4/5 persistent double-buffered tiles,
    6 register-staged tiles, 7 z-marching tiles, 8 register-staged with
    records in shared memory, 9 the same reading one-byte row types,
    11 the TMA z-marching kernel (shapes and conditions in spmvc.h; 10
    needs spmv_set_tile)."""
    _check(library().spmv_set_variant(A, variant, tile_rows))


def spmv_set_spmm_kernel(A: SpmvMatrix, kind: int) -> None:
    """FAST SpMM kernel: 1, 2 or 3 the TMA-fed kernel with that many CTAs an
    SM where it applies (3 by default), 0 one thread a (row, column) pair."""
    _check(library().spmv_set_spmm_kernel(A, kind))


def spmv_set_f32_kernel(A: SpmvMatrix, kind: int) -> None:
    """Binary32 product kernel: 2 TMA-fed with row types (default), 1 row
    types, 0 the row records."""
    _check(library().spmv_set_f32_kernel(A, kind))


def spmv_set_tile(A: SpmvMatrix, variant: int, tile_rows: int, block_threads: int) -> None:
    """spmv_set_variant with the staged kernel's block size (512, or 256 on
    the full 27-slot union); variant 10, the z-block kernel, takes 256 with
    tile_rows = 512 x planes (1536 or 2048); variant 11 takes tile_rows 1 or 2
    (grid lines a thread's 4-column tile spans; 0 keeps the current one) and
    block_threads 2 for two CTAs an SM (blocks of at most 768 rows), any
    other value for one (its block is whole grid lines)."""
    _check(library().spmv_set_tile(A, variant, tile_rows, block_threads))


def spmv_device_error(A: SpmvMatrix) -> int:
    c = _i32(0)
    _check(library().spmv_device_error(A, ctypes.byref(c)))
    return c.value
