"""CPU oracle for the compressed SpMV path (arXiv:1612.00530).

TEST INFRASTRUCTURE ONLY: a plain, slow, obviously correct restatement in C
(oracle.c, binary64, explicit fma) of what the CUDA library computes.  Only
the tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg import
this package; the library never does, and this package never imports the
library.  Each wrapper names the passage of the paper it follows.

Parity status of each function (what pins it is in tests/test_oracle_pins.py):
  hpcg_csr / hpcg_row / hpcg_spmv_rows : pinned (nnz closed form, row classes,
      A*1, symmetry, brute-force dense, Kronecker closed form, eigenpairs)
  spmv / spmv_f32 / spmm              : pinned (integer-x exactness vs dense
      matmul, eigenpairs, brute force)
  value_table / data_table_row        : pinned (Fig. 2 worked example)
  data_table_spmv                     : pinned (exact rational model of its
      fma chain in value-group order on non-integer x, with planted slips;
      integer-x equality with the CSR product; Fig. 2 row)
  data_index_table / listing1_spmv    : pinned (pattern census, integer-x
      equality with the CSR product, byte counts of Sec. V)
  kron_apply                          : pinned (dense Kronecker product)
  cg                                  : pinned (exact solution 1, Krylov
      termination on tiny grids, iteration bound from the closed-form kappa)
  irregular_csr                       : parity unpinned beyond its invariants
      (symmetry, value set, drop rate, M-matrix certificate, brute-force row
      checks of the stated construction) -- the paper prints no values.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build_oracle

_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int
_u64 = ctypes.c_uint64
_dbl = ctypes.c_double
_p = ctypes.c_void_p


def _load():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        lib = ctypes.CDLL(path)
        sig = {
            "orc_hpcg_row": (_i32, [_i32, _i32, _i32, _i64, _p, _p]),
            "orc_hpcg_csr": (_i64, [_i32, _i32, _i32, _i64, _i64, _p, _p, _p]),
            "orc_hpcg_spmv_rows": (None, [_i32, _i32, _i32, _i64, _p, _p, _p]),
            "orc_irregular_csr": (_i64, [_i32, _i32, _i32, _u64, _dbl, _dbl, _i32, _i32, _p, _p, _p, _p]),
            "orc_spmv_csr": (None, [_i64, _p, _p, _p, _p, _p]),
            "orc_spmv_csr_range": (None, [_i64, _i64, _p, _p, _p, _p, _p]),
            "orc_spmv_csr_f32": (None, [_i64, _p, _p, _p, _p, _p]),
            "orc_spmm_csr": (None, [_i64, _i32, _p, _p, _p, _p, _p]),
            "orc_value_table": (_i64, [_i64, _p, _p]),
            "orc_data_table_row": (None, [_i32, _p, _p, _i32, _p, _p, _p, _p]),
            "orc_data_table_spmv": (None, [_i64, _p, _p, _p, _i32, _p, _p, _p]),
            "orc_data_index_table": (_i64, [_i64, _p, _p, _p, _i32, _p, _i32, _i64, _p, _p, _p, _p]),
            "orc_listing1_spmv": (None, [_i64, _p, _p, _i32, _p, _i32, _p, _p, _p]),
            "orc_hpcg_kron_apply": (None, [_i32, _i32, _i32, _p, _p, _p]),
            "orc_cg": (_i32, [_i64, _p, _p, _p, _p, _p, _dbl, _i32, _p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# Sec. III-A: the HPCG 27-point-stencil matrix
# --------------------------------------------------------------------------
def hpcg_row(nx: int, ny: int, nz: int, i: int):
    """Columns (ascending) and values of row i (Sec. III-A, Fig. 2 values)."""
    col = np.zeros(27, np.int32)
    val = np.zeros(27, np.float64)
    k = _load().orc_hpcg_row(nx, ny, nz, i, _ptr(col), _ptr(val))
    return col[:k].copy(), val[:k].copy()


def hpcg_csr(nx: int, ny: int, nz: int, row0: int = 0, row1: int | None = None):
    """CSR (rowptr int64, col int32, val float64) of rows [row0, row1)."""
    n = nx * ny * nz
    row1 = n if row1 is None else row1
    m = row1 - row0
    rowptr = np.zeros(m + 1, np.int64)
    col = np.zeros(27 * m, np.int32)
    val = np.zeros(27 * m, np.float64)
    nnz = _load().orc_hpcg_csr(nx, ny, nz, row0, row1, _ptr(rowptr), _ptr(col), _ptr(val))
    return rowptr, col[:nnz].copy(), val[:nnz].copy()


def hpcg_spmv_rows(nx: int, ny: int, nz: int, rows, x) -> np.ndarray:
    """Eq. (1) on selected rows, each rebuilt from the stencil definition."""
    rows = _c(rows, np.int64)
    x = _c(x, np.float64)
    y = np.zeros(len(rows), np.float64)
    _load().orc_hpcg_spmv_rows(nx, ny, nz, len(rows), _ptr(rows), _ptr(x), _ptr(y))
    return y


def irregular_csr(nx: int, ny: int, nz: int, seed: int, drop_p: float = 0.10,
                  special_frac: float = 0.05, diag_rule: int = 0, permute: bool = True):
    """The irregularised 27-point matrix (see oracle.c for the construction)."""
    n = nx * ny * nz
    rowptr = np.zeros(n + 1, np.int64)
    col = np.zeros(27 * n, np.int32)
    val = np.zeros(27 * n, np.float64)
    perm = np.zeros(n, np.int32)
    nnz = _load().orc_irregular_csr(nx, ny, nz, seed, drop_p, special_frac, diag_rule,
                                    1 if permute else 0, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(perm))
    if nnz < 0:
        raise MemoryError("oracle irregular generator failed")
    return rowptr, col[:nnz].copy(), val[:nnz].copy(), perm


# --------------------------------------------------------------------------
# Eq. (1): y = A x
# --------------------------------------------------------------------------
def spmv(rowptr, col, val, x) -> np.ndarray:
    """y_i = fma chain over row i in ascending column order, from 0."""
    rowptr, col, val, x = _c(rowptr, np.int64), _c(col, np.int32), _c(val, np.float64), _c(x, np.float64)
    n = len(rowptr) - 1
    y = np.zeros(n, np.float64)
    _load().orc_spmv_csr(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
    return y


def spmv_range(row0: int, row1: int, rowptr, col, val, x) -> np.ndarray:
    """Eq. (1) for rows [row0,row1) of a CSR slice whose rowptr starts at row0."""
    rowptr, col, val, x = _c(rowptr, np.int64), _c(col, np.int32), _c(val, np.float64), _c(x, np.float64)
    y = np.zeros(row1 - row0, np.float64)
    _load().orc_spmv_csr_range(row0, row1, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
    return y


def spmv_f32(rowptr, col, val, x32) -> np.ndarray:
    """Eq. (1) in binary32: values rounded to float, fmaf chain from 0."""
    rowptr, col, val = _c(rowptr, np.int64), _c(col, np.int32), _c(val, np.float64)
    x32 = _c(x32, np.float32)
    n = len(rowptr) - 1
    y = np.zeros(n, np.float32)
    _load().orc_spmv_csr_f32(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(x32), _ptr(y))
    return y


def spmm(rowptr, col, val, X) -> np.ndarray:
    """Eq. (1) column by column for a row-major n x k block X."""
    rowptr, col, val = _c(rowptr, np.int64), _c(col, np.int32), _c(val, np.float64)
    X = _c(X, np.float64)
    n = len(rowptr) - 1
    k = X.shape[1]
    Y = np.zeros((n, k), np.float64)
    _load().orc_spmm_csr(n, k, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(X), _ptr(Y))
    return Y


# --------------------------------------------------------------------------
# Sec. V: value table, data table (Fig. 2), data+index table (Listing 1)
# --------------------------------------------------------------------------
def value_table(val) -> np.ndarray:
    """All distinct values, ascending (Sec. V)."""
    val = _c(val, np.float64)
    V = np.zeros(max(len(val), 1), np.float64)
    m = _load().orc_value_table(len(val), _ptr(val), _ptr(V))
    return V[:m].copy()


def data_table_row(col, val, V):
    """(S_i, T_incl, T_end) of one row (Sec. V, Fig. 2)."""
    col, val, V = _c(col, np.int32), _c(val, np.float64), _c(V, np.float64)
    S = np.zeros(len(col), np.int32)
    Ti = np.zeros(len(V), np.int32)
    Te = np.zeros(len(V), np.int32)
    _load().orc_data_table_row(len(col), _ptr(col), _ptr(val), len(V), _ptr(V), _ptr(S), _ptr(Ti), _ptr(Te))
    return S, Ti, Te


def data_table_spmv(rowptr, col, val, V, x) -> np.ndarray:
    """y = A x from each row's (S_i, T_i) over the value table V (Sec. V,
    "Data Table"): value groups ascending, one fma per entry."""
    rowptr, col, val = _c(rowptr, np.int64), _c(col, np.int32), _c(val, np.float64)
    V, x = _c(V, np.float64), _c(x, np.float64)
    n = len(rowptr) - 1
    y = np.zeros(n, np.float64)
    _load().orc_data_table_spmv(n, _ptr(rowptr), _ptr(col), _ptr(val), len(V), _ptr(V), _ptr(x), _ptr(y))
    return y


def data_index_table(rowptr, col, val, V, maxlen: int = 27, maxtypes: int = 4096):
    """Pattern registration of Sec. V: (type, diffs, typelen, valueIdxEnd)."""
    rowptr, col, val, V = _c(rowptr, np.int64), _c(col, np.int32), _c(val, np.float64), _c(V, np.float64)
    n = len(rowptr) - 1
    typ = np.zeros(n, np.int32)
    diffs = np.zeros(maxtypes * maxlen, np.int32)
    typelen = np.zeros(maxtypes, np.int32)
    ends = np.zeros(n * len(V), np.int32)
    nt = _load().orc_data_index_table(n, _ptr(rowptr), _ptr(col), _ptr(val), len(V), _ptr(V), maxlen,
                                      maxtypes, _ptr(typ), _ptr(diffs), _ptr(typelen), _ptr(ends))
    if nt < 0:
        raise ValueError("too many patterns")
    return typ, diffs.reshape(maxtypes, maxlen)[:nt].copy(), typelen[:nt].copy(), ends.reshape(n, len(V))


def listing1_spmv(typ, diffs, ends, V, x) -> np.ndarray:
    """Listing 1's decode loop over value groups and pattern displacements."""
    typ, diffs, ends = _c(typ, np.int32), _c(diffs, np.int32), _c(ends, np.int32)
    V, x = _c(V, np.float64), _c(x, np.float64)
    n = len(typ)
    y = np.zeros(n, np.float64)
    _load().orc_listing1_spmv(n, _ptr(typ), _ptr(diffs), diffs.shape[1], _ptr(ends), len(V), _ptr(V),
                              _ptr(x), _ptr(y))
    return y


def kron_apply(nx: int, ny: int, nz: int, x) -> np.ndarray:
    """y = (27 I - Tz (x) Ty (x) Tx) x via three 1-D 3-point sums."""
    x = _c(x, np.float64)
    n = nx * ny * nz
    y = np.zeros(n, np.float64)
    work = np.zeros(2 * n, np.float64)
    _load().orc_hpcg_kron_apply(nx, ny, nz, _ptr(x), _ptr(y), _ptr(work))
    return y


def cg(rowptr, col, val, b, x0=None, tol: float = 1e-10, maxit: int = 1000):
    """Hestenes-Stiefel CG; returns (x, iterations, relative residual history)."""
    rowptr, col, val, b = _c(rowptr, np.int64), _c(col, np.int32), _c(val, np.float64), _c(b, np.float64)
    n = len(rowptr) - 1
    x = np.zeros(n, np.float64) if x0 is None else _c(x0, np.float64).copy()
    hist = np.zeros(maxit + 1, np.float64)
    it = _load().orc_cg(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b), _ptr(x), tol, maxit, _ptr(hist))
    if it < 0:
        raise MemoryError("oracle cg failed")
    return x, it, hist[: it + 1].copy()
