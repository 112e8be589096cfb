"""spmm_apply_noalloc, the entry point for callers that cannot allocate
device memory, against spmm_apply on the same matrix and data.

It runs the generic FAST SpMM kernels (X converted as it is read) with their
scratch in a fixed device array instead of the matrix handle's own buffer;
spmm_apply takes a faster route for the full 27-point union (a fixed-point
copy of X).  Both are FAST order, so two consecutive calls must agree with
the ordinary entry point within its tolerance (1e-14), and a column holding
a non-finite entry takes the COLUMN order in both, bit for bit.  This file is
collected last so that a run stopping at the first failure has run every
other test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import spmv_inputs

torch = pytest.importorskip("torch")
import paper_1612_00530_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-14


@pytest.fixture(scope="module", autouse=True)
def device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def c_call(A, X, Y):
    """The C entry point itself, through ctypes."""
    lib = P.library()
    fn = lib.spmm_apply_noalloc
    return fn(ctypes.c_void_p(A.handle), X.shape[1], X.data_ptr(), X.stride(0), Y.data_ptr(), Y.stride(0),
              torch.cuda.current_stream().cuda_stream)


# 3 and 7 do not divide the 256 threads of the column-maxima pass, so some
# of its threads hold no column; all widths check the k-strided scratch words
@pytest.mark.parametrize("k", [1, 3, 7, 8, 32])
def test_matches_spmm_apply_on_two_calls(k):
    g = (20, 17, 13)
    rowptr, col, val = oracle.hpcg_csr(*g)
    n = len(rowptr) - 1
    A = P.spmv_compress(P.spmv_build("hpcg", *g), format="pattern", order="fast")
    X_np = spmv_inputs.uniform_matrix(n, k, seed=3)
    X = torch.from_numpy(X_np).cuda()
    Y_ref = torch.full_like(X, float("nan"))
    P.spmm_apply(A, X, Y_ref)          # ordinary entry point: copies A to the device
    torch.cuda.synchronize()
    ref = Y_ref.cpu().numpy()
    for _ in range(2):
        Y = torch.full_like(X, float("nan"))
        assert c_call(A, X, Y) == P.SPMV_OK
        torch.cuda.synchronize()
        got = Y.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))
    # and both against the CPU oracle
    scale = oracle.spmm(rowptr, col, np.abs(val), np.abs(X_np))
    assert np.max(np.abs(got - oracle.spmm(rowptr, col, val, X_np)) / scale) <= TOL


def test_limits_are_reported():
    g = (8, 8, 8)
    n = 512
    A = P.spmv_compress(P.spmv_build("hpcg", *g), format="pattern", order="fast")
    X = torch.zeros((n, 33), dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    # not on the device yet: refused rather than copied
    assert c_call(A, X[:, :4].contiguous(), Y[:, :4].contiguous()) == P.SPMV_EINVAL
    P.spmm_apply(A, X[:, :4].contiguous(), Y[:, :4].contiguous())
    assert c_call(A, X, Y) == P.SPMV_EINVAL          # 33 columns: above the scratch size
    assert b"32" in P.library().spmv_last_error()


def test_non_finite_column_takes_the_exact_path():
    """A column with a NaN and an infinity: its scale is not finite, so both
    entry points sum it in COLUMN order (the same bits, NaN where the oracle
    has NaN); the other columns stay in FAST order within 1e-14."""
    g = (16, 15, 14)
    rowptr, col, val = oracle.hpcg_csr(*g)
    n = len(rowptr) - 1
    k = 5
    A = P.spmv_compress(P.spmv_build("hpcg", *g), format="pattern", order="fast")
    X_np = spmv_inputs.uniform_matrix(n, k, seed=4)
    X_np[17, 2] = np.nan
    X_np[n // 2, 2] = np.inf
    X = torch.from_numpy(X_np).cuda()
    Y_ref = torch.full_like(X, float("nan"))
    P.spmm_apply(A, X, Y_ref)
    torch.cuda.synchronize()
    ref = Y_ref.cpu().numpy()
    want = oracle.spmm(rowptr, col, val, X_np)
    for _ in range(2):
        Y = torch.full_like(X, 7.0)
        assert c_call(A, X, Y) == P.SPMV_OK
        torch.cuda.synchronize()
        got = Y.cpu().numpy()
        assert np.array_equal(np.isnan(got[:, 2]), np.isnan(want[:, 2]))
        assert np.array_equal(got[:, 2], ref[:, 2], equal_nan=True)
        assert np.array_equal(got[:, 2], want[:, 2], equal_nan=True)
        others = [0, 1, 3, 4]
        assert np.max(np.abs(got[:, others] - ref[:, others])) <= TOL * np.max(np.abs(ref[:, others]))


def test_refuses_column_order_and_reordered_handles():
    g = (8, 8, 8)
    n = 512
    X = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    A = P.spmv_compress(P.spmv_build("hpcg", *g), format="pattern", order="column")
    P.spmm_apply(A, X, Y)
    assert c_call(A, X, Y) == P.SPMV_EUNSUPPORTED
    B = P.spmv_compress(P.spmv_build("irregular", 6, 6, 6, seed=2), format="delta", reorder=True)
    assert c_call(B, X[:216].contiguous(), Y[:216].contiguous()) == P.SPMV_EUNSUPPORTED
