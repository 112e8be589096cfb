"""spmm_apply_noalloc, the entry point for callers that cannot allocate
device memory, against spmm_apply on the same matrix and data.

It runs the same kernels with its scratch in a fixed device array instead of
the matrix handle's own buffer, so two consecutive calls must agree with the
ordinary entry point within the FAST-order tolerance (1e-14).  This file is
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


@pytest.mark.parametrize("k", [1, 8, 32])
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
