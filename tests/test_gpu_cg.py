"""CG on the device (Table I's CG iteration without the preconditioner)
against the oracle's Hestenes-Stiefel CG, and the mixed-precision
iterative refinement against the same 1e-10 target."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_1612_00530_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def setup(g, order="column", fmt="pattern"):
    rowptr, col, val = oracle.hpcg_csr(*g)
    n = len(rowptr) - 1
    A = P.spmv_build("hpcg", *g)
    C = A if fmt == "ell" else P.spmv_compress(A, format=fmt, order=order)
    b_np = oracle.spmv(rowptr, col, val, np.ones(n))
    return (rowptr, col, val), C, torch.from_numpy(b_np).cuda(), b_np


@pytest.mark.parametrize("order,fmt", [("column", "pattern"), ("fast", "pattern"), ("column", "ell")])
def test_cg_fp64_matches_oracle_history(order, fmt):
    g = (16, 16, 16)
    csr, C, b, b_np = setup(g, order, fmt)
    x = torch.zeros_like(b)
    res = P.cg_solve(C, b, x, tol=1e-10, mode="fp64", check_every=8)
    assert res["status"] == P.SPMV_OK
    x_ref, it_ref, hist_ref = oracle.cg(*csr, b_np, tol=1e-10, maxit=1000)
    hist = np.array(res["history"])
    assert abs(res["iterations"] - it_ref) <= 1
    m = min(30, len(hist), len(hist_ref))
    assert np.max(np.abs(hist[:m] / hist_ref[:m] - 1)) < 1e-8
    assert res["rel_residual"] <= 1.5e-10
    assert np.max(np.abs(x.cpu().numpy() - 1.0)) < 1e-8


def test_cg_without_graphs_same_history():
    g = (12, 12, 12)
    _, C, b, _ = setup(g)
    x1 = torch.zeros_like(b)
    x2 = torch.zeros_like(b)
    r1 = P.cg_solve(C, b, x1, use_graph=True, check_every=5)
    r2 = P.cg_solve(C, b, x2, use_graph=False, check_every=5)
    assert r1["history"] == r2["history"]
    assert torch.equal(x1, x2)


def test_cg_ir_fp32_reaches_target():
    g = (32, 32, 32)
    _, C, b, _ = setup(g)
    x = torch.zeros_like(b)
    res = P.cg_solve(C, b, x, tol=1e-10, mode="ir_fp32")
    assert res["status"] == P.SPMV_OK
    assert res["rel_residual"] <= 1e-10
    assert res["outer_iterations"] >= 2
    assert np.max(np.abs(x.cpu().numpy() - 1.0)) < 1e-8


def test_cg_reports_not_converged():
    g = (16, 16, 16)
    _, C, b, _ = setup(g)
    x = torch.zeros_like(b)
    res = P.cg_solve(C, b, x, tol=1e-10, max_iter=5)
    assert res["status"] == P.SPMV_ENOTCONVERGED
    assert res["iterations"] == 5


@pytest.mark.parametrize("k,order,g", [(4, "fast", (14, 13, 12)), (8, "column", (14, 13, 12)),
                                       (3, "fast", (14, 13, 12)), (8, "fast", (32, 24, 10)),
                                       (12, "fast", (32, 24, 10))])
def test_batched_cg_columns_match_oracle(k, order, g):
    """k right-hand sides at once against the oracle's CG column by column;
    on the 32 x 24 grid the products run through the TMA-fed SpMM with the
    columns' scales fixed from the update kernel's maxima of |p|."""
    rowptr, col, val = oracle.hpcg_csr(*g)
    n = len(rowptr) - 1
    import spmv_inputs
    V = spmv_inputs.uniform_matrix(n, k, seed=21)
    B_np = oracle.spmm(rowptr, col, val, V)
    A = P.spmv_build("hpcg", *g)
    C = P.spmv_compress(A, format="pattern", order=order)
    B = torch.from_numpy(B_np).cuda()
    X = torch.zeros_like(B)
    res = P.cg_solve(C, B, X, tol=1e-10, check_every=8)
    assert res["status"] == P.SPMV_OK and res["rel_residual"] <= 1.5e-10
    Xh = X.cpu().numpy()
    its = []
    for j in range(k):
        xj, itj, _ = oracle.cg(rowptr, col, val, np.ascontiguousarray(B_np[:, j]), tol=1e-10, maxit=1000)
        its.append(itj)
        assert np.max(np.abs(Xh[:, j] - xj)) < 1e-7
        assert np.max(np.abs(Xh[:, j] - V[:, j])) < 1e-7
    # the batch stops when its slowest column converges
    assert abs(res["iterations"] - max(its)) <= 1


def test_ir_fp32_with_longer_inner_solves():
    g = (32, 32, 32)
    _, C, b, _ = setup(g)
    x = torch.zeros_like(b)
    res = P.cg_solve(C, b, x, tol=1e-10, mode="ir_fp32", inner_max_iter=400, inner_tol=1e-6)
    assert res["status"] == P.SPMV_OK and res["rel_residual"] <= 1e-10
    assert np.max(np.abs(x.cpu().numpy() - 1.0)) < 1e-8



def test_cg_fp64_with_tma_kernel():
    """FP64 CG whose FAST product is the TMA kernel: the history follows the
    oracle's, is the same with and without graphs, and x reaches the
    all-ones solution."""
    g = (32, 64, 6)
    csr, C, b, b_np = setup(g, "fast")
    P.spmv_set_tile(C, 11, 1, 0)
    x1 = torch.zeros_like(b)
    r1 = P.cg_solve(C, b, x1, tol=1e-10, mode="fp64", check_every=8)
    assert r1["status"] == P.SPMV_OK and r1["rel_residual"] <= 1.5e-10
    x_ref, it_ref, hist_ref = oracle.cg(*csr, b_np, tol=1e-10, maxit=2000)
    hist = np.array(r1["history"])
    assert abs(r1["iterations"] - it_ref) <= 1
    m = min(30, len(hist), len(hist_ref))
    assert np.max(np.abs(hist[:m] / hist_ref[:m] - 1)) < 1e-8
    assert np.max(np.abs(x1.cpu().numpy() - 1.0)) < 1e-8
    x2 = torch.zeros_like(b)
    r2 = P.cg_solve(C, b, x2, tol=1e-10, mode="fp64", check_every=8, use_graph=False)
    assert r1["history"] == r2["history"]
    assert torch.equal(x1, x2)
    assert P.spmv_device_error(C) == 0
