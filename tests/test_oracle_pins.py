"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formula: each compares it with
something of different structure (a closed form, a dense brute force built
from the stencil definition, the Kronecker form, eigenpairs, exact integer
arithmetic, the worked example printed in the paper).
"""
import os

import numpy as np
import pytest

import oracle
import spmv_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [float(v) for v in vals]
    return out


def dense_from_definition(nx, ny, nz):
    """Brute force: A[i, j] = 26 if i == j, -1 if the nodes touch (Chebyshev
    distance 1 on the grid), else 0 -- every pair of nodes examined."""
    n = nx * ny * nz
    coords = [(i % nx, (i // nx) % ny, i // (nx * ny)) for i in range(n)]
    A = np.zeros((n, n))
    for i, (ax, ay, az) in enumerate(coords):
        for j, (bx, by, bz) in enumerate(coords):
            d = max(abs(ax - bx), abs(ay - by), abs(az - bz))
            if d == 0:
                A[i, j] = 26.0
            elif d == 1:
                A[i, j] = -1.0
    return A


def csr_to_dense(rowptr, col, val, n):
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            A[i, col[k]] += val[k]
    return A


def tridiag_ones(n):
    return np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)


GRIDS = [(1, 1, 1), (2, 1, 1), (2, 3, 5), (3, 3, 3), (4, 4, 4), (5, 7, 3), (1, 4, 6), (17, 3, 2)]


@pytest.mark.parametrize("g", GRIDS)
def test_nnz_closed_form(g):
    nx, ny, nz = g
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    assert rowptr[-1] == (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2)


def test_nnz_32_cubed():
    rowptr, _, _ = oracle.hpcg_csr(32, 32, 32)
    assert rowptr[-1] == 830584


@pytest.mark.parametrize("g", [(4, 4, 4), (6, 5, 7)])
def test_row_classes(g):
    nx, ny, nz = g
    rowptr, _, _ = oracle.hpcg_csr(nx, ny, nz)
    lens = np.diff(rowptr)
    assert set(np.unique(lens)) <= {8, 12, 18, 27}
    # interior rows (27 entries) are exactly those away from every face
    assert np.sum(lens == 27) == (nx - 2) * (ny - 2) * (nz - 2)
    assert np.sum(lens == 8) == 8


@pytest.mark.parametrize("g", GRIDS)
def test_dense_brute_force(g):
    nx, ny, nz = g
    n = nx * ny * nz
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    assert np.array_equal(csr_to_dense(rowptr, col, val, n), dense_from_definition(nx, ny, nz))
    # columns strictly ascending inside each row
    for i in range(n):
        assert np.all(np.diff(col[rowptr[i]:rowptr[i + 1]]) > 0)


@pytest.mark.parametrize("g", [(4, 4, 4), (3, 4, 5), (2, 3, 1)])
def test_kronecker_closed_form(g):
    nx, ny, nz = g
    n = nx * ny * nz
    K = np.kron(tridiag_ones(nz), np.kron(tridiag_ones(ny), tridiag_ones(nx)))
    A = 27.0 * np.eye(n) - K
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    assert np.array_equal(csr_to_dense(rowptr, col, val, n), A)
    x = spmv_inputs.integer_vector(n, seed=5)
    assert np.array_equal(oracle.kron_apply(nx, ny, nz, x), A @ x)


@pytest.mark.parametrize("g", [(32, 32, 32), (17, 9, 23)])
def test_a_times_ones(g):
    nx, ny, nz = g
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    y = oracle.spmv(rowptr, col, val, np.ones(nx * ny * nz))
    assert np.array_equal(y, 27.0 - np.diff(rowptr))


def test_symmetry_bitexact():
    n = 9 * 8 * 7
    rowptr, col, val = oracle.hpcg_csr(9, 8, 7)
    A = csr_to_dense(rowptr, col, val, n)
    assert np.array_equal(A, A.T)


@pytest.mark.parametrize("g", [(6, 5, 4), (12, 10, 9)])
def test_eigenpairs(g):
    nx, ny, nz = g
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    rng = [(1, 1, 1), (2, 3, 1), (nx, ny, nz), (3, 1, 2)]
    for kx, ky, kz in rng:
        vx = np.sin(kx * np.arange(1, nx + 1) * np.pi / (nx + 1))
        vy = np.sin(ky * np.arange(1, ny + 1) * np.pi / (ny + 1))
        vz = np.sin(kz * np.arange(1, nz + 1) * np.pi / (nz + 1))
        v = np.kron(vz, np.kron(vy, vx))
        lam = 27.0 - np.prod([1 + 2 * np.cos(k * np.pi / (m + 1)) for k, m in ((kx, nx), (ky, ny), (kz, nz))])
        r = oracle.spmv(rowptr, col, val, v) - lam * v
        assert np.max(np.abs(r)) <= 1e-13 * np.max(np.abs(v)) * 54


def test_integer_x_is_exact_in_any_order():
    nx, ny, nz = 8, 8, 8
    n = nx * ny * nz
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    x = spmv_inputs.integer_vector(n, seed=11)
    A = dense_from_definition(nx, ny, nz).astype(np.int64)
    y_int = A @ x.astype(np.int64)
    assert np.array_equal(oracle.spmv(rowptr, col, val, x), y_int.astype(np.float64))
    big = 40
    xb = spmv_inputs.integer_vector(big ** 3, seed=12)
    rp, c, v = oracle.hpcg_csr(big, big, big)
    assert np.array_equal(oracle.spmv(rp, c, v, xb), oracle.kron_apply(big, big, big, xb))


def test_sampled_rows_match_full_csr():
    nx, ny, nz = 20, 13, 11
    n = nx * ny * nz
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    x = spmv_inputs.uniform_vector(n, seed=1)
    y = oracle.spmv(rowptr, col, val, x)
    rows = np.array([0, 1, nx - 1, nx, n // 2, n - 1, n - nx])
    assert np.array_equal(oracle.hpcg_spmv_rows(nx, ny, nz, rows, x), y[rows])
    # a row range of the CSR
    rp2, c2, v2 = oracle.hpcg_csr(nx, ny, nz, 100, 900)
    assert np.array_equal(oracle.spmv_range(100, 900, rp2, c2, v2, x), y[100:900])


def test_random_x_close_to_dense_product():
    nx, ny, nz = 5, 6, 7
    n = nx * ny * nz
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    x = spmv_inputs.uniform_vector(n, seed=0)
    A = dense_from_definition(nx, ny, nz)
    y = oracle.spmv(rowptr, col, val, x)
    scale = np.abs(A) @ np.abs(x)
    assert np.max(np.abs(y - A @ x) / scale) < 1e-15 * 30


def test_spmv_f32_matches_float_arithmetic():
    nx, ny, nz = 6, 6, 6
    n = nx * ny * nz
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    x = spmv_inputs.integer_vector(n, seed=3).astype(np.float32)
    y = oracle.spmv_f32(rowptr, col, val, x)
    assert y.dtype == np.float32
    assert np.array_equal(y, oracle.spmv(rowptr, col, val, x.astype(np.float64)).astype(np.float32))


def pow2(e):
    from fractions import Fraction
    return Fraction(2) ** e if e >= 0 else Fraction(1, 2 ** -e)


def round_binary32(q):
    """The binary32 number nearest to the rational q, ties to even (IEEE 754
    round-to-nearest-even), subnormals included; overflow is not reached by
    the inputs used here."""
    from fractions import Fraction
    if q == 0:
        return Fraction(0)
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if pow2(e) > a:
        e -= 1                       # now 2^e <= a < 2^(e+1)
    e = max(e, -126)                 # subnormal range: fixed quantum 2^-149
    quantum = pow2(e - 23)
    m = a / quantum
    f = m.numerator // m.denominator
    rest = m - f
    if rest > Fraction(1, 2) or (rest == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return (f * quantum) if q > 0 else -(f * quantum)


def exact_binary32_csr(rowptr, col, val, x32):
    """Each row: s = 0; s = RN32(RN32(a_ij) * x_j + s) in ascending column
    order, every step evaluated exactly in rationals and rounded once, which
    is what an fmaf chain computes."""
    from fractions import Fraction
    xs = [Fraction(float(v)) for v in x32.tolist()]
    vs = [round_binary32(Fraction(float(v))) for v in val.tolist()]
    out = np.empty(len(rowptr) - 1, np.float32)
    for i in range(len(rowptr) - 1):
        s = Fraction(0)
        for k in range(rowptr[i], rowptr[i + 1]):
            s = round_binary32(vs[k] * xs[col[k]] + s)
        out[i] = np.float32(float(s))
    return out


def test_round_binary32_against_numpy():
    from fractions import Fraction
    rng = np.random.default_rng(5)
    for d in np.concatenate([rng.uniform(-3, 3, 300), rng.uniform(-1e-40, 1e-40, 50), [1.0 + 2.0 ** -24]]):
        assert np.float32(float(round_binary32(Fraction(float(d))))) == np.float32(d)


@pytest.mark.parametrize("which", ["hpcg", "irregular"])
def test_spmv_f32_rounds_every_fma_step(which):
    """Non-integer x: the binary32 product equals the exact model of an fmaf
    chain (one rounding per step) bit for bit.  The irregular matrix's values
    (-1.5 + k/15, U[-2,-0.1)) are not binary32 numbers, so the rounding of
    each value to binary32 is pinned too."""
    if which == "hpcg":
        rowptr, col, val = oracle.hpcg_csr(5, 4, 6)
    else:
        rowptr, col, val, _ = oracle.irregular_csr(6, 5, 4, seed=2)
    n = len(rowptr) - 1
    x32 = spmv_inputs.uniform_vector(n, seed=11).astype(np.float32)
    want = exact_binary32_csr(rowptr, col, val, x32)
    got = oracle.spmv_f32(rowptr, col, val, x32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # planted slips, each of which this pin must tell apart from the model:
    # (a) accumulation in binary64, one rounding at the end
    v32 = val.astype(np.float32).astype(np.float64)
    slip_a = oracle.spmv(rowptr, col, v32, x32.astype(np.float64)).astype(np.float32)
    assert not np.array_equal(slip_a, want)
    # (b) separate binary32 multiply and add (no fused multiply-add)
    slip_b = np.empty(n, np.float32)
    for i in range(n):
        s = np.float32(0)
        for k in range(rowptr[i], rowptr[i + 1]):
            s = np.float32(np.float32(np.float32(val[k]) * x32[col[k]]) + s)
        slip_b[i] = s
    assert not np.array_equal(slip_b, want)


def test_spmm_columns_match_spmv():
    nx, ny, nz = 7, 5, 6
    n = nx * ny * nz
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    X = spmv_inputs.uniform_matrix(n, 4, seed=3)
    Y = oracle.spmm(rowptr, col, val, X)
    for c in range(4):
        assert np.array_equal(Y[:, c], oracle.spmv(rowptr, col, val, X[:, c].copy()))


# --------------------------------------------------------------------------
# Sec. V worked example and byte counts
# --------------------------------------------------------------------------
def test_fig2_worked_example():
    g = read_golden("fig2_worked_example.txt")
    val = np.array(g["values"])
    col = np.array(g["columns"], dtype=np.int32)
    V = oracle.value_table(val)
    assert np.array_equal(V, np.array(g["V"]))
    S, T_incl, T_end = oracle.data_table_row(col, val, V)
    assert np.array_equal(S, np.array(g["S"], dtype=np.int32))
    assert np.array_equal(T_incl, np.array(g["T"], dtype=np.int32))
    assert np.array_equal(T_end, T_incl + 1)


def exact_data_table_spmv(rowptr, col, val, x):
    """Each row: entries ordered by value (ascending), ties by ascending
    column; s = 0; s = RN64(a * x_j + s) per entry, every step evaluated
    exactly in rationals and rounded once to binary64 (Python's float of a
    Fraction rounds correctly), which is what an fma chain computes."""
    from fractions import Fraction
    xs = [Fraction(float(v)) for v in x.tolist()]
    out = np.empty(len(rowptr) - 1, np.float64)
    for i in range(len(rowptr) - 1):
        ks = sorted(range(rowptr[i], rowptr[i + 1]), key=lambda k: (val[k], col[k]))
        s = Fraction(0)
        for k in ks:
            s = Fraction(float(Fraction(float(val[k])) * xs[col[k]] + s))
        out[i] = float(s)
    return out


@pytest.mark.parametrize("which", ["hpcg", "irregular"])
def test_data_table_spmv_is_the_value_group_fma_chain(which):
    """Non-integer x: the Data Table product equals the exact model of an
    fma chain in value-group order bit for bit; two plausible slips (the
    column-order chain, separate multiply and add) both differ from it."""
    if which == "hpcg":
        rowptr, col, val = oracle.hpcg_csr(5, 4, 6)
    else:
        # no unique-valued rows: the table holds the 16 levels and the diagonals
        rowptr, col, val, _ = oracle.irregular_csr(6, 5, 4, seed=2, special_frac=0.0, diag_rule=1)
    n = len(rowptr) - 1
    x = spmv_inputs.uniform_vector(n, seed=13)
    V = oracle.value_table(val)
    want = exact_data_table_spmv(rowptr, col, val, x)
    got = oracle.data_table_spmv(rowptr, col, val, V, x)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    slip_col = oracle.spmv(rowptr, col, val, x)                 # ascending columns
    assert not np.array_equal(slip_col, want)
    slip_sep = np.empty(n)
    for i in range(n):
        s = 0.0
        for k in sorted(range(rowptr[i], rowptr[i + 1]), key=lambda k: (val[k], col[k])):
            s = float(np.float64(val[k]) * np.float64(x[col[k]])) + s
        slip_sep[i] = s
    assert not np.array_equal(slip_sep, want)


def test_data_table_spmv_integer_x_and_fig2_row():
    # integer x: every partial sum is exact, so any order gives the CSR product
    rowptr, col, val = oracle.hpcg_csr(6, 7, 5)
    n = len(rowptr) - 1
    x = np.random.default_rng(4).integers(-50, 50, n).astype(np.float64)
    V = oracle.value_table(val)
    assert np.array_equal(oracle.data_table_spmv(rowptr, col, val, V, x), oracle.spmv(rowptr, col, val, x))
    ones = np.ones(n)
    assert np.array_equal(oracle.data_table_spmv(rowptr, col, val, V, ones), 27.0 - np.diff(rowptr))
    # the Fig. 2 row as a one-row matrix over 66 columns, x_j = j
    g = read_golden("fig2_worked_example.txt")
    fcol = np.array(g["columns"], dtype=np.int32)
    fval = np.array(g["values"], dtype=np.float64)
    xj = np.arange(66, dtype=np.float64)
    y = oracle.data_table_spmv(np.array([0, len(fcol)]), fcol, fval, oracle.value_table(fval), xj)
    assert y[0] == -(45 + 49 + 51 + 65) + 26 * 50


def test_value_table_of_hpcg():
    _, _, val = oracle.hpcg_csr(7, 7, 7)
    assert np.array_equal(oracle.value_table(val), np.array([-1.0, 26.0]))


def test_sec5_byte_counts_and_table2():
    g = read_golden("sec5_table2.txt")
    nx = ny = nz = 5
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    V = oracle.value_table(val)
    typ, diffs, typelen, ends = oracle.data_index_table(rowptr, col, val, V)
    i = 2 + nx * (2 + ny * 2)  # an interior row
    nnz_row = rowptr[i + 1] - rowptr[i]
    S, Ti, Te = oracle.data_table_row(col[rowptr[i]:rowptr[i + 1]], val[rowptr[i]:rowptr[i + 1]], V)
    original = nnz_row * (8 + 4)            # FP64 value + int32 column per entry
    data_table = (len(S) + len(Ti)) * 4     # S_i and T_i as 4-byte words
    data_index = (1 + len(Ti)) * 4          # pattern number + T_i
    assert original == g["original_ell_bytes_per_row"][0]
    assert data_table == g["data_table_bytes_per_row"][0]
    assert data_index == g["data_index_table_bytes_per_row"][0]
    bw = g["measured_read_bandwidth_gbs"][0]
    flops_row = 2 * nnz_row
    assert bw / g["ell_bytes_per_flop"][0] == g["table2_theoretical_original"][0]
    assert bw * flops_row / original == pytest.approx(g["table2_theoretical_original"][0])
    # the paper prints 34.8 for 75*54/116 = 34.91 (a rounding of the paper)
    assert bw * flops_row / data_table == pytest.approx(g["table2_theoretical_data_table"][0], abs=0.15)
    # 326 in Table II does not follow from 12 B/row (75*54/12 = 337.5); kept
    # as printed, within 4 percent
    assert bw * flops_row / data_index == pytest.approx(g["table2_theoretical_data_index"][0], rel=0.04)


@pytest.mark.parametrize("g,ntypes", [((5, 5, 5), 27), ((3, 4, 6), 27), ((2, 2, 2), 8), ((1, 3, 3), 9), ((1, 1, 1), 1)])
def test_pattern_census(g, ntypes):
    nx, ny, nz = g
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    V = oracle.value_table(val)
    typ, diffs, typelen, ends = oracle.data_index_table(rowptr, col, val, V)
    assert len(typelen) == ntypes
    # every row's value ends: n-1 entries of -1 then the single 26
    lens = np.diff(rowptr)
    if len(V) == 2:
        assert np.array_equal(ends[:, 0], lens - 1)
        assert np.array_equal(ends[:, 1], lens)


@pytest.mark.parametrize("g", [(6, 6, 6), (9, 4, 7)])
def test_listing1_equals_csr(g):
    nx, ny, nz = g
    n = nx * ny * nz
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    V = oracle.value_table(val)
    typ, diffs, typelen, ends = oracle.data_index_table(rowptr, col, val, V)
    xi = spmv_inputs.integer_vector(n, seed=4)
    assert np.array_equal(oracle.listing1_spmv(typ, diffs, ends, V, xi), oracle.spmv(rowptr, col, val, xi))
    x = spmv_inputs.uniform_vector(n, seed=4)
    y1 = oracle.listing1_spmv(typ, diffs, ends, V, x)
    y0 = oracle.spmv(rowptr, col, val, x)
    assert np.max(np.abs(y1 - y0)) <= 1e-14 * np.max(np.abs(y0))


# --------------------------------------------------------------------------
# CG
# --------------------------------------------------------------------------
def kappa_hpcg(nx, ny, nz):
    ev = lambda k, m: 1 + 2 * np.cos(k * np.pi / (m + 1))
    lams = []
    for kx in (1, nx):
        for ky in (1, ny):
            for kz in (1, nz):
                lams.append(27.0 - ev(kx, nx) * ev(ky, ny) * ev(kz, nz))
    # extreme eigenvalues are attained at the extreme wave numbers
    return max(lams) / min(lams)


def test_cg_converges_to_ones_within_bound():
    nx = ny = nz = 16
    n = nx * ny * nz
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    b = oracle.spmv(rowptr, col, val, np.ones(n))
    x, it, hist = oracle.cg(rowptr, col, val, b, tol=1e-10, maxit=500)
    kap = kappa_hpcg(nx, ny, nz)
    bound = 0.5 * np.sqrt(kap) * np.log(2 / 1e-10)
    assert hist[-1] <= 1e-10
    assert it <= bound
    assert np.max(np.abs(x - 1.0)) < 1e-8
    # true residual agrees with the recurrence
    r = b - oracle.spmv(rowptr, col, val, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-9


def test_cg_energy_norm_monotone():
    nx, ny, nz = 10, 9, 8
    n = nx * ny * nz
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    A = csr_to_dense(rowptr, col, val, n)
    xs = spmv_inputs.uniform_vector(n, seed=9)
    b = A @ xs
    errs = []
    for k in range(1, 30):
        x, it, _ = oracle.cg(rowptr, col, val, b, tol=0.0, maxit=k)
        e = x - xs
        errs.append(e @ A @ e)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))


def test_cg_krylov_termination_2x2x2():
    # eigenvalues of the 2x2x2 matrix are {19, 27}: exact CG stops in 2 steps
    rowptr, col, val = oracle.hpcg_csr(2, 2, 2)
    b = spmv_inputs.uniform_vector(8, seed=2)
    x, it, hist = oracle.cg(rowptr, col, val, b, tol=1e-14, maxit=20)
    assert it <= 3
    A = csr_to_dense(rowptr, col, val, 8)
    assert np.allclose(A @ x, b, rtol=0, atol=1e-13)


def test_cg_krylov_termination_4x4x4():
    """On 4^3 the closed-form spectrum 27 - prod_d (1 + 2 cos(k_d pi / 5))
    has 19 distinct values, so exact CG ends within 19 steps for any b; the
    oracle's CG reaches 1e-13 within that count."""
    import math
    f = [1 + 2 * math.cos(k * math.pi / 5) for k in range(1, 5)]
    distinct = len({round(27 - a * b * c, 9) for a in f for b in f for c in f})
    assert distinct == 19
    rowptr, col, val = oracle.hpcg_csr(4, 4, 4)
    A = csr_to_dense(rowptr, col, val, 64)
    assert len(np.unique(np.round(np.linalg.eigvalsh(A), 9))) == distinct
    b = spmv_inputs.uniform_vector(64, seed=3)
    x, it, hist = oracle.cg(rowptr, col, val, b, tol=1e-13, maxit=200)
    assert hist[-1] <= 1e-13 and it <= distinct
    assert np.allclose(A @ x, b, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# Irregular variant: construction invariants
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def irregular_small():
    nx = ny = nz = 20
    return (nx, ny, nz) + oracle.irregular_csr(nx, ny, nz, seed=2)


def test_irregular_symmetric_and_signs(irregular_small):
    nx, ny, nz, rowptr, col, val, perm = irregular_small
    n = nx * ny * nz
    A = csr_to_dense(rowptr, col, val, n)
    assert np.array_equal(A, A.T)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    off = val[col != rows]
    # special links are U[-2,-0.1), ordinary ones the levels -1.5 .. -0.5
    assert np.all(off < -0.1) and np.all(off >= -2.0)
    levels = -1.5 + np.arange(16) / 15.0
    on_level = np.isin(off, levels)
    assert 0 < np.sum(~on_level) < off.size
    assert np.max(off[~on_level]) < -0.1 and np.min(off[~on_level]) >= -2.0
    assert np.all(np.diff(col)[np.diff(rows) == 0] > 0)


def test_irregular_unpermuted_structure(irregular_small):
    nx, ny, nz, rowptr, col, val, perm = irregular_small
    n = nx * ny * nz
    # undo the renumbering and compare with the stencil: every stored link is
    # a stencil link, about 10 percent of stencil links are missing
    A = csr_to_dense(rowptr, col, val, n)[np.ix_(perm, perm)]
    rp0, c0, v0 = oracle.hpcg_csr(nx, ny, nz)
    stencil = csr_to_dense(rp0, c0, v0, n) != 0
    assert np.all((A != 0) <= stencil)
    nlinks = (np.sum(stencil) - n) // 2
    kept = (np.sum(A != 0) - n) // 2
    drop = 1 - kept / nlinks
    sd = np.sqrt(0.1 * 0.9 / nlinks)
    assert abs(drop - 0.10) < 5 * sd
    diag = np.diag(A)
    offsum = np.sum(np.abs(A), axis=1) - np.abs(diag)
    special = np.abs(diag - 1.05 * offsum) <= 1e-12 * diag
    normal = diag == 26.0
    assert np.all(special | normal)
    assert np.sum(special & ~normal) == int(np.floor(0.05 * n))
    levels = -1.5 + np.arange(16) / 15.0
    for i in np.nonzero(normal & ~special)[0][:200]:
        for j in np.nonzero(A[i])[0]:
            if j != i and diag[j] == 26.0 and not special[j]:
                assert np.any(A[i, j] == levels)


def test_irregular_m_matrix_certificate(irregular_small):
    """A symmetric Z-matrix with some v > 0 and A v > 0 is positive definite."""
    nx, ny, nz, rowptr, col, val, perm = irregular_small
    n = nx * ny * nz
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    diag = val[col == rows]
    v = np.ones(n)
    for _ in range(60):
        v = (diag * v - oracle.spmv(rowptr, col, val, v) + diag) / diag
    Av = oracle.spmv(rowptr, col, val, v)
    assert np.all(v > 0) and np.min(Av) > 1e-6 * np.max(np.abs(Av))


def test_irregular_deterministic():
    a = oracle.irregular_csr(6, 5, 4, seed=7)
    b = oracle.irregular_csr(6, 5, 4, seed=7)
    c = oracle.irregular_csr(6, 5, 4, seed=8)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    assert not np.array_equal(a[2], c[2])


# --------------------------------------------------------------------------
# Planted mistakes: each plausible slip in the oracle fails some pin
# --------------------------------------------------------------------------
def test_planted_mistakes_are_caught():
    nx, ny, nz = 5, 4, 6
    n = nx * ny * nz
    rowptr, col, val = oracle.hpcg_csr(nx, ny, nz)
    ref = dense_from_definition(nx, ny, nz)
    x = spmv_inputs.integer_vector(n, seed=1)

    def caught(rp, c, v):
        A = csr_to_dense(rp, c, v, n)
        y = oracle.spmv(rp, c, v, np.ones(n))
        return (not np.array_equal(A, ref)) or (not np.array_equal(y, 27.0 - np.diff(rowptr))) \
            or (not np.array_equal(oracle.spmv(rp, c, v, x), oracle.kron_apply(nx, ny, nz, x)))

    # wrong diagonal value
    v = val.copy(); v[col == np.repeat(np.arange(n), np.diff(rowptr))] = 27.0
    assert caught(rowptr, col, v)
    # wrong sign on one neighbour
    v = val.copy(); v[1] = 1.0
    assert caught(rowptr, col, v)
    # shifted column index (wrong neighbour)
    c = col.copy(); c[5] = (c[5] + 1) % n
    assert caught(rowptr, c, val)
    # a dropped entry
    rp = rowptr.copy(); rp[1:] -= 1; rp[0] = 0
    c = np.delete(col, 0); v = np.delete(val, 0)
    assert caught(rp, c, v)
    # SpMV reading x at the row instead of the column: y = (A 1) * x
    y_bad = oracle.spmv(rowptr, col, val, np.ones(n)) * x
    assert not np.array_equal(y_bad, oracle.kron_apply(nx, ny, nz, x))


# --------------------------------------------------------------------------
# The shared input generator against its published definition
# --------------------------------------------------------------------------
def test_splitmix64_known_answers():
    # first outputs of SplitMix64 seeded with 1234567, as published with the
    # generator's reference code
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(v) for v in spmv_inputs.splitmix64_block(1234567, 5)] == want
    s = 1234567
    for w in want:
        s, out = spmv_inputs.splitmix64_next(s)
        assert out == w


def test_inputs_ranges():
    x = spmv_inputs.uniform_vector(100000, seed=1)
    assert x.min() >= -1.0 and x.max() < 1.0 and abs(x.mean()) < 0.02
    e = spmv_inputs.grid_edges(24, seed=4)
    assert len(e) == 24 and min(e) >= 16 and max(e) <= 96
    xi = spmv_inputs.integer_vector(1000, seed=1)
    assert set(np.unique(xi)) <= set(range(-3, 4))
