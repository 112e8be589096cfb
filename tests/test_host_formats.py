"""Host-side logic of the library, checked against the oracle on the CPU:
generators (bit-exact CSR), compression/decompression round trips, the
pattern census of Sec. V, byte accounting, export/import and corruption
detection."""
import numpy as np
import pytest

import oracle
import paper_1612_00530_gb300 as P
import spmv_inputs
from paper_1612_00530_gb300 import build as lib_build


@pytest.fixture(scope="module", autouse=True)
def built():
    lib_build.build()


GRIDS = [(1, 1, 1), (2, 3, 5), (3, 3, 3), (4, 4, 4), (17, 5, 3), (32, 32, 32)]


def same_csr(a, b):
    return all(np.array_equal(u, v) for u, v in zip(a, b))


@pytest.mark.parametrize("g", GRIDS)
def test_hpcg_generator_matches_oracle(g):
    A = P.spmv_build("hpcg", *g)
    assert same_csr(P.spmv_decompress(A), oracle.hpcg_csr(*g))


@pytest.mark.parametrize("g,seed", [((6, 5, 4), 2), ((12, 12, 12), 2), ((9, 7, 11), 13)])
def test_irregular_generator_matches_oracle(g, seed):
    A = P.spmv_build("irregular", *g, seed=seed)
    rp, c, v, _ = oracle.irregular_csr(*g, seed=seed)
    got = P.spmv_decompress(A)
    assert np.array_equal(got[0], rp) and np.array_equal(got[1], c)
    assert np.array_equal(got[2].view(np.uint64), v.view(np.uint64))


def test_irregular_diag_rule_and_no_permutation():
    g = (7, 6, 5)
    A = P.spmv_build("irregular", *g, seed=3, diag_rule=1, permute=False)
    rp, c, v, perm = oracle.irregular_csr(*g, seed=3, diag_rule=1, permute=False)
    assert np.array_equal(perm, np.arange(len(perm)))
    assert same_csr(P.spmv_decompress(A), (rp, c, v))


@pytest.mark.parametrize("g", GRIDS)
def test_pattern_round_trip_and_census(g):
    A = P.spmv_build("hpcg", *g)
    C = P.spmv_compress(A, format="pattern")
    info = P.spmv_info(C)
    assert info["format_name"] == "pattern"
    ntypes = int(np.prod([min(d, 3) for d in g]))
    assert info["n_patterns"] == ntypes
    assert info["dict_size"] == (1 if g == (1, 1, 1) else 2)
    assert info["fast_eligible"] == 1
    assert same_csr(P.spmv_decompress(C), oracle.hpcg_csr(*g))
    if min(g) >= 3:
        assert info["union_size"] == 27 and info["record_bytes"] == 28


def test_pattern_census_matches_oracle_registry():
    g = (6, 7, 5)
    rp, c, v = oracle.hpcg_csr(*g)
    V = oracle.value_table(v)
    typ, diffs, typelen, ends = oracle.data_index_table(rp, c, v, V)
    C = P.spmv_compress(P.spmv_build("hpcg", *g), format="pattern")
    assert P.spmv_info(C)["n_patterns"] == len(typelen)


@pytest.mark.parametrize("g", [(4, 4, 4), (33, 9, 2), (64, 64, 8)])
def test_delta_round_trip(g):
    A = P.spmv_build("hpcg", *g)
    C = P.spmv_compress(A, format="delta", min_count=1)
    info = P.spmv_info(C)
    assert info["format_name"] == "delta" and info["slices_value_raw"] == 0
    assert same_csr(P.spmv_decompress(C), oracle.hpcg_csr(*g))


def test_delta_irregular_fallback_fractions():
    g = (40, 40, 40)
    A = P.spmv_build("irregular", *g, seed=2)
    C = P.spmv_compress(A)  # AUTO: too many patterns, goes to delta
    info = P.spmv_info(C)
    assert info["format_name"] == "delta"
    rp, c, v, _ = oracle.irregular_csr(*g, seed=2)
    got = P.spmv_decompress(C)
    assert np.array_equal(got[0], rp) and np.array_equal(got[1], c)
    assert np.array_equal(got[2].view(np.uint64), v.view(np.uint64))
    # random renumbering spreads columns beyond int16: almost every slice
    # takes 24-bit deltas (n < 2^23, so none needs raw int32 columns)
    assert info["slices_col24"] >= 0.9 * info["n_slices"] and info["slices_col_raw"] == 0
    # 16 levels + 26.0 make the table; the unique values of the special rows'
    # links are escaped entry by entry, so few slices store raw values
    assert info["dict_size"] >= 17
    assert info["slices_value_raw"] <= 0.05 * info["n_slices"]
    assert info["format_bytes"] / info["nnz"] < 6.5


def test_delta_encodings_round_trip():
    """Every delta encoding bit-exact through decompress: int16, 24-bit and
    raw int32 columns (a column 2^23 away from its row), table codes, codes
    with a few escaped entries, raw values where most entries escape."""
    n = (1 << 23) + 64
    rng = np.random.default_rng(3)
    cols = [np.array([i]) for i in range(n)]
    # slice 0: row 0 reaches the last column (a delta above 2^23 - 1)
    cols[0] = np.array([0, n - 1])
    # slice 1: deltas of +-40000 (24-bit)
    for i in range(32, 64):
        cols[i] = np.array([i, i + 40000])
    # slice 2: int16 deltas
    for i in range(64, 96):
        cols[i] = np.unique(np.array([i - 3, i, i + 5]))
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(c) for c in cols])
    col = np.concatenate(cols).astype(np.int32)
    val = np.full(len(col), 2.0)
    val[col == np.arange(n).repeat(np.diff(rowptr))] = 26.0
    # slice 3: two entries outside the table (escaped)
    k3 = rowptr[96]
    val[k3] = 0.123456789
    val[k3 + 5] = -7.5e-300
    # slice 4: every entry a unique value (raw)
    k4a, k4b = rowptr[128], rowptr[160]
    val[k4a:k4b] = rng.uniform(-1, 1, k4b - k4a)
    A = P.spmv_build_csr(rowptr, col, val)
    C = P.spmv_compress(A, format="delta", min_count=64)
    info = P.spmv_info(C)
    assert info["format_name"] == "delta"
    assert info["slices_col_raw"] == 1 and info["slices_col24"] == 1
    assert info["slices_value_raw"] == 1
    got = P.spmv_decompress(C)
    assert np.array_equal(got[0], rowptr) and np.array_equal(got[1], col)
    assert np.array_equal(got[2].view(np.uint64), val.view(np.uint64))
    # and through a stream (every field checked on import)
    D = P.spmv_import(P.spmv_export(C))
    got = P.spmv_decompress(D)
    assert np.array_equal(got[2].view(np.uint64), val.view(np.uint64))


def test_round_trip_random_csr_with_signed_zeros():
    rng = np.random.default_rng(0)
    n = 300
    rows = []
    for i in range(n):
        cols = np.unique(np.concatenate([[i], rng.integers(0, n, size=rng.integers(0, 12))]))
        rows.append(cols)
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    val = rng.choice([-0.0, 0.0, 1.5, -2.25, np.inf, 3.0e-310], size=len(col))
    A = P.spmv_build_csr(rowptr, col, val)
    for fmt in ("delta",):
        C = P.spmv_compress(A, format=fmt, min_count=1)
        got = P.spmv_decompress(C)
        assert np.array_equal(got[0], rowptr) and np.array_equal(got[1], col)
        assert np.array_equal(got[2].view(np.uint64), val.view(np.uint64))
    with pytest.raises(P.SpmvError) as e:
        P.spmv_compress(A, format="pattern")
    assert e.value.status == P.SPMV_EUNSUPPORTED


def test_ell_padding_accounting():
    g = (5, 5, 5)
    A = P.spmv_build("hpcg", *g)
    info = P.spmv_info(A)
    nnz = (3 * 5 - 2) ** 3
    assert info["nnz"] == nnz
    slots = (info["format_bytes"] - info["n_slices"] * 12) // 12
    assert info["padding_bytes"] == (slots - nnz) * 12


def test_pattern_bytes_per_row_192():
    # 27 one-byte codes + the pattern byte: 28 bytes per row, 1.0 per nonzero
    # plus 1/27 for the pattern, against 12 for ELL (Sec. IV-B, Table II)
    A = P.spmv_build("hpcg", 20, 20, 20)
    C = P.spmv_compress(A, format="pattern")
    info = P.spmv_info(C)
    assert info["format_bytes"] == 28 * info["n"]


@pytest.mark.parametrize("fmt", ["ell", "pattern", "delta"])
def test_export_import_round_trip(fmt):
    A = P.spmv_build("hpcg", 7, 6, 5)
    C = A if fmt == "ell" else P.spmv_compress(A, format=fmt, min_count=1)
    blob = P.spmv_export(C)
    D = P.spmv_import(blob)
    assert P.spmv_info(D)["checksum"] == P.spmv_info(C)["checksum"]
    assert same_csr(P.spmv_decompress(D), oracle.hpcg_csr(7, 6, 5))
    if fmt == "pattern":
        assert P.spmv_info(D)["fast_eligible"] == 1


@pytest.mark.parametrize("fmt", ["pattern", "delta"])
def test_corrupted_stream_rejected(fmt):
    A = P.spmv_build("hpcg", 7, 6, 5)
    C = P.spmv_compress(A, format=fmt, min_count=1)
    blob = bytearray(P.spmv_export(C))
    rng = np.random.default_rng(1)
    for pos in list(rng.integers(8, len(blob), size=24)) + [len(blob) - 1, 40]:
        bad = bytearray(blob)
        bad[pos] ^= 0x5A
        with pytest.raises(P.SpmvError) as e:
            P.spmv_import(bytes(bad))
        assert e.value.status == P.SPMV_ECORRUPT
    with pytest.raises(P.SpmvError) as e:
        P.spmv_import(bytes(blob[:-3]))
    assert e.value.status == P.SPMV_ECORRUPT


def test_empty_matrix():
    A = P.spmv_build_csr(np.array([0]), np.array([], np.int32), np.array([]))
    assert P.spmv_info(A)["n"] == 0
    C = P.spmv_compress(A, format="delta")
    assert P.spmv_decompress(C)[0].tolist() == [0]


@pytest.mark.parametrize("g", [(1, 1, 1), (2, 3, 5), (4, 4, 4), (17, 5, 3), (32, 32, 32)])
def test_data_index_table_round_trip_and_type_census(g):
    """Sec. V's Data+Index Table: bit-exact round trip, one type per distinct
    value-grouped displacement list (the oracle's registry), 1 + |V| bytes a row."""
    rowptr, col, val = oracle.hpcg_csr(*g)
    D = P.spmv_compress(P.spmv_build("hpcg", *g), format="dit")
    assert same_csr(P.spmv_decompress(D), (rowptr, col, val))
    V = oracle.value_table(val)
    typ, diffs, typelen, ends = oracle.data_index_table(rowptr, col, val, V)
    info = P.spmv_info(D)
    assert info["format_name"] == "dit"
    assert info["n_patterns"] == len(typelen)
    assert info["dict_size"] == len(V)
    assert info["record_bytes"] == 1 + len(V)
    assert info["union_size"] == typelen.max()


def test_data_index_table_signed_zeros_and_refusals():
    rng = np.random.default_rng(1)
    n = 400
    rows = [np.unique(np.concatenate([[i], rng.integers(0, n, size=rng.integers(0, 9))])) for i in range(n)]
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    val = rng.choice([-0.0, 0.0, 1.5, -2.25, np.inf, 3.0e-310], size=len(col))
    A = P.spmv_build_csr(rowptr, col, val)
    # random columns: more than 256 value-grouped displacement lists
    with pytest.raises(P.SpmvError) as e:
        P.spmv_compress(A, format="dit")
    assert e.value.status == P.SPMV_EUNSUPPORTED
    # a banded matrix with the same values: few types, exact round trip
    band = [np.arange(max(0, i - 2), min(n, i + 3)) for i in range(n)]
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in band])
    col = np.concatenate(band).astype(np.int32)
    val = np.where((col % 3) == 0, -0.0, np.where((col % 3) == 1, 0.0, 1.5))
    D = P.spmv_compress(P.spmv_build_csr(rowptr, col, val), format="dit")
    got = P.spmv_decompress(D)
    assert np.array_equal(got[0], rowptr) and np.array_equal(got[1], col)
    assert np.array_equal(got[2].view(np.uint64), val.view(np.uint64))
    # no stream form, no FAST order
    with pytest.raises(P.SpmvError):
        P.spmv_export(D)
    with pytest.raises(P.SpmvError):
        P.spmv_set_order(D, "fast")


def data_table_bytes(rowptr, nv):
    """S: 4 B for each slot of a 32-row slice, the slice as wide as its
    longest row; ends: 1 B for each value and row."""
    lens = np.diff(rowptr)
    n = len(lens)
    width = sum(int(lens[s:s + 32].max()) for s in range(0, n, 32)) if n else 0
    return 4 * 32 * width + nv * n, 4 * (32 * width - int(lens.sum()))


@pytest.mark.parametrize("g", [(1, 1, 1), (2, 3, 5), (17, 5, 3), (32, 32, 32)])
def test_data_table_round_trip_and_sizes(g):
    """Sec. V's Data Table (Fig. 2): bit-exact round trip, the value table of
    the oracle, S_i at 4 B an entry in 32-row slices, 1 B a value a row."""
    rowptr, col, val = oracle.hpcg_csr(*g)
    D = P.spmv_compress(P.spmv_build("hpcg", *g), format="data_table")
    assert same_csr(P.spmv_decompress(D), (rowptr, col, val))
    info = P.spmv_info(D)
    V = oracle.value_table(val)
    assert info["format_name"] == "data_table"
    assert info["dict_size"] == len(V)
    fb, pad = data_table_bytes(rowptr, len(V))
    assert info["format_bytes"] == fb and info["padding_bytes"] == pad


def test_data_table_irregular_signed_zeros_and_refusals():
    # seventeen values (16 levels and the diagonal 26), permuted numbering
    g = (9, 7, 11)
    rowptr, col, val, _ = oracle.irregular_csr(*g, seed=13, special_frac=0.0)
    A = P.spmv_build("irregular", *g, seed=13, special_frac=0.0)
    D = P.spmv_compress(A, format="data_table")
    assert same_csr(P.spmv_decompress(D), (rowptr, col, val))
    assert P.spmv_info(D)["dict_size"] == len(oracle.value_table(val)) == 17
    # with reordering the stored matrix is P A P^T; decompress gives A back
    R = P.spmv_compress(A, format="data_table", reorder=True)
    assert same_csr(P.spmv_decompress(R), (rowptr, col, val))
    # -0.0 and +0.0 are two values
    n = 300
    band = [np.arange(max(0, i - 2), min(n, i + 3)) for i in range(n)]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in band])
    c = np.concatenate(band).astype(np.int32)
    v = np.where((c % 3) == 0, -0.0, np.where((c % 3) == 1, 0.0, 1.5))
    got = P.spmv_decompress(P.spmv_compress(P.spmv_build_csr(rp, c, v), format="data_table"))
    assert np.array_equal(got[0], rp) and np.array_equal(got[1], c)
    assert np.array_equal(got[2].view(np.uint64), v.view(np.uint64))
    # unique-valued rows: more than 255 distinct values
    with pytest.raises(P.SpmvError) as e:
        P.spmv_compress(P.spmv_build("irregular", 12, 12, 12, seed=2), format="data_table")
    assert e.value.status == P.SPMV_EUNSUPPORTED
    # no stream form, no FAST order
    with pytest.raises(P.SpmvError):
        P.spmv_export(D)
    with pytest.raises(P.SpmvError):
        P.spmv_set_order(D, "fast")


@pytest.mark.parametrize("g,seed", [((8, 8, 8), 2), ((16, 16, 16), 5)])
def test_reorder_round_trip_and_locality(g, seed):
    """Locality reordering inside spmv_compress: a permutation, the exact
    original matrix back from decompress, a narrower band, no more raw-value
    or wide-column slices and fewer bytes than the random numbering gives."""
    A = P.spmv_build("irregular", *g, seed=seed)
    C0 = P.spmv_compress(A, format="delta")
    C = P.spmv_compress(A, format="delta", reorder=True)
    n = P.spmv_info(C)["n"]
    perm = P.spmv_permutation(C)
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert same_csr(P.spmv_decompress(C), P.spmv_decompress(A))
    i0, i1 = P.spmv_info(C0), P.spmv_info(C)
    assert i1["reordered"] == 1 and i0["reordered"] == 0
    assert i1["bandwidth"] < i0["bandwidth"] / 2
    assert i1["slices_value_raw"] <= i0["slices_value_raw"]
    assert i1["slices_col24"] + i1["slices_col_raw"] <= i0["slices_col24"] + i0["slices_col_raw"]
    assert i1["format_bytes"] < i0["format_bytes"]
    # the stored matrix is P A P^T: its band is what info reports
    rowptr, col, val = P.spmv_decompress(A)
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    assert np.abs(inv[col] - inv[rows]).max() == i1["bandwidth"]
    with pytest.raises(P.SpmvError):
        P.spmv_export(C)
    with pytest.raises(P.SpmvError):
        P.spmv_permutation(C0)
