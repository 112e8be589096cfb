/*
 * oracle.c -- plain, slow, obviously correct CPU restatement of what the
 * compressed-SpMV path computes (Yoshifuji et al., arXiv:1612.00530).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load, link or
 * call this file: only the tests, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py use it.  It shares no code, header, table or
 * constant generator with the CUDA library; the two meet only through the
 * seeded input vectors of the spmv_inputs module.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no -ffast-math);
 * every multiply-add is an explicit fma(), evaluated in IEEE binary64 with
 * round-to-nearest-even, so the results do not depend on the compiler.
 *
 * Contents and the passage each restates:
 *   hpcg row / CSR        Sec. III-A (27-point stencil on an nx*ny*nz grid)
 *                         and Fig. 2 (diagonal 26, neighbours -1)
 *   irregular CSR         the irregularised variant of the HPCG matrix; its
 *                         random choices follow the readings listed in the
 *                         design notes (SplitMix64 streams, link drops,
 *                         special rows, 16-level values, renumbering)
 *   spmv (f64, f32)       Eq. (1), y = A x, each row summed in ascending
 *                         column order as y = fma(a_ij, x_j, y) from 0
 *   value table           Sec. V: all distinct values, sorted ascending
 *   data table row        Sec. V and Fig. 2: columns sorted by value (S_i)
 *                         and the terminal index of each value (T_i)
 *   data+index table      Sec. V: displacements relative to the diagonal,
 *                         registered as patterns; decoded as in Listing 1
 *   kron apply            closed form A = 27 I - T (x) T (x) T of the HPCG
 *                         matrix (T = tridiag(1,1,1)), a second oracle of
 *                         different structure
 *   cg                    textbook unpreconditioned CG (Hestenes-Stiefel),
 *                         the Krylov solver of Sec. III-A without the
 *                         preconditioner (Table I's Dot/Waxpby/SpMV steps)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), written from its    */
/* published definition.                                                */
/* ------------------------------------------------------------------ */
static uint64_t sm64(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ull;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Stream for one purpose: first output of a SplitMix64 started at
 * seed XOR (purpose name as little-endian ASCII). */
static uint64_t purpose_stream(uint64_t seed, const char *name)
{
    uint64_t tag = 0, s;
    for (int i = 0; name[i] != 0 && i < 8; ++i)
        tag |= (uint64_t)(unsigned char)name[i] << (8 * i);
    s = seed ^ tag;
    return sm64(&s);
}

static double unit_draw(uint64_t *state)
{
    return (double)(sm64(state) >> 11) * 0x1.0p-53;
}

/* integer in [0, m): floor(u * m), kept below m */
static int64_t index_draw(uint64_t *state, int64_t m)
{
    int64_t k = (int64_t)floor(unit_draw(state) * (double)m);
    return k < m ? k : m - 1;
}

/* ------------------------------------------------------------------ */
/* HPCG matrix, Sec. III-A: node i = ix + nx*(iy + ny*iz); row i has one */
/* entry per neighbour (dx,dy,dz) in {-1,0,1}^3 inside the grid; the     */
/* diagonal is 26 and every other entry -1 (Fig. 2 values).  Looping dz, */
/* dy, dx upward visits the columns in ascending order.                   */
/* ------------------------------------------------------------------ */
int orc_hpcg_row(int nx, int ny, int nz, int64_t i, int32_t *col, double *val)
{
    int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / ((int64_t)nx * ny);
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int64_t jx = ix + dx, jy = iy + dy, jz = iz + dz;
                if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz)
                    continue;
                col[cnt] = (int32_t)(jx + (int64_t)nx * (jy + (int64_t)ny * jz));
                val[cnt] = (dx == 0 && dy == 0 && dz == 0) ? 26.0 : -1.0;
                ++cnt;
            }
    return cnt;
}

/* CSR of rows [row0, row1); rowptr has row1-row0+1 entries starting at 0;
 * col/val need room for 27 entries per row.  Returns the nonzero count. */
int64_t orc_hpcg_csr(int nx, int ny, int nz, int64_t row0, int64_t row1,
                     int64_t *rowptr, int32_t *col, double *val)
{
    int64_t k = 0;
    rowptr[0] = 0;
    for (int64_t i = row0; i < row1; ++i) {
        k += orc_hpcg_row(nx, ny, nz, i, col + k, val + k);
        rowptr[i - row0 + 1] = k;
    }
    return k;
}

/* y_i for selected rows straight from the row definition (no stored matrix):
 * the check used on sampled rows of grids too large to hold as CSR. */
void orc_hpcg_spmv_rows(int nx, int ny, int nz, int64_t count, const int64_t *rows,
                        const double *x, double *y)
{
    int32_t col[27];
    double val[27];
    for (int64_t t = 0; t < count; ++t) {
        int len = orc_hpcg_row(nx, ny, nz, rows[t], col, val);
        double s = 0.0;
        for (int k = 0; k < len; ++k)
            s = fma(val[k], x[col[k]], s);
        y[t] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Irregularised HPCG matrix.  Steps, in this order:                    */
/*  1. special rows: floor(special_frac*N) nodes chosen by a partial    */
/*     Fisher-Yates shuffle of 0..N-1 ("special" stream);                */
/*  2. links: every stencil pair i<j, enumerated by i ascending then j   */
/*     ascending, is dropped when a "drop" draw is < drop_p; a kept link */
/*     takes U[-2,-0.1) if either end is special, else the level         */
/*     -1.5 + k/15 with k = floor(16 u) ("val" stream), the same value   */
/*     for (i,j) and (j,i);                                             */
/*  3. diagonal: special rows 1.05 * sum|a_ij| (off-diagonals summed in  */
/*     ascending column order); other rows 26, or max(26, that) when     */
/*     diag_rule = 1;                                                    */
/*  4. renumbering: a full Fisher-Yates shuffle p ("perm" stream, t from */
/*     N-1 down to 1, partner floor(u*(t+1))); old node k becomes p[k].  */
/* Output: CSR of P A P^T with columns ascending; perm_out[k] = p[k].    */
/* ------------------------------------------------------------------ */
typedef struct { int32_t c; double v; } orc_entry;

static int cmp_entry(const void *a, const void *b)
{
    int32_t x = ((const orc_entry *)a)->c, y = ((const orc_entry *)b)->c;
    return (x > y) - (x < y);
}

int64_t orc_irregular_csr(int nx, int ny, int nz, uint64_t seed, double drop_p,
                          double special_frac, int diag_rule, int permute,
                          int64_t *rowptr, int32_t *col, double *val, int32_t *perm_out)
{
    int64_t n = (int64_t)nx * ny * nz;
    int64_t nspecial = (int64_t)floor(special_frac * (double)n);
    uint64_t st_special = purpose_stream(seed, "special");
    uint64_t st_drop = purpose_stream(seed, "drop");
    uint64_t st_val = purpose_stream(seed, "val");
    uint64_t st_perm = purpose_stream(seed, "perm");
    int32_t *order = malloc(sizeof(int32_t) * n);
    char *special = calloc(n, 1);
    int *deg = calloc(n, sizeof(int));
    orc_entry *adj = malloc(sizeof(orc_entry) * 27 * n);
    int32_t *p = malloc(sizeof(int32_t) * n);
    if (!order || !special || !deg || !adj || !p)
        return -1;

    for (int64_t k = 0; k < n; ++k)
        order[k] = (int32_t)k;
    for (int64_t t = 0; t < nspecial; ++t) {
        int64_t j = t + index_draw(&st_special, n - t);
        int32_t tmp = order[t];
        order[t] = order[j];
        order[j] = tmp;
        special[order[t]] = 1;
    }

    for (int64_t i = 0; i < n; ++i) {
        int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / ((int64_t)nx * ny);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t jx = ix + dx, jy = iy + dy, jz = iz + dz, j;
                    double v;
                    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz)
                        continue;
                    j = jx + (int64_t)nx * (jy + (int64_t)ny * jz);
                    if (j <= i)
                        continue;
                    if (unit_draw(&st_drop) < drop_p)
                        continue;
                    if (special[i] || special[j]) {
                        double lo = -2.0, hi = -0.1;
                        v = lo + (hi - lo) * unit_draw(&st_val);
                    } else {
                        int64_t lvl = index_draw(&st_val, 16);
                        v = -1.5 + (double)lvl / 15.0;
                    }
                    adj[27 * i + deg[i]].c = (int32_t)j;
                    adj[27 * i + deg[i]].v = v;
                    deg[i]++;
                    adj[27 * j + deg[j]].c = (int32_t)i;
                    adj[27 * j + deg[j]].v = v;
                    deg[j]++;
                }
    }

    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0, d;
        qsort(adj + 27 * i, deg[i], sizeof(orc_entry), cmp_entry);
        for (int k = 0; k < deg[i]; ++k)
            s = s + fabs(adj[27 * i + k].v);
        if (special[i])
            d = 1.05 * s;
        else if (diag_rule == 1)
            d = fmax(26.0, 1.05 * s);
        else
            d = 26.0;
        adj[27 * i + deg[i]].c = (int32_t)i;
        adj[27 * i + deg[i]].v = d;
        deg[i]++;
    }

    for (int64_t k = 0; k < n; ++k)
        p[k] = (int32_t)k;
    if (permute) {
        for (int64_t t = n - 1; t >= 1; --t) {
            int64_t j = index_draw(&st_perm, t + 1);
            int32_t tmp = p[t];
            p[t] = p[j];
            p[j] = tmp;
        }
    }

    /* row p[k] of the output is row k of A with columns renamed by p */
    {
        int64_t *len_new = calloc(n, sizeof(int64_t));
        if (!len_new)
            return -1;
        for (int64_t k = 0; k < n; ++k)
            len_new[p[k]] = deg[k];
        rowptr[0] = 0;
        for (int64_t r = 0; r < n; ++r)
            rowptr[r + 1] = rowptr[r] + len_new[r];
        for (int64_t k = 0; k < n; ++k) {
            orc_entry row[27];
            int64_t base = rowptr[p[k]];
            for (int e = 0; e < deg[k]; ++e) {
                row[e].c = p[adj[27 * k + e].c];
                row[e].v = adj[27 * k + e].v;
            }
            qsort(row, deg[k], sizeof(orc_entry), cmp_entry);
            for (int e = 0; e < deg[k]; ++e) {
                col[base + e] = row[e].c;
                val[base + e] = row[e].v;
            }
        }
        free(len_new);
    }
    if (perm_out)
        memcpy(perm_out, p, sizeof(int32_t) * n);
    {
        int64_t nnz = rowptr[n];
        free(order); free(special); free(deg); free(adj); free(p);
        return nnz;
    }
}

/* ------------------------------------------------------------------ */
/* Eq. (1): y = A x.  Row i: y_i = 0, then y_i = fma(a_ij, x_j, y_i) over */
/* the row's entries in their stored (ascending-column) order.            */
/* ------------------------------------------------------------------ */
void orc_spmv_csr(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                  const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            s = fma(val[k], x[col[k]], s);
        y[i] = s;
    }
}

/* Eq. (1) for a row range [row0,row1) of a CSR whose rowptr starts at row0. */
void orc_spmv_csr_range(int64_t row0, int64_t row1, const int64_t *rowptr, const int32_t *col,
                        const double *val, const double *x, double *y)
{
    for (int64_t i = row0; i < row1; ++i) {
        double s = 0.0;
        for (int64_t k = rowptr[i - row0]; k < rowptr[i - row0 + 1]; ++k)
            s = fma(val[k], x[col[k]], s);
        y[i - row0] = s;
    }
}

/* Eq. (1) in binary32: values rounded to float, y_i = fmaf chain from 0. */
void orc_spmv_csr_f32(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                      const float *x, float *y)
{
    for (int64_t i = 0; i < n; ++i) {
        float s = 0.0f;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            s = fmaf((float)val[k], x[col[k]], s);
        y[i] = s;
    }
}

/* Eq. (1) with k right-hand sides, X and Y row-major n x k. */
void orc_spmm_csr(int64_t n, int k, const int64_t *rowptr, const int32_t *col, const double *val,
                  const double *X, double *Y)
{
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < k; ++c) {
            double s = 0.0;
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
                s = fma(val[e], X[(int64_t)col[e] * k + c], s);
            Y[i * k + c] = s;
        }
}

/* ------------------------------------------------------------------ */
/* Sec. V: the value table V lists every distinct matrix value once, in */
/* ascending order (v_i < v_{i+1}).  Returns |V|; V needs nnz slots.     */
/* ------------------------------------------------------------------ */
static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int64_t orc_value_table(int64_t nnz, const double *val, double *V)
{
    int64_t m = 0;
    if (nnz == 0)
        return 0;
    memcpy(V, val, sizeof(double) * nnz);
    qsort(V, nnz, sizeof(double), cmp_double);
    for (int64_t k = 0; k < nnz; ++k)
        if (m == 0 || V[k] != V[m - 1])
            V[m++] = V[k];
    return m;
}

/* Sec. V / Fig. 2: the row's entries sorted by value, ties kept in their
 * ascending column order (a stable sort); S lists the columns in that
 * order; T_incl[v] is the last position (0-based) holding a value <= V[v]
 * (-1 if none) and T_end[v] = T_incl[v] + 1 the exclusive end used by the
 * decode loop of Listing 1. */
void orc_data_table_row(int len, const int32_t *col, const double *val, int nV, const double *V,
                        int32_t *S, int32_t *T_incl, int32_t *T_end)
{
    int pos = 0;
    for (int v = 0; v < nV; ++v) {
        for (int k = 0; k < len; ++k)
            if (val[k] == V[v])
                S[pos++] = col[k];
        T_end[v] = pos;
        T_incl[v] = pos - 1;
    }
}

/* Sec. V, first scheme ("Data Table" of Table II): each row kept as its
 * value-sorted column list S_i and terminal indices T_i over the value
 * table V.  y_i walks the value groups in ascending order and, inside a
 * group, S_i in order; each entry adds V[v] * x[S_i[idx]] with one fma. */
void orc_data_table_spmv(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                         int nV, const double *V, const double *x, double *y)
{
    int maxlen = 1;
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] - rowptr[i] > maxlen)
            maxlen = (int)(rowptr[i + 1] - rowptr[i]);
    int32_t *S = malloc(sizeof(int32_t) * maxlen);
    int32_t *Ti = malloc(sizeof(int32_t) * (nV > 0 ? nV : 1));
    int32_t *Te = malloc(sizeof(int32_t) * (nV > 0 ? nV : 1));
    if (!S || !Ti || !Te) {
        free(S); free(Ti); free(Te);
        return;
    }
    for (int64_t i = 0; i < n; ++i) {
        int len = (int)(rowptr[i + 1] - rowptr[i]);
        orc_data_table_row(len, col + rowptr[i], val + rowptr[i], nV, V, S, Ti, Te);
        double s = 0.0;
        int idx = 0;
        for (int v = 0; v < nV; ++v)
            for (; idx < Te[v]; ++idx)
                s = fma(V[v], x[S[idx]], s);
        y[i] = s;
    }
    free(S);
    free(Ti);
    free(Te);
}

/* Sec. V, second scheme: within each row the value-sorted column list S_i
 * is made relative to the diagonal (S_i - i) and the displacement list is
 * registered in a table of patterns; the row keeps only its pattern number
 * (columnDiffType) and its value ends (valueIdxEnd).  maxlen bounds a
 * pattern's length; diffs holds maxtypes*maxlen entries.  Returns the
 * number of patterns, or -1 when maxtypes is exceeded. */
int64_t orc_data_index_table(int64_t n, const int64_t *rowptr, const int32_t *col,
                             const double *val, int nV, const double *V, int maxlen,
                             int64_t maxtypes, int32_t *type, int32_t *diffs, int32_t *typelen,
                             int32_t *valueIdxEnd)
{
    int64_t ntypes = 0;
    int32_t *S = malloc(sizeof(int32_t) * maxlen);
    int32_t *Ti = malloc(sizeof(int32_t) * nV);
    if (!S || !Ti)
        return -1;
    for (int64_t i = 0; i < n; ++i) {
        int len = (int)(rowptr[i + 1] - rowptr[i]);
        int64_t t;
        orc_data_table_row(len, col + rowptr[i], val + rowptr[i], nV, V, S, Ti,
                           valueIdxEnd + i * nV);
        for (int k = 0; k < len; ++k)
            S[k] = (int32_t)(S[k] - i);
        for (t = 0; t < ntypes; ++t)
            if (typelen[t] == len && memcmp(diffs + t * maxlen, S, sizeof(int32_t) * len) == 0)
                break;
        if (t == ntypes) {
            if (ntypes == maxtypes) {
                free(S); free(Ti);
                return -1;
            }
            memcpy(diffs + t * maxlen, S, sizeof(int32_t) * len);
            typelen[t] = len;
            ++ntypes;
        }
        type[i] = (int32_t)t;
    }
    free(S);
    free(Ti);
    return ntypes;
}

/* Listing 1: for each row, walk the value groups in order; entries idx of
 * group v (idx below valueIdxEnd[i][v]) use column i + columnDiff[type][idx]
 * and the value V[v]; accumulate with fma. */
void orc_listing1_spmv(int64_t n, const int32_t *type, const int32_t *diffs, int maxlen,
                       const int32_t *valueIdxEnd, int nV, const double *V, const double *x,
                       double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        const int32_t *d = diffs + (int64_t)type[i] * maxlen;
        int idx = 0;
        double s = 0.0;
        for (int v = 0; v < nV; ++v) {
            double a = V[v];
            for (; idx < valueIdxEnd[i * nV + v]; ++idx)
                s = fma(a, x[i + d[idx]], s);
        }
        y[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Closed form of the HPCG matrix: A = 27 I - Tz (x) Ty (x) Tx with       */
/* T = tridiag(1,1,1), i.e. y = 27 x - w where w sums x over the 3x3x3    */
/* box around each node, formed as three one-dimensional 3-point sums.    */
/* work needs 2n doubles.                                                 */
/* ------------------------------------------------------------------ */
void orc_hpcg_kron_apply(int nx, int ny, int nz, const double *x, double *y, double *work)
{
    int64_t n = (int64_t)nx * ny * nz, sxy = (int64_t)nx * ny;
    double *a = work, *b = work + n;
    for (int64_t i = 0; i < n; ++i) {
        int64_t ix = i % nx;
        double s = x[i];
        if (ix > 0) s += x[i - 1];
        if (ix < nx - 1) s += x[i + 1];
        a[i] = s;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t iy = (i / nx) % ny;
        double s = a[i];
        if (iy > 0) s += a[i - nx];
        if (iy < ny - 1) s += a[i + nx];
        b[i] = s;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t iz = i / sxy;
        double s = b[i];
        if (iz > 0) s += b[i - sxy];
        if (iz < nz - 1) s += b[i + sxy];
        y[i] = 27.0 * x[i] - s;
    }
}

/* ------------------------------------------------------------------ */
/* Unpreconditioned CG (Hestenes-Stiefel) in binary64.  x holds x0 on    */
/* entry.  r = b - A x; p = r; per step: q = A p, alpha = r.r / p.q,       */
/* x += alpha p, r -= alpha q, beta = r'.r' / r.r, p = r + beta p.  Dots   */
/* are sequential fma sums in index order.  hist[k] = |r_k| / |b| for      */
/* k = 0..iterations.  Stops when hist[k] <= tol or after maxit steps;     */
/* returns the number of steps taken.                                      */
/* ------------------------------------------------------------------ */
static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        s = fma(a[i], b[i], s);
    return s;
}

int orc_cg(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
           const double *b, double *x, double tol, int maxit, double *hist)
{
    double *r = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n);
    double *q = malloc(sizeof(double) * n);
    double bnorm, rr;
    int k;
    if (!r || !p || !q)
        return -1;
    orc_spmv_csr(n, rowptr, col, val, x, q);
    for (int64_t i = 0; i < n; ++i) {
        r[i] = b[i] - q[i];
        p[i] = r[i];
    }
    bnorm = sqrt(dot(n, b, b));
    rr = dot(n, r, r);
    hist[0] = sqrt(rr) / bnorm;
    for (k = 1; k <= maxit && hist[k - 1] > tol; ++k) {
        double alpha, beta, rr_new;
        orc_spmv_csr(n, rowptr, col, val, p, q);
        alpha = rr / dot(n, p, q);
        for (int64_t i = 0; i < n; ++i) {
            x[i] = fma(alpha, p[i], x[i]);
            r[i] = fma(-alpha, q[i], r[i]);
        }
        rr_new = dot(n, r, r);
        hist[k] = sqrt(rr_new) / bnorm;
        beta = rr_new / rr;
        for (int64_t i = 0; i < n; ++i)
            p[i] = fma(beta, p[i], r[i]);
        rr = rr_new;
    }
    free(r);
    free(p);
    free(q);
    return k - 1;
}
