// Host-side matrix generators (Sec. III-A of arXiv:1612.00530) and CSR
// validation.  The HPCG matrix: 27-point stencil on an nx*ny*nz grid, node
// i = ix + nx*(iy + ny*iz), value 26 on the diagonal and -1 for each
// neighbour inside the grid (Fig. 2).  The irregular variant removes links,
// gives a fraction of rows unique values and renumbers the nodes.
#include <algorithm>
#include <cmath>
#include <thread>

#include "spmvc_internal.h"

namespace spmvc {

namespace {

// Neighbour (dx,dy,dz) of node (ix,iy,iz), or -1 when outside the grid.
struct Grid {
    int64_t nx, ny, nz;
    int64_t n() const { return nx * ny * nz; }
    int64_t neighbour(int64_t i, int d) const {  // d in 0..26, (dz,dy,dx) lexicographic
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const int64_t ix = i % nx + dx, iy = (i / nx) % ny + dy, iz = i / (nx * ny) + dz;
        if (ix < 0 || ix >= nx || iy < 0 || iy >= ny || iz < 0 || iz >= nz) return -1;
        return ix + nx * (iy + ny * iz);
    }
};

template <class F>
void parallel_rows(int64_t n, F&& f) {
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (n < 65536) nt = 1;
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) {
        const int64_t a = n * t / nt, b = n * (t + 1) / nt;
        th.emplace_back([&f, a, b] { f(a, b); });
    }
    for (auto& x : th) x.join();
}

// SplitMix64 (Steele, Lea and Flood 2014).
struct SplitMix64 {
    uint64_t s;
    uint64_t next() {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double unit() { return static_cast<double>(next() >> 11) * 0x1.0p-53; }
    int64_t below(int64_t m) {  // floor(u*m), kept below m
        const int64_t k = static_cast<int64_t>(std::floor(unit() * static_cast<double>(m)));
        return std::min(k, m - 1);
    }
};

// The independent stream for one purpose: first output of a SplitMix64
// started at seed ^ (the purpose name's bytes, little-endian).
SplitMix64 stream_for(uint64_t seed, const char* purpose) {
    uint64_t tag = 0;
    for (int i = 0; purpose[i] && i < 8; ++i) tag |= uint64_t(uint8_t(purpose[i])) << (8 * i);
    SplitMix64 g{seed ^ tag};
    return SplitMix64{g.next()};
}

}  // namespace

int generate_hpcg(int nx, int ny, int nz, Csr* out) {
    if (nx < 1 || ny < 1 || nz < 1) return fail(SPMV_EINVAL, "grid edges must be >= 1");
    const Grid g{nx, ny, nz};
    const int64_t n = g.n();
    if (n >= (int64_t(1) << 31)) return fail(SPMV_EINVAL, "grid too large for int32 columns");
    out->n = n;
    out->rowptr.assign(n + 1, 0);
    // row lengths first: product of per-dimension neighbour counts
    auto span = [](int64_t c, int64_t m) { return int64_t(1) + (c > 0) + (c < m - 1); };
    for (int64_t i = 0; i < n; ++i) {
        const int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / (int64_t(nx) * ny);
        out->rowptr[i + 1] = span(ix, nx) * span(iy, ny) * span(iz, nz);
    }
    for (int64_t i = 0; i < n; ++i) out->rowptr[i + 1] += out->rowptr[i];
    out->col.resize(out->rowptr[n]);
    out->val.resize(out->rowptr[n]);
    parallel_rows(n, [&](int64_t a, int64_t b) {
        for (int64_t i = a; i < b; ++i) {
            int64_t k = out->rowptr[i];
            for (int d = 0; d < 27; ++d) {
                const int64_t j = g.neighbour(i, d);
                if (j < 0) continue;
                out->col[k] = static_cast<int32_t>(j);
                out->val[k] = (j == i) ? 26.0 : -1.0;
                ++k;
            }
        }
    });
    return SPMV_OK;
}

int generate_irregular(const spmv_gen_desc& d, Csr* out) {
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return fail(SPMV_EINVAL, "grid edges must be >= 1");
    if (!(d.drop_prob >= 0.0 && d.drop_prob <= 1.0) || !(d.special_frac >= 0.0 && d.special_frac <= 1.0))
        return fail(SPMV_EINVAL, "drop_prob and special_frac must lie in [0, 1]");
    const Grid g{d.nx, d.ny, d.nz};
    const int64_t n = g.n();
    if (n >= (int64_t(1) << 31)) return fail(SPMV_EINVAL, "grid too large for int32 columns");

    // 1. special rows: partial Fisher-Yates over 0..n-1
    SplitMix64 rs = stream_for(d.seed, "special");
    const int64_t nspecial = static_cast<int64_t>(std::floor(d.special_frac * static_cast<double>(n)));
    std::vector<int32_t> idx(n);
    for (int64_t k = 0; k < n; ++k) idx[k] = static_cast<int32_t>(k);
    std::vector<uint8_t> special(n, 0);
    for (int64_t t = 0; t < nspecial; ++t) {
        std::swap(idx[t], idx[t + rs.below(n - t)]);
        special[idx[t]] = 1;
    }

    // 2. links i < j in (i, then j) ascending order; drop or give a value
    SplitMix64 rd = stream_for(d.seed, "drop");
    SplitMix64 rv = stream_for(d.seed, "val");
    std::vector<int32_t> deg(n, 0);
    std::vector<int32_t> adj_col(27 * n);
    std::vector<double> adj_val(27 * n);
    const double ulo = -2.0, uhi = -0.1;
    for (int64_t i = 0; i < n; ++i) {
        for (int dd = 0; dd < 27; ++dd) {
            const int64_t j = g.neighbour(i, dd);
            if (j <= i) continue;
            if (rd.unit() < d.drop_prob) continue;
            double v;
            if (special[i] || special[j]) {
                v = ulo + (uhi - ulo) * rv.unit();
            } else {
                v = -1.5 + static_cast<double>(rv.below(16)) / 15.0;
            }
            adj_col[27 * i + deg[i]] = static_cast<int32_t>(j);
            adj_val[27 * i + deg[i]++] = v;
            adj_col[27 * j + deg[j]] = static_cast<int32_t>(i);
            adj_val[27 * j + deg[j]++] = v;
        }
    }

    // 3. diagonal from the off-diagonals in ascending column order
    for (int64_t i = 0; i < n; ++i) {
        int32_t* c = &adj_col[27 * i];
        double* v = &adj_val[27 * i];
        const int m = deg[i];
        // insertion sort by column (at most 26 entries)
        for (int a = 1; a < m; ++a)
            for (int b = a; b > 0 && c[b - 1] > c[b]; --b) {
                std::swap(c[b - 1], c[b]);
                std::swap(v[b - 1], v[b]);
            }
        double s = 0.0;
        for (int a = 0; a < m; ++a) s = s + std::fabs(v[a]);
        double diag = 26.0;
        if (special[i]) diag = 1.05 * s;
        else if (d.diag_rule == 1) diag = std::fmax(26.0, 1.05 * s);
        c[m] = static_cast<int32_t>(i);
        v[m] = diag;
        deg[i] = m + 1;
    }

    // 4. renumbering: full Fisher-Yates, old node k becomes p[k]
    std::vector<int32_t> p(n);
    for (int64_t k = 0; k < n; ++k) p[k] = static_cast<int32_t>(k);
    if (d.permute) {
        SplitMix64 rp = stream_for(d.seed, "perm");
        for (int64_t t = n - 1; t >= 1; --t) std::swap(p[t], p[rp.below(t + 1)]);
    }
    out->n = n;
    out->rowptr.assign(n + 1, 0);
    for (int64_t k = 0; k < n; ++k) out->rowptr[p[k] + 1] = deg[k];
    for (int64_t r = 0; r < n; ++r) out->rowptr[r + 1] += out->rowptr[r];
    out->col.resize(out->rowptr[n]);
    out->val.resize(out->rowptr[n]);
    parallel_rows(n, [&](int64_t a, int64_t b) {
        std::vector<std::pair<int32_t, double>> row;
        for (int64_t k = a; k < b; ++k) {
            row.clear();
            for (int e = 0; e < deg[k]; ++e) row.emplace_back(p[adj_col[27 * k + e]], adj_val[27 * k + e]);
            std::sort(row.begin(), row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
            int64_t base = out->rowptr[p[k]];
            for (const auto& e : row) {
                out->col[base] = e.first;
                out->val[base++] = e.second;
            }
        }
    });
    return SPMV_OK;
}

int validate_csr(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val) {
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(SPMV_EINVAL, "n out of range");
    if (!rowptr || (n > 0 && rowptr[n] > 0 && (!col || !val))) return fail(SPMV_EINVAL, "null CSR array");
    if (rowptr[0] != 0) return fail(SPMV_EINVAL, "rowptr[0] must be 0");
    for (int64_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return fail(SPMV_EINVAL, "rowptr must be nondecreasing");
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (col[k] < 0 || col[k] >= n) return fail(SPMV_EINVAL, "column index out of range");
            if (k > rowptr[i] && col[k] <= col[k - 1])
                return fail(SPMV_EINVAL, "columns must be strictly ascending within a row");
        }
    }
    return SPMV_OK;
}

}  // namespace spmvc
