// Locality reordering inside spmv_compress (the reordering Sec. V names as
// the way to cut the cost of the indirect, far-flung x accesses): reverse
// Cuthill-McKee brings every row's columns close to the diagonal, so the
// delta format's int16 column deltas fit again, and inside each
// breadth-first level the rows whose values all sit in the value table go
// first, so that table-coded slices and raw-value slices cluster.  The
// permutation is applied as B = P A P^T; products gather x and scatter y.
#include <algorithm>
#include <cstring>
#include <vector>

#include "host_par.h"
#include "spmvc_internal.h"

namespace spmvc {

namespace {

// Row i of P A P^T (perm[i] = old row) or of P^T B P (the inverse map):
// row `src` of m with every column c mapped to colmap[c], columns sorted.
void permute_rows(const Csr& m, const std::vector<int32_t>& rowsrc, const std::vector<int32_t>& colmap, Csr* out) {
    const int64_t n = m.n;
    out->n = n;
    out->rowptr.assign(static_cast<size_t>(n) + 1, 0);
    for (int64_t i = 0; i < n; ++i) out->rowptr[i + 1] = out->rowptr[i] + (m.rowptr[rowsrc[i] + 1] - m.rowptr[rowsrc[i]]);
    out->col.resize(m.col.size());
    out->val.resize(m.val.size());
    parallel_ranges(n, 1 << 15, [&](int64_t a, int64_t b, int) {
        std::vector<std::pair<int32_t, double>> row;
        for (int64_t i = a; i < b; ++i) {
            const int32_t o = rowsrc[i];
            row.clear();
            for (int64_t k = m.rowptr[o]; k < m.rowptr[o + 1]; ++k) row.emplace_back(colmap[m.col[k]], m.val[k]);
            std::sort(row.begin(), row.end(), [](const auto& p, const auto& q) { return p.first < q.first; });
            int64_t pos = out->rowptr[i];
            for (const auto& e : row) {
                out->col[pos] = e.first;
                out->val[pos] = e.second;
                ++pos;
            }
        }
    });
}

// Breadth-first levels from `start` over unvisited nodes; returns the nodes
// in visiting order (neighbours by ascending degree) and their levels.
void bfs(const Csr& a, int64_t start, std::vector<uint8_t>& seen, std::vector<int32_t>& order,
         std::vector<int32_t>& level, const std::vector<int32_t>& deg) {
    std::vector<int32_t> nb;
    const size_t first = order.size();
    order.push_back(static_cast<int32_t>(start));
    seen[start] = 1;
    level[start] = 0;
    for (size_t h = first; h < order.size(); ++h) {
        const int32_t u = order[h];
        nb.clear();
        for (int64_t k = a.rowptr[u]; k < a.rowptr[u + 1]; ++k) {
            const int32_t v = a.col[k];
            if (!seen[v]) {
                seen[v] = 1;
                nb.push_back(v);
            }
        }
        std::sort(nb.begin(), nb.end(), [&](int32_t p, int32_t q) { return deg[p] != deg[q] ? deg[p] < deg[q] : p < q; });
        for (int32_t v : nb) {
            level[v] = level[u] + 1;
            order.push_back(v);
        }
    }
}

}  // namespace

int reorder_rcm(const Csr& a, const std::vector<double>& dict, std::vector<int32_t>* perm) {
    const int64_t n = a.n;
    if (n >= (int64_t(1) << 31)) return fail(SPMV_EUNSUPPORTED, "reordering needs fewer than 2^31 rows");
    std::vector<int32_t> deg(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) deg[i] = static_cast<int32_t>(a.rowptr[i + 1] - a.rowptr[i]);
    // rows holding a value outside the table
    BitsTable in_table;
    for (double v : dict) in_table.at(value_bits(v)) = 1;
    std::vector<uint8_t> dirty(static_cast<size_t>(n), 0);
    parallel_ranges(n, 1 << 15, [&](int64_t r0, int64_t r1, int) {
        for (int64_t i = r0; i < r1; ++i)
            for (int64_t k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k)
                if (!in_table.get(value_bits(a.val[k]), 0)) { dirty[i] = 1; break; }
    });
    // nodes by ascending degree: each component starts from its first one,
    // moved to a pseudo-peripheral node (last level, smallest degree) by two
    // extra sweeps
    std::vector<int32_t> by_deg(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) by_deg[i] = static_cast<int32_t>(i);
    std::stable_sort(by_deg.begin(), by_deg.end(), [&](int32_t p, int32_t q) { return deg[p] < deg[q]; });
    std::vector<uint8_t> seen(static_cast<size_t>(n), 0), probe(static_cast<size_t>(n), 0);
    std::vector<int32_t> level(static_cast<size_t>(n), 0), order, comp, lev2(static_cast<size_t>(n), 0);
    order.reserve(static_cast<size_t>(n));
    std::vector<int32_t> cm;                      // Cuthill-McKee order
    std::vector<int32_t> cm_level;
    cm.reserve(static_cast<size_t>(n));
    cm_level.reserve(static_cast<size_t>(n));
    int32_t level_base = 0;
    for (int32_t s0 : by_deg) {
        if (seen[s0]) continue;
        int64_t start = s0;
        for (int sweep = 0; sweep < 2; ++sweep) {
            comp.clear();
            bfs(a, start, probe, comp, lev2, deg);
            const int32_t last = lev2[comp.back()];
            int64_t best = start;
            for (int32_t v : comp)
                if (lev2[v] == last && (best == start || deg[v] < deg[best])) best = v;
            for (int32_t v : comp) probe[v] = 0;
            start = best;
        }
        const size_t first = order.size();
        bfs(a, start, seen, order, level, deg);
        int32_t top = 0;
        for (size_t h = first; h < order.size(); ++h) {
            cm.push_back(order[h]);
            cm_level.push_back(level_base + level[order[h]]);
            top = std::max(top, level[order[h]]);
        }
        level_base += top + 1;
    }
    // reverse, then clean rows ahead of dirty ones inside each level
    std::reverse(cm.begin(), cm.end());
    std::reverse(cm_level.begin(), cm_level.end());
    std::vector<int32_t> idx(cm.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = static_cast<int32_t>(i);
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t p, int32_t q) {
        if (cm_level[p] != cm_level[q]) return cm_level[p] > cm_level[q];
        return dirty[cm[p]] < dirty[cm[q]];
    });
    perm->resize(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) (*perm)[i] = cm[idx[i]];
    return SPMV_OK;
}

void permute_csr(const Csr& a, const std::vector<int32_t>& perm, Csr* out) {
    std::vector<int32_t> inv(perm.size());
    for (size_t i = 0; i < perm.size(); ++i) inv[perm[i]] = static_cast<int32_t>(i);
    permute_rows(a, perm, inv, out);
}

// A = P^T B P: row o of A is row inv[o] of B with columns mapped back
void unpermute_csr(const Csr& b, const std::vector<int32_t>& perm, Csr* out) {
    std::vector<int32_t> inv(perm.size());
    for (size_t i = 0; i < perm.size(); ++i) inv[perm[i]] = static_cast<int32_t>(i);
    permute_rows(b, inv, perm, out);
}

}  // namespace spmvc
