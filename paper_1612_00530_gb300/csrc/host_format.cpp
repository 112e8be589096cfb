// Host-side storage formats of arXiv:1612.00530, Sec. V, as laid out for a
// GB300: plain sliced ELL ("Original" of Table II), the pattern format
// (value table + registered displacement patterns, the "Data+Index Table"
// idea) and the delta format with a raw per-slice fallback.  Compression is
// done once on the host (its cost is amortised over many products, Sec. V);
// decompression is bit-exact and doubles as the validation of imported
// streams.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_map>

#include "spmvc_internal.h"

namespace spmvc {

namespace {

uint64_t bits_of(double v) {
    uint64_t b;
    std::memcpy(&b, &v, 8);
    return b;
}

// Value table of Sec. V: the distinct values in ascending order.  Values are
// told apart by their bit patterns so that -0.0 and +0.0 both survive a
// round trip; NaN is refused.
int value_table(const std::vector<double>& val, std::vector<double>* dict,
                std::unordered_map<uint64_t, int64_t>* counts) {
    counts->clear();
    for (double v : val) {
        if (std::isnan(v)) return fail(SPMV_EUNSUPPORTED, "NaN matrix values cannot be tabled");
        (*counts)[bits_of(v)]++;
    }
    dict->clear();
    for (const auto& kv : *counts) {
        double v;
        std::memcpy(&v, &kv.first, 8);
        dict->push_back(v);
    }
    std::sort(dict->begin(), dict->end(), [](double a, double b) {
        if (a != b) return a < b;
        return std::signbit(a) > std::signbit(b);  // -0.0 before +0.0
    });
    return SPMV_OK;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace

// ------------------------------------------------------------------ ELL ---
int pack_ell(const Csr& a, EllFormat* out) {
    const int64_t n = a.n;
    out->nslices = (n + kSliceRows - 1) / kSliceRows;
    out->slice_off.assign(out->nslices + 1, 0);
    out->slice_w.assign(out->nslices, 0);
    for (int64_t s = 0; s < out->nslices; ++s) {
        int64_t w = 0;
        for (int64_t r = s * kSliceRows; r < std::min(n, (s + 1) * kSliceRows); ++r)
            w = std::max<int64_t>(w, a.rowptr[r + 1] - a.rowptr[r]);
        out->slice_w[s] = static_cast<int32_t>(w);
        out->slice_off[s + 1] = out->slice_off[s] + w * kSliceRows;
    }
    out->val.assign(out->slice_off.back(), 0.0);
    out->col.assign(out->slice_off.back(), -1);
    for (int64_t r = 0; r < n; ++r) {
        const int64_t s = r / kSliceRows, l = r % kSliceRows;
        int64_t t = 0;
        for (int64_t k = a.rowptr[r]; k < a.rowptr[r + 1]; ++k, ++t) {
            out->val[out->slice_off[s] + t * kSliceRows + l] = a.val[k];
            out->col[out->slice_off[s] + t * kSliceRows + l] = a.col[k];
        }
    }
    return SPMV_OK;
}


// Exact fixed-point order: every table value an integer multiple m_v
// (|m_v| <= 127) of one power of two, at most kMaxFastDict values, and row
// sums of |m| below 2^10 so that 53-bit fixed-point sums cannot overflow.
void derive_fast_order(int64_t n, PatternFormat* p) {
    p->fast_ok = false;
    p->mult.clear();
    p->mult_exp = 0;
    p->max_row_abs = 0;
    if (p->dict.empty() || static_cast<int>(p->dict.size()) > kMaxFastDict) return;
    int e_min = 100000;
    for (double v : p->dict) {
        if (!std::isfinite(v)) return;
        if (v == 0.0) continue;
        int e;
        const double f = std::frexp(std::fabs(v), &e);           // |v| = f * 2^e, f in [0.5, 1)
        int64_t m = static_cast<int64_t>(std::ldexp(f, 53));    // exact 53-bit integer
        int tz = 0;
        while ((m & 1) == 0) { m >>= 1; ++tz; }
        e_min = std::min(e_min, e - 53 + tz);
    }
    if (e_min == 100000) e_min = 0;
    for (double v : p->dict) {
        const double m = std::ldexp(v, -e_min);
        if (!(std::fabs(m) <= 127.0) || m != std::floor(m)) { p->mult.clear(); return; }
        p->mult.push_back(static_cast<int32_t>(m));
    }
    const int nu = static_cast<int>(p->uoff.size());
    int64_t worst = 0;
    for (int64_t r = 0; r < n; ++r) {
        const uint8_t* b = reinterpret_cast<const uint8_t*>(&p->rec[static_cast<size_t>(r) * p->words]);
        const uint32_t mask = p->pmask[b[nu]];
        int64_t s = 0;
        for (int u = 0; u < nu; ++u)
            if ((mask >> u) & 1u) s += std::abs(p->mult[b[u]]);
        worst = std::max(worst, s);
    }
    p->max_row_abs = worst;
    p->mult_exp = e_min;
    p->fast_ok = worst < 1024;
}

// Values registered in the pattern (Sec. V): a row's whole record -- its
// codes and its pattern number -- becomes one of at most 256 row types.
bool build_row_types(int64_t n, PatternFormat* p) {
    p->rtype.clear();
    p->rtypes.clear();
    if (p->words != 7) return false;
    std::map<std::vector<uint32_t>, int> types;
    std::vector<uint8_t> rtype(static_cast<size_t>(n));
    std::vector<uint32_t> table;
    std::vector<uint32_t> key(7);
    for (int64_t r = 0; r < n; ++r) {
        std::copy(&p->rec[static_cast<size_t>(r) * 7], &p->rec[static_cast<size_t>(r) * 7] + 7, key.begin());
        auto it = types.find(key);
        if (it == types.end()) {
            if (types.size() == 256) return false;
            it = types.emplace(key, static_cast<int>(types.size())).first;
            table.insert(table.end(), key.begin(), key.end());
            table.push_back(0u);                       // 8 words a type
        }
        rtype[r] = static_cast<uint8_t>(it->second);
    }
    p->rtype = std::move(rtype);
    p->rtypes = std::move(table);
    return true;
}

// -------------------------------------------------------------- pattern ---
int compress_pattern(const Csr& a, int max_dict, PatternFormat* out) {
    const int64_t n = a.n;
    std::unordered_map<uint64_t, int64_t> counts;
    int st = value_table(a.val, &out->dict, &counts);
    if (st) return st;
    if (static_cast<int>(out->dict.size()) > max_dict)
        return fail(SPMV_EUNSUPPORTED, "value table larger than max_dict");
    std::unordered_map<uint64_t, int> code_of;
    for (size_t v = 0; v < out->dict.size(); ++v) code_of[bits_of(out->dict[v])] = static_cast<int>(v);

    // Register each row's displacement list (columns relative to the
    // diagonal) in the pattern table (Sec. V).
    std::map<std::vector<int32_t>, int> registry;
    std::vector<std::vector<int32_t>> patterns;
    std::vector<uint8_t> row_pat(n);
    std::vector<int32_t> disp;
    int last = -1;
    for (int64_t r = 0; r < n; ++r) {
        disp.clear();
        for (int64_t k = a.rowptr[r]; k < a.rowptr[r + 1]; ++k) disp.push_back(static_cast<int32_t>(a.col[k] - r));
        int id;
        if (last >= 0 && patterns[last] == disp) {
            id = last;
        } else {
            auto it = registry.find(disp);
            if (it == registry.end()) {
                if (static_cast<int>(patterns.size()) == kMaxPatterns)
                    return fail(SPMV_EUNSUPPORTED, "more than 32 displacement patterns");
                id = static_cast<int>(patterns.size());
                registry.emplace(disp, id);
                patterns.push_back(disp);
            } else {
                id = it->second;
            }
        }
        row_pat[r] = static_cast<uint8_t>(id);
        last = id;
    }
    // union of displacements and per-pattern slot masks
    std::vector<int32_t> uni;
    for (const auto& p : patterns) uni.insert(uni.end(), p.begin(), p.end());
    std::sort(uni.begin(), uni.end());
    uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
    if (static_cast<int>(uni.size()) > kMaxUnion) return fail(SPMV_EUNSUPPORTED, "displacement union above 31 slots");
    if (out->dict.size() > 254) return fail(SPMV_EUNSUPPORTED, "value table above 254 entries");
    const int nu = static_cast<int>(uni.size());
    out->uoff = uni;
    out->pmask.assign(patterns.size(), 0u);
    std::vector<std::vector<int>> slot_of(patterns.size());
    for (size_t p = 0; p < patterns.size(); ++p)
        for (int32_t dlt : patterns[p]) {
            const int u = static_cast<int>(std::lower_bound(uni.begin(), uni.end(), dlt) - uni.begin());
            out->pmask[p] |= 1u << u;
            slot_of[p].push_back(u);
        }
    out->words = (nu + 1 + 3) / 4;
    out->rec.assign(static_cast<size_t>(n) * out->words, 0u);
    const uint8_t absent = static_cast<uint8_t>(out->dict.size());
    std::vector<uint8_t> bytes(4 * out->words);
    for (int64_t r = 0; r < n; ++r) {
        std::fill(bytes.begin(), bytes.end(), 0);
        std::fill(bytes.begin(), bytes.begin() + nu, absent);
        const int p = row_pat[r];
        int64_t k = a.rowptr[r];
        for (int u : slot_of[p]) bytes[u] = static_cast<uint8_t>(code_of[bits_of(a.val[k++])]);
        bytes[nu] = static_cast<uint8_t>(p);
        std::memcpy(&out->rec[static_cast<size_t>(r) * out->words], bytes.data(), bytes.size());
    }

    derive_fast_order(n, out);
    return SPMV_OK;
}

// ------------------------------------------------------ Data+Index Table ---
// Sec. V: each row's nonzeros sorted by value (columns ascending inside a
// value), made relative to the row (column - row), and the displacement
// list registered as a type; the row keeps its type and the end of each
// value group (Fig. 2's terminal indices, stored exclusive).
int compress_dit(const Csr& a, DitFormat* out) {
    const int64_t n = a.n;
    std::unordered_map<uint64_t, int64_t> counts;
    int st = value_table(a.val, &out->dict, &counts);
    if (st) return st;
    const int nv = static_cast<int>(out->dict.size());
    if (nv > 255) return fail(SPMV_EUNSUPPORTED, "Data+Index Table: more than 255 distinct values");
    std::unordered_map<uint64_t, int> code_of;
    for (int v = 0; v < nv; ++v) code_of[bits_of(out->dict[v])] = v;
    std::map<std::vector<int32_t>, int> types;
    std::vector<std::vector<int32_t>> lists;
    out->type.assign(static_cast<size_t>(n), 0);
    out->ends.assign(static_cast<size_t>(n) * nv, 0);
    std::vector<std::vector<int32_t>> groups(nv);
    std::vector<int32_t> disp;
    for (int64_t r = 0; r < n; ++r) {
        const int64_t len = a.rowptr[r + 1] - a.rowptr[r];
        if (len > 255) return fail(SPMV_EUNSUPPORTED, "Data+Index Table: a row holds more than 255 entries");
        for (auto& g : groups) g.clear();
        for (int64_t k = a.rowptr[r]; k < a.rowptr[r + 1]; ++k)
            groups[code_of[bits_of(a.val[k])]].push_back(static_cast<int32_t>(a.col[k] - r));
        disp.clear();
        for (int v = 0; v < nv; ++v) {
            disp.insert(disp.end(), groups[v].begin(), groups[v].end());
            out->ends[static_cast<size_t>(v) * n + r] = static_cast<uint8_t>(disp.size());
        }
        auto it = types.find(disp);
        if (it == types.end()) {
            if (types.size() == 256) return fail(SPMV_EUNSUPPORTED, "Data+Index Table: more than 256 row types");
            it = types.emplace(disp, static_cast<int>(lists.size())).first;
            lists.push_back(disp);
        }
        out->type[r] = static_cast<uint8_t>(it->second);
    }
    out->maxlen = 0;
    for (const auto& l : lists) out->maxlen = std::max<int32_t>(out->maxlen, static_cast<int32_t>(l.size()));
    out->disp.assign(lists.size() * static_cast<size_t>(std::max(out->maxlen, 1)), 0);
    out->tlen.assign(lists.size(), 0);
    for (size_t t = 0; t < lists.size(); ++t) {
        std::copy(lists[t].begin(), lists[t].end(), out->disp.begin() + t * std::max(out->maxlen, 1));
        out->tlen[t] = static_cast<int32_t>(lists[t].size());
    }
    return SPMV_OK;
}

// ---------------------------------------------------------------- delta ---
// The delta format's value table: the most frequent values with at least
// min_count uses, at most max_dict of them, in ascending order.
void delta_dictionary(const std::vector<double>& val, int max_dict, int min_count, std::vector<double>* dict) {
    std::unordered_map<uint64_t, int64_t> counts;
    std::vector<double> all;
    if (value_table(val, &all, &counts)) {
        // NaN values: no table at all, every slice raw
        all.clear();
        counts.clear();
    }
    std::vector<std::pair<int64_t, double>> freq;
    for (double v : all) {
        const int64_t c = counts[bits_of(v)];
        if (c >= min_count) freq.emplace_back(-c, v);
    }
    std::sort(freq.begin(), freq.end(), [](const auto& x, const auto& y) {
        if (x.first != y.first) return x.first < y.first;
        return x.second < y.second;
    });
    if (static_cast<int>(freq.size()) > max_dict) freq.resize(max_dict);
    dict->clear();
    for (const auto& f : freq) dict->push_back(f.second);
    std::sort(dict->begin(), dict->end(), [](double x, double y) {
        if (x != y) return x < y;
        return std::signbit(x) > std::signbit(y);
    });
}

int compress_delta(const Csr& a, int max_dict, int min_count, DeltaFormat* out) {
    const int64_t n = a.n;
    delta_dictionary(a.val, max_dict, min_count, &out->dict);
    std::unordered_map<uint64_t, int> code_of;
    for (size_t v = 0; v < out->dict.size(); ++v) code_of[bits_of(out->dict[v])] = static_cast<int>(v);

    out->nslices = (n + kSliceRows - 1) / kSliceRows;
    out->hdr.assign(out->nslices, DeltaSlice{0, 0, 0});
    uint64_t off = 0;
    for (int64_t s = 0; s < out->nslices; ++s) {
        const int64_t r0 = s * kSliceRows, r1 = std::min(n, r0 + kSliceRows);
        int64_t w = 0;
        uint32_t flags = 0;
        for (int64_t r = r0; r < r1; ++r) {
            w = std::max<int64_t>(w, a.rowptr[r + 1] - a.rowptr[r]);
            for (int64_t k = a.rowptr[r]; k < a.rowptr[r + 1]; ++k) {
                const int64_t dlt = static_cast<int64_t>(a.col[k]) - r;
                if (dlt < -32768 || dlt > 32767) flags |= kSliceColRaw;
                if (std::isnan(a.val[k]) || code_of.find(bits_of(a.val[k])) == code_of.end()) flags |= kSliceValRaw;
            }
        }
        if (w > 255) return fail(SPMV_EUNSUPPORTED, "delta format holds at most 255 entries per row");
        const int64_t cb = (flags & kSliceColRaw) ? 4 : 2, vb = (flags & kSliceValRaw) ? 8 : 1;
        out->hdr[s] = DeltaSlice{off, static_cast<uint32_t>(w), flags};
        off += round_up(32 + w * kSliceRows * cb, 16) + round_up(w * kSliceRows * vb, 16);
    }
    out->payload.assign(off, 0);
    for (int64_t s = 0; s < out->nslices; ++s) {
        const DeltaSlice h = out->hdr[s];
        const int64_t r0 = s * kSliceRows, r1 = std::min(n, r0 + kSliceRows);
        uint8_t* base = out->payload.data() + h.off;
        const bool craw = h.flags & kSliceColRaw, vraw = h.flags & kSliceValRaw;
        uint8_t* cols = base + 32;
        uint8_t* vals = base + round_up(32 + int64_t(h.w) * kSliceRows * (craw ? 4 : 2), 16);
        for (int64_t r = r0; r < r1; ++r) {
            const int64_t l = r - r0;
            base[l] = static_cast<uint8_t>(a.rowptr[r + 1] - a.rowptr[r]);
            int64_t t = 0;
            for (int64_t k = a.rowptr[r]; k < a.rowptr[r + 1]; ++k, ++t) {
                const int64_t slot = t * kSliceRows + l;
                if (craw) {
                    const int32_t c = a.col[k];
                    std::memcpy(cols + 4 * slot, &c, 4);
                } else {
                    const int16_t d16 = static_cast<int16_t>(a.col[k] - r);
                    std::memcpy(cols + 2 * slot, &d16, 2);
                }
                if (vraw) std::memcpy(vals + 8 * slot, &a.val[k], 8);
                else vals[slot] = static_cast<uint8_t>(code_of[bits_of(a.val[k])]);
            }
        }
    }
    return SPMV_OK;
}

}  // namespace spmvc
