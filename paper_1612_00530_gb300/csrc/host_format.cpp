// Host-side storage formats of arXiv:1612.00530, Sec. V, as laid out for a
// GB300: plain sliced ELL ("Original" of Table II), the pattern format
// (value table + registered displacement patterns, the "Data+Index Table"
// idea) and the delta format with a raw per-slice fallback.  Compression is
// done once on the host (its cost is amortised over many products, Sec. V);
// decompression is bit-exact and doubles as the validation of imported
// streams.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>

#include "host_par.h"
#include "spmvc_internal.h"

namespace spmvc {

namespace {

double value_of(uint64_t bits) {
    double v;
    std::memcpy(&v, &bits, 8);
    return v;
}

// Ascending values, -0.0 before +0.0.
bool value_less(double a, double b) {
    if (a != b) return a < b;
    return std::signbit(a) > std::signbit(b);
}

// Value table of Sec. V: the distinct values in ascending order.  Values are
// told apart by their bit patterns so that -0.0 and +0.0 both survive a
// round trip; NaN is refused, and so is a table above `limit` entries
// (limit 0: no limit).  *counts receives every value's count.
int value_table(const std::vector<double>& val, size_t limit, std::vector<double>* dict, BitsTable* counts,
                const char* over_msg) {
    bool over = false, nan = false;
    count_values(val, limit, counts, &over, &nan);
    if (nan) return fail(SPMV_EUNSUPPORTED, "NaN matrix values cannot be tabled");
    if (over) return fail(SPMV_EUNSUPPORTED, over_msg);
    dict->clear();
    counts->for_each([&](uint64_t k, int64_t) { dict->push_back(value_of(k)); });
    std::sort(dict->begin(), dict->end(), value_less);
    return SPMV_OK;
}

// dict[v] -> v, looked up by bit pattern (-1 when absent)
BitsTable code_table(const std::vector<double>& dict) {
    BitsTable t;
    for (size_t v = 0; v < dict.size(); ++v) t.at(value_bits(dict[v])) = int64_t(v);
    return t;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Numbers the distinct keys of rows 0..n-1 in order of first appearance
// (the row order, as one sequential pass would), chunks of rows in
// parallel and their local tables merged in chunk order.  key_of(r, key)
// fills row r's key and returns false to abort.  ids[r] receives row r's
// number.  Returns 0, 1 when there are more than `limit` keys, 2 when
// key_of aborted.
template <class Key, class KeyOf>
int register_first_seen(int64_t n, size_t limit, KeyOf&& key_of, std::vector<uint8_t>* ids, std::vector<Key>* keys) {
    constexpr int64_t kGrain = 1 << 16;
    const int parts = parallel_parts(n, kGrain);
    std::vector<std::vector<Key>> local(parts);
    std::vector<int> bad(parts, 0);
    std::vector<int32_t> lid(static_cast<size_t>(n));
    parallel_ranges(n, kGrain, [&](int64_t a, int64_t b, int t) {
        std::map<Key, int32_t> reg;
        Key k;
        int32_t last = -1;
        for (int64_t r = a; r < b; ++r) {
            if (!key_of(r, k)) { bad[t] = 2; return; }
            int32_t id;
            if (last >= 0 && local[t][last] == k) {
                id = last;
            } else {
                auto it = reg.find(k);
                if (it == reg.end()) {
                    if (local[t].size() == limit) { bad[t] = 1; return; }
                    id = static_cast<int32_t>(local[t].size());
                    reg.emplace(k, id);
                    local[t].push_back(k);
                } else {
                    id = it->second;
                }
            }
            lid[r] = id;
            last = id;
        }
    });
    for (int t = 0; t < parts; ++t)
        if (bad[t]) return bad[t];
    std::map<Key, int32_t> glob;
    std::vector<std::vector<uint8_t>> remap(parts);
    keys->clear();
    for (int t = 0; t < parts; ++t)
        for (const Key& k : local[t]) {
            auto it = glob.find(k);
            if (it == glob.end()) {
                if (keys->size() == limit) return 1;
                it = glob.emplace(k, static_cast<int32_t>(keys->size())).first;
                keys->push_back(k);
            }
            remap[t].push_back(static_cast<uint8_t>(it->second));
        }
    ids->resize(static_cast<size_t>(n));
    parallel_ranges(n, kGrain, [&](int64_t a, int64_t b, int t) {
        for (int64_t r = a; r < b; ++r) (*ids)[r] = remap[t][lid[r]];
    });
    return 0;
}

}  // namespace

// ------------------------------------------------------------------ ELL ---
int pack_ell(const Csr& a, EllFormat* out) {
    const int64_t n = a.n;
    const int64_t ns = (n + kSliceRows - 1) / kSliceRows;
    out->nslices = ns;
    out->slice_off.assign(ns + 1, 0);
    out->slice_w.assign(ns, 0);
    parallel_ranges(ns, 4096, [&](int64_t s0, int64_t s1, int) {
        for (int64_t s = s0; s < s1; ++s) {
            int64_t w = 0;
            for (int64_t r = s * kSliceRows; r < std::min(n, (s + 1) * kSliceRows); ++r)
                w = std::max<int64_t>(w, a.rowptr[r + 1] - a.rowptr[r]);
            out->slice_w[s] = static_cast<int32_t>(w);
        }
    });
    for (int64_t s = 0; s < ns; ++s) out->slice_off[s + 1] = out->slice_off[s] + int64_t(out->slice_w[s]) * kSliceRows;
    out->val.resize(out->slice_off.back());
    out->col.resize(out->slice_off.back());
    // every slot written once: a row's entries, then padding (value 0,
    // column -1) up to the slice width
    parallel_ranges(ns, 4096, [&](int64_t s0, int64_t s1, int) {
        for (int64_t s = s0; s < s1; ++s) {
            const int64_t w = out->slice_w[s], base = out->slice_off[s];
            for (int64_t l = 0; l < kSliceRows; ++l) {
                const int64_t r = s * kSliceRows + l;
                int64_t t = 0;
                if (r < n)
                    for (int64_t k = a.rowptr[r]; k < a.rowptr[r + 1]; ++k, ++t) {
                        out->val[base + t * kSliceRows + l] = a.val[k];
                        out->col[base + t * kSliceRows + l] = a.col[k];
                    }
                for (; t < w; ++t) {
                    out->val[base + t * kSliceRows + l] = 0.0;
                    out->col[base + t * kSliceRows + l] = -1;
                }
            }
        }
    });
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
    std::vector<int64_t> part_worst(parallel_parts(n, 1 << 16), 0);
    parallel_ranges(n, 1 << 16, [&](int64_t a, int64_t b, int t) {
        int64_t w = 0;
        for (int64_t r = a; r < b; ++r) {
            const uint8_t* rb = reinterpret_cast<const uint8_t*>(&p->rec[static_cast<size_t>(r) * p->words]);
            const uint32_t mask = p->pmask[rb[nu]];
            int64_t s = 0;
            for (int u = 0; u < nu; ++u)
                if ((mask >> u) & 1u) s += std::abs(p->mult[rb[u]]);
            w = std::max(w, s);
        }
        part_worst[t] = w;
    });
    int64_t worst = 0;
    for (int64_t w : part_worst) worst = std::max(worst, w);
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
    std::vector<std::array<uint32_t, 7>> types;
    std::vector<uint8_t> rtype;
    auto rec_of = [&](int64_t r, std::array<uint32_t, 7>& key) {
        std::copy(&p->rec[static_cast<size_t>(r) * 7], &p->rec[static_cast<size_t>(r) * 7] + 7, key.begin());
        return true;
    };
    if (register_first_seen(n, 256, rec_of, &rtype, &types)) return false;
    std::vector<uint32_t> table;
    for (const auto& t : types) {
        table.insert(table.end(), t.begin(), t.end());
        table.push_back(0u);                       // 8 words a type
    }
    p->rtype = std::move(rtype);
    p->rtypes = std::move(table);
    return true;
}

// -------------------------------------------------------------- pattern ---
int compress_pattern(const Csr& a, int max_dict, PatternFormat* out) {
    const int64_t n = a.n;
    BitsTable counts;
    int st = value_table(a.val, static_cast<size_t>(max_dict), &out->dict, &counts, "value table larger than max_dict");
    if (st) return st;
    const BitsTable code = code_table(out->dict);

    // Register each row's displacement list (columns relative to the
    // diagonal) in the pattern table (Sec. V).
    std::vector<std::vector<int32_t>> patterns;
    std::vector<uint8_t> row_pat;
    auto disp_of = [&](int64_t r, std::vector<int32_t>& disp) {
        disp.clear();
        for (int64_t k = a.rowptr[r]; k < a.rowptr[r + 1]; ++k) disp.push_back(static_cast<int32_t>(a.col[k] - r));
        return true;
    };
    if (register_first_seen(n, kMaxPatterns, disp_of, &row_pat, &patterns))
        return fail(SPMV_EUNSUPPORTED, "more than 32 displacement patterns");
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
    out->rec.resize(static_cast<size_t>(n) * out->words);
    const uint8_t absent = static_cast<uint8_t>(out->dict.size());
    parallel_ranges(n, 1 << 16, [&](int64_t r0, int64_t r1, int) {
        std::vector<uint8_t> bytes(4 * out->words);
        for (int64_t r = r0; r < r1; ++r) {
            std::fill(bytes.begin(), bytes.end(), 0);
            std::fill(bytes.begin(), bytes.begin() + nu, absent);
            const int p = row_pat[r];
            int64_t k = a.rowptr[r];
            for (int u : slot_of[p]) bytes[u] = static_cast<uint8_t>(code.get(value_bits(a.val[k++]), 0));
            bytes[nu] = static_cast<uint8_t>(p);
            std::memcpy(&out->rec[static_cast<size_t>(r) * out->words], bytes.data(), bytes.size());
        }
    });

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
    BitsTable counts;
    int st = value_table(a.val, 255, &out->dict, &counts, "Data+Index Table: more than 255 distinct values");
    if (st) return st;
    const int nv = static_cast<int>(out->dict.size());
    const BitsTable code = code_table(out->dict);
    out->ends.resize(static_cast<size_t>(n) * nv);
    // a row's displacement list, its entries grouped by value code (value
    // groups ascending, columns ascending inside a group), and the end of
    // each group
    auto disp_of = [&](int64_t r, std::vector<int32_t>& disp) {
        const int64_t k0 = a.rowptr[r], len = a.rowptr[r + 1] - k0;
        if (len > 255) return false;
        uint8_t c[255];
        int32_t pos[257];
        std::fill(pos, pos + nv + 1, 0);
        for (int64_t i = 0; i < len; ++i) {
            c[i] = static_cast<uint8_t>(code.get(value_bits(a.val[k0 + i]), 0));
            ++pos[c[i] + 1];
        }
        for (int v = 0; v < nv; ++v) pos[v + 1] += pos[v];
        disp.resize(static_cast<size_t>(len));
        for (int64_t i = 0; i < len; ++i) disp[pos[c[i]]++] = static_cast<int32_t>(a.col[k0 + i] - r);
        for (int v = 0; v < nv; ++v) out->ends[static_cast<size_t>(v) * n + r] = static_cast<uint8_t>(pos[v]);
        return true;
    };
    std::vector<std::vector<int32_t>> lists;
    st = register_first_seen(n, 256, disp_of, &out->type, &lists);
    if (st == 2) return fail(SPMV_EUNSUPPORTED, "Data+Index Table: a row holds more than 255 entries");
    if (st == 1) return fail(SPMV_EUNSUPPORTED, "Data+Index Table: more than 256 row types");
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

// ------------------------------------------------------------ Data Table ---
// Sec. V, first scheme: per row the columns in value order (S_i) and the end
// of every value group, rows packed in 32-row slices for coalesced reads.
int compress_data_table(const Csr& a, DataTableFormat* out) {
    const int64_t n = a.n;
    BitsTable counts;
    int st = value_table(a.val, 255, &out->dict, &counts, "Data Table: more than 255 distinct values");
    if (st) return st;
    const int nv = static_cast<int>(out->dict.size());
    const BitsTable code = code_table(out->dict);
    const int64_t ns = (n + kSliceRows - 1) / kSliceRows;
    out->nslices = ns;
    out->slice_w.assign(ns, 0);
    out->slice_off.assign(ns + 1, 0);
    std::atomic<bool> too_long{false};
    parallel_ranges(ns, 4096, [&](int64_t s0, int64_t s1, int) {
        for (int64_t s = s0; s < s1; ++s) {
            int64_t w = 0;
            for (int64_t r = s * kSliceRows; r < std::min(n, (s + 1) * kSliceRows); ++r)
                w = std::max<int64_t>(w, a.rowptr[r + 1] - a.rowptr[r]);
            if (w > 255) too_long = true;
            out->slice_w[s] = static_cast<uint8_t>(std::min<int64_t>(w, 255));
        }
    });
    if (too_long) return fail(SPMV_EUNSUPPORTED, "Data Table: a row holds more than 255 entries");
    for (int64_t s = 0; s < ns; ++s) out->slice_off[s + 1] = out->slice_off[s] + int64_t(out->slice_w[s]) * kSliceRows;
    out->S.resize(out->slice_off.back());
    out->ends.resize(static_cast<size_t>(n) * nv);
    parallel_ranges(ns, 4096, [&](int64_t s0, int64_t s1, int) {
        for (int64_t s = s0; s < s1; ++s) {
            const int64_t w = out->slice_w[s], base = out->slice_off[s];
            for (int64_t l = 0; l < kSliceRows; ++l) {
                const int64_t r = s * kSliceRows + l;
                int64_t len = 0;
                if (r < n) {
                    // a stable counting sort of the row's entries by value code
                    const int64_t k0 = a.rowptr[r];
                    len = a.rowptr[r + 1] - k0;
                    uint8_t c[255];
                    int32_t pos[257];
                    std::fill(pos, pos + nv + 1, 0);
                    for (int64_t i = 0; i < len; ++i) {
                        c[i] = static_cast<uint8_t>(code.get(value_bits(a.val[k0 + i]), 0));
                        ++pos[c[i] + 1];
                    }
                    for (int v = 0; v < nv; ++v) pos[v + 1] += pos[v];
                    for (int64_t i = 0; i < len; ++i) out->S[base + int64_t(pos[c[i]]++) * kSliceRows + l] = a.col[k0 + i];
                    for (int v = 0; v < nv; ++v) out->ends[static_cast<size_t>(v) * n + r] = static_cast<uint8_t>(pos[v]);
                }
                for (int64_t t = len; t < w; ++t) out->S[base + t * kSliceRows + l] = -1;
            }
        }
    });
    return SPMV_OK;
}

// ---------------------------------------------------------------- delta ---
// The delta format's value table: the most frequent values with at least
// min_count uses, at most max_dict of them, in ascending order.
void delta_dictionary(const std::vector<double>& val, int max_dict, int min_count, std::vector<double>* dict) {
    BitsTable counts;
    bool over = false, nan = false;
    count_values(val, 0, &counts, &over, &nan);
    std::vector<std::pair<int64_t, double>> freq;
    // NaN values: no table at all, every slice raw
    if (!nan)
        counts.for_each([&](uint64_t k, int64_t c) {
            if (c >= min_count) freq.emplace_back(-c, value_of(k));
        });
    std::sort(freq.begin(), freq.end(), [](const auto& x, const auto& y) {
        if (x.first != y.first) return x.first < y.first;
        return value_less(x.second, y.second);
    });
    if (static_cast<int>(freq.size()) > max_dict) freq.resize(max_dict);
    dict->clear();
    for (const auto& f : freq) dict->push_back(f.second);
    std::sort(dict->begin(), dict->end(), value_less);
}

int compress_delta(const Csr& a, int max_dict, int min_count, DeltaFormat* out) {
    const int64_t n = a.n;
    delta_dictionary(a.val, std::min(max_dict, 254), min_count, &out->dict);
    const BitsTable code = code_table(out->dict);
    const int nd = static_cast<int>(out->dict.size());

    const int64_t ns = (n + kSliceRows - 1) / kSliceRows;
    out->nslices = ns;
    out->hdr.assign(ns, DeltaSlice{0, 0, 0});
    std::vector<uint64_t> bytes(static_cast<size_t>(ns));
    std::atomic<bool> too_wide{false};
    // per slice: the narrowest column encoding that holds every delta, and
    // global codes, global and local codes, or raw values, whichever fits
    // and is smallest (a local table holds the slice's distinct values that
    // the global table lacks, at most 256 - |global table| of them)
    parallel_ranges(ns, 2048, [&](int64_t s0, int64_t s1, int) {
        BitsTable loc;
        for (int64_t s = s0; s < s1; ++s) {
            const int64_t r0 = s * kSliceRows, r1 = std::min(n, r0 + kSliceRows);
            int64_t w = 0, maxd = 0;
            loc.reset(8);
            for (int64_t r = r0; r < r1; ++r) {
                w = std::max<int64_t>(w, a.rowptr[r + 1] - a.rowptr[r]);
                for (int64_t k = a.rowptr[r]; k < a.rowptr[r + 1]; ++k) {
                    const int64_t dlt = static_cast<int64_t>(a.col[k]) - r;
                    maxd = std::max<int64_t>(maxd, dlt < 0 ? -dlt - 1 : dlt);   // two's complement range
                    if (code.get(value_bits(a.val[k]), -1) < 0) loc.at(value_bits(a.val[k])) = 0;
                }
            }
            if (w > 255) too_wide = true;
            w = std::min<int64_t>(w, 255);
            const int64_t nloc = int64_t(loc.size());
            uint32_t flags = maxd <= 32767 ? 0u : maxd <= 8388607 ? kSliceCol24 : kSliceColRaw;
            if (nloc > 0) {
                const bool fits = nloc <= 256 - nd;
                flags |= fits && 16 + 8 * nloc < w * kSliceRows * 7 ? kSliceValLocal : kSliceValRaw;
            }
            out->hdr[s] = DeltaSlice{0, static_cast<uint32_t>(w), flags};
            const DeltaParts pt = delta_parts(uint32_t(w), flags);
            bytes[s] = (flags & kSliceValLocal) ? delta_up16(pt.local + 16 + 8 * uint64_t(nloc)) : pt.local;
        }
    });
    if (too_wide) return fail(SPMV_EUNSUPPORTED, "delta format holds at most 255 entries per row");
    uint64_t off = 0;
    for (int64_t s = 0; s < ns; ++s) {
        out->hdr[s].off = off;
        off += bytes[s];
    }
    out->payload.assign(off, 0);
    parallel_ranges(ns, 2048, [&](int64_t s0, int64_t s1, int) {
        BitsTable loc;
        for (int64_t s = s0; s < s1; ++s) {
            const DeltaSlice h = out->hdr[s];
            const DeltaParts pt = delta_parts(h.w, h.flags);
            const int64_t r0 = s * kSliceRows, r1 = std::min(n, r0 + kSliceRows);
            uint8_t* base = out->payload.data() + h.off;
            const bool craw = h.flags & kSliceColRaw, c24 = h.flags & kSliceCol24;
            const bool vraw = h.flags & kSliceValRaw, vloc = h.flags & kSliceValLocal;
            loc.reset(8);
            uint32_t nloc = 0;
            for (int64_t r = r0; r < r1; ++r) {
                const int64_t l = r - r0;
                base[l] = static_cast<uint8_t>(a.rowptr[r + 1] - a.rowptr[r]);
                int64_t t = 0;
                for (int64_t k = a.rowptr[r]; k < a.rowptr[r + 1]; ++k, ++t) {
                    const int64_t slot = t * kSliceRows + l;
                    if (craw) {
                        const int32_t c = a.col[k];
                        std::memcpy(base + pt.cols + 4 * slot, &c, 4);
                    } else {
                        const int32_t d = static_cast<int32_t>(a.col[k] - r);
                        const int16_t lo = static_cast<int16_t>(static_cast<uint16_t>(uint32_t(d) & 0xFFFFu));
                        std::memcpy(base + pt.cols + 2 * slot, &lo, 2);
                        if (c24) base[pt.hi + slot] = static_cast<uint8_t>(static_cast<int8_t>(d >> 16));
                    }
                    if (vraw) {
                        std::memcpy(base + pt.vals + 8 * slot, &a.val[k], 8);
                        continue;
                    }
                    int64_t cv = code.get(value_bits(a.val[k]), -1);
                    if (cv < 0 && vloc) {   // the slice's own table, in order of first use
                        int64_t& e = loc.at(value_bits(a.val[k]));
                        if (e == 0) {
                            e = ++nloc;
                            std::memcpy(base + pt.local + 16 + 8 * (nloc - 1), &a.val[k], 8);
                        }
                        cv = int64_t(out->dict.size()) + e - 1;
                    }
                    base[pt.vals + slot] = static_cast<uint8_t>(cv);
                }
            }
            if (vloc) std::memcpy(base + pt.local, &nloc, 4);
        }
    });
    return SPMV_OK;
}

}  // namespace spmvc
