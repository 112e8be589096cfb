// Decompression of every stored format back to CSR (bit-exact: values are
// copied, never recomputed), stream checksums, and export/import of a
// matrix's stored form.  Decompression checks every decoded index, so it is
// also how an imported stream is validated before any kernel can see it.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "spmvc_internal.h"

namespace spmvc {

int decompress_ell(int64_t n, const EllFormat& e, Csr* out);
int decompress_pattern(int64_t n, const PatternFormat& p, Csr* out);
int decompress_delta(int64_t n, const DeltaFormat& d, Csr* out);
int decompress_dit(int64_t n, const DitFormat& d, Csr* out);
int decompress_data_table(int64_t n, const DataTableFormat& d, Csr* out);
uint64_t checksum_of(const spmv_mat_s& m);
int export_stream(const spmv_mat_s& m, void* buf, size_t* len);
int import_stream(const void* buf, size_t len, spmv_mat_s* m);

namespace {

int corrupt(const char* what) { return fail(SPMV_ECORRUPT, std::string("corrupt stream: ") + what); }

int finish_csr(Csr* out) {
    // columns must be strictly ascending in every row
    for (int64_t i = 0; i < out->n; ++i)
        for (int64_t k = out->rowptr[i] + 1; k < out->rowptr[i + 1]; ++k)
            if (out->col[k] <= out->col[k - 1]) return corrupt("columns not ascending");
    return SPMV_OK;
}

// FNV-1a over 64-bit words (then the tail bytes).
struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t len) {
        const uint8_t* b = static_cast<const uint8_t*>(p);
        size_t i = 0;
        for (; i + 8 <= len; i += 8) {
            uint64_t w;
            std::memcpy(&w, b + i, 8);
            h = (h ^ w) * 1099511628211ull;
        }
        for (; i < len; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
    template <class T> void vec(const std::vector<T>& v) {
        const uint64_t k = v.size();
        add(&k, 8);
        if (!v.empty()) add(v.data(), v.size() * sizeof(T));
    }
    template <class T> void pod(const T& v) { add(&v, sizeof(T)); }
};

}  // namespace

int decompress_ell(int64_t n, const EllFormat& e, Csr* out) {
    out->n = n;
    out->rowptr.assign(n + 1, 0);
    out->col.clear();
    out->val.clear();
    if (e.nslices != (n + kSliceRows - 1) / kSliceRows || (int64_t)e.slice_off.size() != e.nslices + 1 ||
        (int64_t)e.slice_w.size() != e.nslices)
        return corrupt("ELL slice table size");
    for (int64_t r = 0; r < n; ++r) {
        const int64_t s = r / kSliceRows, l = r % kSliceRows;
        const int64_t w = e.slice_w[s];
        if (w < 0 || e.slice_off[s] + w * kSliceRows > (int64_t)e.val.size()) return corrupt("ELL slice bounds");
        for (int64_t t = 0; t < w; ++t) {
            const int64_t k = e.slice_off[s] + t * kSliceRows + l;
            if (e.col[k] < 0) continue;
            if (e.col[k] >= n) return corrupt("ELL column out of range");
            out->col.push_back(e.col[k]);
            out->val.push_back(e.val[k]);
        }
        out->rowptr[r + 1] = static_cast<int64_t>(out->col.size());
    }
    return finish_csr(out);
}

int decompress_pattern(int64_t n, const PatternFormat& p, Csr* out) {
    const int nu = static_cast<int>(p.uoff.size());
    if (nu > kMaxUnion || p.words != (nu + 4) / 4 || (int64_t)p.rec.size() != n * p.words ||
        p.pmask.size() > (size_t)kMaxPatterns || p.dict.size() > 254)
        return corrupt("pattern table sizes");
    for (size_t q = 0; q < p.pmask.size(); ++q)
        if (nu < 32 && (p.pmask[q] >> nu) != 0) return corrupt("pattern mask outside the union");
    out->n = n;
    out->rowptr.assign(n + 1, 0);
    out->col.clear();
    out->val.clear();
    const uint32_t ndict = static_cast<uint32_t>(p.dict.size());
    for (int64_t r = 0; r < n; ++r) {
        const uint8_t* b = reinterpret_cast<const uint8_t*>(&p.rec[static_cast<size_t>(r) * p.words]);
        const uint32_t pat = b[nu];
        if (pat >= p.pmask.size()) return corrupt("pattern number out of range");
        for (int u = 0; u < nu; ++u) {
            if (!((p.pmask[pat] >> u) & 1u)) {
                if (b[u] != ndict) return corrupt("absent slot without the absent code");
                continue;
            }
            const int64_t c = r + p.uoff[u];
            if (c < 0 || c >= n) return corrupt("pattern column out of range");
            if (b[u] >= ndict) return corrupt("value code out of range");
            out->col.push_back(static_cast<int32_t>(c));
            out->val.push_back(p.dict[b[u]]);
        }
        out->rowptr[r + 1] = static_cast<int64_t>(out->col.size());
    }
    return finish_csr(out);
}

// Data+Index Table -> CSR: walk each row's value groups (Listing 1), then
// put the entries back in column order.  Every index is checked.
int decompress_dit(int64_t n, const DitFormat& d, Csr* out) {
    const int nv = static_cast<int>(d.dict.size());
    const int64_t ntypes = static_cast<int64_t>(d.tlen.size());
    const int64_t stride = std::max<int32_t>(d.maxlen, 1);
    if (static_cast<int64_t>(d.type.size()) != n || static_cast<int64_t>(d.ends.size()) != n * nv ||
        static_cast<int64_t>(d.disp.size()) != ntypes * stride)
        return corrupt("Data+Index Table sizes");
    out->n = n;
    out->rowptr.assign(static_cast<size_t>(n) + 1, 0);
    out->col.clear();
    out->val.clear();
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t r = 0; r < n; ++r) {
        const int64_t t = d.type[r];
        if (t >= ntypes) return corrupt("row type");
        row.clear();
        int idx = 0;
        for (int v = 0; v < nv; ++v) {
            const int end = d.ends[static_cast<size_t>(v) * n + r];
            if (end < idx || end > d.tlen[t]) return corrupt("value group end");
            for (; idx < end; ++idx) {
                const int64_t c = r + d.disp[t * stride + idx];
                if (c < 0 || c >= n) return corrupt("column outside the matrix");
                row.emplace_back(static_cast<int32_t>(c), d.dict[v]);
            }
        }
        if (idx != d.tlen[t]) return corrupt("row length");
        std::sort(row.begin(), row.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        for (const auto& e : row) {
            out->col.push_back(e.first);
            out->val.push_back(e.second);
        }
        out->rowptr[r + 1] = static_cast<int64_t>(out->col.size());
    }
    return finish_csr(out);
}

// Data Table -> CSR: walk each row's value groups over S_i, then put the
// entries back in column order.  Every index is checked.
int decompress_data_table(int64_t n, const DataTableFormat& d, Csr* out) {
    const int nv = static_cast<int>(d.dict.size());
    const int64_t ns = (n + kSliceRows - 1) / kSliceRows;
    if (d.nslices != ns || static_cast<int64_t>(d.slice_w.size()) != ns ||
        static_cast<int64_t>(d.slice_off.size()) != ns + 1 || static_cast<int64_t>(d.ends.size()) != n * nv ||
        d.slice_off[0] != 0)
        return corrupt("Data Table sizes");
    for (int64_t s = 0; s < ns; ++s)
        if (d.slice_off[s + 1] - d.slice_off[s] != int64_t(d.slice_w[s]) * kSliceRows) return corrupt("Data Table slices");
    if (d.slice_off[ns] != static_cast<int64_t>(d.S.size())) return corrupt("Data Table column list size");
    out->n = n;
    out->rowptr.assign(static_cast<size_t>(n) + 1, 0);
    out->col.clear();
    out->val.clear();
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t r = 0; r < n; ++r) {
        const int64_t s = r / kSliceRows, l = r % kSliceRows;
        row.clear();
        int idx = 0;
        for (int v = 0; v < nv; ++v) {
            const int end = d.ends[static_cast<size_t>(v) * n + r];
            if (end < idx || end > d.slice_w[s]) return corrupt("value group end");
            for (; idx < end; ++idx) {
                const int64_t c = d.S[d.slice_off[s] + int64_t(idx) * kSliceRows + l];
                if (c < 0 || c >= n) return corrupt("column outside the matrix");
                row.emplace_back(static_cast<int32_t>(c), d.dict[v]);
            }
        }
        std::sort(row.begin(), row.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        for (const auto& e : row) {
            out->col.push_back(e.first);
            out->val.push_back(e.second);
        }
        out->rowptr[r + 1] = static_cast<int64_t>(out->col.size());
    }
    return finish_csr(out);
}

int decompress_delta(int64_t n, const DeltaFormat& d, Csr* out) {
    if (d.nslices != (n + kSliceRows - 1) / kSliceRows || (int64_t)d.hdr.size() != d.nslices || d.dict.size() > 254)
        return corrupt("delta slice table size");
    out->n = n;
    out->rowptr.assign(n + 1, 0);
    out->col.clear();
    out->val.clear();
    const uint32_t nd = static_cast<uint32_t>(d.dict.size());
    for (int64_t s = 0; s < d.nslices; ++s) {
        const DeltaSlice h = d.hdr[s];
        const bool craw = h.flags & kSliceColRaw, c24 = h.flags & kSliceCol24;
        const bool vraw = h.flags & kSliceValRaw, vloc = h.flags & kSliceValLocal;
        if ((h.flags & ~15u) || (craw && c24) || (vraw && vloc)) return corrupt("slice flags");
        if (h.w > 255 || h.off % 16 != 0) return corrupt("slice header");
        const DeltaParts pt = delta_parts(h.w, h.flags);
        if (h.off + pt.local > d.payload.size()) return corrupt("slice payload bounds");
        const uint8_t* base = d.payload.data() + h.off;
        uint32_t nloc = 0;
        if (vloc) {
            if (h.off + pt.local + 16 > d.payload.size()) return corrupt("slice payload bounds");
            std::memcpy(&nloc, base + pt.local, 4);
            if (nloc > 256 - nd || h.off + pt.local + 16 + 8 * uint64_t(nloc) > d.payload.size())
                return corrupt("slice value table");
        }
        for (int64_t r = s * kSliceRows; r < std::min(n, (s + 1) * kSliceRows); ++r) {
            const int64_t l = r - s * kSliceRows;
            const uint32_t len = base[l];
            if (len > h.w) return corrupt("row length above slice width");
            for (uint32_t t = 0; t < len; ++t) {
                const int64_t slot = int64_t(t) * kSliceRows + l;
                int64_t c;
                if (craw) {
                    int32_t c32;
                    std::memcpy(&c32, base + pt.cols + 4 * slot, 4);
                    c = c32;
                } else {
                    int16_t lo;
                    std::memcpy(&lo, base + pt.cols + 2 * slot, 2);
                    int64_t dlt = lo;
                    if (c24) dlt = int64_t(int8_t(base[pt.hi + slot])) * 65536 + int64_t(uint16_t(lo));
                    c = r + dlt;
                }
                if (c < 0 || c >= n) return corrupt("delta column out of range");
                double v;
                if (vraw) {
                    std::memcpy(&v, base + pt.vals + 8 * slot, 8);
                } else {
                    const uint32_t cv = base[pt.vals + slot];
                    if (cv < nd) v = d.dict[cv];
                    else if (vloc && cv - nd < nloc) std::memcpy(&v, base + pt.local + 16 + 8 * (cv - nd), 8);
                    else return corrupt("value code out of range");
                }
                out->col.push_back(static_cast<int32_t>(c));
                out->val.push_back(v);
            }
            out->rowptr[r + 1] = static_cast<int64_t>(out->col.size());
        }
    }
    return finish_csr(out);
}

uint64_t checksum_of(const spmv_mat_s& m) {
    Fnv f;
    f.pod(m.fmt);
    f.pod(m.n);
    f.pod(m.nnz);
    if (m.fmt == SPMV_FMT_ELL) {
        f.vec(m.ell.slice_off);
        f.vec(m.ell.slice_w);
        f.vec(m.ell.val);
        f.vec(m.ell.col);
    } else if (m.fmt == SPMV_FMT_PATTERN) {
        f.vec(m.pat.dict);
        f.vec(m.pat.uoff);
        f.vec(m.pat.pmask);
        f.pod(m.pat.words);
        f.vec(m.pat.rec);
    } else if (m.fmt == SPMV_FMT_DATA_TABLE) {
        f.vec(m.dt.dict);
        f.vec(m.dt.slice_off);
        f.vec(m.dt.slice_w);
        f.vec(m.dt.S);
        f.vec(m.dt.ends);
    } else if (m.fmt == SPMV_FMT_DIT) {
        f.vec(m.dit.dict);
        f.pod(m.dit.maxlen);
        f.vec(m.dit.disp);
        f.vec(m.dit.tlen);
        f.vec(m.dit.type);
        f.vec(m.dit.ends);
    } else {
        f.vec(m.dlt.dict);
        f.vec(m.dlt.hdr);
        f.vec(m.dlt.payload);
    }
    return f.h;
}

// ------------------------------------------------------ export / import ---
// Stream: "SPMVC\0v1" | fmt | n | nnz | checksum | arrays, each as
// (uint64 element count, raw bytes).
namespace {
struct Writer {
    uint8_t* p;
    size_t pos = 0, cap;
    bool dry;
    void put(const void* src, size_t len) {
        if (!dry && pos + len <= cap) std::memcpy(p + pos, src, len);
        pos += len;
    }
    template <class T> void pod(const T& v) { put(&v, sizeof(T)); }
    template <class T> void vec(const std::vector<T>& v) {
        const uint64_t k = v.size();
        pod(k);
        if (k) put(v.data(), k * sizeof(T));
    }
};
struct Reader {
    const uint8_t* p;
    size_t pos = 0, len;
    bool ok = true;
    void get(void* dst, size_t l) {
        if (!ok || pos + l > len) { ok = false; return; }
        std::memcpy(dst, p + pos, l);
        pos += l;
    }
    template <class T> void pod(T* v) { get(v, sizeof(T)); }
    template <class T> void vec(std::vector<T>* v) {
        uint64_t k = 0;
        pod(&k);
        if (!ok || k > (len - pos) / sizeof(T)) { ok = false; return; }
        v->resize(k);
        if (k) get(v->data(), k * sizeof(T));
    }
};
const char kTag[8] = {'S', 'P', 'M', 'V', 'C', 0, 'v', '1'};
}  // namespace

int export_stream(const spmv_mat_s& m, void* buf, size_t* len) {
    if (m.fmt == SPMV_FMT_DIT) return fail(SPMV_EUNSUPPORTED, "the Data+Index Table format has no stream form");
    if (m.fmt == SPMV_FMT_DATA_TABLE) return fail(SPMV_EUNSUPPORTED, "the Data Table format has no stream form");
    Writer w{static_cast<uint8_t*>(buf), 0, buf ? *len : 0, buf == nullptr};
    w.put(kTag, 8);
    w.pod(m.fmt);
    w.pod(m.n);
    w.pod(m.nnz);
    w.pod(m.checksum);
    if (m.fmt == SPMV_FMT_ELL) {
        w.pod(m.ell.nslices);
        w.vec(m.ell.slice_off);
        w.vec(m.ell.slice_w);
        w.vec(m.ell.val);
        w.vec(m.ell.col);
    } else if (m.fmt == SPMV_FMT_PATTERN) {
        w.vec(m.pat.dict);
        w.vec(m.pat.uoff);
        w.vec(m.pat.pmask);
        w.pod(m.pat.words);
        w.vec(m.pat.rec);
    } else {
        w.pod(m.dlt.nslices);
        w.vec(m.dlt.dict);
        w.vec(m.dlt.hdr);
        w.vec(m.dlt.payload);
    }
    if (!buf) {
        *len = w.pos;
        return SPMV_OK;
    }
    if (w.pos > *len) return fail(SPMV_EINVAL, "export buffer too small");
    *len = w.pos;
    return SPMV_OK;
}

int import_stream(const void* buf, size_t len, spmv_mat_s* m) {
    Reader r{static_cast<const uint8_t*>(buf), 0, len};
    char tag[8];
    r.get(tag, 8);
    if (!r.ok || std::memcmp(tag, kTag, 8) != 0) return corrupt("bad tag");
    uint64_t sum = 0;
    r.pod(&m->fmt);
    r.pod(&m->n);
    r.pod(&m->nnz);
    r.pod(&sum);
    if (!r.ok || m->n < 0 || m->n >= (int64_t(1) << 31)) return corrupt("header");
    if (m->fmt == SPMV_FMT_ELL) {
        r.pod(&m->ell.nslices);
        r.vec(&m->ell.slice_off);
        r.vec(&m->ell.slice_w);
        r.vec(&m->ell.val);
        r.vec(&m->ell.col);
        if (r.ok && m->ell.val.size() != m->ell.col.size()) return corrupt("ELL array sizes");
    } else if (m->fmt == SPMV_FMT_PATTERN) {
        r.vec(&m->pat.dict);
        r.vec(&m->pat.uoff);
        r.vec(&m->pat.pmask);
        r.pod(&m->pat.words);
        r.vec(&m->pat.rec);
    } else if (m->fmt == SPMV_FMT_DELTA) {
        r.pod(&m->dlt.nslices);
        r.vec(&m->dlt.dict);
        r.vec(&m->dlt.hdr);
        r.vec(&m->dlt.payload);
    } else {
        return corrupt("format");
    }
    if (!r.ok || r.pos != len) return corrupt("truncated or trailing bytes");
    m->checksum = checksum_of(*m);
    if (m->checksum != sum) return corrupt("checksum mismatch");
    return SPMV_OK;
}

}  // namespace spmvc
