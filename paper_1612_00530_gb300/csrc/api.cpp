// C ABI of the compressed-SpMV library (declared in include/spmvc.h).
// Handles own host copies of their stored form and, after the first device
// call, device copies.  All errors come back as status codes with a
// thread-local message; nothing throws across the boundary.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>

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
void derive_fast_order(int64_t n, PatternFormat* p);

namespace {
thread_local std::string g_last_error;
constexpr uint32_t kMagic = 0x5350564du;
constexpr int kPartialWords = 152 * 64 + 64;
constexpr int64_t kTileOverhang = 4096;  // rows a staged tile may reach past n
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int status, const std::string& msg) {
    g_last_error = msg;
    return status;
}

namespace {

bool valid(spmv_mat_t m) { return m != nullptr && m->magic == kMagic; }

int cuda_fail(cudaError_t e, const char* what) {
    return fail(SPMV_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SPMVC_CUDA(call)                                     \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

template <class T>
int dev_copy(spmv_mat_s* m, const T* src, size_t count, T** dst) {
    *dst = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(SPMV_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    m->dev_allocs.push_back(p);
    if (count && src) {
        e = cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    } else {
        e = cudaMemset(p, 0, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    }
    *dst = static_cast<T*>(p);
    return SPMV_OK;
}

void free_device(spmv_mat_s* m) {
    for (void* p : m->dev_allocs) cudaFree(p);
    m->dev_allocs.clear();
    if (m->own_stream) cudaStreamDestroy(m->own_stream);
    m->own_stream = nullptr;
    if (m->h2d_stream) cudaStreamDestroy(m->h2d_stream);
    if (m->d2h_stream) cudaStreamDestroy(m->d2h_stream);
    m->h2d_stream = m->d2h_stream = nullptr;
    for (cudaEvent_t e : m->host_events) cudaEventDestroy(e);
    m->host_events.clear();
    m->device = -1;
    m->d_ell_val32 = nullptr;
    m->d_hx = m->d_hy = nullptr;
}

// Autotuner cache: (device name, n, nnz, union size) -> rows per thread of
// the staged FAST kernel.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;          // staged kernel: threads * 16 + rows per thread
std::map<std::string, int> g_tune_variant;  // FAST kernel variant

std::string tune_key(const spmv_mat_s* m) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    return std::string(prop.name) + "|" + std::to_string(m->n) + "|" + std::to_string(m->nnz) + "|" +
           std::to_string(m->pat.uoff.size());
}

int tuned_variant(const spmv_mat_s* m, int fallback) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_variant.find(tune_key(m));
    return it == g_tune_variant.end() ? fallback : it->second;
}

// (threads, rows per thread) of the staged kernel chosen by the autotuner
std::pair<int, int> tuned_stage_shape(const spmv_mat_s* m, int threads, int rows_per_thread) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(tune_key(m));
    if (it == g_tune.end()) return {threads, rows_per_thread};
    return {it->second / 16, it->second % 16};
}

// First device use: copy the stored form to the current device.
int ensure_device(spmv_mat_s* m) {
    int dev = 0;
    SPMVC_CUDA(cudaGetDevice(&dev));
    if (m->device >= 0) {
        if (dev != m->device) return fail(SPMV_EINVAL, "matrix lives on another device");
        return SPMV_OK;
    }
    int st;
    int32_t zero = 0;
    if ((st = dev_copy(m, &zero, 1, &m->d_err))) return st;
    std::vector<uint32_t> zeros(kPartialWords, 0u);
    if ((st = dev_copy(m, zeros.data(), zeros.size(), &m->d_scratch_words))) return st;
    m->scratch_words = kPartialWords;
    if (!m->perm.empty()) {
        if ((st = dev_copy(m, m->perm.data(), m->perm.size(), &m->d_perm))) return st;
        if ((st = dev_copy<double>(m, nullptr, static_cast<size_t>(m->n), &m->d_xp))) return st;
        if ((st = dev_copy<double>(m, nullptr, static_cast<size_t>(m->n), &m->d_yp))) return st;
    }
    if (m->fmt == SPMV_FMT_ELL) {
        EllView& v = m->ell_view;
        v.n = m->n;
        v.nslices = m->ell.nslices;
        int64_t* so;
        int32_t *sw, *col;
        double* val;
        if ((st = dev_copy(m, m->ell.slice_off.data(), m->ell.slice_off.size(), &so))) return st;
        if ((st = dev_copy(m, m->ell.slice_w.data(), m->ell.slice_w.size(), &sw))) return st;
        if ((st = dev_copy(m, m->ell.val.data(), m->ell.val.size(), &val))) return st;
        if ((st = dev_copy(m, m->ell.col.data(), m->ell.col.size(), &col))) return st;
        v.slice_off = so;
        v.slice_w = sw;
        v.val = val;
        v.col = col;
        v.val32 = nullptr;
    } else if (m->fmt == SPMV_FMT_PATTERN) {
        const PatternFormat& p = m->pat;
        PatternView& v = m->pat_view;
        std::memset(&v, 0, sizeof(v));
        v.n = m->n;
        v.nu = static_cast<int32_t>(p.uoff.size());
        v.words = p.words;
        v.dict_size = static_cast<int32_t>(p.dict.size());
        v.npat = static_cast<int32_t>(p.pmask.size());
        for (int u = 0; u < v.nu; ++u) v.uoff[u] = p.uoff[u];
        for (int q = 0; q < v.npat; ++q) v.pmask[q] = p.pmask[q];
        const int64_t n = m->n;
        const int q16 = p.words / 4, rem = p.words % 4;
        std::vector<uint32_t> plane;
        auto upload_plane = [&](int first, int width, const void** out) -> int {
            plane.assign(static_cast<size_t>(n) * width, 0u);
            for (int64_t r = 0; r < n; ++r)
                for (int k = 0; k < width; ++k) plane[r * width + k] = p.rec[r * p.words + first + k];
            uint32_t* d;
            int s2 = dev_copy(m, plane.data(), plane.size(), &d);
            *out = d;
            return s2;
        };
        const void* ptr;
        if (q16 >= 1) { if ((st = upload_plane(0, 4, &ptr))) return st; v.p16a = static_cast<const uint4*>(ptr); }
        if (q16 >= 2) { if ((st = upload_plane(4, 4, &ptr))) return st; v.p16b = static_cast<const uint4*>(ptr); }
        if (rem >= 2) { if ((st = upload_plane(4 * q16, 2, &ptr))) return st; v.p8 = static_cast<const uint2*>(ptr); }
        if (rem & 1) { if ((st = upload_plane(p.words - 1, 1, &ptr))) return st; v.p4 = static_cast<const uint32_t*>(ptr); }
        {
            std::vector<uint32_t> pm(32, 0u);
            for (int q = 0; q < v.npat; ++q) pm[q] = p.pmask[q];
            uint32_t* d;
            if ((st = dev_copy(m, pm.data(), pm.size(), &d))) return st;
            v.pmask_dev = d;
        }
        std::vector<double> dict(p.dict);
        std::vector<float> dict32;
        for (double d : dict) dict32.push_back(static_cast<float>(d));
        double* dd;
        float* df;
        if ((st = dev_copy(m, dict.data(), dict.size(), &dd))) return st;
        if ((st = dev_copy(m, dict32.data(), dict32.size(), &df))) return st;
        v.dict = dd;
        v.dict32 = df;
        uint8_t tbl[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (p.fast_ok)
            for (size_t k = 0; k < p.mult.size() && k < 7; ++k) tbl[k] = static_cast<uint8_t>(int8_t(p.mult[k]));
        std::memcpy(&v.mult_lo, tbl, 4);
        std::memcpy(&v.mult_hi, tbl + 4, 4);
        v.mult_exp = p.mult_exp;
        v.rtype = nullptr;              // row types are uploaded on request (variant 9)
        v.rtypes = nullptr;
        v.ntypes = 0;
        v.err = m->d_err;
        // the dominant record (most frequent; its slots must all be present)
        v.dom_ok = 0;
        if (n > 0) {
            std::map<std::vector<uint32_t>, int64_t> freq;
            std::vector<uint32_t> key(p.words);
            const int64_t step = std::max<int64_t>(1, n / 65536);   // a sample is enough to find it
            for (int64_t r = 0; r < n; r += step) {
                std::copy(&p.rec[r * p.words], &p.rec[r * p.words] + p.words, key.begin());
                freq[key]++;
            }
            const auto best = std::max_element(freq.begin(), freq.end(),
                                               [](const auto& a2, const auto& b2) { return a2.second < b2.second; });
            const uint8_t* bytes = reinterpret_cast<const uint8_t*>(best->first.data());
            bool all_present = true;
            for (int u = 0; u < v.nu; ++u) all_present = all_present && bytes[u] < p.dict.size();
            if (all_present) {
                v.dom_ok = 1;
                for (int k2 = 0; k2 < p.words; ++k2) v.dom_w[k2] = best->first[k2];
                for (int u = 0; u < v.nu; ++u) {
                    v.dom_m[u] = p.fast_ok ? p.mult[bytes[u]] : 0;
                    v.dom_v32[u] = static_cast<float>(p.dict[bytes[u]]);
                }
            }
        }
        v.dom_uni = 0;
        if (v.dom_ok && p.fast_ok && v.nu == 27 && p.uoff[13] == 0) {
            bool uni = true;
            for (int u = 0; u < 27; ++u)
                if (u != 13 && v.dom_m[u] != v.dom_m[0]) uni = false;
            if (uni) {
                v.dom_uni = 1;
                v.dom_mo = v.dom_m[0];
                v.dom_mc = v.dom_m[13];
            }
        }
        // runs of consecutive displacements, all of one length
        v.run_len = 0;
        for (int len : {3}) {
            bool ok = v.nu > 0 && v.nu % len == 0;
            for (int u = 0; ok && u < v.nu; ++u)
                if (u % len != 0 && p.uoff[u] != p.uoff[u - 1] + 1) ok = false;
            for (int u = len; ok && u < v.nu; u += len)
                if (p.uoff[u] == p.uoff[u - 1] + 1) ok = false;  // runs are maximal
            if (ok) v.run_len = len;
        }
        m->stage_ok = false;
        m->fast_variant = 0;
        if (p.fast_ok && stage_supported(v.nu)) {
            // fixed-point copy of x with zero guard zones as wide as the
            // largest displacement
            // leading guard: the largest displacement plus the element of
            // padding an odd window start adds; trailing guard: the same plus
            // the overhang of the last shared-memory tile (at most 2048 rows)
            int64_t guard = 0;
            for (int32_t d : p.uoff) guard = std::max<int64_t>(guard, d < 0 ? -int64_t(d) : int64_t(d));
            guard = (guard + 2 + 15) / 16 * 16;
            int2* xf;
            if ((st = dev_copy<int2>(m, nullptr, static_cast<size_t>(n + 2 * guard + kTileOverhang), &xf))) return st;
            m->d_xfixed = xf;
            m->xfixed_guard = guard;
            m->fast_variant = tuned_variant(m, 2);
        }
        if (stage_supported(v.nu)) {
            const std::pair<int, int> prefer = tuned_stage_shape(m, 512, 4);
            for (std::pair<int, int> sh : {prefer, std::make_pair(512, 4), std::make_pair(512, 2), std::make_pair(512, 1)})
                if (make_stage_plan(p.uoff, sh.second, sh.first, 12288, &m->stage)) { m->stage_ok = true; break; }
        }
        // persistent double-buffered kernel: 1024-row tiles, two buffers must fit
        m->async_ok = false;
        if (p.fast_ok && v.run_len == 3 && v.nu == 27 && v.words == 7 &&
            make_stage_plan(p.uoff, 1, 1024, 12288, &m->async_plan)) {
            const size_t xbytes = (size_t(m->async_plan.elems) * 8 + 15) / 16 * 16;
            const size_t xpbytes = (size_t(std::max(m->async_plan.elems, m->async_plan.elems_padded)) * 8 + 15) / 16 * 16;
            m->async_ok = 2 * (std::max(xbytes, xpbytes) + 1024 * 28) <= 220 * 1024;
        }
        {
            int d = 0, sms = 0;
            cudaGetDevice(&d);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
            m->num_sms = sms > 0 ? sms : 152;
        }
        m->zplan_ok = false;
        if (p.fast_ok && v.run_len == 3 && v.nu == 27 && v.words == 7) {
            const std::pair<int, int> zs = tuned_stage_shape(m, 256, 2);
            for (std::pair<int, int> sh : {zs, std::make_pair(256, 2)})
                if (make_zplan(p.uoff, m->n, sh.second, sh.first, m->num_sms, &m->zplan) &&
                    zmarch_supported(m->zplan)) {
                    m->zplan_ok = true;
                    break;
                }
        }
        // z-block kernel: only when the autotuner picked it for a matrix of
        // this shape (planes a CTA recorded with the pick)
        m->zbplan_ok = false;
        if (m->fast_variant == 10 && p.fast_ok && v.run_len == 3 && v.nu == 27 && v.words == 7)
            m->zbplan_ok = make_zblock_plan(p.uoff, m->n, tuned_stage_shape(m, 256, 3).second, 256, &m->zbplan);
        // TMA z-marching kernel: its plan and the table of the record each
        // boundary class of grid position implies
        m->tplan_ok = false;
        m->tplan_cg_ok = false;
        {
            std::vector<uint32_t> tab;
            // lines a compute thread's tile and CTAs an SM: the autotuner's
            // pick for matrices of this shape (ty + 4 (ctas - 1)), else 1 and 1
            const int code = m->fast_variant == 11 ? tuned_stage_shape(m, 0, 1).second : 1;
            const int ty = code & 3, ctas = 1 + (code >> 2);
            if (make_tma_plan(p, v, m->n, m->num_sms, ty, ctas, &m->tplan, &tab) ||
                make_tma_plan(p, v, m->n, m->num_sms, 1, 1, &m->tplan, &tab) ||
                make_tma_plan(p, v, m->n, m->num_sms, 2, 1, &m->tplan, &tab)) {
                uint32_t* dt;
                if ((st = dev_copy(m, tab.data(), tab.size(), &dt))) return st;
                m->tplan.expected = dt;
                m->tplan_ok = true;
                // the CG step's product, which also forms p.q, runs faster
                // with two CTAs an SM (its binary64 work then overlaps the
                // other CTA's steps); the plain product with one
                m->tplan_cg_ok = make_tma_plan(p, v, m->n, m->num_sms, 1, 2, &m->tplan_cg, &tab);
                m->tplan_cg.expected = dt;
            }
        }
        // TMA SpMM plans, sharing the expected-record table
        {
            const uint32_t* table = m->tplan_ok ? m->tplan.expected : nullptr;
            bool any = false;
            for (int ki = 0; ki < 2; ++ki)
                for (int c = 0; c < 3; ++c) {
                    m->splan_ok[ki][c] = make_tma_spmm_plan(p, v, m->n, m->num_sms, ki ? 8 : 4, c + 1, &m->splan[ki][c]);
                    any = any || m->splan_ok[ki][c];
                }
            if (any && !table) {
                std::vector<uint32_t> tab;
                expected_records(p, v, &tab);
                uint32_t* dt;
                if ((st = dev_copy(m, tab.data(), tab.size(), &dt))) return st;
                table = dt;
            }
            for (int ki = 0; ki < 2; ++ki)
                for (int c = 0; c < 3; ++c) m->splan[ki][c].expected = table;
        }
        m->f32plan_ok = make_tma_f32_plan(p, v, m->n, m->num_sms, &m->f32plan);
        if (m->fast_variant == 11 && !m->tplan_ok) m->fast_variant = 1;
        if (m->fast_variant == 7 && !m->zplan_ok) m->fast_variant = 1;
        if (m->fast_variant == 10 && !m->zbplan_ok) m->fast_variant = 1;
        if ((m->fast_variant == 4 || m->fast_variant == 5) && !m->async_ok) m->fast_variant = 2;
        if (m->fast_variant == 9) m->fast_variant = 6;   // row types are built on request only
        if ((m->fast_variant == 6 || m->fast_variant == 8) && !(m->stage_ok && rstage_supported(m->stage)))
            m->fast_variant = 1;
        if ((m->fast_variant == 1 || m->fast_variant == 3) && !m->stage_ok) m->fast_variant = m->d_xfixed ? 2 : 0;
        if (m->fast_variant == 0 && m->stage_ok) m->fast_variant = 1;
    } else if (m->fmt == SPMV_FMT_DATA_TABLE) {
        const DataTableFormat& d = m->dt;
        DataTableView& v = m->dt_view;
        v.n = m->n;
        v.nslices = d.nslices;
        v.nv = static_cast<int32_t>(d.dict.size());
        int64_t* so;
        uint8_t *sw, *en;
        int32_t* S;
        double* dd;
        if ((st = dev_copy(m, d.slice_off.data(), d.slice_off.size(), &so))) return st;
        if ((st = dev_copy(m, d.slice_w.data(), d.slice_w.size(), &sw))) return st;
        if ((st = dev_copy(m, d.S.data(), d.S.size(), &S))) return st;
        if ((st = dev_copy(m, d.ends.data(), d.ends.size(), &en))) return st;
        if ((st = dev_copy(m, d.dict.data(), d.dict.size(), &dd))) return st;
        v.slice_off = so;
        v.slice_w = sw;
        v.S = S;
        v.ends = en;
        v.dict = dd;
        v.err = m->d_err;
    } else if (m->fmt == SPMV_FMT_DIT) {
        const DitFormat& d = m->dit;
        DitView& v = m->dit_view;
        v.n = m->n;
        v.nv = static_cast<int32_t>(d.dict.size());
        v.ntypes = static_cast<int32_t>(d.tlen.size());
        v.maxlen = std::max<int32_t>(d.maxlen, 1);
        uint8_t *ty, *en;
        int32_t* ds;
        double* dd;
        if ((st = dev_copy(m, d.type.data(), d.type.size(), &ty))) return st;
        if ((st = dev_copy(m, d.ends.data(), d.ends.size(), &en))) return st;
        if ((st = dev_copy(m, d.disp.data(), d.disp.size(), &ds))) return st;
        if ((st = dev_copy(m, d.dict.data(), d.dict.size(), &dd))) return st;
        v.type = ty;
        v.ends = en;
        v.disp = ds;
        v.dict = dd;
        v.err = m->d_err;
    } else {
        const DeltaFormat& d = m->dlt;
        DeltaView& v = m->dlt_view;
        v.n = m->n;
        v.nslices = d.nslices;
        v.dict_size = static_cast<int32_t>(d.dict.size());
        DeltaSlice* h;
        uint8_t* pl;
        double* dd;
        float* df;
        std::vector<float> dict32;
        for (double x : d.dict) dict32.push_back(static_cast<float>(x));
        if ((st = dev_copy(m, d.hdr.data(), d.hdr.size(), &h))) return st;
        if ((st = dev_copy(m, d.payload.data(), d.payload.size(), &pl))) return st;
        if ((st = dev_copy(m, d.dict.data(), d.dict.size(), &dd))) return st;
        if ((st = dev_copy(m, dict32.data(), dict32.size(), &df))) return st;
        v.hdr = h;
        v.payload = pl;
        v.dict = dd;
        v.dict32 = df;
        v.err = m->d_err;
    }
    m->device = dev;
    return SPMV_OK;
}

int new_handle(spmv_mat_t* out, spmv_mat_s** m) {
    if (!out) return fail(SPMV_EINVAL, "null output handle");
    *out = nullptr;
    *m = new (std::nothrow) spmv_mat_s();
    if (!*m) return fail(SPMV_ENOMEM, "host allocation failed");
    (*m)->magic = kMagic;
    return SPMV_OK;
}

void stats_from_csr(spmv_mat_s* m, const Csr& c) {
    m->n = c.n;
    m->nnz = c.nnz();
    m->max_row_nnz = 0;
    m->bandwidth = 0;
    for (int64_t i = 0; i < c.n; ++i) {
        m->max_row_nnz = std::max<int32_t>(m->max_row_nnz, static_cast<int32_t>(c.rowptr[i + 1] - c.rowptr[i]));
        for (int64_t k = c.rowptr[i]; k < c.rowptr[i + 1]; ++k)
            m->bandwidth = std::max<int64_t>(m->bandwidth, c.col[k] > i ? c.col[k] - i : i - c.col[k]);
    }
}

int finish_plain(spmv_mat_s* m, spmv_mat_t* out) {
    stats_from_csr(m, m->csr);
    m->fmt = SPMV_FMT_ELL;
    int st = pack_ell(m->csr, &m->ell);
    if (st) { delete m; return st; }
    m->checksum = checksum_of(*m);
    *out = m;
    return SPMV_OK;
}

// The stored matrix as CSR (B = P A P^T for a reordered handle).
int stored_csr(spmv_mat_s* a, Csr* c) {
    if (a->fmt == SPMV_FMT_ELL && a->csr.n == a->n && !a->csr.rowptr.empty()) {
        *c = a->csr;
        return SPMV_OK;
    }
    if (a->fmt == SPMV_FMT_ELL) return decompress_ell(a->n, a->ell, c);
    if (a->fmt == SPMV_FMT_PATTERN) return decompress_pattern(a->n, a->pat, c);
    if (a->fmt == SPMV_FMT_DIT) return decompress_dit(a->n, a->dit, c);
    if (a->fmt == SPMV_FMT_DATA_TABLE) return decompress_data_table(a->n, a->dt, c);
    return decompress_delta(a->n, a->dlt, c);
}

// A itself, in its own numbering.
int to_csr(spmv_mat_s* a, Csr* c) {
    int st = stored_csr(a, c);
    if (st || a->perm.empty()) return st;
    Csr orig;
    unpermute_csr(*c, a->perm, &orig);
    *c = std::move(orig);
    return SPMV_OK;
}

cudaStream_t as_stream(spmv_stream_t s) { return static_cast<cudaStream_t>(s); }

// Variant 11 needs x and y 16-byte aligned (TMA box, bulk store); other
// vectors take the direct FAST kernel.
cudaError_t launch_tma_or_direct(spmv_mat_s* A, const TmaPlan& tp, const double* x, double* y, cudaStream_t s) {
    const cudaError_t e = launch_pattern_fast_tma(A->pat_view, tp, x, y, s);
    if (e != cudaErrorNotSupported) return e;
    return launch_pattern_fast_f64(A->pat_view, x, y, A->d_scratch_words, s);
}

// The stored matrix's product on device vectors (no permutation).
int apply_stored(spmv_mat_s* A, const double* x, double* y, cudaStream_t s) {
    cudaError_t e;
    if (A->fmt == SPMV_FMT_ELL) e = launch_ell_f64(A->ell_view, x, y, s);
    else if (A->fmt == SPMV_FMT_PATTERN)
        e = A->order != SPMV_ORDER_FAST ? launch_pattern_col_f64(A->pat_view, x, y, s)
            : A->fast_variant == 5 ? launch_pattern_fast_async_x(A->pat_view, A->async_plan, x, y, A->d_scratch_words,
                                                                 A->d_xfixed, A->xfixed_guard, A->num_sms, s)
            : A->fast_variant == 4 ? launch_pattern_fast_async(A->pat_view, A->async_plan, x, y, A->num_sms, s)
            : A->fast_variant == 3 ? launch_pattern_fast_xstaged(A->pat_view, A->stage, x, y, A->d_scratch_words,
                                                                 A->d_xfixed, A->xfixed_guard, s)
            : A->fast_variant == 2 ? launch_pattern_fast_x(A->pat_view, x, y, A->d_scratch_words, A->d_xfixed,
                                                           A->xfixed_guard, s)
            : A->fast_variant == 7 ? launch_pattern_fast_zmarch(A->pat_view, A->zplan, x, y, A->d_scratch_words, s)
            : A->fast_variant == 10 ? launch_pattern_fast_zblock(A->pat_view, A->zbplan, x, y, A->d_scratch_words, s)
            : A->fast_variant == 11 ? launch_tma_or_direct(A, A->tplan, x, y, s)
            : A->fast_variant == 6 ? launch_pattern_fast_rstaged(A->pat_view, A->stage, x, y, 0, s)
            : A->fast_variant == 8 ? launch_pattern_fast_rstaged(A->pat_view, A->stage, x, y, 1, s)
            : A->fast_variant == 9 ? launch_pattern_fast_rstaged(A->pat_view, A->stage, x, y, 2, s)
            : A->fast_variant == 1 ? launch_pattern_fast_staged(A->pat_view, A->stage, x, y, s)
                                   : launch_pattern_fast_f64(A->pat_view, x, y, A->d_scratch_words, s);
    else if (A->fmt == SPMV_FMT_DIT) e = launch_dit_f64(A->dit_view, x, y, s);
    else if (A->fmt == SPMV_FMT_DATA_TABLE) e = launch_data_table_f64(A->dt_view, x, y, s);
    else e = launch_delta_f64(A->dlt_view, x, y, s);
    if (e != cudaSuccess) return cuda_fail(e, "spmv launch");
    return SPMV_OK;
}


// Values registered in the pattern: the row types, built and uploaded once
// (false when the matrix has more than 256 distinct records or is not on
// the device yet).
bool ensure_row_types(spmv_mat_s* A) {
    if (A->pat_view.rtype) return true;
    if (A->fmt != SPMV_FMT_PATTERN || A->device < 0 || A->types_failed) return false;
    if (!build_row_types(A->n, &A->pat)) {
        A->types_failed = true;
        return false;
    }
    uint8_t* rt;
    uint32_t* tt;
    if (dev_copy(A, A->pat.rtype.data(), A->pat.rtype.size(), &rt)) return false;
    if (dev_copy(A, A->pat.rtypes.data(), A->pat.rtypes.size(), &tt)) return false;
    A->pat_view.rtype = rt;
    A->pat_view.rtypes = tt;
    A->pat_view.ntypes = static_cast<int32_t>(A->pat.rtypes.size() / 8);
    // the type whose record is the dominant one, if any
    A->pat_view.dom_type = -1;
    if (A->pat_view.dom_ok)
        for (int32_t t = 0; t < A->pat_view.ntypes; ++t)
            if (std::equal(A->pat.rtypes.begin() + t * 8, A->pat.rtypes.begin() + t * 8 + 7, A->pat_view.dom_w)) {
                A->pat_view.dom_type = t;
                break;
            }
    // the type of the record each boundary class of grid position implies
    // (the binary32 TMA kernel's fast rows)
    for (int c = 0; c < 64; ++c) A->f32plan.exp_type[c] = -1;
    // (an out-of-grid slot adds its value times a zero, a no-op only for a
    // finite value)
    bool dom_finite = A->pat_view.dom_ok != 0;
    for (int u = 0; u < A->pat_view.nu && dom_finite; ++u) dom_finite = std::isfinite(A->pat_view.dom_v32[u]);
    if (A->f32plan_ok && dom_finite) {
        std::vector<uint32_t> tab;
        expected_records(A->pat, A->pat_view, &tab);
        for (int c = 0; c < 64; ++c)
            for (int32_t t = 0; t < A->pat_view.ntypes; ++t)
                if (std::equal(A->pat.rtypes.begin() + t * 8, A->pat.rtypes.begin() + t * 8 + 7, tab.begin() + c * 8)) {
                    A->f32plan.exp_type[c] = int16_t(t);
                    break;
                }
    }
    return true;
}

}  // namespace
}  // namespace spmvc

using namespace spmvc;

extern "C" {

int spmv_build(const spmv_gen_desc* desc, spmv_mat_t* out) {
    if (!desc) return fail(SPMV_EINVAL, "null generator description");
    spmv_mat_s* m;
    int st = new_handle(out, &m);
    if (st) return st;
    if (desc->kind == SPMV_GEN_HPCG) st = generate_hpcg(desc->nx, desc->ny, desc->nz, &m->csr);
    else if (desc->kind == SPMV_GEN_IRREGULAR) st = generate_irregular(*desc, &m->csr);
    else st = fail(SPMV_EINVAL, "unknown generator kind");
    if (st) { delete m; return st; }
    return finish_plain(m, out);
}

int spmv_build_csr(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, spmv_mat_t* out) {
    int st = validate_csr(n, rowptr, col, val);
    if (st) return st;
    spmv_mat_s* m;
    if ((st = new_handle(out, &m))) return st;
    m->csr.n = n;
    m->csr.rowptr.assign(rowptr, rowptr + n + 1);
    m->csr.col.assign(col, col + rowptr[n]);
    m->csr.val.assign(val, val + rowptr[n]);
    return finish_plain(m, out);
}

int spmv_compress(spmv_mat_t A, const spmv_opts* opts, spmv_mat_t* out) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    spmv_opts o{SPMV_FMT_AUTO, SPMV_ORDER_COLUMN, 254, 64, 0};
    if (opts) o = *opts;
    if (o.reorder != 0 && o.reorder != 1) return fail(SPMV_EINVAL, "reorder must be 0 or 1");
    if (o.max_dict <= 0) o.max_dict = 254;
    if (o.min_count <= 0) o.min_count = 64;
    if (o.max_dict > 254) return fail(SPMV_EINVAL, "max_dict above 254");
    if (o.format != SPMV_FMT_AUTO && o.format != SPMV_FMT_PATTERN && o.format != SPMV_FMT_DELTA &&
        o.format != SPMV_FMT_DIT && o.format != SPMV_FMT_DATA_TABLE)
        return fail(SPMV_EINVAL, "compress format must be AUTO, PATTERN, DELTA, DIT or DATA_TABLE");
    Csr c;
    int st = to_csr(A, &c);
    if (st) return st;
    std::vector<int32_t> perm;
    if (o.reorder) {
        // B = P A P^T: reverse Cuthill-McKee with table-coded rows clustered
        std::vector<double> dict;
        delta_dictionary(c.val, o.max_dict, o.min_count, &dict);
        if ((st = reorder_rcm(c, dict, &perm))) return st;
        Csr b;
        permute_csr(c, perm, &b);
        c = std::move(b);
    }
    spmv_mat_s* m;
    if ((st = new_handle(out, &m))) return st;
    m->perm = std::move(perm);
    stats_from_csr(m, c);
    st = SPMV_EUNSUPPORTED;
    if (o.format == SPMV_FMT_DIT) {
        st = compress_dit(c, &m->dit);
        if (st) { delete m; return st; }
        m->fmt = SPMV_FMT_DIT;
    } else if (o.format == SPMV_FMT_DATA_TABLE) {
        st = compress_data_table(c, &m->dt);
        if (st) { delete m; return st; }
        m->fmt = SPMV_FMT_DATA_TABLE;
    } else if (o.format == SPMV_FMT_AUTO || o.format == SPMV_FMT_PATTERN) {
        st = compress_pattern(c, o.max_dict, &m->pat);
        if (st == SPMV_OK) m->fmt = SPMV_FMT_PATTERN;
        else if (o.format == SPMV_FMT_PATTERN) { delete m; return st; }
    }
    if (st != SPMV_OK) {
        m->pat = PatternFormat{};
        st = compress_delta(c, o.max_dict, o.min_count, &m->dlt);
        if (st) { delete m; return st; }
        m->fmt = SPMV_FMT_DELTA;
    }
    m->checksum = checksum_of(*m);
    *out = m;
    if (o.order != SPMV_ORDER_COLUMN) {
        st = spmv_set_order(m, o.order);
        if (st) { delete m; *out = nullptr; return st; }
    }
    return SPMV_OK;
}

int spmv_set_order(spmv_mat_t A, int32_t order) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (order == SPMV_ORDER_COLUMN) { A->order = order; return SPMV_OK; }
    if (order != SPMV_ORDER_FAST) return fail(SPMV_EINVAL, "unknown order");
    if (A->fmt != SPMV_FMT_PATTERN || !A->pat.fast_ok)
        return fail(SPMV_EUNSUPPORTED, "FAST order needs the pattern format with a small integer value table");
    A->order = order;
    return SPMV_OK;
}

int spmv_info(spmv_mat_t A, spmv_info_t* out) {
    if (!valid(A) || !out) return fail(SPMV_EINVAL, "invalid argument");
    std::memset(out, 0, sizeof(*out));
    out->n = A->n;
    out->nnz = A->nnz;
    out->format = A->fmt;
    out->order = A->order;
    out->max_row_nnz = A->max_row_nnz;
    out->checksum = A->checksum;
    out->reordered = A->perm.empty() ? 0 : 1;
    out->bandwidth = A->bandwidth;
    if (A->fmt == SPMV_FMT_ELL) {
        out->n_slices = A->ell.nslices;
        out->format_bytes = static_cast<int64_t>(A->ell.val.size() * 12 + A->ell.slice_off.size() * 8 +
                                                 A->ell.slice_w.size() * 4);
        out->padding_bytes = static_cast<int64_t>((A->ell.val.size() - A->nnz) * 12);
        out->device_bytes = out->format_bytes;
    } else if (A->fmt == SPMV_FMT_PATTERN) {
        out->dict_size = static_cast<int32_t>(A->pat.dict.size());
        out->n_patterns = static_cast<int32_t>(A->pat.pmask.size());
        out->union_size = static_cast<int32_t>(A->pat.uoff.size());
        out->record_bytes = 4 * A->pat.words;
        out->fast_eligible = A->pat.fast_ok ? 1 : 0;
        out->fast_tile_rows = A->fast_variant == 7 && A->zplan_ok ? A->zplan.rows
                            : A->fast_variant == 10 && A->zbplan_ok ? A->zbplan.rows * A->zbplan.zc
                            : A->fast_variant == 11 && A->tplan_ok ? A->tplan.C
                            : A->stage_ok ? A->stage.rows : 0;
        out->fast_variant = A->device >= 0 ? A->fast_variant : -1;
        out->fast_block_threads = A->fast_variant == 7 && A->zplan_ok ? A->zplan.threads
                                  : A->fast_variant == 10 && A->zbplan_ok ? A->zbplan.threads
                                  : A->fast_variant == 11 && A->tplan_ok ? A->tplan.threads
                                  : A->stage_ok ? A->stage.rows / A->stage.rows_per_thread : 0;
        out->row_types = static_cast<int32_t>(A->pat.rtypes.size() / 8);
        out->format_bytes = A->n * 4 * A->pat.words;
        out->padding_bytes = out->format_bytes - A->nnz - A->n;
        out->device_bytes = out->format_bytes + static_cast<int64_t>(A->pat.dict.size() * 12);
    } else if (A->fmt == SPMV_FMT_DATA_TABLE) {
        out->dict_size = static_cast<int32_t>(A->dt.dict.size());
        out->n_slices = A->dt.nslices;
        out->format_bytes = static_cast<int64_t>(A->dt.S.size() * 4 + A->dt.ends.size());
        out->record_bytes = A->n ? static_cast<int32_t>((out->format_bytes + A->n - 1) / A->n) : 0;
        out->padding_bytes = static_cast<int64_t>(A->dt.S.size() - A->nnz) * 4;
        out->device_bytes = out->format_bytes +
                            static_cast<int64_t>(A->dt.slice_off.size() * 8 + A->dt.slice_w.size() + A->dt.dict.size() * 8);
    } else if (A->fmt == SPMV_FMT_DIT) {
        out->dict_size = static_cast<int32_t>(A->dit.dict.size());
        out->n_patterns = static_cast<int32_t>(A->dit.tlen.size());
        out->union_size = A->dit.maxlen;
        out->record_bytes = 1 + out->dict_size;
        out->format_bytes = A->n * out->record_bytes;
        out->device_bytes = out->format_bytes + static_cast<int64_t>(A->dit.disp.size() * 4 + A->dit.dict.size() * 8);
    } else {
        out->dict_size = static_cast<int32_t>(A->dlt.dict.size());
        out->n_slices = A->dlt.nslices;
        for (const auto& h : A->dlt.hdr) {
            out->slices_value_raw += (h.flags & kSliceValRaw) ? 1 : 0;
            out->slices_col_raw += (h.flags & kSliceColRaw) ? 1 : 0;
            out->slices_col24 += (h.flags & kSliceCol24) ? 1 : 0;
        }
        out->format_bytes = static_cast<int64_t>(A->dlt.payload.size() + A->dlt.hdr.size() * sizeof(DeltaSlice));
        int64_t useful = A->n;  // row lengths
        for (int64_t s = 0; s < A->dlt.nslices; ++s) {
            const auto& h = A->dlt.hdr[s];
            const int64_t r0 = s * kSliceRows, r1 = std::min<int64_t>(A->n, r0 + kSliceRows);
            const int64_t per = ((h.flags & kSliceColRaw) ? 4 : (h.flags & kSliceCol24) ? 3 : 2) +
                                ((h.flags & kSliceValRaw) ? 8 : 1);
            const uint8_t* base = A->dlt.payload.data() + h.off;
            for (int64_t r = r0; r < r1; ++r) useful += per * base[r - r0];
            if (h.flags & kSliceValLocal) {   // the slice's own value table
                const DeltaParts pt = delta_parts(h.w, h.flags);
                uint32_t nloc;
                std::memcpy(&nloc, base + pt.local, 4);
                useful += 8 * int64_t(nloc);
            }
        }
        out->padding_bytes = out->format_bytes - useful - static_cast<int64_t>(A->dlt.hdr.size() * sizeof(DeltaSlice));
        out->device_bytes = out->format_bytes + static_cast<int64_t>(A->dlt.dict.size() * 12);
    }
    return SPMV_OK;
}

int spmv_decompress(spmv_mat_t A, int64_t* rowptr, int32_t* col, double* val) {
    if (!valid(A) || !rowptr || (A->nnz > 0 && (!col || !val))) return fail(SPMV_EINVAL, "invalid argument");
    Csr c;
    int st = to_csr(A, &c);
    if (st) return st;
    if (c.nnz() != A->nnz) return fail(SPMV_ECORRUPT, "decompressed nonzero count differs");
    std::memcpy(rowptr, c.rowptr.data(), sizeof(int64_t) * (A->n + 1));
    if (A->nnz) {
        std::memcpy(col, c.col.data(), sizeof(int32_t) * A->nnz);
        std::memcpy(val, c.val.data(), sizeof(double) * A->nnz);
    }
    return SPMV_OK;
}

int spmv_export(spmv_mat_t A, void* buf, size_t* len) {
    if (!valid(A) || !len) return fail(SPMV_EINVAL, "invalid argument");
    if (!A->perm.empty()) return fail(SPMV_EUNSUPPORTED, "a reordered handle has no stream form");
    return export_stream(*A, buf, len);
}

int spmv_import(const void* buf, size_t len, spmv_mat_t* out) {
    if (!buf || !out) return fail(SPMV_EINVAL, "invalid argument");
    spmv_mat_s* m;
    int st = new_handle(out, &m);
    if (st) return st;
    st = import_stream(buf, len, m);
    Csr c;
    if (!st) {
        if (m->fmt == SPMV_FMT_ELL) st = decompress_ell(m->n, m->ell, &c);
        else if (m->fmt == SPMV_FMT_PATTERN) st = decompress_pattern(m->n, m->pat, &c);
        else st = decompress_delta(m->n, m->dlt, &c);
    }
    if (!st && c.nnz() != m->nnz) st = fail(SPMV_ECORRUPT, "corrupt stream: nonzero count");
    if (st) { delete m; return st; }
    stats_from_csr(m, c);
    if (m->fmt == SPMV_FMT_ELL) m->csr = std::move(c);
    if (m->fmt == SPMV_FMT_PATTERN) derive_fast_order(m->n, &m->pat);
    *out = m;
    return SPMV_OK;
}

int spmv_apply(spmv_mat_t A, const double* x, double* y, spmv_stream_t stream) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (A->n > 0 && (!x || !y)) return fail(SPMV_EINVAL, "null vector");
    if (x == y && A->n > 0) return fail(SPMV_EINVAL, "x and y must not alias");
    int st = ensure_device(A);
    if (st) return st;
    cudaError_t e;
    const cudaStream_t s = as_stream(stream);
    if (!A->perm.empty() && A->n > 0) {
        // reordered: xp = P x, yp = B xp, y = P^T yp
        if ((e = launch_gather(A->d_perm, A->n, x, A->d_xp, s)) != cudaSuccess) return cuda_fail(e, "gather launch");
        x = A->d_xp;
        if (A->fmt == SPMV_FMT_DELTA) {   // the scatter folded into the product
            if ((e = launch_delta_f64_scatter(A->dlt_view, x, y, A->d_perm, s)) != cudaSuccess)
                return cuda_fail(e, "spmv launch");
            return SPMV_OK;
        }
        double* const y_user = y;
        y = A->d_yp;
        st = apply_stored(A, x, y, s);
        if (st) return st;
        if ((e = launch_scatter(A->d_perm, A->n, A->d_yp, y_user, s)) != cudaSuccess) return cuda_fail(e, "scatter launch");
        return SPMV_OK;
    }
    return apply_stored(A, x, y, s);
}

int spmv_permutation(spmv_mat_t A, int32_t* perm) {
    if (!valid(A) || (A->n > 0 && !perm)) return fail(SPMV_EINVAL, "invalid argument");
    if (A->perm.empty()) return fail(SPMV_EINVAL, "the handle is not reordered");
    std::memcpy(perm, A->perm.data(), sizeof(int32_t) * A->perm.size());
    return SPMV_OK;
}

int spmv_apply_host(spmv_mat_t A, const double* x, double* y) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (A->n > 0 && (!x || !y)) return fail(SPMV_EINVAL, "null vector");
    int st = ensure_device(A);
    if (st) return st;
    if (!A->own_stream) SPMVC_CUDA(cudaStreamCreateWithFlags(&A->own_stream, cudaStreamNonBlocking));
    if (!A->d_hx) {
        if ((st = dev_copy<double>(A, nullptr, A->n, &A->d_hx))) return st;
        if ((st = dev_copy<double>(A, nullptr, A->n, &A->d_hy))) return st;
    }
    const size_t bytes = sizeof(double) * A->n;
    const bool fast = A->fmt == SPMV_FMT_PATTERN && A->order == SPMV_ORDER_FAST && A->perm.empty();
    const bool zblock = fast && A->fast_variant == 10 && A->zbplan_ok;
    const bool tma = fast && A->fast_variant == 11 && A->tplan_ok &&
                     ((reinterpret_cast<uintptr_t>(A->d_hx) | reinterpret_cast<uintptr_t>(A->d_hy)) & 15u) == 0;
    const bool tiled = zblock || tma || (fast && A->stage_ok && (A->fast_variant == 1 || A->fast_variant == 6 ||
                                                                 A->fast_variant == 8 || A->fast_variant == 9));
    // the unit a chunk is made of: a tile, a z-block chunk of planes, or a plane
    const int64_t rows = zblock ? int64_t(A->zbplan.zc) * A->zbplan.S : tma ? A->tplan.S : int64_t(A->stage.rows);
    constexpr int kChunks = 8;
    if (!tiled || A->n < int64_t(kChunks) * (zblock ? 1 : 4) * rows) {
        SPMVC_CUDA(cudaMemcpyAsync(A->d_hx, x, bytes, cudaMemcpyHostToDevice, A->own_stream));
        if ((st = spmv_apply(A, A->d_hx, A->d_hy, A->own_stream))) return st;
        SPMVC_CUDA(cudaMemcpyAsync(y, A->d_hy, bytes, cudaMemcpyDeviceToHost, A->own_stream));
        SPMVC_CUDA(cudaStreamSynchronize(A->own_stream));
        return SPMV_OK;
    }
    // Pipelined by row chunks (whole tiles): x chunk j goes in on
    // one stream; the rows of chunk i are computed once every x chunk up to
    // row end + the largest displacement has arrived; y chunk i goes out on
    // a third stream while later chunks are still coming in.  The tiles
    // are those of the one-shot product, so the result is the same bits.
    if (!A->h2d_stream) SPMVC_CUDA(cudaStreamCreateWithFlags(&A->h2d_stream, cudaStreamNonBlocking));
    if (!A->d2h_stream) SPMVC_CUDA(cudaStreamCreateWithFlags(&A->d2h_stream, cudaStreamNonBlocking));
    while (A->host_events.size() < 2 * kChunks) {
        cudaEvent_t e;
        SPMVC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        A->host_events.push_back(e);
    }
    const int64_t n = A->n;
    // chunk ends in whole tiles, equal chunks (measured best against
    // chunks growing from small ones: the last chunk's copy-out is the tail)
    const int64_t tiles = (n + rows - 1) / rows;
    int64_t bound[kChunks + 1];
    for (int j = 0; j <= kChunks; ++j) bound[j] = std::min(n, (tiles * j + kChunks - 1) / kChunks * rows);
    bound[kChunks] = n;
    int64_t halo = 0;
    for (int32_t d : A->pat.uoff) halo = std::max<int64_t>(halo, d < 0 ? -int64_t(d) : int64_t(d));
    for (int j = 0; j < kChunks; ++j) {
        const int64_t b = bound[j], e = bound[j + 1];
        if (e > b)
            SPMVC_CUDA(cudaMemcpyAsync(A->d_hx + b, x + b, sizeof(double) * (e - b), cudaMemcpyHostToDevice,
                                       A->h2d_stream));
        SPMVC_CUDA(cudaEventRecord(A->host_events[j], A->h2d_stream));
    }
    for (int i = 0; i < kChunks; ++i) {
        const int64_t b = bound[i], e = bound[i + 1];
        if (e <= b) continue;
        // the windows of a chunk's last tiles reach one element past the
        // largest displacement (a 16-byte pair that starts on an odd
        // element); that element enters the tile's exponent, so it must have
        // arrived too
        const int64_t need = std::min(n, e + halo + 2);
        int jx = i;
        while (jx + 1 < kChunks && bound[jx + 1] < need) ++jx;     // last x chunk the rows read
        SPMVC_CUDA(cudaStreamWaitEvent(A->own_stream, A->host_events[jx], 0));
        cudaError_t ce;
        if (tma) {
            TmaPlan tp = A->tplan;
            tp.z_lo = int32_t(b / rows);
            tp.z_hi = int32_t((e + rows - 1) / rows);
            ce = launch_pattern_fast_tma(A->pat_view, tp, A->d_hx, A->d_hy, A->own_stream);
        } else if (zblock) {
            ZPlan zp = A->zbplan;
            zp.chunk0 = int32_t(b / rows);
            zp.nchunks = int32_t((e - b + rows - 1) / rows);
            ce = launch_pattern_fast_zblock(A->pat_view, zp, A->d_hx, A->d_hy, A->d_scratch_words, A->own_stream);
        } else {
            StagePlan plan = A->stage;
            plan.tile0 = b / rows;
            plan.ntiles = (e - b + rows - 1) / rows;
            ce = A->fast_variant == 1 ? launch_pattern_fast_staged(A->pat_view, plan, A->d_hx, A->d_hy, A->own_stream)
                                      : launch_pattern_fast_rstaged(A->pat_view, plan, A->d_hx, A->d_hy,
                                                                    A->fast_variant == 6 ? 0 : A->fast_variant == 8 ? 1 : 2,
                                                                    A->own_stream);
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "spmv chunk launch");
        SPMVC_CUDA(cudaEventRecord(A->host_events[kChunks + i], A->own_stream));
        SPMVC_CUDA(cudaStreamWaitEvent(A->d2h_stream, A->host_events[kChunks + i], 0));
        SPMVC_CUDA(cudaMemcpyAsync(y + b, A->d_hy + b, sizeof(double) * (e - b), cudaMemcpyDeviceToHost,
                                   A->d2h_stream));
    }
    SPMVC_CUDA(cudaStreamSynchronize(A->d2h_stream));
    return SPMV_OK;
}

// binary32 product from the stored records (or ELL values)
static int apply_f32_records(spmv_mat_t A, const float* x, float* y, spmv_stream_t stream) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (A->fmt == SPMV_FMT_DIT) return fail(SPMV_EUNSUPPORTED, "no binary32 product for the Data+Index Table format");
    if (A->fmt == SPMV_FMT_DATA_TABLE) return fail(SPMV_EUNSUPPORTED, "no binary32 product for the Data Table format");
    if (!A->perm.empty()) return fail(SPMV_EUNSUPPORTED, "no binary32 product for a reordered handle");
    if (A->n > 0 && (!x || !y)) return fail(SPMV_EINVAL, "null vector");
    int st = ensure_device(A);
    if (st) return st;
    const cudaStream_t s = as_stream(stream);
    cudaError_t e;
    if (A->fmt == SPMV_FMT_ELL) {
        if (!A->d_ell_val32) {
            std::vector<float> v32(A->ell.val.size());
            for (size_t k = 0; k < v32.size(); ++k) v32[k] = static_cast<float>(A->ell.val[k]);
            if ((st = dev_copy(A, v32.data(), v32.size(), &A->d_ell_val32))) return st;
            A->ell_view.val32 = A->d_ell_val32;
        }
        e = launch_ell_f32(A->ell_view, x, y, s);
    } else if (A->fmt == SPMV_FMT_PATTERN) {
        e = launch_pattern_col_f32(A->pat_view, x, y, s);
    } else {
        e = launch_delta_f32(A->dlt_view, x, y, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "spmv_f32 launch");
    return SPMV_OK;
}

int spmv_apply_f32(spmv_mat_t A, const float* x, float* y, spmv_stream_t stream) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (A->fmt == SPMV_FMT_PATTERN && A->perm.empty() && A->n > 0 && x && y) {
        // one byte a row: the binary32 chain from the row types where the
        // matrix has at most 256 distinct records
        int st = ensure_device(A);
        if (st) return st;
        if (A->f32_kind >= 1 && ensure_row_types(A)) {
            cudaError_t e = cudaErrorNotSupported;
            if (A->f32_kind == 2 && A->f32plan_ok)
                e = launch_pattern_f32_tma(A->pat_view, A->f32plan, x, y, as_stream(stream));
            if (e == cudaErrorNotSupported) e = launch_pattern_types_f32(A->pat_view, x, y, as_stream(stream));
            if (e == cudaSuccess) return SPMV_OK;
            if (e != cudaErrorNotSupported) return cuda_fail(e, "spmv_f32 launch");
        }
    }
    return apply_f32_records(A, x, y, stream);
}

int spmm_apply(spmv_mat_t A, int32_t k, const double* X, int64_t ldx, double* Y, int64_t ldy,
               spmv_stream_t stream) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (k < 1 || k > 64 || ldx < k || ldy < k) return fail(SPMV_EINVAL, "need 1 <= k <= 64, ldx >= k, ldy >= k");
    if (A->fmt == SPMV_FMT_DIT) return fail(SPMV_EUNSUPPORTED, "no SpMM for the Data+Index Table format");
    if (A->fmt == SPMV_FMT_DATA_TABLE) return fail(SPMV_EUNSUPPORTED, "no SpMM for the Data Table format");
    if (!A->perm.empty()) return fail(SPMV_EUNSUPPORTED, "no SpMM for a reordered handle");
    if (A->n > 0 && (!X || !Y)) return fail(SPMV_EINVAL, "null block");
    int st = ensure_device(A);
    if (st) return st;
    const cudaStream_t s = as_stream(stream);
    cudaError_t e;
    if (A->fmt == SPMV_FMT_PATTERN && A->order == SPMV_ORDER_FAST && A->n > 0) {
        // the TMA-fed kernel: 8 columns a pass from k = 8, else 4 from k = 4
        const int c = A->spmm_kind - 1;
        const TmaSpmmPlan* tp = c < 0 ? nullptr
                                : k >= 8 && A->splan_ok[1][c] ? &A->splan[1][c]
                                : k >= 4 && A->splan_ok[0][c] ? &A->splan[0][c]
                                                              : nullptr;
        if (tp) {
            e = launch_pattern_spmm_tma(A->pat_view, *tp, k, X, ldx, Y, ldy, s);
            if (e == cudaSuccess) return SPMV_OK;
            if (e != cudaErrorNotSupported) return cuda_fail(e, "spmm launch");
        }
    }
    if (A->fmt == SPMV_FMT_ELL) e = launch_ell_spmm(A->ell_view, k, X, ldx, Y, ldy, s);
    else if (A->fmt == SPMV_FMT_PATTERN && A->order == SPMV_ORDER_FAST && A->d_xfixed &&
             A->pat_view.run_len == 3 && A->pat_view.nu == 27) {
        // fixed-point copy of X with guard rows, grown to the widest k seen
        if (A->xfixed_block_cols < k) {
            int2* xf;
            const int kc = k <= 8 ? 8 : (k <= 32 ? 32 : 64);
            if ((st = dev_copy<int2>(A, nullptr, static_cast<size_t>(A->n + 2 * A->xfixed_guard) * kc, &xf))) return st;
            A->d_xfixed_block = xf;
            A->xfixed_block_cols = kc;
        }
        e = launch_pattern_spmm_fast_x(A->pat_view, k, X, ldx, Y, ldy, A->d_scratch_words, A->d_xfixed_block,
                                       A->xfixed_guard, s);
    } else if (A->fmt == SPMV_FMT_PATTERN)
        e = A->order == SPMV_ORDER_FAST
                ? launch_pattern_spmm_fast(A->pat_view, k, X, ldx, Y, ldy, A->d_scratch_words, s)
                : launch_pattern_spmm_col(A->pat_view, k, X, ldx, Y, ldy, s);
    else e = launch_delta_spmm(A->dlt_view, k, X, ldx, Y, ldy, s);
    if (e != cudaSuccess) return cuda_fail(e, "spmm launch");
    return SPMV_OK;
}

int spmv_autotune(spmv_mat_t A, const double* x, double* y, int32_t reps, int32_t* choice) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (A->n > 0 && (!x || !y)) return fail(SPMV_EINVAL, "null vector");
    if (reps <= 0) reps = 10;
    int st = ensure_device(A);
    if (st) return st;
    if (choice) *choice = 0;
    if (A->fmt != SPMV_FMT_PATTERN || A->order != SPMV_ORDER_FAST || A->n == 0) return SPMV_OK;
    struct Cand { int variant; StagePlan plan; ZPlan zplan; TmaPlan tplan; };
    std::vector<Cand> cands;
    if (A->d_xfixed) cands.push_back(Cand{2, A->stage, {}, {}});
    if (A->async_ok) cands.push_back(Cand{4, A->async_plan, {}, {}});
    if (A->async_ok && A->d_xfixed) cands.push_back(Cand{5, A->async_plan, {}, {}});
    if (A->stage_ok) {
        const bool full27 = A->pat_view.run_len == 3 && A->pat_view.nu == 27;
        for (int rpt : {1, 2, 4}) {
            StagePlan plan;
            if (make_stage_plan(A->pat.uoff, rpt, 512, 12288, &plan)) {
                cands.push_back(Cand{1, plan, {}, {}});
                if (A->d_xfixed && full27) cands.push_back(Cand{3, plan, {}, {}});
            }
        }
        // 256-thread tiles (six resident CTAs per SM) and the register-staged
        // kernel for the full 27-point union
        if (full27) {
            for (int rpt : {2, 4, 8}) {
                StagePlan plan;
                if (make_stage_plan(A->pat.uoff, rpt, 256, 12288, &plan)) cands.push_back(Cand{1, plan, {}, {}});
            }
            for (std::pair<int, int> sh : {std::make_pair(256, 4), std::make_pair(256, 2), std::make_pair(512, 2)}) {
                StagePlan plan;
                if (make_stage_plan(A->pat.uoff, sh.second, sh.first, 12288, &plan) && rstage_supported(plan)) {
                    cands.push_back(Cand{6, plan, {}, {}});
                    cands.push_back(Cand{8, plan, {}, {}});
                }
            }
            for (std::pair<int, int> sh : {std::make_pair(256, 2), std::make_pair(256, 4), std::make_pair(512, 2)}) {
                ZPlan zp;
                if (A->pat_view.words == 7 && make_zplan(A->pat.uoff, A->n, sh.second, sh.first, A->num_sms, &zp) &&
                    zmarch_supported(zp))
                    cands.push_back(Cand{7, {}, zp, {}});
            }
            for (int planes : {3, 4}) {
                ZPlan zp;
                if (A->pat_view.words == 7 && make_zblock_plan(A->pat.uoff, A->n, planes, 256, &zp))
                    cands.push_back(Cand{10, {}, zp, {}});
            }
            if (A->tplan_ok && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) == 0)
                for (int ctas : {1, 2})
                    for (int ty : {1, 2}) {
                        TmaPlan tp;
                        std::vector<uint32_t> tab;
                        if (make_tma_plan(A->pat, A->pat_view, A->n, A->num_sms, ty, ctas, &tp, &tab)) {
                            tp.expected = A->tplan.expected;   // the same table for every shape
                            cands.push_back(Cand{11, {}, {}, tp});
                        }
                    }
        }
    }
    if (cands.size() <= 1) return SPMV_OK;
    // Every candidate's result is checked against the COLUMN-order product
    // before it may be picked: |y - y_col| <= R max|x| 2^-46 + 2^-50 |y_col|,
    // R the largest absolute row sum of A (the FAST bound plus the COLUMN
    // chain's own rounding, with margin).  A kernel that disagrees is never
    // chosen.
    double* y_ref = nullptr;
    unsigned long long* words = nullptr;          // [0] max |x| bits, [1] mismatch count
    SPMVC_CUDA(cudaMalloc(&y_ref, sizeof(double) * A->n));
    struct Freer {
        double* a = nullptr;
        unsigned long long* b = nullptr;
        ~Freer() { cudaFree(a); cudaFree(b); }
    } freer;
    freer.a = y_ref;
    SPMVC_CUDA(cudaMalloc(&words, 2 * sizeof(unsigned long long)));
    freer.b = words;
    SPMVC_CUDA(cudaMemset(words, 0, 2 * sizeof(unsigned long long)));
    {
        const cudaError_t ce = launch_pattern_col_f64(A->pat_view, x, y_ref, nullptr);
        if (ce != cudaSuccess) return cuda_fail(ce, "autotune reference launch");
        const cudaError_t me = launch_absmax(x, A->n, words, nullptr);
        if (me != cudaSuccess) return cuda_fail(me, "autotune max launch");
    }
    unsigned long long xbits = 0;
    SPMVC_CUDA(cudaMemcpy(&xbits, words, sizeof(xbits), cudaMemcpyDeviceToHost));
    double xmax;
    std::memcpy(&xmax, &xbits, sizeof(xmax));
    const double row_abs = std::ldexp(double(A->pat.max_row_abs), A->pat.mult_exp);
    const double abs_tol = row_abs * xmax * std::ldexp(1.0, -46), rel_tol = std::ldexp(1.0, -50);
    cudaEvent_t e0, e1;
    SPMVC_CUDA(cudaEventCreate(&e0));
    SPMVC_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    Cand pick = cands[0];
    bool picked = false;
    for (const Cand& c : cands) {
        auto launch = [&]() {
            if (c.variant == 4) return launch_pattern_fast_async(A->pat_view, c.plan, x, y, A->num_sms, nullptr);
            if (c.variant == 6) return launch_pattern_fast_rstaged(A->pat_view, c.plan, x, y, 0, nullptr);
            if (c.variant == 8) return launch_pattern_fast_rstaged(A->pat_view, c.plan, x, y, 1, nullptr);
            if (c.variant == 7)
                return launch_pattern_fast_zmarch(A->pat_view, c.zplan, x, y, A->d_scratch_words, nullptr);
            if (c.variant == 10)
                return launch_pattern_fast_zblock(A->pat_view, c.zplan, x, y, A->d_scratch_words, nullptr);
            if (c.variant == 11) return launch_pattern_fast_tma(A->pat_view, c.tplan, x, y, nullptr);
            if (c.variant == 5)
                return launch_pattern_fast_async_x(A->pat_view, c.plan, x, y, A->d_scratch_words, A->d_xfixed,
                                                   A->xfixed_guard, A->num_sms, nullptr);
            return c.variant == 2 ? launch_pattern_fast_x(A->pat_view, x, y, A->d_scratch_words, A->d_xfixed,
                                                          A->xfixed_guard, nullptr)
                 : c.variant == 3 ? launch_pattern_fast_xstaged(A->pat_view, c.plan, x, y, A->d_scratch_words,
                                                                A->d_xfixed, A->xfixed_guard, nullptr)
                                  : launch_pattern_fast_staged(A->pat_view, c.plan, x, y, nullptr);
        };
        cudaError_t e = launch();
        if (e != cudaSuccess) return cuda_fail(e, "autotune launch");
        SPMVC_CUDA(cudaMemsetAsync(words + 1, 0, sizeof(unsigned long long), nullptr));
        if ((e = launch_check_close(y, y_ref, A->n, abs_tol, rel_tol, words + 1, nullptr)) != cudaSuccess)
            return cuda_fail(e, "autotune check launch");
        unsigned long long bad = 0;
        SPMVC_CUDA(cudaMemcpy(&bad, words + 1, sizeof(bad), cudaMemcpyDeviceToHost));
        if (bad != 0) continue;                       // wrong results: never a candidate
        SPMVC_CUDA(cudaEventRecord(e0, nullptr));
        for (int k = 0; k < reps; ++k) launch();
        SPMVC_CUDA(cudaEventRecord(e1, nullptr));
        SPMVC_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; pick = c; picked = true; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!picked) return fail(SPMV_EDEVICE, "autotune: no FAST kernel matched the COLUMN-order product");
    A->fast_variant = pick.variant;
    const bool staged_pick = pick.variant == 1 || pick.variant == 3 || pick.variant == 6 || pick.variant == 8;
    if (staged_pick) A->stage = pick.plan;
    if (pick.variant == 4 || pick.variant == 5) A->async_plan = pick.plan;
    if (pick.variant == 7) {
        A->zplan = pick.zplan;
        A->zplan_ok = true;
    }
    if (pick.variant == 10) {
        A->zbplan = pick.zplan;
        A->zbplan_ok = true;
    }
    if (pick.variant == 11) A->tplan = pick.tplan;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_variant[tune_key(A)] = pick.variant;
        if (pick.variant == 7)
            g_tune[tune_key(A)] = pick.zplan.threads * 16 + pick.zplan.rows_per_thread;
        else if (pick.variant == 10)
            g_tune[tune_key(A)] = pick.zplan.threads * 16 + pick.zplan.zc;
        else if (pick.variant == 11)
            g_tune[tune_key(A)] = pick.tplan.ty + 4 * (pick.tplan.ctas - 1);
        else if (staged_pick)
            g_tune[tune_key(A)] = (pick.plan.rows / pick.plan.rows_per_thread) * 16 + pick.plan.rows_per_thread;
    }
    if (choice) *choice = staged_pick ? pick.plan.rows : pick.variant == 7 ? pick.zplan.rows
                        : pick.variant == 10 ? pick.zplan.rows * pick.zplan.zc
                        : pick.variant == 11 ? A->tplan.C
                        : (pick.variant >= 4 ? pick.variant : 1);
    return SPMV_OK;
}

int spmv_set_f32_kernel(spmv_mat_t A, int32_t kind) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (kind < 0 || kind > 2) return fail(SPMV_EINVAL, "binary32 kernel kind must be 0, 1 or 2");
    A->f32_kind = kind;
    return SPMV_OK;
}

int spmv_set_spmm_kernel(spmv_mat_t A, int32_t kind) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (kind < 0 || kind > 3) return fail(SPMV_EINVAL, "SpMM kernel kind must be 0 to 3");
    A->spmm_kind = kind;
    return SPMV_OK;
}

int spmv_set_tile(spmv_mat_t A, int32_t variant, int32_t tile_rows, int32_t block_threads) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (A->fmt != SPMV_FMT_PATTERN || !A->pat.fast_ok) return fail(SPMV_EUNSUPPORTED, "no FAST kernels for this matrix");
    int st = ensure_device(A);
    if (st) return st;
    if (variant == 0) { A->fast_variant = 0; return SPMV_OK; }
    if (variant == 2) {
        if (!A->d_xfixed) return fail(SPMV_EUNSUPPORTED, "no pre-converted kernel for this union size");
        A->fast_variant = 2;
        return SPMV_OK;
    }
    if (variant == 4 || variant == 5) {
        if (!A->async_ok || (variant == 5 && !A->d_xfixed))
            return fail(SPMV_EUNSUPPORTED, "no persistent double-buffered kernel for this union");
        A->fast_variant = variant;
        return SPMV_OK;
    }
    if (variant == 7) {
        ZPlan zp;
        const int rpt = block_threads > 0 ? tile_rows / block_threads : 0;
        if (block_threads != 256 && block_threads != 512) return fail(SPMV_EINVAL, "block_threads must be 256 or 512");
        if (A->pat_view.words != 7 || tile_rows <= 0 || tile_rows % block_threads != 0 ||
            !make_zplan(A->pat.uoff, A->n, rpt, block_threads, A->num_sms, &zp) || !zmarch_supported(zp))
            return fail(SPMV_EUNSUPPORTED, "no z-marching kernel for this union and tile (tile_rows/threads "
                                           "512/256, 1024/256 or 1024/512, plane stride a multiple of tile_rows)");
        A->zplan = zp;
        A->zplan_ok = true;
        A->fast_variant = 7;
        return SPMV_OK;
    }
    if (variant == 10) {
        ZPlan zp;
        if (block_threads != 256 && block_threads != 512) return fail(SPMV_EINVAL, "block_threads must be 256 or 512");
        if (A->pat_view.words != 7 || tile_rows <= 0 || tile_rows % 512 != 0 ||
            !make_zblock_plan(A->pat.uoff, A->n, tile_rows / 512, block_threads, &zp))
            return fail(SPMV_EUNSUPPORTED, "no z-block kernel for this union and tile (tile_rows 1536 or 2048 with "
                                           "256 threads; plane stride a multiple of 512)");
        A->zbplan = zp;
        A->zbplan_ok = true;
        A->fast_variant = 10;
        return SPMV_OK;
    }
    if (variant == 11) {
        // tile_rows: lines of a compute thread's tile, 1 or 2 (0: keep the
        // current plan's); block_threads 2: two CTAs an SM, else one
        if (!A->tplan_ok)
            return fail(SPMV_EUNSUPPORTED, "no TMA z-marching kernel for this matrix (the full 27-point box of an "
                                           "nx*ny*nz grid with uniform neighbour weights, nx a multiple of 4 up "
                                           "to 252, a column block of whole lines dividing ny)");
        if (tile_rows != 0) {
            TmaPlan tp;
            std::vector<uint32_t> tab;
            if (tile_rows != 1 && tile_rows != 2) return fail(SPMV_EINVAL, "variant 11 takes tiles of 1 or 2 lines");
            const int ctas = block_threads == 2 ? 2 : 1;
            if (!make_tma_plan(A->pat, A->pat_view, A->n, A->num_sms, tile_rows, ctas, &tp, &tab))
                return fail(SPMV_EUNSUPPORTED, "no TMA z-marching kernel with that tile here");
            tp.expected = A->tplan.expected;
            A->tplan = tp;
        }
        A->fast_variant = 11;
        return SPMV_OK;
    }
    if (variant != 1 && variant != 3 && variant != 6 && variant != 8 && variant != 9)
        return fail(SPMV_EINVAL, "variant must be 0..11");
    const bool full27 = A->pat_view.run_len == 3 && A->pat_view.nu == 27;
    const bool rstaged = variant == 6 || variant == 8 || variant == 9;
    if (variant == 3 && !(A->d_xfixed && full27))
        return fail(SPMV_EUNSUPPORTED, "no staged pre-converted kernel for this union");
    if (!stage_supported(static_cast<int>(A->pat.uoff.size()))) return fail(SPMV_EUNSUPPORTED, "no staged kernel for this union size");
    if (block_threads != 512 && block_threads != 256) return fail(SPMV_EINVAL, "block_threads must be 256 or 512");
    if (rstaged && !(full27 && A->pat_view.words == 7))
        return fail(SPMV_EUNSUPPORTED, "no register-staged kernel for this union");
    if (block_threads == 256 && !((variant == 1 || rstaged) && full27))
        return fail(SPMV_EUNSUPPORTED, "256-thread tiles exist for the full 27-point union only");
    const int rpt = tile_rows / block_threads;
    const bool shape_ok = tile_rows > 0 && tile_rows % block_threads == 0 &&
                          (block_threads == 512 ? (rpt == 1 || rpt == 2 || rpt == 4) : (rpt == 2 || rpt == 4 || rpt == 8));
    StagePlan plan;
    if (!shape_ok || !make_stage_plan(A->pat.uoff, rpt, block_threads, 12288, &plan))
        return fail(SPMV_EUNSUPPORTED, "tile does not fit shared memory (tile_rows 512, 1024 or 2048)");
    if (rstaged && !rstage_supported(plan))
        return fail(SPMV_EUNSUPPORTED, "register-staged kernel: tile_rows/threads 1024/256, 512/256 or 1024/512 "
                                       "with windows of at most 2*pairs*threads elements");
    if (variant == 9 && !ensure_row_types(A))
        return fail(SPMV_EUNSUPPORTED, "more than 256 distinct row records: no row types");
    A->stage = plan;
    A->stage_ok = true;
    A->fast_variant = variant;
    return SPMV_OK;
}

int spmv_set_variant(spmv_mat_t A, int32_t variant, int32_t tile_rows) {
    return spmv_set_tile(A, variant, tile_rows, 512);
}

int spmv_free(spmv_mat_t A) {
    if (!A) return SPMV_OK;
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    free_device(A);
    A->magic = 0;
    delete A;
    return SPMV_OK;
}

const char* spmv_strerror(int status) {
    switch (status) {
        case SPMV_OK: return "ok";
        case SPMV_EINVAL: return "invalid argument";
        case SPMV_ENOMEM: return "out of memory";
        case SPMV_ECUDA: return "CUDA error";
        case SPMV_ECORRUPT: return "corrupt compressed stream";
        case SPMV_EUNSUPPORTED: return "unsupported for this matrix or format";
        case SPMV_ENOTCONVERGED: return "not converged";
        case SPMV_ETIMEOUT: return "device wait timed out";
        case SPMV_EDEVICE: return "device-side decoding error";
        default: return "unknown status";
    }
}

const char* spmv_last_error(void) { return g_last_error.c_str(); }

int spmv_device_error(spmv_mat_t A, int32_t* code) {
    if (!valid(A) || !code) return fail(SPMV_EINVAL, "invalid argument");
    *code = 0;
    if (A->device < 0) return SPMV_OK;
    SPMVC_CUDA(cudaDeviceSynchronize());
    SPMVC_CUDA(cudaMemcpy(code, A->d_err, 4, cudaMemcpyDeviceToHost));
    SPMVC_CUDA(cudaMemset(A->d_err, 0, 4));
    return SPMV_OK;
}

const char* spmv_version(void) { return "spmvc 0.1 (sm_103a)"; }

}  // extern "C"

// Accessors used by the solver and batch translation units.
namespace spmvc {
int api_ensure_device(spmv_mat_s* m) { return ensure_device(m); }
// Before timed binary32 work: the device copy and, for the pattern format,
// the one-byte row types (built on the host once).
int api_prepare_f32(spmv_mat_s* m) {
    const int st = ensure_device(m);
    if (st == SPMV_OK && m->fmt == SPMV_FMT_PATTERN && m->perm.empty() && m->f32_kind >= 1) ensure_row_types(m);
    return st;
}
bool api_valid(spmv_mat_t m) { return valid(m); }

// y = A x where the caller also has the partial maxima of x's high words
// (xmax_n words, sign cleared): the TMA kernel then scales by the whole
// vector's exponent (no rescaling of windows); other kernels ignore them.
// With dot_part, the kernel that can also writes per-CTA partial sums of
// x.y there and *dot_n their count; *dot_n = 0 means the caller forms x.y.
int api_apply_xmax(spmv_mat_s* A, const double* x, double* y, const uint32_t* xmax_part, int xmax_n,
                   cudaStream_t s, double* dot_part, int* dot_n) {
    if (dot_n) *dot_n = 0;
    int st = ensure_device(A);
    if (st) return st;
    if (A->fmt == SPMV_FMT_PATTERN && A->order == SPMV_ORDER_FAST && A->perm.empty() && A->fast_variant == 11 &&
        A->tplan_ok && A->n > 0 && x != y) {
        const TmaPlan& tp = dot_part && A->tplan_cg_ok ? A->tplan_cg : A->tplan;
        const cudaError_t e = launch_pattern_fast_tma(A->pat_view, tp, x, y, s, xmax_part, xmax_n, dot_part, dot_n);
        if (e == cudaSuccess) return SPMV_OK;
        if (e != cudaErrorNotSupported) return cuda_fail(e, "spmv launch");
    }
    return spmv_apply(A, x, y, s);
}

// Y = A X where the caller also has partial maxima of the high words of
// |X| by column (xmax_n rows of k words): the TMA-fed SpMM then scales each
// column by its whole-vector exponent; other kernels ignore them.
int api_spmm_xmax(spmv_mat_s* A, int32_t k, const double* X, int64_t ldx, double* Y, int64_t ldy, cudaStream_t s,
                  const uint32_t* xmax_part, int xmax_n) {
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    int st = ensure_device(A);
    if (st) return st;
    if (A->fmt == SPMV_FMT_PATTERN && A->order == SPMV_ORDER_FAST && A->perm.empty() && A->n > 0 && X && Y &&
        k >= 1 && k <= 64 && ldx >= k && ldy >= k) {
        const int c = A->spmm_kind - 1;
        const TmaSpmmPlan* tp = c < 0 ? nullptr
                                : k >= 8 && A->splan_ok[1][c] ? &A->splan[1][c]
                                : k >= 4 && A->splan_ok[0][c] ? &A->splan[0][c]
                                                              : nullptr;
        if (tp) {
            const cudaError_t e = launch_pattern_spmm_tma(A->pat_view, *tp, k, X, ldx, Y, ldy, s, xmax_part, xmax_n);
            if (e == cudaSuccess) return SPMV_OK;
            if (e != cudaErrorNotSupported) return cuda_fail(e, "spmm launch");
        }
    }
    return spmm_apply(A, k, X, ldx, Y, ldy, s);
}

// The binary32 product with x.y as above (the TMA-fed kernel only).
int api_apply_f32_dot(spmv_mat_s* A, const float* x, float* y, cudaStream_t s, double* dot_part, int* dot_n) {
    if (dot_n) *dot_n = 0;
    if (!valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    if (A->fmt == SPMV_FMT_PATTERN && A->perm.empty() && A->n > 0 && x && y && x != y && A->f32_kind == 2) {
        int st = ensure_device(A);
        if (st) return st;
        if (ensure_row_types(A) && A->f32plan_ok) {
            const cudaError_t e = launch_pattern_f32_tma(A->pat_view, A->f32plan, x, y, s, dot_part, dot_n);
            if (e == cudaSuccess) return SPMV_OK;
            if (e != cudaErrorNotSupported) return cuda_fail(e, "spmv_f32 launch");
        }
    }
    return spmv_apply_f32(A, x, y, s);
}
}  // namespace spmvc
