// Ragged batches: y_b = A_b x_b for many pattern-format matrices of
// different sizes in ONE persistent kernel launch.  The host cuts every
// matrix into work items of item_rows rows (256 unless spmv_batch_autotune
// picked another size); each warp of a grid sized to the SM count takes
// items from an atomic ticket counter until none are left (no warp ever
// waits on another).  The counter reset and the launch are captured once
// in a CUDA graph that later calls replay.
//
// Summation order: the matrices' own.  When every matrix of the batch is
// in FAST order (spmv_set_order), a first pass takes the largest exponent
// of each x_b (warps over the items, one atomic maximum an item into the
// matrix's word) and the rows are then summed as exact fixed-point
// integers at that scale and rounded once -- spmv_apply's FAST rule with
// the whole vector's exponent, the scale the single-matrix direct kernel
// uses; a matrix whose x is zero/subnormal only or not finite takes the
// COLUMN order, as there.  Otherwise every row is the COLUMN order's fma
// chain (bit-exact with the CSR product).
#include <cstring>
#include <new>

#include "spmvc_internal.h"

namespace spmvc {
int api_ensure_device(spmv_mat_s* m);
bool api_valid(spmv_mat_t m);

namespace {
#include "fast_fixed.cuh"

constexpr int kItemRows = 256;
constexpr int kBatchBlock = 256;

template <int WORDS>
__device__ __forceinline__ void load_rec(const PatternView& a, int64_t r, uint32_t (&w)[kMaxRecordWords]) {
    constexpr int q16 = WORDS / 4, rem = WORDS % 4;
    if (q16 >= 1) { const uint4 v = __ldcs(a.p16a + r); w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w; }
    if (q16 >= 2) { const uint4 v = __ldcs(a.p16b + r); w[4] = v.x; w[5] = v.y; w[6] = v.z; w[7] = v.w; }
    if (rem >= 2) { const uint2 v = __ldcs(a.p8 + r); w[4 * q16] = v.x; w[4 * q16 + 1] = v.y; }
    if (rem & 1) w[WORDS - 1] = __ldcs(a.p4 + r);
}

template <int WORDS>
__global__ void __launch_bounds__(kBatchBlock) pattern_batch_kernel(const PatternView* __restrict__ mats,
                                                                    const double* const* __restrict__ xs,
                                                                    double* const* __restrict__ ys,
                                                                    const BatchItem* __restrict__ items,
                                                                    int64_t nitems, uint32_t* __restrict__ counter) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t ticket = 0;
        if (lane == 0) ticket = atomicAdd(counter, 1u);
        ticket = __shfl_sync(0xFFFFFFFFu, ticket, 0);
        if (int64_t(ticket) >= nitems) return;
        const BatchItem it = items[ticket];
        const PatternView* a = mats + it.m;
        const int64_t n = a->n;
        const int nu = a->nu, npat = a->npat, nd = a->dict_size;
        const double* __restrict__ x = xs[it.m];
        double* __restrict__ y = ys[it.m];
        for (int64_t r = it.r0 + lane; r < it.r1; r += 32) {
            uint32_t w[kMaxRecordWords];
            load_rec<WORDS>(*a, r, w);
            const uint32_t pat = (w[nu >> 2] >> (8 * (nu & 3))) & 0xFFu;
            if (pat >= uint32_t(npat)) { atomicOr(a->err, 1); continue; }
            const uint32_t mask = a->pmask[pat];
            double acc = 0.0;
#pragma unroll
            for (int u = 0; u < 4 * WORDS - 1; ++u)
                if (u < nu && ((mask >> u) & 1u)) {
                    const uint32_t code = (w[u >> 2] >> (8 * (u & 3))) & 0xFFu;
                    const int64_t c = r + a->uoff[u];
                    if (code >= uint32_t(nd) || uint64_t(c) >= uint64_t(n)) { atomicOr(a->err, 2); continue; }
                    acc = fma(__ldg(a->dict + code), __ldg(x + c), acc);
                }
            y[r] = acc;
        }
    }
}
// Per item, the largest high word of |x| over its rows, folded into its
// matrix's word (atomic maximum; the words are zeroed before the pass).
// Every row of a matrix belongs to one item, so a matrix's word ends as the
// largest high word of its whole x.
__global__ void __launch_bounds__(kBatchBlock) batch_xmax_kernel(const double* const* __restrict__ xs,
                                                                 const BatchItem* __restrict__ items, int64_t nitems,
                                                                 uint32_t* __restrict__ mat_max) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t t = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5); t < nitems; t += warps) {
        const BatchItem it = items[t];
        const double* __restrict__ x = xs[it.m];
        uint32_t m = 0u;
        for (int64_t r = it.r0 + lane; r < it.r1; r += 32)
            m = max(m, uint32_t(__double2hiint(__ldg(x + r))) & 0x7FFFFFFFu);
        m = __reduce_max_sync(0xFFFFFFFFu, m);
        if (lane == 0) atomicMax(mat_max + it.m, m);
    }
}

// FAST order: rows of an item summed exactly in fixed point at their
// matrix's scale (mat_max) and rounded once; COLUMN order for a matrix
// whose x is zero/subnormal only or has a non-finite entry.
template <int WORDS>
__global__ void __launch_bounds__(kBatchBlock) pattern_batch_fast_kernel(const PatternView* __restrict__ mats,
                                                                         const double* const* __restrict__ xs,
                                                                         double* const* __restrict__ ys,
                                                                         const BatchItem* __restrict__ items,
                                                                         int64_t nitems, uint32_t* __restrict__ counter,
                                                                         const uint32_t* __restrict__ mat_max) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t ticket = 0;
        if (lane == 0) ticket = atomicAdd(counter, 1u);
        ticket = __shfl_sync(0xFFFFFFFFu, ticket, 0);
        if (int64_t(ticket) >= nitems) return;
        const BatchItem it = items[ticket];
        const PatternView* a = mats + it.m;
        const int64_t n = a->n;
        const int nu = a->nu, npat = a->npat, nd = a->dict_size;
        const uint32_t mlo = a->mult_lo, mhi = a->mult_hi;
        const int emax = int(__ldg(mat_max + it.m) >> 20);
        const bool fast = emax >= 64 && emax < 2047;
        const int S = emax - 1075 + a->mult_exp;
        const double* __restrict__ x = xs[it.m];
        double* __restrict__ y = ys[it.m];
        for (int64_t r = it.r0 + lane; r < it.r1; r += 32) {
            uint32_t w[kMaxRecordWords];
            load_rec<WORDS>(*a, r, w);
            const uint32_t pat = (w[nu >> 2] >> (8 * (nu & 3))) & 0xFFu;
            if (pat >= uint32_t(npat)) { atomicOr(a->err, 1); continue; }
            const uint32_t mask = a->pmask[pat];
            if (!fast) {
                double acc = 0.0;
#pragma unroll
                for (int u = 0; u < 4 * WORDS - 1; ++u)
                    if (u < nu && ((mask >> u) & 1u)) {
                        const uint32_t code = (w[u >> 2] >> (8 * (u & 3))) & 0xFFu;
                        const int64_t c = r + a->uoff[u];
                        if (code >= uint32_t(nd) || uint64_t(c) >= uint64_t(n)) { atomicOr(a->err, 2); continue; }
                        acc = fma(__ldg(a->dict + code), __ldg(x + c), acc);
                    }
                y[r] = acc;
                continue;
            }
            int64_t ah = 0, al = 0;
#pragma unroll
            for (int u = 0; u < 4 * WORDS - 1; ++u)
                if (u < nu && ((mask >> u) & 1u)) {
                    const uint32_t code = (w[u >> 2] >> (8 * (u & 3))) & 0xFFu;
                    const int64_t c = r + a->uoff[u];
                    if (code >= uint32_t(nd) || uint64_t(c) >= uint64_t(n)) { atomicOr(a->err, 2); continue; }
                    const int32_t m8 = mult_of(mlo, mhi, code);
                    int32_t xh, xl;
                    to_fixed(__ldg(x + c), emax, xh, xl);
                    ah += int64_t(m8) * xh;
                    al += int64_t(m8) * xl;
                }
            y[r] = fixed_to_double(ah * (int64_t(1) << 26) + al, S);
        }
    }
}
}  // namespace

cudaError_t launch_pattern_batch_fast(const PatternView* mats_dev, const double* const* xs_dev,
                                      double* const* ys_dev, const BatchItem* items, int64_t nitems,
                                      uint32_t* counter, uint32_t* mat_max, int count, int words, int grid,
                                      cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mat_max, 0, sizeof(uint32_t) * size_t(count), s);
    if (e != cudaSuccess) return e;
    batch_xmax_kernel<<<grid, kBatchBlock, 0, s>>>(xs_dev, items, nitems, mat_max);
    switch (words) {
#define SPMVC_BATCH_FAST(W) \
    case W: pattern_batch_fast_kernel<W><<<grid, kBatchBlock, 0, s>>>(mats_dev, xs_dev, ys_dev, items, nitems, counter, mat_max); break;
        SPMVC_BATCH_FAST(1) SPMVC_BATCH_FAST(2) SPMVC_BATCH_FAST(3) SPMVC_BATCH_FAST(4)
        SPMVC_BATCH_FAST(5) SPMVC_BATCH_FAST(6) SPMVC_BATCH_FAST(7) SPMVC_BATCH_FAST(8)
#undef SPMVC_BATCH_FAST
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pattern_batch(const PatternView* mats_dev, const double* const* xs_dev, double* const* ys_dev,
                                 const BatchItem* items, int64_t nitems, uint32_t* counter, int words, int grid,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    switch (words) {
        case 1: pattern_batch_kernel<1><<<grid, kBatchBlock, 0, s>>>(mats_dev, xs_dev, ys_dev, items, nitems, counter); break;
        case 2: pattern_batch_kernel<2><<<grid, kBatchBlock, 0, s>>>(mats_dev, xs_dev, ys_dev, items, nitems, counter); break;
        case 3: pattern_batch_kernel<3><<<grid, kBatchBlock, 0, s>>>(mats_dev, xs_dev, ys_dev, items, nitems, counter); break;
        case 4: pattern_batch_kernel<4><<<grid, kBatchBlock, 0, s>>>(mats_dev, xs_dev, ys_dev, items, nitems, counter); break;
        case 5: pattern_batch_kernel<5><<<grid, kBatchBlock, 0, s>>>(mats_dev, xs_dev, ys_dev, items, nitems, counter); break;
        case 6: pattern_batch_kernel<6><<<grid, kBatchBlock, 0, s>>>(mats_dev, xs_dev, ys_dev, items, nitems, counter); break;
        case 7: pattern_batch_kernel<7><<<grid, kBatchBlock, 0, s>>>(mats_dev, xs_dev, ys_dev, items, nitems, counter); break;
        case 8: pattern_batch_kernel<8><<<grid, kBatchBlock, 0, s>>>(mats_dev, xs_dev, ys_dev, items, nitems, counter); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace spmvc

using namespace spmvc;

struct spmv_batch_s {
    uint32_t magic = 0x42415443u;
    int32_t count = 0;
    int words = 0;
    int grid = 0;
    bool fast = false;                 // every matrix in FAST order
    int item_rows = 0;
    std::vector<int64_t> ns;           // rows of each matrix
    int64_t nitems = 0;
    std::vector<void*> allocs;
    PatternView* d_views = nullptr;
    const double** d_xs = nullptr;
    double** d_ys = nullptr;
    BatchItem* d_items = nullptr;
    uint32_t* d_counter = nullptr;
    uint32_t* d_mat_max = nullptr;     // FAST: largest high word of each x_b
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {
int batch_fail_cuda(cudaError_t e, const char* what) {
    return fail(SPMV_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
template <class T>
int batch_alloc(spmv_batch_s* b, const T* src, size_t count, T** out) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(16, count * sizeof(T)));
    if (e != cudaSuccess) return fail(SPMV_ENOMEM, "cudaMalloc for batch plan");
    b->allocs.push_back(p);
    if (src && count) {
        e = cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return batch_fail_cuda(e, "cudaMemcpy");
    }
    *out = static_cast<T*>(p);
    return SPMV_OK;
}
// Cuts every matrix into items of `rows` rows, uploads the list and captures
// the launch (counter reset, for FAST the exponent pass, the kernel) in a
// fresh graph; a previous list and graph are dropped.
int batch_build(spmv_batch_s* p, int rows) {
    std::vector<BatchItem> items;
    for (int32_t b = 0; b < p->count; ++b)
        for (int64_t r0 = 0; r0 < p->ns[b]; r0 += rows) items.push_back(BatchItem{b, 0, r0, std::min<int64_t>(p->ns[b], r0 + rows)});
    BatchItem* d_items = nullptr;
    int st = batch_alloc(p, items.data(), items.size(), &d_items);
    if (st) return st;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    p->d_items = d_items;
    p->nitems = static_cast<int64_t>(items.size());
    p->item_rows = rows;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->grid = std::max(1, std::min<int>(sms * 4, static_cast<int>((p->nitems * 32 + kBatchBlock - 1) / kBatchBlock)));
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return batch_fail_cuda(e, "cudaStreamCreate");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t le =
            p->fast ? launch_pattern_batch_fast(p->d_views, p->d_xs, p->d_ys, p->d_items, p->nitems, p->d_counter,
                                                p->d_mat_max, p->count, p->words, p->grid, cs)
                    : launch_pattern_batch(p->d_views, p->d_xs, p->d_ys, p->d_items, p->nitems, p->d_counter, p->words,
                                           p->grid, cs);
        e = cudaStreamEndCapture(cs, &p->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return batch_fail_cuda(e, "batch graph capture");
    return SPMV_OK;
}

void batch_release(spmv_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void* p : b->allocs) cudaFree(p);
    b->magic = 0;
    delete b;
}
}  // namespace

extern "C" {

int spmv_batch_create(int32_t count, const spmv_mat_t* mats, const double* const* xs, double* const* ys,
                      spmv_batch_t* out) {
    if (!out || count < 1 || !mats || !xs || !ys) return fail(SPMV_EINVAL, "invalid batch arguments");
    *out = nullptr;
    int words = -1;
    bool fast = true;
    std::vector<PatternView> views;
    std::vector<int64_t> ns;
    for (int32_t b = 0; b < count; ++b) {
        spmv_mat_s* m = mats[b];
        if (!api_valid(m)) return fail(SPMV_EINVAL, "invalid matrix handle in batch");
        if (m->fmt != SPMV_FMT_PATTERN || !m->perm.empty())
            return fail(SPMV_EUNSUPPORTED, "batches take pattern-format matrices in their own numbering");
        if (words >= 0 && m->pat.words != words) return fail(SPMV_EUNSUPPORTED, "batch records must have equal size");
        if (m->n > 0 && (!xs[b] || !ys[b])) return fail(SPMV_EINVAL, "null vector in batch");
        words = m->pat.words;
        int st = api_ensure_device(m);
        if (st) return st;
        views.push_back(m->pat_view);
        ns.push_back(m->n);
        fast = fast && m->order == SPMV_ORDER_FAST && m->pat.fast_ok;
    }
    spmv_batch_s* p = new (std::nothrow) spmv_batch_s();
    if (!p) return fail(SPMV_ENOMEM, "host allocation failed");
    p->count = count;
    p->words = words;
    p->fast = fast;
    p->ns = std::move(ns);
    int st = batch_alloc(p, views.data(), views.size(), &p->d_views);
    if (!st) st = batch_alloc(p, xs, static_cast<size_t>(count), &p->d_xs);
    if (!st) st = batch_alloc(p, ys, static_cast<size_t>(count), &p->d_ys);
    if (!st) st = batch_alloc<uint32_t>(p, nullptr, 1, &p->d_counter);
    if (!st) st = batch_alloc<uint32_t>(p, nullptr, static_cast<size_t>(count), &p->d_mat_max);
    if (!st) st = batch_build(p, kItemRows);
    if (st) { batch_release(p); return st; }
    *out = p;
    return SPMV_OK;
}

int spmv_batch_autotune(spmv_batch_t plan, int32_t reps, int32_t* item_rows) {
    if (!plan || plan->magic != 0x42415443u) return fail(SPMV_EINVAL, "invalid batch plan");
    if (reps <= 0) reps = 10;
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return batch_fail_cuda(e, "cudaStreamCreate");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = plan->item_rows, st = SPMV_OK;
    float best_ms = 0.0f;
    for (int rows : {64, 128, 256, 512, 1024}) {
        if ((st = batch_build(plan, rows))) break;
        e = cudaGraphLaunch(plan->exec, cs);   // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
        for (int i = 0; i < reps && e == cudaSuccess; ++i) e = cudaGraphLaunch(plan->exec, cs);
        if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { st = batch_fail_cuda(e, "batch autotune"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_ms == 0.0f || ms < best_ms) {
            best_ms = ms;
            best = rows;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(cs);
    if (!st) st = batch_build(plan, best);
    if (!st && item_rows) *item_rows = best;
    return st;
}

int spmv_batch_launch(spmv_batch_t plan, spmv_stream_t stream) {
    if (!plan || plan->magic != 0x42415443u) return fail(SPMV_EINVAL, "invalid batch plan");
    cudaError_t e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return batch_fail_cuda(e, "cudaGraphLaunch");
    return SPMV_OK;
}

int spmv_batch_free(spmv_batch_t plan) {
    if (!plan) return SPMV_OK;
    if (plan->magic != 0x42415443u) return fail(SPMV_EINVAL, "invalid batch plan");
    batch_release(plan);
    return SPMV_OK;
}

int spmv_apply_batched(int32_t count, const spmv_mat_t* mats, const double* const* xs, double* const* ys,
                       spmv_stream_t stream) {
    spmv_batch_t plan;
    int st = spmv_batch_create(count, mats, xs, ys, &plan);
    if (st) return st;
    st = spmv_batch_launch(plan, stream);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    spmv_batch_free(plan);
    if (st) return st;
    if (e != cudaSuccess) return batch_fail_cuda(e, "cudaStreamSynchronize");
    return SPMV_OK;
}

}  // extern "C"
