// Binary32 compressed SpMV, y = A x (Eq. 1 of arXiv:1612.00530) in the
// binary32 fmaf chain over ascending columns that spmv_apply_f32 defines,
// for the pattern format of a 27-point grid stencil whose rows carry
// one-byte row types (values registered in the pattern, Sec. V), fed by the
// Tensor Memory Accelerator.  It is the product of IR-CG's inner solve.
//
// One persistent CTA an SM walks an equal share of the (column block,
// plane) sequence; a column block is L whole grid lines (C = L*nx rows) and
// a compute thread owns four vertically consecutive rows of one column.  A
// producer warp keeps the copies going: lane 0 loads, for every plane z of
// the block, the window W(z) -- nx+8 values by L+2 lines at (ix = -4,
// iy = first line - 1, z), one TMA tensor copy that fills everything outside
// the grid with zeros (the start at ix = -4 keeps the innermost coordinate
// 16-byte aligned) -- into a ring of twelve stages, and lane 1 the block's row
// types of every plane (one bulk copy of C bytes) into a ring of eight, so
// that many copies are in flight while three windows are being read.
// The compute warps use the raw windows directly (the chain needs no
// conversion), so they synchronise only through the rings' mbarriers, never
// with each other: a warp sums plane q from W(q-1), W(q), W(q+1) and hands
// back W(q-1) and the types of plane q.
// A row whose type is the one its grid position implies (the dominant
// record's codes at the slots inside the grid, absent codes elsewhere) sums
// all 27 window values with the dominant record's values (kernel
// parameters): its out-of-grid slots read zeros.  Any other row takes its
// type's record: from the window when every slot it holds lies inside the
// grid, else from x itself.  In-grid slots of the
// window are the x values the columns name, out-of-grid ones are zero, and
// an fmaf of a zero product leaves a chain started at +0 unchanged, so the
// result is the CSR chain's bit for bit.  Every mbarrier wait is bounded
// (error word bit 16, then a drain of the copies in flight).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "spmvc_internal.h"

namespace spmvc {

namespace {

#include "fast_fixed.cuh"
#include "tma_ptx.cuh"

constexpr int kF32RawStages = 12;
constexpr int kF32TypeStages = 8;
constexpr int kF32MaxThreads = 384;   // compute threads (four rows each)

// With DOT the kernel also forms x.y (the p.q of the inner CG step): each
// thread sums its four rows' products x[row]*y[row] of a step in binary32
// (x from the window's centre) and adds that chunk to a binary64 sum, one
// conversion a step (binary64 work runs on a narrow pipe); the CTA's sum
// goes to dot_part[blockIdx.x].
template <bool DOT>
__global__ void __launch_bounds__(kF32MaxThreads + 32, 1)
    pattern_f32_tma_kernel(const __grid_constant__ CUtensorMap xmap, const PatternView a, const TmaF32Plan tp,
                           const float* __restrict__ x, float* __restrict__ y, double* __restrict__ dot_part) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31;
    const int NC = tp.threads, C = tp.C, nx = tp.nx, pitch = tp.pitch;
    const float* const raw = reinterpret_cast<const float*>(smem + tp.off_raw);
    unsigned char* const typ = smem + tp.off_types;
    uint32_t* const stab = reinterpret_cast<uint32_t*>(smem + tp.off_tab);     // ntypes x 8 words
    uint32_t* const tmask = reinterpret_cast<uint32_t*>(smem + tp.off_tmask);  // [256] slot mask of each type
    uint32_t* const cmask = tmask + 256;                                        // [64] slots inside the grid
    float* const sdict = reinterpret_cast<float*>(smem + tp.off_dict);          // [256]
    uint32_t* const swords = reinterpret_cast<uint32_t*>(smem + tp.off_words);
    volatile uint32_t* const sabort = swords;
    volatile uint32_t* const spdone = swords + 1;
    volatile uint32_t* const siss = swords + 2;                                 // [2] issued
    uint64_t* const raw_full = reinterpret_cast<uint64_t*>(smem + tp.off_mbar);
    uint64_t* const raw_empty = raw_full + kF32RawStages;
    uint64_t* const typ_full = raw_empty + kF32RawStages;
    uint64_t* const typ_empty = typ_full + kF32TypeStages;

    const int ntypes = a.ntypes;
    for (int i = tid; i < ntypes * 8; i += blockDim.x) stab[i] = __ldg(a.rtypes + i);
    for (int i = tid; i < 256; i += blockDim.x) sdict[i] = i < a.dict_size ? a.dict32[i] : 0.0f;
    for (int t = tid; t < 256; t += blockDim.x) {
        uint32_t m = 0;
        if (t < ntypes) {
            const uint32_t pat = (__ldg(a.rtypes + t * 8 + 6) >> 24) & 0xFFu;   // byte 27: the pattern number
            m = pat < uint32_t(a.npat) ? a.pmask[pat] : 0xFFFFFFFFu;
        }
        tmask[t] = m;
    }
    for (int cls = tid; cls < 64; cls += blockDim.x) {
        uint32_t m = 0;
        for (int u = 0; u < 27; ++u) {
            const int d[3] = {u % 3 - 1, (u / 3) % 3 - 1, u / 9 - 1};
            bool in = true;
            for (int k = 0; k < 3; ++k) {
                const int c = (cls >> (2 * k)) & 3;
                if ((d[k] == -1 && !(c & 1)) || (d[k] == 1 && !(c & 2))) in = false;
            }
            if (in) m |= 1u << u;
        }
        cmask[cls] = m;
    }
    if (tid < 4) swords[tid] = 0u;
    if (tid == 0) {
        for (int i = 0; i < kF32RawStages; ++i) {
            mbar_init(raw_full + i, 1);
            mbar_init(raw_empty + i, NC / 32);
        }
        for (int i = 0; i < kF32TypeStages; ++i) {
            mbar_init(typ_full + i, 1);
            mbar_init(typ_empty + i, NC / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const int64_t units = int64_t(tp.nblk) * (tp.nz + kRunCost);
    Share share{units * blockIdx.x / gridDim.x, units * (blockIdx.x + 1) / gridDim.x, tp.nz, 0};

    if (tid >= NC) {
        // ---- producer warp: lane 0 the windows, lane 1 the row types
        if (lane > 1) return;
        const uint64_t policy = evict_first_policy();
        uint32_t n = 0;
        int b, z0, z1;
        bool ok = true;
        while (ok && share.next(b, z0, z1)) {
            for (int w = z0 - 1; ok && w <= z1; ++w) {
                if (lane == 0) {
                    const uint32_t st = n % kF32RawStages, k = n / kF32RawStages;
                    if (k > 0 && !mbar_wait(raw_empty + st, (k - 1) & 1u)) ok = false;
                    if (ok && *sabort) ok = false;
                    if (!ok) break;
                    fence_proxy_async();
                    mbar_expect_tx(raw_full + st, uint32_t(tp.win_floats) * 4u);
                    tma_load_3d(smem + tp.off_raw + st * tp.raw_stride * 4, &xmap, -4, b * tp.L - 1, w, raw_full + st);
                    siss[0] = ++n;
                } else if (w >= z0 && w < z1) {
                    const uint32_t st = n % kF32TypeStages, k = n / kF32TypeStages;
                    if (k > 0 && !mbar_wait(typ_empty + st, (k - 1) & 1u)) ok = false;
                    if (ok && *sabort) ok = false;
                    if (!ok) break;
                    fence_proxy_async();
                    mbar_expect_tx(typ_full + st, uint32_t(C));
                    bulk_g2s(typ + st * C, a.rtype + int64_t(w) * tp.S + int64_t(b) * C, uint32_t(C), typ_full + st,
                             policy);
                    siss[1] = ++n;
                }
            }
        }
        if (!ok && !*sabort) {
            atomicOr(reinterpret_cast<uint32_t*>(swords), 1u);
            raise_error(a.err, kErrWaitTimeout);
        }
        __threadfence_block();
        atomicAdd(reinterpret_cast<uint32_t*>(swords + 1), 1u);
        return;
    }

    // ---- compute threads: rows of block lines 4*vy .. 4*vy+3 at column ix
    const int vy = tid / nx, ix = tid - vy * nx;
    const uint32_t xcls = (ix > 0 ? 1u : 0u) | (ix < nx - 1 ? 2u : 0u);
    uint32_t nraw = 0, ntyp = 0;
    bool aborted = false;
    double dacc = 0.0;   // this thread's part of x.y (DOT)
    auto wait_raw = [&](uint32_t& st) -> bool {
        st = nraw % kF32RawStages;
        const bool okw = mbar_wait(raw_full + st, (nraw / kF32RawStages) & 1u);
        ++nraw;
        return okw;
    };
    auto release = [&](uint64_t* bar) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bar);
    };
    int b, z0, z1;
    while (!aborted && share.next(b, z0, z1)) {
        const int y0 = b * tp.L;
        uint32_t ycls[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int iy = y0 + 4 * vy + j;
            ycls[j] = (iy > 0 ? 1u : 0u) | (iy < tp.ny - 1 ? 2u : 0u);
        }
        uint32_t sA, sB, sC;
        bool okw = wait_raw(sA);
        okw = wait_raw(sB) && okw;
        for (int w = z0 + 1; w <= z1; ++w) {
            const int q = w - 1;                 // plane summed this step
            okw = wait_raw(sC) && okw;
            const uint32_t stT = ntyp % kF32TypeStages;
            okw = mbar_wait(typ_full + stT, (ntyp / kF32TypeStages) & 1u) && okw;
            ++ntyp;
            if (!okw || *sabort) {
                if (!okw) {
                    atomicOr(reinterpret_cast<uint32_t*>(swords), 1u);
                    raise_error(a.err, kErrWaitTimeout);
                }
                aborted = true;
                break;
            }
            const uint32_t zcls = (q > 0 ? 1u : 0u) | (q < tp.nz - 1 ? 2u : 0u);
            const float* P[3] = {raw + sA * tp.raw_stride, raw + sB * tp.raw_stride, raw + sC * tp.raw_stride};
            const unsigned char* tq = typ + stT * C;
            uint32_t t[4], cls[4];
            bool fast = true;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                t[j] = tq[(4 * vy + j) * nx + ix];
                cls[j] = xcls | (ycls[j] << 2) | (zcls << 4);
                fast = fast && int32_t(t[j]) == tp.exp_type[cls[j]];
            }
            const int64_t row0 = int64_t(q) * tp.S + int64_t(y0 + 4 * vy) * nx + ix;
            float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            const int base = 4 * vy * pitch + ix + 4;   // window line 4*vy, column ix
            if (__all_sync(0xFFFFFFFFu, fast)) {
                // every row of the warp holds the record its position implies:
                // 27 slots of six window lines a plane, shared by the four rows
#pragma unroll
                for (int dz = 0; dz < 3; ++dz) {
                    float e[6][3];
#pragma unroll
                    for (int l = 0; l < 6; ++l)
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) e[l][dx] = P[dz][base + l * pitch + dx - 1];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx)
                                acc[j] = fmaf(a.dom_v32[dz * 9 + dy * 3 + dx], e[j + dy][dx], acc[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint32_t mask = 0u;
                    uint32_t wrec[kMaxRecordWords] = {};
                    if (t[j] < uint32_t(ntypes)) {
                        mask = tmask[t[j]];
#pragma unroll
                        for (int k = 0; k < 7; ++k) wrec[k] = stab[t[j] * 8 + k];
                    } else {
                        raise_error(a.err, 2);
                    }
                    if (mask == 0xFFFFFFFFu) {
                        raise_error(a.err, 1);
                        mask = 0u;
                    }
                    float s = 0.0f;
                    if ((mask & ~cmask[cls[j]]) == 0u) {
                        // every slot the row holds lies inside the grid: the window
#pragma unroll
                        for (int u = 0; u < 27; ++u)
                            if ((mask >> u) & 1u) {
                                const int dz = u / 9, dy = (u / 3) % 3, dx = u % 3;
                                s = fmaf(sdict[byte_of(wrec, u)], P[dz][base + (j + dy) * pitch + dx - 1], s);
                            }
                    } else {
                        // a slot outside the grid (not a grid stencil there): x itself
                        const int64_t r = row0 + int64_t(j) * nx;
#pragma unroll
                        for (int u = 0; u < 27; ++u)
                            if ((mask >> u) & 1u) {
                                const int64_t c = r + a.uoff[u];
                                if (uint64_t(c) >= uint64_t(a.n)) {
                                    raise_error(a.err, 2);
                                    continue;
                                }
                                s = fmaf(sdict[byte_of(wrec, u)], __ldg(x + c), s);
                            }
                    }
                    acc[j] = s;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) y[row0 + int64_t(j) * nx] = acc[j];
            if constexpr (DOT) {
                float c = P[1][base + pitch] * acc[0];
#pragma unroll
                for (int j = 1; j < 4; ++j) c = fmaf(P[1][base + (j + 1) * pitch], acc[j], c);
                dacc += double(c);
            }
            release(raw_empty + sA);           // W(q-1) is no longer read
            release(typ_empty + stT);
            sA = sB;
            sB = sC;
        }
        if (aborted) break;
        release(raw_empty + sA);               // the run's last two windows
        release(raw_empty + sB);
    }
    // every compute thread is done with the rings; after an abort one
    // thread waits (bounded) for the producer to stop and for the copies it
    // had issued, which may still be in flight
    compute_sync(NC);
    if (aborted || *sabort) {
        if (tid == 0) {
            const long long t0 = clock64();
            while (*spdone < 2u && clock64() - t0 < kWaitCycles) {
            }
            const uint32_t iw = siss[0], it = siss[1];
            for (uint32_t i = iw > kF32RawStages ? iw - kF32RawStages : 0; i < iw; ++i)
                mbar_wait(raw_full + i % kF32RawStages, (i / kF32RawStages) & 1u);
            for (uint32_t i = it > kF32TypeStages ? it - kF32TypeStages : 0; i < it; ++i)
                mbar_wait(typ_full + i % kF32TypeStages, (i / kF32TypeStages) & 1u);
        }
    }
    if constexpr (DOT) {
        // the CTA's x.y: warp sums, then the warps in order (the value table
        // is no longer read and holds them)
        for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xFFFFFFFFu, dacc, o);
        double* const sred = reinterpret_cast<double*>(sdict);
        if (lane == 0) sred[tid >> 5] = dacc;
        compute_sync(NC);
        if (tid == 0) {
            double s = 0.0;
            for (int i = 0; i < (NC >> 5); ++i) s += sred[i];
            dot_part[blockIdx.x] = s;
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn_f32() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

}  // namespace

bool make_tma_f32_plan(const PatternFormat& p, const PatternView& v, int64_t n, int num_sms, TmaF32Plan* out) {
    if (v.nu != 27 || v.words != 7) return false;
    const std::vector<int32_t>& U = p.uoff;
    if (U.size() != 27) return false;
    const int64_t nx = U[16], S = U[22];
    if (nx < 3 || S <= 2 * nx + 2) return false;
    for (int u = 0; u < 27; ++u) {
        const int64_t dz = u / 9 - 1, dy = (u / 3) % 3 - 1, dx = u % 3 - 1;
        if (U[u] != dz * S + dy * nx + dx) return false;   // the 27-point box of an nx-wide grid
    }
    if (S % nx != 0 || n % S != 0 || S % 16 != 0) return false;
    const int64_t ny = S / nx, nz = n / S;
    if (nx % 4 != 0 || nx + 8 > 256 || nz < 1) return false;
    // the most lines a block (a multiple of four dividing ny) whose four-row
    // columns make whole warps and at most kF32MaxThreads threads
    int L = 0;
    for (int64_t l = 4; l <= ny && l + 2 <= 256; l += 4)
        if (ny % l == 0 && (l * nx) % 128 == 0 && l * nx / 4 <= kF32MaxThreads) L = int(l);
    if (L == 0) return false;
    auto up = [](int64_t v_, int64_t a_) { return (v_ + a_ - 1) / a_ * a_; };
    TmaF32Plan t{};
    t.nx = int32_t(nx);
    t.ny = int32_t(ny);
    t.nz = int32_t(nz);
    t.L = L;
    t.C = int32_t(L * nx);
    t.threads = t.C / 4;
    t.pitch = t.nx + 8;
    t.win_floats = (L + 2) * t.pitch;
    t.raw_stride = int32_t(up(t.win_floats, 32));             // 128-byte aligned stages
    t.nblk = int32_t(ny / L);
    t.S = S;
    t.grid = std::max(num_sms, 1);
    t.off_raw = 0;
    t.off_types = int32_t(up(int64_t(kF32RawStages) * t.raw_stride * 4, 128));
    t.off_tab = int32_t(up(t.off_types + int64_t(kF32TypeStages) * t.C, 128));
    t.off_tmask = t.off_tab + 256 * 8 * 4;
    t.off_dict = t.off_tmask + (256 + 64) * 4;
    t.off_words = t.off_dict + 256 * 4;
    t.off_mbar = t.off_words + 16;
    t.smem_bytes = int32_t(up(t.off_mbar + 8 * 2 * (kF32RawStages + kF32TypeStages), 128));
    if (t.smem_bytes > 227 * 1024) return false;
    for (int c = 0; c < 64; ++c) t.exp_type[c] = -1;   // set with the row types
    *out = t;
    return true;
}

cudaError_t launch_pattern_f32_tma(const PatternView& a, const TmaF32Plan& tp, const float* x, float* y,
                                   cudaStream_t s, double* dot_part, int* dot_n) {
    if (dot_n) *dot_n = 0;
    if (a.n == 0) return cudaSuccess;
    if (!a.rtype || !a.rtypes || a.ntypes < 1 || a.ntypes > 256 || a.dict_size > 256) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0 || (reinterpret_cast<uintptr_t>(a.rtype) & 15u) != 0)
        return cudaErrorNotSupported;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn_f32();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[3] = {cuuint64_t(tp.nx), cuuint64_t(tp.ny), cuuint64_t(tp.nz)};
    const cuuint64_t strides[2] = {cuuint64_t(tp.nx) * 4u, cuuint64_t(tp.S) * 4u};
    const cuuint32_t box[3] = {cuuint32_t(tp.pitch), cuuint32_t(tp.L + 2), 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    auto kernel = dot_part ? pattern_f32_tma_kernel<true> : pattern_f32_tma_kernel<false>;
    {
        static std::mutex mu;
        static bool set[64][2] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> g(mu);
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!set[dev][dot_part != nullptr]) {
            e = cudaFuncSetAttribute(reinterpret_cast<const void*>(kernel),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            if (e != cudaSuccess) return e;
            set[dev][dot_part != nullptr] = true;
        }
    }
    const int64_t units = int64_t(tp.nblk) * tp.nz;
    const unsigned grid = unsigned(std::min<int64_t>(units, tp.grid));
    kernel<<<grid, tp.threads + 32, tp.smem_bytes, s>>>(map, a, tp, x, y, dot_part);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && dot_n) *dot_n = int(grid);
    return e;
}

}  // namespace spmvc
