// SpMV kernels for sm_103a: y = A x (Eq. 1 of arXiv:1612.00530) over the
// library's three stored forms.  None of this is a dense contraction, so
// tensor cores are not used; the kernels stream the matrix once with
// coalesced, vectorised loads (evict-first), keep x in L2, and decode value
// codes and column patterns in registers and shared memory.
//
// Two summation orders:
//  - COLUMN: y_i = fma(a_ij, x_j, y_i) over ascending j from 0, exactly the
//    CPU CSR product, so results are bit-identical.  On GB300 the FP64 pipe
//    issues about 2 fma per clock per SM, which bounds these kernels.
//  - FAST (pattern format, integer-valued value tables): x is turned into
//    53-bit fixed point by integer bit manipulation, every row is summed
//    exactly with 32x32->64-bit integer multiply-adds, and one rounding to
//    nearest makes the double result -- no FP64 instruction per nonzero.
#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <cstdint>

#include "spmvc_internal.h"

namespace spmvc {

namespace {

#include "fast_fixed.cuh"

constexpr int kBlock = 256;
constexpr int kXmaxBlocks = 152;  // partial maxima written by the pre-pass



// true when the row's record equals the matrix's dominant record
template <int WORDS>
__device__ __forceinline__ bool is_dominant(const PatternView& a, const uint32_t (&w)[kMaxRecordWords]) {
    bool eq = a.dom_ok != 0;
#pragma unroll
    for (int k = 0; k < WORDS; ++k) eq = eq && (w[k] == a.dom_w[k]);
    return eq;
}

// Warp vote: true when every row of the warp carries the dominant record.
// All 32 lanes must reach the call (callers never return or break out of a
// row loop before it): a lane whose row lies past the matrix votes true and
// stores nothing, so the full-warp mask is exact.
template <int WORDS>
__device__ __forceinline__ bool warp_dominant(const PatternView& a, const uint32_t (&w)[kMaxRecordWords],
                                              bool valid) {
    return __all_sync(0xFFFFFFFFu, !valid || is_dominant<WORDS>(a, w));
}

// ------------------------------------------------------------- ELL -------
template <typename T>
__global__ void __launch_bounds__(kBlock) ell_kernel(EllView a, const T* __restrict__ x, T* __restrict__ y) {
    const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (r >= a.n) return;
    const int64_t s = r >> 5;
    const int64_t base = a.slice_off[s] + (r & 31);
    const int w = a.slice_w[s];
    T acc = T(0);
#pragma unroll 9
    for (int t = 0; t < w; ++t) {
        const int32_t c = __ldcs(a.col + base + 32 * t);
        T v;
        if constexpr (sizeof(T) == 8) v = __ldcs(a.val + base + 32 * t);
        else v = __ldcs(a.val32 + base + 32 * t);
        if (c >= 0) acc = fma(v, __ldg(x + c), acc);
    }
    y[r] = acc;
}

// ------------------------------------------------ pattern, COLUMN order ---
template <int WORDS, typename T>
__global__ void __launch_bounds__(kBlock) pattern_col_kernel(PatternView a, const T* __restrict__ x,
                                                             T* __restrict__ y) {
    __shared__ T sdict[256];
    __shared__ uint32_t smask[32];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        T v = T(0);
        if (i < a.dict_size) {
            if constexpr (sizeof(T) == 8) v = a.dict[i];
            else v = a.dict32[i];
        }
        sdict[i] = v;
    }
    if (threadIdx.x < 32) smask[threadIdx.x] = threadIdx.x < a.npat ? a.pmask[threadIdx.x] : 0u;
    __syncthreads();
    const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (r >= a.n) return;
    uint32_t w[kMaxRecordWords];
    load_record<WORDS>(a, r, w);
    const uint32_t pat = byte_of(w, a.nu);
    if (pat >= uint32_t(a.npat)) raise_error(a.err, 1);
    const uint32_t mask = smask[pat & 31];
    T acc = T(0);
#pragma unroll
    for (int u = 0; u < 4 * WORDS - 1; ++u) {
        if (u < a.nu && ((mask >> u) & 1u)) {
            const uint32_t code = byte_of(w, u);
            const int64_t c = r + a.uoff[u];
            if (code >= uint32_t(a.dict_size) || uint64_t(c) >= uint64_t(a.n)) {
                raise_error(a.err, 2);
                continue;
            }
            acc = fma(sdict[code], __ldg(x + c), acc);
        }
    }
    y[r] = acc;
}

// ---------------------------------------------------- FAST order ---------
// max over x of the high word with the sign cleared: its exponent field is
// the largest biased exponent E of any x_j.  One partial per block; the
// SpMV kernel reduces the partials itself, so no reset or atomic is needed.
__global__ void __launch_bounds__(1024) xmax_kernel(const double* __restrict__ x, int64_t n,
                                                    uint32_t* __restrict__ partial) {
    uint32_t m = 0;
    // doubles are 8-byte aligned; peel one element when x is not 16-byte
    // aligned, then read two doubles per 16-byte load
    const int64_t head = (n > 0 && (reinterpret_cast<uintptr_t>(x) & 15u)) ? 1 : 0;
    const uint4* __restrict__ x2 = reinterpret_cast<const uint4*>(x + head);
    const int64_t na = n - head, n2 = na / 2, stride = int64_t(gridDim.x) * blockDim.x;
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    for (; i + 3 * stride < n2; i += 4 * stride) {      // four independent loads in flight
        const uint4 a = __ldg(x2 + i), b = __ldg(x2 + i + stride);
        const uint4 c = __ldg(x2 + i + 2 * stride), d = __ldg(x2 + i + 3 * stride);
        m = max(m, max(max(a.y & 0x7FFFFFFFu, a.w & 0x7FFFFFFFu), max(b.y & 0x7FFFFFFFu, b.w & 0x7FFFFFFFu)));
        m = max(m, max(max(c.y & 0x7FFFFFFFu, c.w & 0x7FFFFFFFu), max(d.y & 0x7FFFFFFFu, d.w & 0x7FFFFFFFu)));
    }
    for (; i < n2; i += stride) {
        const uint4 a = __ldg(x2 + i);
        m = max(m, max(a.y & 0x7FFFFFFFu, a.w & 0x7FFFFFFFu));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (head) m = max(m, uint32_t(__double2hiint(__ldg(x))) & 0x7FFFFFFFu);
        if (na > 0 && (na & 1)) m = max(m, uint32_t(__double2hiint(__ldg(x + n - 1))) & 0x7FFFFFFFu);
    }
    m = __reduce_max_sync(0xFFFFFFFFu, m);
    __shared__ uint32_t sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0u;
        v = __reduce_max_sync(0xFFFFFFFFu, v);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

__device__ __forceinline__ int block_emax(const uint32_t* __restrict__ partial, int* s_emax) {
    if (threadIdx.x < 32) {
        uint32_t v = 0;
        for (int i = threadIdx.x; i < kXmaxBlocks; i += 32) v = max(v, __ldg(partial + i));
        v = __reduce_max_sync(0xFFFFFFFFu, v);
        if (threadIdx.x == 0) *s_emax = int(v >> 20);
    }
    __syncthreads();
    return *s_emax;
}

template <int WORDS>
__global__ void __launch_bounds__(kBlock) pattern_fast_kernel(PatternView a, const double* __restrict__ x,
                                                              double* __restrict__ y,
                                                              const uint32_t* __restrict__ partial) {
    __shared__ uint32_t smask[32];
    __shared__ double sdict[8];
    __shared__ int s_emax;
    if (threadIdx.x < 32) smask[threadIdx.x] = threadIdx.x < a.npat ? a.pmask[threadIdx.x] : 0u;
    if (threadIdx.x < 8) sdict[threadIdx.x] = threadIdx.x < a.dict_size ? a.dict[threadIdx.x] : 0.0;
    const int emax = block_emax(partial, &s_emax);
    const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (r >= a.n) return;
    uint32_t w[kMaxRecordWords];
    load_record<WORDS>(a, r, w);
    const uint32_t pat = byte_of(w, a.nu);
    if (pat >= uint32_t(a.npat)) raise_error(a.err, 1);
    const uint32_t mask = smask[pat & 31];
    if (emax < 64 || emax >= 2047) {
        // zero/denormal-only or non-finite x: the COLUMN order, same result rules as IEEE
        double acc = 0.0;
#pragma unroll
        for (int u = 0; u < 4 * WORDS - 1; ++u)
            if (u < a.nu && ((mask >> u) & 1u)) {
                const uint32_t code = byte_of(w, u);
                const int64_t c = r + a.uoff[u];
                if (code < uint32_t(a.dict_size) && uint64_t(c) < uint64_t(a.n))
                    acc = fma(sdict[code & 7], __ldg(x + c), acc);
            }
        y[r] = acc;
        return;
    }
    int64_t acc_h = 0, acc_l = 0;
#pragma unroll
    for (int u = 0; u < 4 * WORDS - 1; ++u) {
        if (u < a.nu) {
            const uint32_t code = byte_of(w, u);
            // multiplier of the code, sign-extended; absent slots map to 0
            const int32_t m = mult_of(a.mult_lo, a.mult_hi, code);
            const int64_t c = r + a.uoff[u];
            const bool inside = uint64_t(c) < uint64_t(a.n);
            const double xv = __ldg(x + (inside ? c : r));
            int32_t xh, xl;
            to_fixed(xv, emax, xh, xl);
            const int32_t mm = ((mask >> u) & 1u) ? m : 0;
            acc_h += int64_t(mm) * xh;
            acc_l += int64_t(mm) * xl;
        }
    }
    const int64_t acc = acc_h * (int64_t(1) << 26) + acc_l;
    y[r] = fixed_to_double(acc, emax - 1075 + a.mult_exp);
}


// ------------------------------------- FAST order, pre-converted x -------
// x is converted once per product into fixed-point limbs stored in a
// scratch copy with zero guard zones of `guard` elements on both sides, so
// that the row kernel reads X[r + d] for every union displacement d without
// a bounds check (out-of-range slots are absent ones, multiplier 0).
__device__ __forceinline__ int2 limbs_of(uint32_t lo, uint32_t hi, uint32_t emax) {
    const uint32_t k = emax - ((hi >> 20) & 0x7FFu);
    const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
    uint64_t v;
    asm("shr.b64 %0, %1, %2;" : "=l"(v) : "l"((uint64_t(mh) << 32) | lo), "r"(k));
    const int32_t s1 = (int32_t(hi) >> 31) | 1;
    return make_int2(int32_t(uint32_t(v) & 0x3FFFFFFu) * s1, int32_t(uint32_t(v >> 26)) * s1);
}

__global__ void __launch_bounds__(256) convert_x_kernel(const uint2* __restrict__ xw, int64_t n,
                                                        uint32_t* __restrict__ partial,
                                                        int2* __restrict__ X) {
    __shared__ int s_emax;
    const uint32_t emax = uint32_t(block_emax(partial, &s_emax));
    if (blockIdx.x == 0 && threadIdx.x == 0) partial[kXmaxBlocks] = emax;
    if (emax < 64u || emax >= 2047u) return;   // the row kernel takes the exact path
    // peel one element when x is not 16-byte aligned, then two per load
    const int64_t head = (n > 0 && (reinterpret_cast<uintptr_t>(xw) & 15u)) ? 1 : 0;
    const uint4* __restrict__ x2 = reinterpret_cast<const uint4*>(xw + head);
    int2* __restrict__ Xh = X + head;
    const int64_t na = n - head, n2 = na / 2, stride = int64_t(gridDim.x) * blockDim.x;
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    for (; i + stride < n2; i += 2 * stride) {
        const uint4 a = __ldcs(x2 + i), b = __ldcs(x2 + i + stride);
        Xh[2 * i] = limbs_of(a.x, a.y, emax);
        Xh[2 * i + 1] = limbs_of(a.z, a.w, emax);
        Xh[2 * (i + stride)] = limbs_of(b.x, b.y, emax);
        Xh[2 * (i + stride) + 1] = limbs_of(b.z, b.w, emax);
    }
    for (; i < n2; i += stride) {
        const uint4 a = __ldcs(x2 + i);
        Xh[2 * i] = limbs_of(a.x, a.y, emax);
        Xh[2 * i + 1] = limbs_of(a.z, a.w, emax);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (head) { const uint2 b = __ldg(xw); X[0] = limbs_of(b.x, b.y, emax); }
        if (na > 0 && (na & 1)) { const uint2 b = __ldg(xw + n - 1); X[n - 1] = limbs_of(b.x, b.y, emax); }
    }
}

template <int WORDS, int NU, int RUN>
__global__ void __launch_bounds__(kBlock, 6) pattern_fast_x_kernel(PatternView a, const double* __restrict__ x,
                                                                const int2* __restrict__ X,
                                                                double* __restrict__ y,
                                                                const uint32_t* __restrict__ partial) {
    // the largest exponent of x, left by the conversion pass
    const int emax = int(__ldg(partial + kXmaxBlocks));
    const int64_t r0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    // every lane stays for the warp vote: a lane past the last row works on
    // the last row and stores nothing
    const bool valid = r0 < a.n;
    const int64_t r = valid ? r0 : a.n - 1;
    uint32_t w[kMaxRecordWords];
    load_record<WORDS>(a, r, w);
    if (emax < 64 || emax >= 2047) {
        if (!valid) return;
        const uint32_t mask = __ldg(a.pmask_dev + (byte_of(w, NU) & 31));
        double acc = 0.0;
#pragma unroll
        for (int u = 0; u < NU; ++u)
            if ((mask >> u) & 1u)
                acc = fma(__ldg(a.dict + (byte_of(w, u) & 7)), __ldg(x + r + a.uoff[u]), acc);
        y[r] = acc;
        return;
    }
    // one pointer per run of RUN consecutive displacements, the run's other
    // slots at immediate offsets; three accumulator pairs shorten the
    // dependency chains
    const int2* __restrict__ Xr = X + r;
    int64_t ah[3] = {0, 0, 0}, al[3] = {0, 0, 0};
    if (warp_dominant<WORDS>(a, w, valid)) {
        // the warp's rows all carry the dominant record: multipliers are
        // kernel parameters
#pragma unroll
        for (int k = 0; k < NU / RUN; ++k) {
            const int2* __restrict__ p = Xr + a.uoff[k * RUN];
#pragma unroll
            for (int j = 0; j < RUN; ++j) {
                const int u = k * RUN + j;
                const int2 v = __ldg(p + j);
                ah[u % 3] += int64_t(a.dom_m[u]) * v.y;
                al[u % 3] += int64_t(a.dom_m[u]) * v.x;
            }
        }
    } else {
        uint32_t mw[(NU + 3) / 4];
#pragma unroll
        for (int k = 0; k < (NU + 3) / 4; ++k) mw[k] = prmt(a.mult_lo, a.mult_hi, prmt(w[k] | (w[k] >> 4), 0u, 0x0020u));
#pragma unroll
        for (int k = 0; k < NU / RUN; ++k) {
            const int2* __restrict__ p = Xr + a.uoff[k * RUN];
#pragma unroll
            for (int j = 0; j < RUN; ++j) {
                const int u = k * RUN + j;
                const int32_t m = int32_t(prmt(mw[u >> 2], 0u, uint32_t(u & 3) * 0x1111u + 0x8880u));
                const int2 v = __ldg(p + j);
                ah[u % 3] += int64_t(m) * v.y;
                al[u % 3] += int64_t(m) * v.x;
            }
        }
    }
    const int64_t acc = (ah[0] + ah[1] + ah[2]) * (int64_t(1) << 26) + (al[0] + al[1] + al[2]);
    if (valid) y[r] = fixed_to_double(acc, emax - 1075 + a.mult_exp);
}

// ---------------------------------------------- FAST order, staged -------
// One CTA per tile of sp.rows consecutive rows.  Phase 1 copies the x
// windows the tile touches (merged segments of the union displacements)
// into shared memory and takes their largest exponent; phase 2 converts
// every staged element once to two-limb fixed point in place; phase 3 sums
// each row slot by slot from shared memory with 32x32->64-bit multiply-adds
// and rounds once.  Windows outside [0, n) read as zero; they are only ever
// addressed by absent slots, whose multiplier is 0.  Everything is integer:
// x is moved as raw 64-bit words and never touches the FP64 pipe.
constexpr int kStageThreads = 512;

// 16-byte cp.async copy global -> shared of the first nbytes (0..16) of the
// source, zero-filling the rest (nbytes == 0 reads nothing).
__device__ __forceinline__ void cp16_zfill(void* sdst, const void* gsrc, uint32_t nbytes) {
    const uint32_t d = uint32_t(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(nbytes));
}

// Row phase of the staged kernels: every thread sums RPT rows (r0 + tid +
// i*THREADS) slot by slot from the tile's converted windows in shared memory
// (raw words on the exact path) and rounds once.  off(u): shared-memory
// index of slot u's element for the tile's first row.  w holds the record of the
// thread's first row (loaded by the caller before the tile's barriers, when
// that row exists); each row's loop issues the next row's record loads
// before it sums, so record latency overlaps the previous row's work.
// Where a row's record comes from (RECS): 0 global memory, the next row's
// record prefetched into registers (w holds the first row's on entry);
// 1 the tile's record planes copied to shared memory (srec, srows rows);
// 2 a one-byte row type indexing a table of distinct records in shared
// memory (srec, 8 words a type; tfirst is the first row's type).
template <int WORDS, int NU, int RPT, int RUN, int THREADS, typename Off, int RECS = 0>
__device__ __forceinline__ void tile_rows(const PatternView& a, Off off, const int2* sx, const uint32_t* smask,
                                          int64_t r0, uint32_t emax, bool exact_path, double* __restrict__ y,
                                          uint32_t (&w)[kMaxRecordWords], const uint32_t* srec = nullptr,
                                          int srows = 0, uint32_t tfirst = 0) {
    const int tid = threadIdx.x;
    uint32_t tcur = tfirst;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int rl = tid + i * THREADS;
        const int64_t r = r0 + rl;
        // rows past the matrix are summed from the tile's (zero-filled)
        // windows like the others, so the whole warp reaches the vote, and
        // are not stored
        const bool valid = r < a.n;
        uint32_t wn[kMaxRecordWords];
        uint32_t tnext = 0;
        if constexpr (RECS == 1) {
            // the tile's records were copied to shared memory: words 0..3, 4..5, 6
            static_assert(WORDS == 7, "shared-memory records are laid out for 7 words");
            const uint4 v = reinterpret_cast<const uint4*>(srec)[rl];
            const uint2 v2 = reinterpret_cast<const uint2*>(srec + 4 * srows)[rl];
            w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
            w[4] = v2.x; w[5] = v2.y;
            w[6] = srec[6 * srows + rl];
        } else if constexpr (RECS == 2) {
            static_assert(WORDS == 7, "typed records are laid out for 7 words");
            if (i + 1 < RPT && r + THREADS < a.n) tnext = __ldg(a.rtype + r + THREADS);
            const uint4 v = reinterpret_cast<const uint4*>(srec)[2 * tcur];
            const uint4 v2 = reinterpret_cast<const uint4*>(srec)[2 * tcur + 1];
            w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
            w[4] = v2.x; w[5] = v2.y; w[6] = v2.z;
        } else {
            if (i + 1 < RPT && r + THREADS < a.n) load_record<WORDS>(a, r + THREADS, wn);
        }
        if (exact_path) {
            // zeros/denormals only, or non-finite values: the COLUMN order
            if (valid) {
                const uint32_t mask = smask[byte_of(w, NU) & 31];
                double acc = 0.0;
#pragma unroll
                for (int u = 0; u < NU; ++u)
                    if ((mask >> u) & 1u) {
                        const int2 b = sx[rl + off(u)];
                        acc = fma(__ldg(a.dict + (byte_of(w, u) & 7)), __hiloint2double(b.y, b.x), acc);
                    }
                y[r] = acc;
            }
            if (RECS == 0 && i + 1 < RPT) {
#pragma unroll
                for (int k = 0; k < WORDS; ++k) w[k] = wn[k];
            }
            tcur = tnext;
            continue;
        }
        int64_t ah[3] = {0, 0, 0}, al[3] = {0, 0, 0};
        const bool dom = warp_dominant<WORDS>(a, w, valid);
        if (NU == 27 && RUN == 3 && dom && a.dom_uni) {
            // uniform neighbour weights: sum the 26 neighbour limbs exactly in
            // 32-bit integers (|xh| < 2^27: two partial sums of 13 terms;
            // |xl| < 2^26: one of 26), then scale once
            int32_t sh0 = 0, sh1 = 0, sl = 0;
            int2 vc = make_int2(0, 0);
#pragma unroll
            for (int k = 0; k < NU / RUN; ++k) {
                const int2* p = sx + rl + off(k * RUN);
#pragma unroll
                for (int j = 0; j < RUN; ++j) {
                    const int u = k * RUN + j;
                    const int2 v = p[j];
                    if (u == 13) { vc = v; continue; }
                    if (u < 13) sh0 += v.y;
                    else sh1 += v.y;
                    sl += v.x;
                }
            }
            ah[0] = int64_t(a.dom_mo) * sh0 + int64_t(a.dom_mo) * sh1;
            ah[1] = int64_t(a.dom_mc) * vc.y;
            al[0] = int64_t(a.dom_mo) * sl;
            al[1] = int64_t(a.dom_mc) * vc.x;
        } else if (dom) {
#pragma unroll
            for (int k = 0; k < NU / RUN; ++k) {
                const int2* p = sx + rl + off(k * RUN);
#pragma unroll
                for (int j = 0; j < RUN; ++j) {
                    const int u = k * RUN + j;
                    const int2 v = p[j];
                    ah[u % 3] += int64_t(a.dom_m[u]) * v.y;
                    al[u % 3] += int64_t(a.dom_m[u]) * v.x;
                }
            }
        } else {
            uint32_t mw[(NU + 3) / 4];
#pragma unroll
            for (int k = 0; k < (NU + 3) / 4; ++k) mw[k] = prmt(a.mult_lo, a.mult_hi, prmt(w[k] | (w[k] >> 4), 0u, 0x0020u));
#pragma unroll
            for (int k = 0; k < NU / RUN; ++k) {
                const int2* p = sx + rl + off(k * RUN);
#pragma unroll
                for (int j = 0; j < RUN; ++j) {
                    const int u = k * RUN + j;
                    const int32_t m = int32_t(prmt(mw[u >> 2], 0u, uint32_t(u & 3) * 0x1111u + 0x8880u));
                    const int2 v = p[j];
                    ah[u % 3] += int64_t(m) * v.y;
                    al[u % 3] += int64_t(m) * v.x;
                }
            }
        }
        const int64_t acc = (ah[0] + ah[1] + ah[2]) * (int64_t(1) << 26) + (al[0] + al[1] + al[2]);
        if (valid) y[r] = fixed_to_double(acc, int(emax) - 1075 + a.mult_exp);
        if (RECS == 0 && i + 1 < RPT) {
#pragma unroll
            for (int k = 0; k < WORDS; ++k) w[k] = wn[k];
        }
        tcur = tnext;
    }
}

// Every shape is held to the register budget of 1536 resident threads a SM
// (40 registers at 256 threads); eight rows a thread then spill a little.
template <int WORDS, int NU, int RPT, int RUN, int THREADS, bool VEC>
__global__ void __launch_bounds__(THREADS, 1536 / THREADS)
    pattern_fast_staged_kernel(PatternView a, StagePlan sp,
                                                                                    const double* __restrict__ x,
                                                                                    double* __restrict__ y) {
    extern __shared__ int4 sx4[];
    int2* const sx = reinterpret_cast<int2*>(sx4);
    __shared__ uint32_t s_red[THREADS / 32];
    __shared__ uint32_t smask[32];
    const int tid = threadIdx.x;
    const int64_t r0 = (sp.tile0 + int64_t(blockIdx.x)) * sp.rows;
    if (tid < 32) smask[tid] = tid < a.npat ? a.pmask[tid] : 0u;
    uint32_t w0[kMaxRecordWords];                  // first row's record, in flight during staging
    if (r0 + tid < a.n) load_record<WORDS>(a, r0 + tid, w0);
    // phase 1: stage raw words of x and find the tile's largest exponent
    uint32_t mx = 0;
#pragma unroll
    for (int sg = 0; sg < kMaxSegments; ++sg) {
        if (sg >= sp.nseg) break;
        if constexpr (VEC) {
            // 16-byte loads on the padded layout (x 16-byte aligned, window
            // starts rounded down to an even element)
            const int64_t g0 = r0 + sp.seg_min[sg] - sp.seg_pad[sg];
            const int len2 = (sp.rows + sp.seg_span[sg] + sp.seg_pad[sg] + 1) / 2;
            const uint4* __restrict__ src = reinterpret_cast<const uint4*>(x + g0);
            int4* dst = sx4 + sp.seg_pbase[sg] / 2;
            const int64_t lo = -g0, hi = a.n - g0;   // valid element range, relative
            for (int e = tid; e < len2; e += THREADS) {
                uint4 b;
                if (2 * e >= lo && 2 * e + 1 < hi) {
                    b = __ldg(src + e);
                } else {
                    b = make_uint4(0u, 0u, 0u, 0u);
                    if (2 * e >= lo && 2 * e < hi) { const uint2 h = __ldg(reinterpret_cast<const uint2*>(x + g0 + 2 * e)); b.x = h.x; b.y = h.y; }
                    if (2 * e + 1 >= lo && 2 * e + 1 < hi) { const uint2 h = __ldg(reinterpret_cast<const uint2*>(x + g0 + 2 * e + 1)); b.z = h.x; b.w = h.y; }
                }
                dst[e] = make_int4(int(b.x), int(b.y), int(b.z), int(b.w));
                mx = max(mx, max(b.y & 0x7FFFFFFFu, b.w & 0x7FFFFFFFu));
            }
        } else {
            const uint2* __restrict__ xw = reinterpret_cast<const uint2*>(x);
            const int64_t g0 = r0 + sp.seg_min[sg];
            const int len = sp.rows + sp.seg_span[sg];
            int2* dst = sx + sp.seg_base[sg];
            for (int e = tid; e < len; e += THREADS) {
                const int64_t idx = g0 + e;
                uint2 b = make_uint2(0u, 0u);
                if (uint64_t(idx) < uint64_t(a.n)) b = __ldg(xw + idx);
                dst[e] = make_int2(int(b.x), int(b.y));
                mx = max(mx, b.y & 0x7FFFFFFFu);
            }
        }
    }
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if ((tid & 31) == 0) s_red[tid >> 5] = mx;
    __syncthreads();
    mx = 0;
#pragma unroll
    for (int w = 0; w < THREADS / 32; ++w) mx = max(mx, s_red[w]);
    const uint32_t emax = mx >> 20;
    const bool exact_path = emax < 64u || emax >= 2047u;
    const int nel = VEC ? sp.elems_padded : sp.elems;
    // phase 2: convert in place, two elements per 16-byte access
    if (!exact_path) {
        for (int e = tid; e < (nel + 1) / 2; e += THREADS) {
            const int4 b = sx4[e];
            const int2 l0 = fixed_limbs(uint32_t(b.x), uint32_t(b.y), emax);
            const int2 l1 = fixed_limbs(uint32_t(b.z), uint32_t(b.w), emax);
            sx4[e] = make_int4(l0.x, l0.y, l1.x, l1.y);
        }
    }
    __syncthreads();
    // phase 3: rows
    tile_rows<WORDS, NU, RPT, RUN, THREADS>(a, [&](int u) { return VEC ? sp.soff_padded[u] : sp.soff[u]; }, sx,
                                            smask, r0, emax, exact_path, y, w0);
}

// ------------------------- FAST order, register-staged tiles (27 slots) ---
// For the full 27-point union, whose tile windows form three merged segments
// (planes z-1, z, z+1), every thread loads its QS 16-byte pairs of each
// window into registers at once -- all 3*QS loads in flight together -- the
// block reduces the tile's largest exponent, and each thread converts its
// own pairs to limbs and writes them to shared memory once.  Rows then sum
// from shared memory as in the staged kernel.  x must be 16-byte aligned;
// the plan must have three segments of at most 2*QS*THREADS elements each.
template <int QS, int RPT, int THREADS, int MINB, int RECS>
__global__ void __launch_bounds__(THREADS, MINB) pattern_fast_rstaged_kernel(PatternView a, StagePlan sp,
                                                                             const double* __restrict__ x,
                                                                             double* __restrict__ y) {
    extern __shared__ int4 sx4[];
    __shared__ uint32_t s_red[THREADS / 32];
    __shared__ uint32_t smask[32];
    const int tid = threadIdx.x;
    const int64_t r0 = (sp.tile0 + int64_t(blockIdx.x)) * sp.rows;
    if (tid < 32) smask[tid] = tid < a.npat ? a.pmask[tid] : 0u;
    const uint4* __restrict__ x4 = reinterpret_cast<const uint4*>(x);
    const uint2* __restrict__ x2 = reinterpret_cast<const uint2*>(x);
    uint32_t* srec = reinterpret_cast<uint32_t*>(sx4 + sp.elems_padded / 2);
    uint32_t w0[kMaxRecordWords];
    uint32_t t0 = 0;
    if constexpr (RECS == 0) {
        // first row's record in flight during the staging
        if (r0 + tid < a.n) load_record<7>(a, r0 + tid, w0);
    } else if constexpr (RECS == 1) {
        // the tile's records (planes of 16, 8 and 4 bytes per row) go to
        // shared memory behind the windows by cp.async, in flight during the
        // staging; rows past n read as zero
        const int64_t left = a.n - r0;             // rows of this tile that exist (>= 1)
        for (int c = tid; c < sp.rows; c += THREADS)
            cp16_zfill(srec + 4 * c, c < left ? static_cast<const void*>(a.p16a + r0 + c) : a.p16a,
                       c < left ? 16u : 0u);
        for (int c = tid; c < sp.rows / 2; c += THREADS) {
            const int64_t k = min(max(left - 2 * int64_t(c), int64_t(0)), int64_t(2));
            cp16_zfill(srec + 4 * sp.rows + 4 * c, k ? static_cast<const void*>(a.p8 + r0 + 2 * c) : a.p8,
                       uint32_t(k) * 8u);
        }
        for (int c = tid; c < sp.rows / 4; c += THREADS) {
            const int64_t k = min(max(left - 4 * int64_t(c), int64_t(0)), int64_t(4));
            cp16_zfill(srec + 6 * sp.rows + 4 * c, k ? static_cast<const void*>(a.p4 + r0 + 4 * c) : a.p4,
                       uint32_t(k) * 4u);
        }
        asm volatile("cp.async.commit_group;");
    } else {
        // the table of distinct records (8 words a type) behind the windows,
        // and the first row's type
        for (int i = tid; i < a.ntypes * 8; i += THREADS) srec[i] = __ldg(a.rtypes + i);
        if (r0 + tid < a.n) t0 = __ldg(a.rtype + r0 + tid);
    }
    // phase 1: every pair of the three windows this thread owns, in flight
    // together; a tile whose windows lie inside [0, n) skips the bounds tests
    uint4 b[3][QS];
    const bool interior = r0 + sp.seg_min[0] - sp.seg_pad[0] >= 0 &&
                          r0 + sp.seg_min[2] + sp.seg_span[2] + sp.rows + 1 < a.n;
#pragma unroll
    for (int sg = 0; sg < 3; ++sg) {
        const int64_t g0 = r0 + sp.seg_min[sg] - sp.seg_pad[sg];   // even
        const int len2 = (sp.rows + sp.seg_span[sg] + sp.seg_pad[sg] + 1) / 2;
        if (interior) {
            const uint4* __restrict__ w4 = x4 + (g0 >> 1);
#pragma unroll
            for (int j = 0; j < QS; ++j) {
                const int q = tid + j * THREADS;
                b[sg][j] = q < len2 ? __ldg(w4 + q) : make_uint4(0u, 0u, 0u, 0u);
            }
            continue;
        }
#pragma unroll
        for (int j = 0; j < QS; ++j) {
            const int q = tid + j * THREADS;
            const int64_t g = g0 + 2 * q;                               // first element of the pair
            b[sg][j] = make_uint4(0u, 0u, 0u, 0u);
            if (q < len2) {
                if (uint64_t(g) < uint64_t(a.n - 1)) {                  // 0 <= g and g + 1 < n
                    b[sg][j] = __ldg(x4 + (g >> 1));
                } else if (g == a.n - 1) {                              // odd n: the last element alone
                    const uint2 h = __ldg(x2 + g);
                    b[sg][j].x = h.x;
                    b[sg][j].y = h.y;
                }
            }
        }
    }
    uint32_t mx = 0;
#pragma unroll
    for (int sg = 0; sg < 3; ++sg)
#pragma unroll
        for (int j = 0; j < QS; ++j) mx = max(mx, max(b[sg][j].y & 0x7FFFFFFFu, b[sg][j].w & 0x7FFFFFFFu));
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if ((tid & 31) == 0) s_red[tid >> 5] = mx;
    __syncthreads();
    mx = 0;
#pragma unroll
    for (int w = 0; w < THREADS / 32; ++w) mx = max(mx, s_red[w]);
    const uint32_t emax = mx >> 20;
    const bool exact_path = emax < 64u || emax >= 2047u;
    // phase 2: convert the pairs in registers, one shared-memory write each
#pragma unroll
    for (int sg = 0; sg < 3; ++sg) {
        const int len2 = (sp.rows + sp.seg_span[sg] + sp.seg_pad[sg] + 1) / 2;
        int4* dst = sx4 + sp.seg_pbase[sg] / 2;
#pragma unroll
        for (int j = 0; j < QS; ++j) {
            const int q = tid + j * THREADS;
            if (q >= len2) continue;
            const uint4 v = b[sg][j];
            if (exact_path) {
                dst[q] = make_int4(int(v.x), int(v.y), int(v.z), int(v.w));
            } else {
                const int2 l0 = fixed_limbs(v.x, v.y, emax);
                const int2 l1 = fixed_limbs(v.z, v.w, emax);
                dst[q] = make_int4(l0.x, l0.y, l1.x, l1.y);
            }
        }
    }
    if constexpr (RECS == 1) asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    auto off = [&](int u) { return sp.soff_padded[u]; };
    tile_rows<7, 27, RPT, 3, THREADS, decltype(off), RECS>(a, off, reinterpret_cast<const int2*>(sx4), smask, r0,
                                                           emax, exact_path, y, w0, srec, sp.rows, t0);
}

// ------------------------------------- FAST order, z-marching tiles ------
// The full 27-point union's tile windows are three copies of one window
// shape spaced by the plane stride S.  A CTA keeps the windows of planes
// z-1, z, z+1 of its column block converted in a ring of three shared-memory
// slots and walks z upward: each step computes plane z's rows while the
// 16-byte loads of window W(z+2) are in flight, then converts W(z+2) into
// the slot W(z-1) leaves.  Every x element is loaded and converted about
// once per column block instead of three times.  The exponent is the
// vector's largest one (a pre-pass), so all windows share one scale.
template <int QS, int THREADS>
__device__ __forceinline__ void zmarch_load(const PatternView& a, const ZPlan& zp, const double* __restrict__ x,
                                            int64_t z, int64_t col0, uint4 (&b)[QS]) {
    const int64_t g = z * zp.S + col0 + zp.m1;
    const int64_t g0 = g - (g & 1);                       // even: 16-byte aligned
    const uint4* __restrict__ x4 = reinterpret_cast<const uint4*>(x);
    const uint2* __restrict__ x2 = reinterpret_cast<const uint2*>(x);
#pragma unroll
    for (int j = 0; j < QS; ++j) {
        const int q = threadIdx.x + j * THREADS;
        const int64_t e = g0 + 2 * q;
        b[j] = make_uint4(0u, 0u, 0u, 0u);
        if (q < zp.pairs) {
            if (uint64_t(e) < uint64_t(a.n - 1)) {
                b[j] = __ldg(x4 + (e >> 1));
            } else if (e == a.n - 1) {
                const uint2 h = __ldg(x2 + e);
                b[j].x = h.x;
                b[j].y = h.y;
            }
        }
    }
}

template <int QS, int THREADS>
__device__ __forceinline__ void zmarch_store(const ZPlan& zp, int4* sx4, int64_t z, const uint4 (&b)[QS],
                                             uint32_t emax, bool exact_path) {
    int4* dst = sx4 + int((z + 3) % 3) * (zp.slot / 2);
#pragma unroll
    for (int j = 0; j < QS; ++j) {
        const int q = threadIdx.x + j * THREADS;
        if (q >= zp.pairs) continue;
        const uint4 v = b[j];
        if (exact_path) {
            dst[q] = make_int4(int(v.x), int(v.y), int(v.z), int(v.w));
        } else {
            const int2 l0 = fixed_limbs(v.x, v.y, emax);
            const int2 l1 = fixed_limbs(v.z, v.w, emax);
            dst[q] = make_int4(l0.x, l0.y, l1.x, l1.y);
        }
    }
}

template <int RPT, int THREADS, int MINB, int QS>
__global__ void __launch_bounds__(THREADS, MINB) pattern_fast_zmarch_kernel(PatternView a, ZPlan zp,
                                                                            const double* __restrict__ x,
                                                                            double* __restrict__ y,
                                                                            const uint32_t* __restrict__ partial) {
    extern __shared__ int4 sx4[];
    __shared__ uint32_t smask[32];
    __shared__ int s_emax;
    const int tid = threadIdx.x;
    const int blk = int(blockIdx.x % unsigned(zp.nblk));
    const int64_t z0 = int64_t(blockIdx.x / unsigned(zp.nblk)) * zp.zc;
    const int64_t z1 = min(zp.nplanes, z0 + zp.zc);
    const int64_t col0 = int64_t(blk) * zp.rows;
    if (tid < 32) smask[tid] = tid < a.npat ? a.pmask[tid] : 0u;
    const uint32_t emax = uint32_t(block_emax(partial, &s_emax));   // also orders smask
    const bool exact_path = emax < 64u || emax >= 2047u;
    uint4 b[QS];
    // the ring starts with W(z0-1), W(z0), W(z0+1)
    for (int64_t z = z0 - 1; z <= z0 + 1; ++z) {
        zmarch_load<QS, THREADS>(a, zp, x, z, col0, b);
        zmarch_store<QS, THREADS>(zp, sx4, z, b, emax, exact_path);
    }
    __syncthreads();
    const int2* sx = reinterpret_cast<const int2*>(sx4);
    uint32_t w0[kMaxRecordWords];                        // first row's record of the step
    if (z0 * zp.S + col0 + tid < a.n) load_record<7>(a, z0 * zp.S + col0 + tid, w0);
    for (int64_t z = z0; z < z1; ++z) {
        const bool more = z + 2 <= z1;                   // plane z+1 is this CTA's: it needs W(z+2)
        if (more) zmarch_load<QS, THREADS>(a, zp, x, z + 2, col0, b);
        const int64_t r0 = z * zp.S + col0;
        // shared-memory index of each segment's window start for local row 0
        int base[3];
#pragma unroll
        for (int sg = 0; sg < 3; ++sg) {
            const int64_t zz = z - 1 + sg;
            base[sg] = int((zz + 3) % 3) * zp.slot + int((zz * zp.S + col0 + zp.m1) & 1);
        }
        tile_rows<7, 27, RPT, 3, THREADS>(a, [&](int u) { return base[u / 9] + zp.rel[u]; }, sx, smask, r0, emax,
                                          exact_path, y, w0);
        // the next step's first record, in flight across the barriers
        if (z + 1 < z1 && r0 + zp.S + tid < a.n) load_record<7>(a, r0 + zp.S + tid, w0);
        __syncthreads();                                 // W(z-1)'s slot is free
        if (more) zmarch_store<QS, THREADS>(zp, sx4, z + 2, b, emax, exact_path);
        __syncthreads();
    }
}

// --------------------------------------------- FAST order, z-block tiles -
// A CTA owns a column block of zp.rows rows in ZC consecutive planes
// z0 .. z0+ZC-1 (the z-marching plan's window shape).  Those planes need the
// ZC+2 windows W(z0-1) .. W(z0+ZC): every thread loads its QS 16-byte pairs
// of each window into registers at once, the block reduces the largest
// exponent over all of them, and each thread converts its pairs and writes
// them to shared memory once.  The ZC planes' rows then sum from shared
// memory with no further barrier.  Each x element is loaded and converted
// (ZC+2)/ZC times per column block instead of three times, and the exponent
// is the CTA's own (no pre-pass).  x must be 16-byte aligned.
template <int ZC, int QS, int RPT, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) pattern_fast_zblock_kernel(PatternView a, ZPlan zp,
                                                                           const double* __restrict__ x,
                                                                           double* __restrict__ y) {
    extern __shared__ int4 sx4[];
    __shared__ uint32_t s_red[THREADS / 32];
    __shared__ uint32_t smask[32];
    const int tid = threadIdx.x;
    const int64_t z0 = (int64_t(blockIdx.x / unsigned(zp.nblk)) + zp.chunk0) * ZC;
    const int64_t col0 = int64_t(blockIdx.x % unsigned(zp.nblk)) * zp.rows;
    if (tid < 32) smask[tid] = tid < a.npat ? a.pmask[tid] : 0u;
    const uint4* __restrict__ x4 = reinterpret_cast<const uint4*>(x);
    const uint2* __restrict__ x2 = reinterpret_cast<const uint2*>(x);
    // window W(z) covers the pairs from the even element at or below
    // z*S + col0 + m1; a CTA whose windows all lie inside [0, n) skips the
    // bounds tests
    const int64_t gfirst = (z0 - 1) * zp.S + col0 + zp.m1;
    const int64_t glast = (z0 + ZC) * zp.S + col0 + zp.m1;
    const bool interior = gfirst >= 1 && glast + 2 * int64_t(zp.pairs) <= a.n;
    uint4 b[ZC + 2][QS];
#pragma unroll
    for (int w = 0; w < ZC + 2; ++w) {
        const int64_t g = gfirst + int64_t(w) * zp.S;
        const int64_t g0 = g - (g & 1);
#pragma unroll
        for (int j = 0; j < QS; ++j) {
            const int q = tid + j * THREADS;
            const int64_t e = g0 + 2 * q;
            b[w][j] = make_uint4(0u, 0u, 0u, 0u);
            if (q < zp.pairs) {
                if (interior || uint64_t(e) < uint64_t(a.n - 1)) {        // 0 <= e and e + 1 < n
                    b[w][j] = __ldg(x4 + (e >> 1));
                } else if (e == a.n - 1) {                                 // odd n: the last element alone
                    const uint2 h = __ldg(x2 + e);
                    b[w][j].x = h.x;
                    b[w][j].y = h.y;
                }
            }
        }
    }
    uint32_t mx = 0;
#pragma unroll
    for (int w = 0; w < ZC + 2; ++w)
#pragma unroll
        for (int j = 0; j < QS; ++j) mx = max(mx, max(b[w][j].y & 0x7FFFFFFFu, b[w][j].w & 0x7FFFFFFFu));
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if ((tid & 31) == 0) s_red[tid >> 5] = mx;
    __syncthreads();
    mx = 0;
#pragma unroll
    for (int w = 0; w < THREADS / 32; ++w) mx = max(mx, s_red[w]);
    const uint32_t emax = mx >> 20;
    const bool exact_path = emax < 64u || emax >= 2047u;
#pragma unroll
    for (int w = 0; w < ZC + 2; ++w) {
        int4* dst = sx4 + w * (zp.slot / 2);
#pragma unroll
        for (int j = 0; j < QS; ++j) {
            const int q = tid + j * THREADS;
            if (q >= zp.pairs) continue;
            const uint4 v = b[w][j];
            if (exact_path) {
                dst[q] = make_int4(int(v.x), int(v.y), int(v.z), int(v.w));
            } else {
                const int2 l0 = fixed_limbs(v.x, v.y, emax);
                const int2 l1 = fixed_limbs(v.z, v.w, emax);
                dst[q] = make_int4(l0.x, l0.y, l1.x, l1.y);
            }
        }
    }
    __syncthreads();
    const int2* sx = reinterpret_cast<const int2*>(sx4);
#pragma unroll 1
    for (int k = 0; k < ZC; ++k) {
        const int64_t z = z0 + k;
        if (z >= zp.nplanes) break;
        const int64_t r0 = z * zp.S + col0;
        // shared-memory index of each segment's window start for local row 0
        int base[3];
#pragma unroll
        for (int sg = 0; sg < 3; ++sg)
            base[sg] = (k + sg) * zp.slot + int((gfirst + int64_t(k + sg) * zp.S) & 1);
        uint32_t w0[kMaxRecordWords];
        if (r0 + tid < a.n) load_record<7>(a, r0 + tid, w0);
        tile_rows<7, 27, RPT, 3, THREADS>(a, [&](int u) { return base[u / 9] + zp.rel[u]; }, sx, smask, r0, emax,
                                          exact_path, y, w0);
    }
}

// ------------------- FAST order, staged tiles of the pre-converted copy ---
// As the staged kernel, but the tile's windows are copied from the
// fixed-point copy X (guard zones make every window index valid), so the
// CTA neither reduces an exponent nor converts: phase 1 is a plain 16-byte
// copy into shared memory, phase 2 the rows.
template <int WORDS, int NU, int RPT, int RUN>
__global__ void __launch_bounds__(kStageThreads, 3) pattern_fast_xstaged_kernel(PatternView a, StagePlan sp,
                                                                             const double* __restrict__ x,
                                                                             const int2* __restrict__ X,
                                                                             double* __restrict__ y,
                                                                             const uint32_t* __restrict__ partial) {
    extern __shared__ int4 sx4[];
    const int2* sx = reinterpret_cast<const int2*>(sx4);
    const int tid = threadIdx.x;
    const int64_t r0 = int64_t(blockIdx.x) * sp.rows;
    const int emax = int(__ldg(partial + kXmaxBlocks));
    const bool exact_path = emax < 64 || emax >= 2047;
    if (!exact_path) {
#pragma unroll
        for (int sg = 0; sg < kMaxSegments; ++sg) {
            if (sg >= sp.nseg) break;
            // segment windows start at an even element (the plan keeps seg_base even
            // and rounds the global start down), so both sides are 16-byte aligned
            const int64_t g0 = r0 + sp.seg_min[sg] - sp.seg_pad[sg];
            const int len2 = (sp.rows + sp.seg_span[sg] + sp.seg_pad[sg] + 1) / 2;
            const int4* src = reinterpret_cast<const int4*>(X + g0);
            int4* dst = sx4 + sp.seg_pbase[sg] / 2;
            for (int e = tid; e < len2; e += kStageThreads) dst[e] = __ldg(src + e);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int rl = tid + i * kStageThreads;
        // a row past the matrix reads the last row's record, is summed from
        // the tile's windows so the whole warp reaches the vote, and is not
        // stored
        const bool valid = r0 + rl < a.n;
        const int64_t r = valid ? r0 + rl : a.n - 1;
        uint32_t w[kMaxRecordWords];
        load_record<WORDS>(a, r, w);
        if (exact_path) {
            if (!valid) continue;
            const uint32_t mask = __ldg(a.pmask_dev + (byte_of(w, NU) & 31));
            double acc = 0.0;
#pragma unroll
            for (int u = 0; u < NU; ++u)
                if ((mask >> u) & 1u)
                    acc = fma(__ldg(a.dict + (byte_of(w, u) & 7)), __ldg(x + r + a.uoff[u]), acc);
            y[r] = acc;
            continue;
        }
        int64_t ah[3] = {0, 0, 0}, al[3] = {0, 0, 0};
        if (warp_dominant<WORDS>(a, w, valid)) {
#pragma unroll
            for (int k = 0; k < NU / RUN; ++k) {
                const int2* p = sx + rl + sp.soff_padded[k * RUN];
#pragma unroll
                for (int j = 0; j < RUN; ++j) {
                    const int u = k * RUN + j;
                    const int2 v = p[j];
                    ah[u % 3] += int64_t(a.dom_m[u]) * v.y;
                    al[u % 3] += int64_t(a.dom_m[u]) * v.x;
                }
            }
        } else {
            uint32_t mw[(NU + 3) / 4];
#pragma unroll
            for (int k = 0; k < (NU + 3) / 4; ++k) mw[k] = prmt(a.mult_lo, a.mult_hi, prmt(w[k] | (w[k] >> 4), 0u, 0x0020u));
#pragma unroll
            for (int k = 0; k < NU / RUN; ++k) {
                const int2* p = sx + rl + sp.soff_padded[k * RUN];
#pragma unroll
                for (int j = 0; j < RUN; ++j) {
                    const int u = k * RUN + j;
                    const int32_t m = int32_t(prmt(mw[u >> 2], 0u, uint32_t(u & 3) * 0x1111u + 0x8880u));
                    const int2 v = p[j];
                    ah[u % 3] += int64_t(m) * v.y;
                    al[u % 3] += int64_t(m) * v.x;
                }
            }
        }
        const int64_t acc = (ah[0] + ah[1] + ah[2]) * (int64_t(1) << 26) + (al[0] + al[1] + al[2]);
        if (valid) y[r] = fixed_to_double(acc, emax - 1075 + a.mult_exp);
    }
}


// ------------------------------- FAST order, persistent, double-buffered --
// One CTA of 1024 threads per SM walks tiles of 1024 rows.  While it
// converts and sums tile t from shared memory, the cp.async copies of tile
// t+1 -- the x windows of its merged segments (8-byte copies, zero-filled
// outside [0, n)) and its row records (16/8/4-byte planes, zero-filled past
// n) -- are already in flight into the other buffer.  cp.async groups and
// block barriers order everything; the kernel has no spin-wait of its own.
constexpr int kAsyncThreads = 1024;
constexpr int kAsyncRows = 1024;

__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, bool valid) {
    const uint32_t d = uint32_t(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gsrc), "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc, bool valid) {
    const uint32_t d = uint32_t(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gsrc), "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
    const uint32_t d = uint32_t(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

struct AsyncBuf {
    int2* xw;        // staged x windows, elems entries
    uint4* r16;      // record words 0..3
    uint2* r8;       // words 4..5
    uint32_t* r4;    // word 6
};

// Issues the copies of tile `tile` into `b` (WORDS == 7 record layout).
__device__ __forceinline__ void async_issue(const PatternView& a, const StagePlan& sp, const double* __restrict__ x,
                                            int64_t tile, const AsyncBuf& b) {
    const int tid = threadIdx.x;
    const int64_t r0 = tile * kAsyncRows;
#pragma unroll
    for (int sg = 0; sg < kMaxSegments; ++sg) {
        if (sg >= sp.nseg) break;
        const int64_t g0 = r0 + sp.seg_min[sg];
        const int len = kAsyncRows + sp.seg_span[sg];
        int2* dst = b.xw + sp.seg_base[sg];
        for (int e = tid; e < len; e += kAsyncThreads) {
            const int64_t idx = g0 + e;
            const bool ok = uint64_t(idx) < uint64_t(a.n);
            cp_async8(dst + e, x + (ok ? idx : 0), ok);
        }
    }
    const int64_t r = r0 + tid;
    const bool ok = r < a.n;
    const int64_t rs = ok ? r : 0;
    cp_async16(b.r16 + tid, a.p16a + rs, ok);
    cp_async8(b.r8 + tid, a.p8 + rs, ok);
    cp_async4(b.r4 + tid, a.p4 + rs, ok);
    cp_async_commit();
}

// Issues the copies of tile `tile` of the pre-converted copy X (guard zones
// make every window index valid; 16-byte copies on the padded layout).
__device__ __forceinline__ void async_issue_x(const PatternView& a, const StagePlan& sp, const int2* __restrict__ X,
                                              int64_t tile, const AsyncBuf& b) {
    const int tid = threadIdx.x;
    const int64_t r0 = tile * kAsyncRows;
#pragma unroll
    for (int sg = 0; sg < kMaxSegments; ++sg) {
        if (sg >= sp.nseg) break;
        const int4* src = reinterpret_cast<const int4*>(X + (r0 + sp.seg_min[sg] - sp.seg_pad[sg]));
        int4* dst = reinterpret_cast<int4*>(b.xw + sp.seg_pbase[sg]);
        const int len2 = (kAsyncRows + sp.seg_span[sg] + sp.seg_pad[sg] + 1) / 2;
        for (int e = tid; e < len2; e += kAsyncThreads) cp_async16(dst + e, src + e, true);
    }
    const int64_t r = r0 + tid;
    const bool ok = r < a.n;
    const int64_t rs = ok ? r : 0;
    cp_async16(b.r16 + tid, a.p16a + rs, ok);
    cp_async8(b.r8 + tid, a.p8 + rs, ok);
    cp_async4(b.r4 + tid, a.p4 + rs, ok);
    cp_async_commit();
}

template <int NU, int RUN, bool PRECONVERTED>
__global__ void __launch_bounds__(kAsyncThreads, 1) pattern_fast_async_kernel(PatternView a, StagePlan sp,
                                                                              const double* __restrict__ x,
                                                                              const int2* __restrict__ X,
                                                                              double* __restrict__ y,
                                                                              int64_t ntiles,
                                                                              const uint32_t* __restrict__ partial) {
    constexpr int WORDS = 7;
    extern __shared__ int4 smem4[];
    __shared__ uint32_t s_red[kAsyncThreads / 32];
    __shared__ double sdict[8];
    __shared__ uint32_t smask[32];
    const int tid = threadIdx.x;
    if (tid < 8) sdict[tid] = tid < a.dict_size ? a.dict[tid] : 0.0;
    if (tid < 32) smask[tid] = tid < a.npat ? a.pmask[tid] : 0u;
    // two buffers, each [x windows | r16 | r8 | r4]; pointers computed from
    // the buffer index (no runtime-indexed local arrays)
    const uint32_t xbytes = (uint32_t(PRECONVERTED ? sp.elems_padded : sp.elems) * 8u + 15u) / 16u * 16u;
    const uint32_t bbytes = xbytes + uint32_t(kAsyncRows) * 28u;
    char* const smem = reinterpret_cast<char*>(smem4);
    // FAST order scale: the largest exponent of x (left by the conversion
    // pass) for the pre-converted copy; per tile otherwise
    const uint32_t emax_x = PRECONVERTED ? __ldg(partial + kXmaxBlocks) : 0u;
    auto buffer = [&](int q) {
        AsyncBuf bb;
        char* base = smem + q * bbytes;
        bb.xw = reinterpret_cast<int2*>(base);
        bb.r16 = reinterpret_cast<uint4*>(base + xbytes);
        bb.r8 = reinterpret_cast<uint2*>(base + xbytes + kAsyncRows * 16);
        bb.r4 = reinterpret_cast<uint32_t*>(base + xbytes + kAsyncRows * 24);
        return bb;
    };
    const bool x_exact = PRECONVERTED && (emax_x < 64u || emax_x >= 2047u);
    auto issue = [&](int64_t t, const AsyncBuf& bb) {
        if (PRECONVERTED && !x_exact) async_issue_x(a, sp, X, t, bb);
        else async_issue(a, sp, x, t, bb);
    };
    int64_t tile = blockIdx.x;
    if (tile < ntiles) issue(tile, buffer(0));
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const AsyncBuf cur = buffer(it & 1);
        cp_async_wait<0>();              // this thread's copies of `tile` have landed
        __syncthreads();                 // everybody's have, and the other buffer is free
        const int64_t next = tile + gridDim.x;
        if (next < ntiles) issue(next, buffer((it + 1) & 1));
        uint32_t emax;
        bool exact_path;
        int soff_shift;     // pre-converted copy: padded layout
        if constexpr (PRECONVERTED) {
            emax = emax_x;
            exact_path = x_exact;
            soff_shift = 1;
        } else {
            soff_shift = 0;
            // largest exponent of the staged windows
            uint32_t mx = 0;
            for (int e = tid; e < sp.elems; e += kAsyncThreads) mx = max(mx, uint32_t(cur.xw[e].y) & 0x7FFFFFFFu);
            mx = __reduce_max_sync(0xFFFFFFFFu, mx);
            if ((tid & 31) == 0) s_red[tid >> 5] = mx;
            __syncthreads();
            mx = 0;
#pragma unroll
            for (int w = 0; w < kAsyncThreads / 32; ++w) mx = max(mx, s_red[w]);
            emax = mx >> 20;
            exact_path = emax < 64u || emax >= 2047u;
            if (!exact_path)
                for (int e = tid; e < sp.elems; e += kAsyncThreads) {
                    const int2 b = cur.xw[e];
                    cur.xw[e] = limbs_of(uint32_t(b.x), uint32_t(b.y), emax);
                }
            __syncthreads();
        }
        const int64_t r = tile * kAsyncRows + tid;
        // rows past the matrix read the zero-filled end of the tile's buffer,
        // so the whole warp reaches the vote; they are not stored
        const bool valid = r < a.n;
        {
            uint32_t w[kMaxRecordWords];
            {
                const uint4 v16 = cur.r16[tid];
                const uint2 v8 = cur.r8[tid];
                w[0] = v16.x; w[1] = v16.y; w[2] = v16.z; w[3] = v16.w;
                w[4] = v8.x; w[5] = v8.y; w[6] = cur.r4[tid];
            }
            if (exact_path) {
                const uint32_t mask = smask[byte_of(w, NU) & 31];
                double acc = 0.0;
#pragma unroll
                for (int u = 0; u < NU; ++u)
                    if ((mask >> u) & 1u) {
                        const int2 b = cur.xw[tid + sp.soff[u]];   // raw copies (unpadded layout)
                        acc = fma(sdict[byte_of(w, u) & 7], __hiloint2double(b.y, b.x), acc);
                    }
                if (valid) y[r] = acc;
            } else {
                int64_t ah[3] = {0, 0, 0}, al[3] = {0, 0, 0};
                if (warp_dominant<WORDS>(a, w, valid)) {
#pragma unroll
                    for (int k = 0; k < NU / RUN; ++k) {
                        const int2* p = cur.xw + tid + (soff_shift ? sp.soff_padded[k * RUN] : sp.soff[k * RUN]);
#pragma unroll
                        for (int j = 0; j < RUN; ++j) {
                            const int u = k * RUN + j;
                            const int2 v = p[j];
                            ah[u % 3] += int64_t(a.dom_m[u]) * v.y;
                            al[u % 3] += int64_t(a.dom_m[u]) * v.x;
                        }
                    }
                } else {
                    uint32_t mw[(NU + 3) / 4];
#pragma unroll
                    for (int k = 0; k < (NU + 3) / 4; ++k)
                        mw[k] = prmt(a.mult_lo, a.mult_hi, prmt(w[k] | (w[k] >> 4), 0u, 0x0020u));
#pragma unroll
                    for (int k = 0; k < NU / RUN; ++k) {
                        const int2* p = cur.xw + tid + (soff_shift ? sp.soff_padded[k * RUN] : sp.soff[k * RUN]);
#pragma unroll
                        for (int j = 0; j < RUN; ++j) {
                            const int u = k * RUN + j;
                            const int32_t m = int32_t(prmt(mw[u >> 2], 0u, uint32_t(u & 3) * 0x1111u + 0x8880u));
                            const int2 v = p[j];
                            ah[u % 3] += int64_t(m) * v.y;
                            al[u % 3] += int64_t(m) * v.x;
                        }
                    }
                }
                const int64_t acc = (ah[0] + ah[1] + ah[2]) * (int64_t(1) << 26) + (al[0] + al[1] + al[2]);
                if (valid) y[r] = fixed_to_double(acc, int(emax) - 1075 + a.mult_exp);
            }
        }
        // the barrier at the top of the next iteration keeps `cur` from being
        // refilled while any thread still reads it
    }
}

// ------------------------------ SpMM, FAST order, pre-converted block X ---
// Per-column largest exponents (one word per column, from the partial
// maxima of xmax_cols_kernel), then X converted once into a fixed-point
// copy with guard rows, then Y = A X with one thread per (row, column).
__global__ void cols_emax_kernel(const uint32_t* __restrict__ partial, int k, uint32_t* __restrict__ emax) {
    const int j = threadIdx.x;
    if (j >= k) return;
    uint32_t v = 0;
    for (int b = 0; b < kXmaxBlocks; ++b) v = max(v, __ldg(partial + b * k + j));
    emax[j] = v >> 20;
}

__global__ void __launch_bounds__(256) convert_cols_kernel(const double* __restrict__ X, int64_t ldx, int64_t n, int k,
                                                           const uint32_t* __restrict__ emax,
                                                           int2* __restrict__ Xf) {
    const int64_t total = n * k, stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += stride) {
        const int64_t r = e / k;
        const int j = int(e - r * k);
        const uint32_t E = __ldg(emax + j);
        if (E < 64u || E >= 2047u) continue;   // that column takes the exact path
        const uint2 b = __ldg(reinterpret_cast<const uint2*>(X + r * ldx + j));
        Xf[e] = limbs_of(b.x, b.y, E);
    }
}

template <int WORDS, int NU, int RUN>
__global__ void __launch_bounds__(kBlock) pattern_spmm_fast_x_kernel(PatternView a, int k, const double* __restrict__ X,
                                                                     int64_t ldx, const int2* __restrict__ Xf,
                                                                     double* __restrict__ Y, int64_t ldy,
                                                                     const uint32_t* __restrict__ emax_cols) {
    const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t r = idx / k;
    const int j = int(idx - r * k);
    if (r >= a.n) return;
    const int emax = int(__ldg(emax_cols + j));
    uint32_t w[kMaxRecordWords];
    load_record<WORDS>(a, r, w);
    if (emax < 64 || emax >= 2047) {
        const uint32_t mask = __ldg(a.pmask_dev + (byte_of(w, NU) & 31));
        double acc = 0.0;
#pragma unroll
        for (int u = 0; u < NU; ++u)
            if ((mask >> u) & 1u)
                acc = fma(__ldg(a.dict + (byte_of(w, u) & 7)), __ldg(X + (r + a.uoff[u]) * ldx + j), acc);
        Y[r * ldy + j] = acc;
        return;
    }
    uint32_t mw[(NU + 3) / 4];
#pragma unroll
    for (int q = 0; q < (NU + 3) / 4; ++q) mw[q] = prmt(a.mult_lo, a.mult_hi, prmt(w[q] | (w[q] >> 4), 0u, 0x0020u));
    const int2* __restrict__ Xr = Xf + idx;   // row r, column j
    int64_t ah[3] = {0, 0, 0}, al[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < NU / RUN; ++q) {
        const int2* __restrict__ p = Xr + int64_t(a.uoff[q * RUN]) * k;
#pragma unroll
        for (int i = 0; i < RUN; ++i) {
            const int u = q * RUN + i;
            const int32_t m = int32_t(prmt(mw[u >> 2], 0u, uint32_t(u & 3) * 0x1111u + 0x8880u));
            const int2 v = __ldg(p + int64_t(i) * k);
            ah[u % 3] += int64_t(m) * v.y;
            al[u % 3] += int64_t(m) * v.x;
        }
    }
    const int64_t acc = (ah[0] + ah[1] + ah[2]) * (int64_t(1) << 26) + (al[0] + al[1] + al[2]);
    Y[r * ldy + j] = fixed_to_double(acc, emax - 1075 + a.mult_exp);
}


// SpMM, FAST order, one thread per (row, group of KC columns): the record,
// the dominant-record vote and the multipliers are decoded once per KC
// columns, and X is read as 16-byte pairs of columns.
template <int KC, int NU, int RUN>
__global__ void __launch_bounds__(kBlock, 2) pattern_spmm_rows_kernel(PatternView a, int k, const double* __restrict__ X,
                                                                   int64_t ldx, const int2* __restrict__ Xf,
                                                                   double* __restrict__ Y, int64_t ldy,
                                                                   const uint32_t* __restrict__ emax_cols) {
    constexpr int WORDS = (NU + 4) / 4;
    const int ng = k / KC;
    const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t r0 = idx / ng;
    const int g = int(idx - r0 * ng);
    // every lane stays for the warp vote below: a lane past the last row
    // reads the last row's record and returns after the vote
    const bool valid = r0 < a.n;
    const int64_t r = valid ? r0 : a.n - 1;
    const int c0 = g * KC;
    int em[KC];
    bool exact = false;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
        em[c] = int(__ldg(emax_cols + c0 + c));
        exact = exact || em[c] < 64 || em[c] >= 2047;
    }
    uint32_t w[kMaxRecordWords];
    load_record<WORDS>(a, r, w);
    // lanes on the exact path (their columns hold no finite nonzero scale)
    // vote true: they do not use the multipliers
    const bool dom = warp_dominant<WORDS>(a, w, valid && !exact);
    if (!valid) return;
    if (exact) {
        const uint32_t mask = __ldg(a.pmask_dev + (byte_of(w, NU) & 31));
#pragma unroll 1
        for (int c = 0; c < KC; ++c) {
            double acc = 0.0;
#pragma unroll
            for (int u = 0; u < NU; ++u)
                if ((mask >> u) & 1u)
                    acc = fma(__ldg(a.dict + (byte_of(w, u) & 7)), __ldg(X + (r + a.uoff[u]) * ldx + c0 + c), acc);
            Y[r * ldy + c0 + c] = acc;
        }
        return;
    }
    // the row's multipliers, once (kernel parameters when the whole warp
    // carries the dominant record)
    int32_t mult[NU];
    if (dom) {
#pragma unroll
        for (int u = 0; u < NU; ++u) mult[u] = a.dom_m[u];
    } else {
        uint32_t mw[(NU + 3) / 4];
#pragma unroll
        for (int q = 0; q < (NU + 3) / 4; ++q) mw[q] = prmt(a.mult_lo, a.mult_hi, prmt(w[q] | (w[q] >> 4), 0u, 0x0020u));
#pragma unroll
        for (int u = 0; u < NU; ++u) mult[u] = int32_t(prmt(mw[u >> 2], 0u, uint32_t(u & 3) * 0x1111u + 0x8880u));
    }
    const int2* __restrict__ Xr = Xf + r * k + c0;
    if constexpr (KC >= 2) {
        // a pair of columns per pass over the slots
#pragma unroll 1
        for (int c = 0; c < KC; c += 2) {
            int64_t ah0 = 0, al0 = 0, ah1 = 0, al1 = 0;
#pragma unroll
            for (int q = 0; q < NU / RUN; ++q) {
                const int2* __restrict__ p = Xr + int64_t(a.uoff[q * RUN]) * k + c;
#pragma unroll
                for (int i = 0; i < RUN; ++i) {
                    const int32_t m = mult[q * RUN + i];
                    const int4 v = __ldg(reinterpret_cast<const int4*>(p + int64_t(i) * k));
                    ah0 += int64_t(m) * v.y;
                    al0 += int64_t(m) * v.x;
                    ah1 += int64_t(m) * v.w;
                    al1 += int64_t(m) * v.z;
                }
            }
            Y[r * ldy + c0 + c] = fixed_to_double(ah0 * (int64_t(1) << 26) + al0, em[c] - 1075 + a.mult_exp);
            Y[r * ldy + c0 + c + 1] = fixed_to_double(ah1 * (int64_t(1) << 26) + al1, em[c + 1] - 1075 + a.mult_exp);
        }
    } else {
        int64_t ah = 0, al = 0;
#pragma unroll
        for (int q = 0; q < NU / RUN; ++q) {
            const int2* __restrict__ p = Xr + int64_t(a.uoff[q * RUN]) * k;
#pragma unroll
            for (int i = 0; i < RUN; ++i) {
                const int2 v = __ldg(p + int64_t(i) * k);
                ah += int64_t(mult[q * RUN + i]) * v.y;
                al += int64_t(mult[q * RUN + i]) * v.x;
            }
        }
        Y[r * ldy + c0] = fixed_to_double(ah * (int64_t(1) << 26) + al, em[0] - 1075 + a.mult_exp);
    }
}

// ------------------------------------ binary32 COLUMN order, specialised -
// y_i = fmaf chain over present slots in ascending column order (bit-equal
// to the binary32 CSR product).  The union size is a compile-time constant;
// runs of RUN consecutive displacements share one pointer; absent slots are
// predicated off (their column may be outside [0, n)).
template <int WORDS, int NU, int RUN>
__global__ void __launch_bounds__(kBlock) pattern_f32_kernel(PatternView a, const float* __restrict__ x,
                                                             float* __restrict__ y) {
    __shared__ float sdict[256];
    __shared__ uint32_t smask[32];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sdict[i] = i < a.dict_size ? a.dict32[i] : 0.0f;
    if (threadIdx.x < 32) smask[threadIdx.x] = threadIdx.x < a.npat ? a.pmask[threadIdx.x] : 0u;
    __syncthreads();
    const int64_t r0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    // every lane stays for the warp vote: a lane past the last row reads the
    // last row's record and returns after the vote
    const bool valid = r0 < a.n;
    const int64_t r = valid ? r0 : a.n - 1;
    uint32_t w[kMaxRecordWords];
    load_record<WORDS>(a, r, w);
    const float* __restrict__ xr = x + r;
    float acc = 0.0f;
    const bool dom = warp_dominant<WORDS>(a, w, valid);
    if (!valid) return;
    if (dom) {
        // every row of the warp carries the dominant record: all slots
        // present, values are kernel parameters
#pragma unroll
        for (int k = 0; k < NU / RUN; ++k) {
            const float* __restrict__ p = xr + a.uoff[k * RUN];
#pragma unroll
            for (int j = 0; j < RUN; ++j) acc = fmaf(a.dom_v32[k * RUN + j], __ldg(p + j), acc);
        }
        y[r] = acc;
        return;
    }
    const uint32_t pat = byte_of(w, NU);
    if (pat >= uint32_t(a.npat)) raise_error(a.err, 1);
    const uint32_t mask = smask[pat & 31];
#pragma unroll
    for (int k = 0; k < NU / RUN; ++k) {
        const float* __restrict__ p = xr + a.uoff[k * RUN];
#pragma unroll
        for (int j = 0; j < RUN; ++j) {
            const int u = k * RUN + j;
            if ((mask >> u) & 1u) acc = fmaf(sdict[byte_of(w, u)], __ldg(p + j), acc);
        }
    }
    y[r] = acc;
}

// ------------------------------------------------------------ delta ------
// A load of the slice payload: from shared memory (SH, the slice staged
// there) or streamed from global memory.
template <bool SH, typename V>
__device__ __forceinline__ V ldp(const V* p) {
    if constexpr (SH) return *p;
    else return __ldcs(p);
}

// One row of a delta slice.  CM: column encoding (0 int16 delta, 1 24-bit
// delta, 2 raw int32); VM: value encoding (0 code, 1 code into the global
// table or, from dict_size up, into the slice's own table, 2 raw double).
// base: the slice payload (in shared memory when SH), gbase: the same in
// global memory (the slice's own value table is read from there).
template <typename T, int CM, int VM, bool SH>
__device__ __forceinline__ T delta_row(const DeltaView& a, const uint8_t* base, const uint8_t* gbase, uint32_t w,
                                       uint32_t flags, int64_t r, int l, int len, const T* sdict,
                                       const T* __restrict__ x, int64_t ldx, int j) {
    const DeltaParts pt = delta_parts(w, flags);
    const double* local = reinterpret_cast<const double*>(gbase + pt.local) + 2;   // after its 16-byte count
    T acc = T(0);
    // the slice's full width, the same for every lane of the warp, so the
    // loop unrolls and independent loads overlap; a lane's slots past its
    // row's length (zero padding inside the slice) are loaded but skipped
#pragma unroll 4
    for (int t = 0; t < int(w); ++t) {
        const bool on = t < len;
        const int64_t slot = int64_t(t) * 32 + l;
        int64_t c;
        if constexpr (CM == 2) {
            c = ldp<SH>(reinterpret_cast<const int32_t*>(base + pt.cols) + slot);
        } else {
            const int16_t lo = ldp<SH>(reinterpret_cast<const int16_t*>(base + pt.cols) + slot);
            if constexpr (CM == 1)
                c = r + int64_t(int8_t(ldp<SH>(base + pt.hi + slot))) * 65536 + int64_t(uint16_t(lo));
            else
                c = r + lo;
        }
        bool ok = on;
        T v = T(0);
        if constexpr (VM == 2) {
            v = T(ldp<SH>(reinterpret_cast<const double*>(base + pt.vals) + slot));
        } else {
            const uint32_t code = ldp<SH>(base + pt.vals + slot);
            if (code < uint32_t(a.dict_size)) {
                v = sdict[code];
            } else if (VM == 1) {
                if (on) v = T(__ldg(local + (code - uint32_t(a.dict_size))));
            } else {
                if (on) raise_error(a.err, 2);
                ok = false;
            }
        }
        if (uint64_t(c) >= uint64_t(a.n)) {
            if (on) raise_error(a.err, 2);
            ok = false;
        }
        const T xv = ok ? __ldg(x + c * ldx + j) : T(0);
        if (ok) acc = fma(v, xv, acc);
    }
    return acc;
}

template <typename T, bool SH = false>
__device__ __forceinline__ T delta_row_any(const DeltaView& a, const uint8_t* base, const uint8_t* gbase,
                                           const DeltaSlice& h, int64_t r, int l, int len, const T* sdict,
                                           const T* __restrict__ x, int64_t ldx, int j) {
    const int cm = (h.flags & kSliceColRaw) ? 2 : (h.flags & kSliceCol24) ? 1 : 0;
    const int vm = (h.flags & kSliceValRaw) ? 2 : (h.flags & kSliceValLocal) ? 1 : 0;
#define SPMVC_DELTA_ROW(C_, V_) \
    if (cm == C_ && vm == V_)   \
        return delta_row<T, C_, V_, SH>(a, base, gbase, h.w, h.flags, r, l, len, sdict, x, ldx, j);
    SPMVC_DELTA_ROW(0, 0) SPMVC_DELTA_ROW(0, 1) SPMVC_DELTA_ROW(0, 2)
    SPMVC_DELTA_ROW(1, 0) SPMVC_DELTA_ROW(1, 1) SPMVC_DELTA_ROW(1, 2)
    SPMVC_DELTA_ROW(2, 0) SPMVC_DELTA_ROW(2, 1) SPMVC_DELTA_ROW(2, 2)
#undef SPMVC_DELTA_ROW
    return T(0);
}

// y[r] = row r, or y[scatter[r]] = row r for a reordered handle (the
// scatter of P^T folded into the product).  A warp first copies its slice's
// row lengths, columns and codes (everything before the slice's own value
// table, when at most kDeltaStage bytes) into its part of shared memory with
// 16-byte loads, so that the slot loop's only global loads are the x
// gathers (and the rare slice-local values).
constexpr int kDeltaStage = 5632;   // bytes a warp: 8 warps plus the value table stay under 48 KB
template <typename T>
__global__ void __launch_bounds__(kBlock) delta_kernel(DeltaView a, const T* __restrict__ x, T* __restrict__ y,
                                                     const int32_t* __restrict__ scatter) {
    __shared__ uint4 sstage[kBlock / 32][kDeltaStage / 16];
    __shared__ T sdict[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        T v = T(0);
        if (i < a.dict_size) {
            if constexpr (sizeof(T) == 8) v = a.dict[i];
            else v = a.dict32[i];
        }
        sdict[i] = v;
    }
    __syncthreads();
    const int64_t s = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    const int l = threadIdx.x & 31;
    if (s >= a.nslices) return;
    const DeltaSlice h = a.hdr[s];
    const uint8_t* base = a.payload + h.off;
    const int64_t r = s * 32 + l;
    const uint64_t sb = delta_parts(h.w, h.flags).local;   // a multiple of 16: every part is 16-byte aligned
    T acc;
    if (sb <= uint64_t(kDeltaStage)) {
        uint4* st = sstage[threadIdx.x >> 5];
        const uint4* src = reinterpret_cast<const uint4*>(base);
        for (int i = l; i < int(sb >> 4); i += 32) st[i] = __ldcs(src + i);
        __syncwarp();
        const uint8_t* sbase = reinterpret_cast<const uint8_t*>(st);
        int len = r < a.n ? int(sbase[l]) : 0;
        if (uint32_t(len) > h.w) { raise_error(a.err, 4); len = 0; }
        acc = delta_row_any<T, true>(a, sbase, base, h, r, l, len, sdict, x, 1, 0);
    } else {
        int len = r < a.n ? int(base[l]) : 0;
        if (uint32_t(len) > h.w) { raise_error(a.err, 4); len = 0; }
        acc = delta_row_any<T, false>(a, base, base, h, r, l, len, sdict, x, 1, 0);
    }
    if (r < a.n) y[scatter ? int64_t(__ldg(scatter + r)) : r] = acc;
}

// ------------------------------------------------------------ SpMM -------
// Y = A X, X and Y row-major n x k.  One thread per (row, column) pair,
// column fastest, so X rows are read as contiguous runs.
template <int WORDS>
__global__ void __launch_bounds__(kBlock) pattern_spmm_col_kernel(PatternView a, int k, const double* __restrict__ X,
                                                                  int64_t ldx, double* __restrict__ Y, int64_t ldy) {
    __shared__ double sdict[256];
    __shared__ uint32_t smask[32];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sdict[i] = i < a.dict_size ? a.dict[i] : 0.0;
    if (threadIdx.x < 32) smask[threadIdx.x] = threadIdx.x < a.npat ? a.pmask[threadIdx.x] : 0u;
    __syncthreads();
    const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t r = idx / k;
    const int j = int(idx - r * k);
    if (r >= a.n) return;
    uint32_t w[kMaxRecordWords];
    load_record<WORDS>(a, r, w);
    const uint32_t pat = byte_of(w, a.nu);
    const uint32_t mask = smask[pat & 31];
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < 4 * WORDS - 1; ++u)
        if (u < a.nu && ((mask >> u) & 1u)) {
            const uint32_t code = byte_of(w, u);
            const int64_t c = r + a.uoff[u];
            if (code >= uint32_t(a.dict_size) || uint64_t(c) >= uint64_t(a.n)) { raise_error(a.err, 2); continue; }
            acc = fma(sdict[code], __ldg(X + c * ldx + j), acc);
        }
    Y[r * ldy + j] = acc;
}

// per-column partial maxima: partial[b * k + j]
__global__ void __launch_bounds__(256) xmax_cols_kernel(const double* __restrict__ X, int64_t n, int k, int64_t ldx,
                                                        uint32_t* __restrict__ partial) {
    // block b handles rows b, b + G, ...; thread t handles column t % k of row group t / k
    const int j = threadIdx.x % k, sub = threadIdx.x / k, nsub = blockDim.x / k;
    uint32_t m = 0;
    if (sub < nsub)
        for (int64_t r = blockIdx.x * int64_t(nsub) + sub; r < n; r += int64_t(gridDim.x) * nsub)
            m = max(m, uint32_t(__double2hiint(__ldg(X + r * ldx + j))) & 0x7FFFFFFFu);
    __shared__ uint32_t sm[256];
    sm[threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.x < k) {
        uint32_t v = 0;
        for (int s2 = 0; s2 < nsub; ++s2) v = max(v, sm[s2 * k + threadIdx.x]);
        partial[blockIdx.x * k + threadIdx.x] = v;
    }
}

template <int WORDS>
__global__ void __launch_bounds__(kBlock) pattern_spmm_fast_kernel(PatternView a, int k, const double* __restrict__ X,
                                                                   int64_t ldx, double* __restrict__ Y, int64_t ldy,
                                                                   const uint32_t* __restrict__ partial) {
    __shared__ uint32_t smask[32];
    __shared__ double sdict[8];
    __shared__ int s_emax[64];
    if (threadIdx.x < 32) smask[threadIdx.x] = threadIdx.x < a.npat ? a.pmask[threadIdx.x] : 0u;
    if (threadIdx.x < 8) sdict[threadIdx.x] = threadIdx.x < a.dict_size ? a.dict[threadIdx.x] : 0.0;
    if (threadIdx.x < k) {
        uint32_t v = 0;
        for (int b = 0; b < kXmaxBlocks; ++b) v = max(v, __ldg(partial + b * k + threadIdx.x));
        s_emax[threadIdx.x] = int(v >> 20);
    }
    __syncthreads();
    const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t r = idx / k;
    const int j = int(idx - r * k);
    if (r >= a.n) return;
    const int emax = s_emax[j];
    uint32_t w[kMaxRecordWords];
    load_record<WORDS>(a, r, w);
    const uint32_t pat = byte_of(w, a.nu);
    const uint32_t mask = smask[pat & 31];
    if (emax < 64 || emax >= 2047) {
        double acc = 0.0;
#pragma unroll
        for (int u = 0; u < 4 * WORDS - 1; ++u)
            if (u < a.nu && ((mask >> u) & 1u)) {
                const uint32_t code = byte_of(w, u);
                const int64_t c = r + a.uoff[u];
                if (code < uint32_t(a.dict_size) && uint64_t(c) < uint64_t(a.n))
                    acc = fma(sdict[code & 7], __ldg(X + c * ldx + j), acc);
            }
        Y[r * ldy + j] = acc;
        return;
    }
    int64_t acc_h = 0, acc_l = 0;
#pragma unroll
    for (int u = 0; u < 4 * WORDS - 1; ++u)
        if (u < a.nu) {
            const uint32_t code = byte_of(w, u);
            const int32_t m = mult_of(a.mult_lo, a.mult_hi, code);
            const int64_t c = r + a.uoff[u];
            const bool inside = uint64_t(c) < uint64_t(a.n);
            int32_t xh, xl;
            to_fixed(__ldg(X + (inside ? c : r) * ldx + j), emax, xh, xl);
            const int32_t mm = ((mask >> u) & 1u) ? m : 0;
            acc_h += int64_t(mm) * xh;
            acc_l += int64_t(mm) * xl;
        }
    Y[r * ldy + j] = fixed_to_double(acc_h * (int64_t(1) << 26) + acc_l, emax - 1075 + a.mult_exp);
}

__global__ void __launch_bounds__(kBlock) ell_spmm_kernel(EllView a, int k, const double* __restrict__ X, int64_t ldx,
                                                          double* __restrict__ Y, int64_t ldy) {
    const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t r = idx / k;
    const int j = int(idx - r * k);
    if (r >= a.n) return;
    const int64_t s = r >> 5;
    const int64_t base = a.slice_off[s] + (r & 31);
    const int w = a.slice_w[s];
    double acc = 0.0;
    for (int t = 0; t < w; ++t) {
        const int32_t c = __ldg(a.col + base + 32 * t);
        if (c >= 0) acc = fma(__ldg(a.val + base + 32 * t), __ldg(X + int64_t(c) * ldx + j), acc);
    }
    Y[r * ldy + j] = acc;
}

__global__ void __launch_bounds__(kBlock) delta_spmm_kernel(DeltaView a, int k, const double* __restrict__ X,
                                                            int64_t ldx, double* __restrict__ Y, int64_t ldy) {
    __shared__ double sdict[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sdict[i] = i < a.dict_size ? a.dict[i] : 0.0;
    __syncthreads();
    const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t r = idx / k;
    const int j = int(idx - r * k);
    if (r >= a.n) return;
    const int64_t s = r >> 5;
    const int l = int(r & 31);
    const DeltaSlice h = a.hdr[s];
    const uint8_t* base = a.payload + h.off;
    int len = base[l];
    if (uint32_t(len) > h.w) { raise_error(a.err, 4); len = 0; }
    Y[r * ldy + j] = delta_row_any<double>(a, base, base, h, r, l, len, sdict, X, ldx, j);
}

__global__ void fill_u32_kernel(uint32_t* p, uint32_t v, int64_t n) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i < n) p[i] = v;
}

unsigned grid_of(int64_t threads) { return unsigned((threads + kBlock - 1) / kBlock); }

// Opens a kernel's dynamic shared memory to the device's per-block limit and
// prefers the largest shared-memory carveout, once per kernel and device:
// the two attribute calls cost more than a launch, and a pipelined product
// launches a kernel many times.
cudaError_t prepare_kernel(const void* kernel) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static std::unordered_map<const void*, uint64_t> done;   // kernel -> devices prepared
    std::lock_guard<std::mutex> g(mu);
    uint64_t& mask = done[kernel];
    const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
    if (bit && (mask & bit)) return cudaSuccess;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
    const int dyn = optin - int(fa.sharedSizeBytes);     // the limit counts the kernel's static shared memory
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  int(cudaSharedmemCarveoutMaxShared))) != cudaSuccess)
        return e;
    mask |= bit;
    return cudaSuccess;
}


}  // namespace

// --------------------------------------------------------- launchers -----
#define SPMVC_DISPATCH_WORDS(WORDS_VAL, CALL)                     \
    switch (WORDS_VAL) {                                          \
        case 1: { constexpr int W = 1; CALL; } break;             \
        case 2: { constexpr int W = 2; CALL; } break;             \
        case 3: { constexpr int W = 3; CALL; } break;             \
        case 4: { constexpr int W = 4; CALL; } break;             \
        case 5: { constexpr int W = 5; CALL; } break;             \
        case 6: { constexpr int W = 6; CALL; } break;             \
        case 7: { constexpr int W = 7; CALL; } break;             \
        case 8: { constexpr int W = 8; CALL; } break;             \
        default: return cudaErrorInvalidValue;                    \
    }

cudaError_t launch_ell_f64(const EllView& a, const double* x, double* y, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    ell_kernel<double><<<grid_of(a.n), kBlock, 0, s>>>(a, x, y);
    return cudaGetLastError();
}
cudaError_t launch_ell_f32(const EllView& a, const float* x, float* y, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    ell_kernel<float><<<grid_of(a.n), kBlock, 0, s>>>(a, x, y);
    return cudaGetLastError();
}
cudaError_t launch_pattern_col_f64(const PatternView& a, const double* x, double* y, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    SPMVC_DISPATCH_WORDS(a.words, (pattern_col_kernel<W, double><<<grid_of(a.n), kBlock, 0, s>>>(a, x, y)));
    return cudaGetLastError();
}
// Binary32 product from the one-byte row types (values registered in the
// pattern, Sec. V): a row's record is the type's, held in shared memory, so
// the matrix costs one byte a row.  The same fmaf chain over ascending
// columns as the record kernel above, so the same bits.
constexpr int kTypeWords = 256 * 8;

template <int NU, int RUN>
__global__ void __launch_bounds__(kBlock) pattern_types_f32_kernel(PatternView a, const float* __restrict__ x,
                                                                   float* __restrict__ y) {
    __shared__ uint32_t stypes[kTypeWords];
    __shared__ float sdict[256];
    __shared__ uint32_t smask[32];
    for (int i = threadIdx.x; i < a.ntypes * 8; i += blockDim.x) stypes[i] = __ldg(a.rtypes + i);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sdict[i] = i < a.dict_size ? a.dict32[i] : 0.0f;
    if (threadIdx.x < 32) smask[threadIdx.x] = threadIdx.x < a.npat ? a.pmask[threadIdx.x] : 0u;
    __syncthreads();
    const int64_t r0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    // every lane stays for the warp vote: a lane past the last row reads the
    // last row's type and returns after the vote
    const bool valid = r0 < a.n;
    const int64_t r = valid ? r0 : a.n - 1;
    uint32_t t = __ldg(a.rtype + r);
    if (t >= uint32_t(a.ntypes)) {
        raise_error(a.err, 2);
        t = 0;
    }
    const float* __restrict__ xr = x + r;
    float acc = 0.0f;
    const bool dom = __all_sync(0xFFFFFFFFu, !valid || int32_t(t) == a.dom_type);
    if (!valid) return;
    if (dom) {
        // every row of the warp carries the dominant record
#pragma unroll
        for (int k = 0; k < NU / RUN; ++k) {
            const float* __restrict__ p = xr + a.uoff[k * RUN];
#pragma unroll
            for (int j = 0; j < RUN; ++j) acc = fmaf(a.dom_v32[k * RUN + j], __ldg(p + j), acc);
        }
        y[r] = acc;
        return;
    }
    uint32_t w[kMaxRecordWords];
#pragma unroll
    for (int k = 0; k < 7; ++k) w[k] = stypes[t * 8 + k];
    const uint32_t pat = byte_of(w, NU);
    if (pat >= uint32_t(a.npat)) raise_error(a.err, 1);
    const uint32_t mask = smask[pat & 31];
#pragma unroll
    for (int k = 0; k < NU / RUN; ++k) {
        const float* __restrict__ p = xr + a.uoff[k * RUN];
#pragma unroll
        for (int j = 0; j < RUN; ++j) {
            const int u = k * RUN + j;
            if ((mask >> u) & 1u) acc = fmaf(sdict[byte_of(w, u)], __ldg(p + j), acc);
        }
    }
    y[r] = acc;
}

cudaError_t launch_pattern_types_f32(const PatternView& a, const float* x, float* y, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    // the 27-slot union of a 3-D grid stencil, nine runs of three columns
    if (a.words != 7 || a.nu != 27 || a.run_len != 3 || !a.rtype || !a.rtypes || a.ntypes < 1 || a.ntypes > 256 ||
        a.dict_size > 256)
        return cudaErrorNotSupported;
    pattern_types_f32_kernel<27, 3><<<grid_of(a.n), kBlock, 0, s>>>(a, x, y);
    return cudaGetLastError();
}

cudaError_t launch_pattern_col_f32(const PatternView& a, const float* x, float* y, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (a.run_len == 3 && a.nu == 27) {
        pattern_f32_kernel<7, 27, 3><<<grid_of(a.n), kBlock, 0, s>>>(a, x, y);
        return cudaGetLastError();
    }
    SPMVC_DISPATCH_WORDS(a.words, (pattern_col_kernel<W, float><<<grid_of(a.n), kBlock, 0, s>>>(a, x, y)));
    return cudaGetLastError();
}
cudaError_t launch_pattern_fast_f64(const PatternView& a, const double* x, double* y, uint32_t* partial,
                                    cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    xmax_kernel<<<kXmaxBlocks, 1024, 0, s>>>(x, a.n, partial);
    SPMVC_DISPATCH_WORDS(a.words, (pattern_fast_kernel<W><<<grid_of(a.n), kBlock, 0, s>>>(a, x, y, partial)));
    return cudaGetLastError();
}

cudaError_t launch_pattern_fast_staged(const PatternView& a, const StagePlan& sp, const double* x, double* y,
                                       cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    // 16-byte staging needs x itself 16-byte aligned
    const bool vec = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
    const int threads = sp.rows / sp.rows_per_thread;
    const int64_t tiles = (a.n + sp.rows - 1) / sp.rows - sp.tile0;
    if (tiles <= 0) return cudaSuccess;
    const unsigned grid = unsigned(sp.ntiles > 0 && sp.ntiles < tiles ? sp.ntiles : tiles);
    const size_t smem = size_t((std::max(sp.elems, sp.elems_padded) + 1) / 2 * 2) * sizeof(int2);
    auto go = [&](auto kernel) -> cudaError_t {
        const cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kernel));
        if (e != cudaSuccess) return e;
        kernel<<<grid, threads, smem, s>>>(a, sp, x, y);
        return cudaGetLastError();
    };
#define SPMVC_STAGED(W, NUV, RUN, RPT, T)                                                       \
    if (sp.rows_per_thread == RPT && threads == T)                                              \
        return vec ? go(pattern_fast_staged_kernel<W, NUV, RPT, RUN, T, true>)                  \
                   : go(pattern_fast_staged_kernel<W, NUV, RPT, RUN, T, false>);
    if (a.run_len == 3 && a.nu == 27) {
        SPMVC_STAGED(7, 27, 3, 1, 512)
        SPMVC_STAGED(7, 27, 3, 2, 512)
        SPMVC_STAGED(7, 27, 3, 4, 512)
        SPMVC_STAGED(7, 27, 3, 2, 256)
        SPMVC_STAGED(7, 27, 3, 4, 256)
        SPMVC_STAGED(7, 27, 3, 8, 256)
        return cudaErrorInvalidValue;
    }
    // union sizes of the 3-D 27-, 19- and 7-point stencils and the 2-D 9- and
    // 5-point ones are compiled with a fixed slot count, 512 threads
#define SPMVC_NU_CASE(NUV)                                                                      \
    case NUV:                                                                                   \
        SPMVC_STAGED((NUV + 4) / 4, NUV, 1, 1, 512)                                             \
        SPMVC_STAGED((NUV + 4) / 4, NUV, 1, 2, 512)                                             \
        SPMVC_STAGED((NUV + 4) / 4, NUV, 1, 4, 512)                                             \
        return cudaErrorInvalidValue;
    switch (a.nu) {
        SPMVC_NU_CASE(27)
        SPMVC_NU_CASE(19)
        SPMVC_NU_CASE(9)
        SPMVC_NU_CASE(7)
        SPMVC_NU_CASE(5)
        default: return cudaErrorNotSupported;
    }
#undef SPMVC_NU_CASE
#undef SPMVC_STAGED
}

cudaError_t launch_pattern_fast_x(const PatternView& a, const double* x, double* y, uint32_t* partial,
                                  int2* X_guarded, int64_t guard, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    int2* X = X_guarded + guard;
    xmax_kernel<<<kXmaxBlocks, 1024, 0, s>>>(x, a.n, partial);
    convert_x_kernel<<<kXmaxBlocks * 8, 256, 0, s>>>(reinterpret_cast<const uint2*>(x), a.n, partial, X);
    const unsigned grid = grid_of(a.n);
#define SPMVC_NU_X(NUV) \
    case NUV: pattern_fast_x_kernel<(NUV + 4) / 4, NUV, 1><<<grid, kBlock, 0, s>>>(a, x, X, y, partial); break;
    if (a.run_len == 3 && a.nu == 27)
        pattern_fast_x_kernel<7, 27, 3><<<grid, kBlock, 0, s>>>(a, x, X, y, partial);
    else if (a.run_len == 3 && a.nu == 9)
        pattern_fast_x_kernel<3, 9, 3><<<grid, kBlock, 0, s>>>(a, x, X, y, partial);
    else switch (a.nu) {
        SPMVC_NU_X(27)
        SPMVC_NU_X(19)
        SPMVC_NU_X(9)
        SPMVC_NU_X(7)
        SPMVC_NU_X(5)
        default: return cudaErrorNotSupported;
    }
#undef SPMVC_NU_X
    return cudaGetLastError();
}


cudaError_t launch_pattern_fast_xstaged(const PatternView& a, const StagePlan& sp, const double* x, double* y,
                                        uint32_t* partial, int2* X_guarded, int64_t guard, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (!(a.run_len == 3 && a.nu == 27)) return cudaErrorNotSupported;
    int2* X = X_guarded + guard;
    xmax_kernel<<<kXmaxBlocks, 1024, 0, s>>>(x, a.n, partial);
    convert_x_kernel<<<kXmaxBlocks * 8, 256, 0, s>>>(reinterpret_cast<const uint2*>(x), a.n, partial, X);
    const unsigned grid = unsigned((a.n + sp.rows - 1) / sp.rows);
    const size_t smem = size_t(sp.elems_padded) * sizeof(int2);
    auto go = [&](auto kernel) -> cudaError_t {
        const cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kernel));
        if (e != cudaSuccess) return e;
        kernel<<<grid, kStageThreads, smem, s>>>(a, sp, x, X, y, partial);
        return cudaGetLastError();
    };
    if (sp.rows_per_thread == 1) return go(pattern_fast_xstaged_kernel<7, 27, 1, 3>);
    if (sp.rows_per_thread == 2) return go(pattern_fast_xstaged_kernel<7, 27, 2, 3>);
    if (sp.rows_per_thread == 4) return go(pattern_fast_xstaged_kernel<7, 27, 4, 3>);
    return cudaErrorInvalidValue;
}


cudaError_t launch_pattern_fast_async(const PatternView& a, const StagePlan& sp, const double* x, double* y,
                                      int num_sms, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (!(a.run_len == 3 && a.nu == 27 && a.words == 7) || sp.rows != kAsyncRows) return cudaErrorNotSupported;
    const int64_t ntiles = (a.n + kAsyncRows - 1) / kAsyncRows;
    const size_t xbytes = (size_t(sp.elems) * 8 + 15) / 16 * 16;
    const size_t smem = 2 * (xbytes + size_t(kAsyncRows) * 28);
    auto kernel = pattern_fast_async_kernel<27, 3, false>;
    const cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kernel));
    if (e != cudaSuccess) return e;
    const unsigned grid = unsigned(std::min<int64_t>(ntiles, num_sms));
    kernel<<<grid, kAsyncThreads, smem, s>>>(a, sp, x, nullptr, y, ntiles, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_pattern_fast_async_x(const PatternView& a, const StagePlan& sp, const double* x, double* y,
                                        uint32_t* partial, int2* X_guarded, int64_t guard, int num_sms,
                                        cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (!(a.run_len == 3 && a.nu == 27 && a.words == 7) || sp.rows != kAsyncRows) return cudaErrorNotSupported;
    int2* X = X_guarded + guard;
    xmax_kernel<<<kXmaxBlocks, 1024, 0, s>>>(x, a.n, partial);
    convert_x_kernel<<<kXmaxBlocks * 8, 256, 0, s>>>(reinterpret_cast<const uint2*>(x), a.n, partial, X);
    const int64_t ntiles = (a.n + kAsyncRows - 1) / kAsyncRows;
    // both layouts must fit: raw windows for the exact fallback, padded ones otherwise
    const size_t xbytes = (size_t(std::max(sp.elems, sp.elems_padded)) * 8 + 15) / 16 * 16;
    const size_t smem = 2 * (xbytes + size_t(kAsyncRows) * 28);
    auto kernel = pattern_fast_async_kernel<27, 3, true>;
    const cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kernel));
    if (e != cudaSuccess) return e;
    const unsigned grid = unsigned(std::min<int64_t>(ntiles, num_sms));
    kernel<<<grid, kAsyncThreads, smem, s>>>(a, sp, x, X, y, ntiles, partial);
    return cudaGetLastError();
}

// Register-staged shapes: (threads, rows per thread, pairs per window per thread)
bool rstage_supported(const StagePlan& sp) {
    const int threads = sp.rows / sp.rows_per_thread;
    int qs = 0;
    if (threads == 256 && sp.rows_per_thread == 4) qs = 3;
    else if (threads == 256 && sp.rows_per_thread == 2) qs = 2;
    else if (threads == 512 && sp.rows_per_thread == 2) qs = 2;
    if (qs == 0 || sp.nseg != 3) return false;
    for (int sg = 0; sg < 3; ++sg)
        if ((sp.rows + sp.seg_span[sg] + sp.seg_pad[sg] + 1) / 2 > qs * threads) return false;
    return int64_t(sp.elems_padded) * 8 + int64_t(sp.rows) * 28 <= 200 * 1024;   // windows + records
}

cudaError_t launch_pattern_fast_rstaged(const PatternView& a, const StagePlan& sp, const double* x, double* y,
                                        int recs, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (!(a.run_len == 3 && a.nu == 27 && a.words == 7) || !rstage_supported(sp)) return cudaErrorNotSupported;
    if (recs < 0 || recs > 2 || (recs == 2 && !(a.rtype && a.ntypes > 0 && a.ntypes <= 256)))
        return cudaErrorInvalidValue;
    // the 16-byte loads need x itself 16-byte aligned: otherwise the staged
    // kernel on the same plan
    if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0) return launch_pattern_fast_staged(a, sp, x, y, s);
    const int threads = sp.rows / sp.rows_per_thread;
    const int64_t tiles = (a.n + sp.rows - 1) / sp.rows - sp.tile0;
    if (tiles <= 0) return cudaSuccess;
    const unsigned grid = unsigned(sp.ntiles > 0 && sp.ntiles < tiles ? sp.ntiles : tiles);
    // converted windows, then the tile's records (28 bytes a row) or the
    // table of row types (32 bytes a type)
    const size_t smem = size_t(sp.elems_padded) * sizeof(int2) +
                        (recs == 1 ? size_t(sp.rows) * 28 : recs == 2 ? size_t(a.ntypes) * 32 : 0);
    auto go = [&](auto kernel) -> cudaError_t {
        const cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kernel));
        if (e != cudaSuccess) return e;
        kernel<<<grid, threads, smem, s>>>(a, sp, x, y);
        return cudaGetLastError();
    };
#define SPMVC_RSTAGED(QSV, RPTV, TV, MB)                                                           \
    if (threads == TV && sp.rows_per_thread == RPTV)                                               \
        return recs == 0 ? go(pattern_fast_rstaged_kernel<QSV, RPTV, TV, MB, 0>)                  \
             : recs == 1 ? go(pattern_fast_rstaged_kernel<QSV, RPTV, TV, MB, 1>)                  \
                         : go(pattern_fast_rstaged_kernel<QSV, RPTV, TV, MB, 2>);
    SPMVC_RSTAGED(3, 4, 256, 4)
    SPMVC_RSTAGED(2, 2, 256, 5)
    SPMVC_RSTAGED(2, 2, 512, 2)
#undef SPMVC_RSTAGED
    return cudaErrorInvalidValue;
}

bool make_zplan(const std::vector<int32_t>& uoff, int64_t n, int rows_per_thread, int threads, int num_sms,
                ZPlan* out) {
    if (uoff.size() != 27 || n <= 0) return false;
    StagePlan sp;
    if (!make_stage_plan(uoff, rows_per_thread, threads, 1 << 30, &sp) || sp.nseg != 3) return false;
    ZPlan z{};
    z.rows = sp.rows;
    z.rows_per_thread = rows_per_thread;
    z.threads = threads;
    const int64_t S = int64_t(sp.seg_min[1]) - sp.seg_min[0];
    if (S <= 0 || int64_t(sp.seg_min[2]) - sp.seg_min[1] != S) return false;
    if (sp.seg_span[0] != sp.seg_span[1] || sp.seg_span[1] != sp.seg_span[2]) return false;
    if (S % sp.rows != 0) return false;
    // nine slots per segment, in order
    for (int u = 0; u < 27; ++u) {
        const int sg = u / 9;
        if (uoff[u] < sp.seg_min[sg] || uoff[u] > sp.seg_min[sg] + sp.seg_span[sg]) return false;
        z.rel[u] = uoff[u] - sp.seg_min[sg];
    }
    z.S = S;
    z.m1 = sp.seg_min[1];
    z.pairs = (sp.rows + sp.seg_span[1] + 1 + 1) / 2;
    z.slot = 2 * z.pairs;
    if (3 * int64_t(z.slot) * 8 > 200 * 1024) return false;
    z.nplanes = (n + S - 1) / S;
    z.nblk = int32_t(S / sp.rows);
    // about four CTAs per SM in one wave
    int64_t chunks = std::max<int64_t>(1, (int64_t(num_sms) * 4 + z.nblk / 2) / z.nblk);
    chunks = std::min<int64_t>(chunks, z.nplanes);
    z.zc = int32_t((z.nplanes + chunks - 1) / chunks);
    z.nchunks = int32_t((z.nplanes + z.zc - 1) / z.zc);
    if (int64_t(z.nblk) * z.nchunks >= (int64_t(1) << 31)) return false;
    *out = z;
    return true;
}

bool zmarch_supported(const ZPlan& zp) {
    if (zp.threads == 256 && zp.rows_per_thread == 2) return zp.pairs <= 2 * 256;
    if (zp.threads == 256 && zp.rows_per_thread == 4) return zp.pairs <= 3 * 256;
    if (zp.threads == 512 && zp.rows_per_thread == 2) return zp.pairs <= 2 * 512;
    return false;
}

cudaError_t launch_pattern_fast_zmarch(const PatternView& a, const ZPlan& zp, const double* x, double* y,
                                       uint32_t* partial, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (!(a.run_len == 3 && a.nu == 27 && a.words == 7) || !zmarch_supported(zp)) return cudaErrorNotSupported;
    // the 16-byte loads need x 16-byte aligned: otherwise the direct kernel
    if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0) return launch_pattern_fast_f64(a, x, y, partial, s);
    xmax_kernel<<<kXmaxBlocks, 1024, 0, s>>>(x, a.n, partial);
    const unsigned grid = unsigned(int64_t(zp.nblk) * zp.nchunks);
    const size_t smem = size_t(3) * zp.slot * sizeof(int2);
    auto go = [&](auto kernel) -> cudaError_t {
        const cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kernel));
        if (e != cudaSuccess) return e;
        kernel<<<grid, zp.threads, smem, s>>>(a, zp, x, y, partial);
        return cudaGetLastError();
    };
    if (zp.threads == 256 && zp.rows_per_thread == 2) return go(pattern_fast_zmarch_kernel<2, 256, 4, 2>);
    if (zp.threads == 256 && zp.rows_per_thread == 4) return go(pattern_fast_zmarch_kernel<4, 256, 4, 3>);
    return go(pattern_fast_zmarch_kernel<2, 512, 2, 2>);
}

bool make_zblock_plan(const std::vector<int32_t>& uoff, int64_t n, int planes, int threads, ZPlan* out) {
    // column blocks of 512 rows, two rows a thread per plane
    if (threads != 256) return false;
    ZPlan zp;
    if (!make_zplan(uoff, n, 2, threads, 1, &zp)) return false;
    zp.zc = planes;
    zp.nchunks = int32_t((zp.nplanes + planes - 1) / planes);
    zp.chunk0 = 0;
    if (int64_t(zp.nblk) * zp.nchunks >= (int64_t(1) << 31)) return false;
    *out = zp;
    return zblock_supported(zp);
}

bool zblock_supported(const ZPlan& zp) {
    if ((zp.zc != 3 && zp.zc != 4) || zp.rows != 512 || zp.threads != 256 || zp.rows_per_thread != 2) return false;
    if ((zp.zc + 2) * int64_t(zp.slot) * 8 > 200 * 1024) return false;
    return zp.pairs <= 2 * 256;
}

cudaError_t launch_pattern_fast_zblock(const PatternView& a, const ZPlan& zp, const double* x, double* y,
                                       uint32_t* partial, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (!(a.run_len == 3 && a.nu == 27 && a.words == 7) || !zblock_supported(zp)) return cudaErrorNotSupported;
    // the 16-byte loads need x 16-byte aligned: otherwise the direct kernel
    if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0) return launch_pattern_fast_f64(a, x, y, partial, s);
    // chunks chunk0 .. chunk0 + nchunks - 1 of zc planes (all of them for a
    // whole product; a row range of them for a pipelined one)
    if (zp.nchunks <= 0 || zp.chunk0 < 0) return cudaSuccess;
    const unsigned grid = unsigned(int64_t(zp.nblk) * zp.nchunks);
    const size_t smem = size_t(zp.zc + 2) * zp.slot * sizeof(int2);
    auto go = [&](auto kernel) -> cudaError_t {
        const cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kernel));
        if (e != cudaSuccess) return e;
        kernel<<<grid, zp.threads, smem, s>>>(a, zp, x, y);
        return cudaGetLastError();
    };
    return zp.zc == 3 ? go(pattern_fast_zblock_kernel<3, 2, 2, 256, 4>) : go(pattern_fast_zblock_kernel<4, 2, 2, 256, 4>);
}

bool stage_supported(int nu) { return nu == 27 || nu == 19 || nu == 9 || nu == 7 || nu == 5; }

bool make_stage_plan(const std::vector<int32_t>& uoff, int rows_per_thread, int threads, int max_elems,
                     StagePlan* out) {
    StagePlan p{};
    p.rows = rows_per_thread * threads;
    p.rows_per_thread = rows_per_thread;
    p.tile0 = 0;
    p.ntiles = 0;
    const int nu = int(uoff.size());
    if (nu == 0 || nu > 31) return false;
    int seg = -1;
    for (int u = 0; u < nu; ++u) {
        if (u == 0 || int64_t(uoff[u]) - uoff[u - 1] > p.rows) {
            if (++seg >= kMaxSegments) return false;
            p.seg_min[seg] = uoff[u];
        }
        p.seg_span[seg] = uoff[u] - p.seg_min[seg];
    }
    p.nseg = seg + 1;
    int64_t base = 0;
    for (int sg = 0; sg < p.nseg; ++sg) {
        p.seg_base[sg] = int32_t(base);
        base += int64_t(p.rows) + p.seg_span[sg];
    }
    if (base > max_elems) return false;
    p.elems = int32_t(base);
    for (int u = 0, sg = 0; u < nu; ++u) {
        while (sg + 1 < p.nseg && uoff[u] >= p.seg_min[sg + 1]) ++sg;
        p.soff[u] = p.seg_base[sg] + (uoff[u] - p.seg_min[sg]);
    }
    // 16-byte staging of an int2 copy: each segment window starts at an even
    // global element (one element of padding in front when seg_min is odd;
    // tile starts are multiples of 512 and so even) and at an even position
    // in shared memory
    int64_t pbase = 0;
    for (int sg = 0; sg < p.nseg; ++sg) {
        p.seg_pad[sg] = (p.seg_min[sg] % 2 != 0) ? 1 : 0;
        p.seg_pbase[sg] = int32_t(pbase);
        pbase += (int64_t(p.rows) + p.seg_span[sg] + p.seg_pad[sg] + 1) / 2 * 2;
    }
    p.elems_padded = int32_t(pbase);
    for (int u = 0, sg = 0; u < nu; ++u) {
        while (sg + 1 < p.nseg && uoff[u] >= p.seg_min[sg + 1]) ++sg;
        p.soff_padded[u] = p.seg_pbase[sg] + p.seg_pad[sg] + (uoff[u] - p.seg_min[sg]);
    }
    *out = p;
    return true;
}

// ------------------------------------------------- Data+Index Table ------
// Listing 1 on the GPU, one thread per row: the row's type selects its
// value-grouped displacement list (staged in shared memory when the table
// fits), and the value groups are walked in ascending order with one fma per
// entry, so the result is bit-identical to Listing 1's chain.  x is read
// through the read-only cache.  A displacement leaving [0, n) can only come
// from a corrupt table: it sets the matrix's error word and is skipped.
constexpr int kDitSmemInts = 8192;   // 32 KB of displacements

__global__ void __launch_bounds__(kBlock) dit_kernel(DitView a, const double* __restrict__ x,
                                                    double* __restrict__ y) {
    __shared__ int32_t sdisp[kDitSmemInts];
    __shared__ double sdict[256];
    const int table = a.ntypes * a.maxlen;
    const bool staged = table <= kDitSmemInts;
    if (staged)
        for (int i = threadIdx.x; i < table; i += blockDim.x) sdisp[i] = __ldg(a.disp + i);
    for (int i = threadIdx.x; i < a.nv; i += blockDim.x) sdict[i] = __ldg(a.dict + i);
    __syncthreads();
    const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (r >= a.n) return;
    const int t = __ldg(a.type + r);
    const int32_t* d = (staged ? static_cast<const int32_t*>(sdisp) : a.disp) + t * a.maxlen;
    int idx = 0;
    double acc = 0.0;
    for (int v = 0; v < a.nv; ++v) {
        const double av = sdict[v];
        const int end = __ldg(a.ends + int64_t(v) * a.n + r);
        for (; idx < end; ++idx) {
            const int64_t j = r + (staged ? d[idx] : __ldg(d + idx));
            if (uint64_t(j) >= uint64_t(a.n)) {
                atomicOr(a.err, 1);
                continue;
            }
            acc = fma(av, __ldg(x + j), acc);
        }
    }
    y[r] = acc;
}

// ------------------------------------------------------- Data Table ------
// Sec. V's first scheme on the GPU, one thread per row, a warp per 32-row
// slice: slot t of the slice's rows is one coalesced 128-byte read of S.  The
// value groups are walked in ascending order with one fma per entry, so the
// result is bit-identical to the oracle's Data Table chain.  A column outside
// [0, n) or a group end past the slice width can only come from a corrupt
// table: it sets the matrix's error word and the entry is skipped.
__global__ void __launch_bounds__(kBlock) data_table_kernel(DataTableView a, const double* __restrict__ x,
                                                           double* __restrict__ y) {
    __shared__ double sdict[256];
    for (int i = threadIdx.x; i < a.nv; i += blockDim.x) sdict[i] = __ldg(a.dict + i);
    __syncthreads();
    const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (r >= a.n) return;
    const int64_t sl = r >> 5;
    const int w = __ldg(a.slice_w + sl);
    const int32_t* S = a.S + __ldg(a.slice_off + sl) + (r & 31);
    int idx = 0;
    double acc = 0.0;
    for (int v = 0; v < a.nv; ++v) {
        const double av = sdict[v];
        int end = __ldg(a.ends + int64_t(v) * a.n + r);
        if (end > w) {
            atomicOr(a.err, 1);
            end = w;
        }
        for (; idx < end; ++idx) {
            const int32_t j = __ldg(S + idx * 32);
            if (uint32_t(j) >= uint64_t(a.n)) {
                atomicOr(a.err, 1);
                continue;
            }
            acc = fma(av, __ldg(x + j), acc);
        }
    }
    y[r] = acc;
}

cudaError_t launch_data_table_f64(const DataTableView& a, const double* x, double* y, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (a.nv > 256) return cudaErrorInvalidValue;
    data_table_kernel<<<grid_of(a.n), kBlock, 0, s>>>(a, x, y);
    return cudaGetLastError();
}

cudaError_t launch_dit_f64(const DitView& a, const double* x, double* y, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (a.nv > 256) return cudaErrorInvalidValue;
    dit_kernel<<<grid_of(a.n), kBlock, 0, s>>>(a, x, y);
    return cudaGetLastError();
}

cudaError_t launch_delta_f64(const DeltaView& a, const double* x, double* y, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    delta_kernel<double><<<grid_of(a.nslices * 32), kBlock, 0, s>>>(a, x, y, nullptr);
    return cudaGetLastError();
}
cudaError_t launch_delta_f32(const DeltaView& a, const float* x, float* y, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    delta_kernel<float><<<grid_of(a.nslices * 32), kBlock, 0, s>>>(a, x, y, nullptr);
    return cudaGetLastError();
}
cudaError_t launch_delta_f64_scatter(const DeltaView& a, const double* x, double* y, const int32_t* perm,
                                     cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    delta_kernel<double><<<grid_of(a.nslices * 32), kBlock, 0, s>>>(a, x, y, perm);
    return cudaGetLastError();
}
cudaError_t launch_pattern_spmm_col(const PatternView& a, int k, const double* X, int64_t ldx, double* Y,
                                    int64_t ldy, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    SPMVC_DISPATCH_WORDS(a.words,
                         (pattern_spmm_col_kernel<W><<<grid_of(a.n * k), kBlock, 0, s>>>(a, k, X, ldx, Y, ldy)));
    return cudaGetLastError();
}
cudaError_t launch_pattern_spmm_fast(const PatternView& a, int k, const double* X, int64_t ldx, double* Y,
                                     int64_t ldy, uint32_t* partial, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (k > 64) return cudaErrorInvalidValue;
    xmax_cols_kernel<<<kXmaxBlocks, 256, 0, s>>>(X, a.n, k, ldx, partial);
    SPMVC_DISPATCH_WORDS(a.words, (pattern_spmm_fast_kernel<W><<<grid_of(a.n * k), kBlock, 0, s>>>(
                                      a, k, X, ldx, Y, ldy, partial)));
    return cudaGetLastError();
}

cudaError_t launch_pattern_spmm_fast_x(const PatternView& a, int k, const double* X, int64_t ldx, double* Y,
                                       int64_t ldy, uint32_t* partial, int2* Xf_guarded, int64_t guard_rows,
                                       cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (k > 64) return cudaErrorInvalidValue;
    uint32_t* emax = partial + kXmaxBlocks * 64;   // k words after the partial maxima
    int2* Xf = Xf_guarded + guard_rows * k;
    xmax_cols_kernel<<<kXmaxBlocks, 256, 0, s>>>(X, a.n, k, ldx, partial);
    cols_emax_kernel<<<1, 64, 0, s>>>(partial, k, emax);
    convert_cols_kernel<<<kXmaxBlocks * 16, 256, 0, s>>>(X, ldx, a.n, k, emax, Xf);
    if (!(a.run_len == 3 && a.nu == 27)) return cudaErrorNotSupported;
    // columns per thread: 4 or 2 for narrow blocks (measured faster there);
    // wider blocks use one thread per (row, column)
    const int kc = (k == 4) ? 4 : (k == 2) ? 2 : 1;
    const unsigned grid = grid_of(a.n * (k / kc));
    switch (kc) {
        case 8: pattern_spmm_rows_kernel<8, 27, 3><<<grid, kBlock, 0, s>>>(a, k, X, ldx, Xf, Y, ldy, emax); break;
        case 4: pattern_spmm_rows_kernel<4, 27, 3><<<grid, kBlock, 0, s>>>(a, k, X, ldx, Xf, Y, ldy, emax); break;
        case 2: pattern_spmm_rows_kernel<2, 27, 3><<<grid, kBlock, 0, s>>>(a, k, X, ldx, Xf, Y, ldy, emax); break;
        default: pattern_spmm_fast_x_kernel<7, 27, 3><<<grid_of(a.n * k), kBlock, 0, s>>>(a, k, X, ldx, Xf, Y, ldy, emax);
    }
    return cudaGetLastError();
}

cudaError_t launch_ell_spmm(const EllView& a, int k, const double* X, int64_t ldx, double* Y, int64_t ldy,
                            cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    ell_spmm_kernel<<<grid_of(a.n * k), kBlock, 0, s>>>(a, k, X, ldx, Y, ldy);
    return cudaGetLastError();
}
cudaError_t launch_delta_spmm(const DeltaView& a, int k, const double* X, int64_t ldx, double* Y, int64_t ldy,
                              cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    delta_spmm_kernel<<<grid_of(a.n * k), kBlock, 0, s>>>(a, k, X, ldx, Y, ldy);
    return cudaGetLastError();
}
cudaError_t launch_fill_u32(uint32_t* p, uint32_t v, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    fill_u32_kernel<<<grid_of(n), kBlock, 0, s>>>(p, v, n);
    return cudaGetLastError();
}

}  // namespace spmvc
