// Conjugate gradients on the device: the CG iteration of Table I of
// arXiv:1612.00530 (Dot, Waxpby, SpMV) without the preconditioner.
// Every vector and scalar stays in device memory; `check_every` steps are
// captured in a CUDA graph and replayed, and the host reads one convergence
// flag per replay.  Reductions use a fixed grid and a fixed tree, so results
// are the same on every run.
//
// Modes: FP64 (all in binary64) and IR_FP32 (iterative refinement: the
// residual b - A x, its norm and the update x += d in binary64, the inner
// correction solve A d = r with the binary32 product and binary32 vectors;
// inner dot products sum 8 products in binary32 and accumulate those chunks
// in binary64, or, where the product forms p.q itself, chunks of 4).
//
// A step is three launches: the product q = A p, which also returns
// per-CTA partial sums of p.q where its kernel can (else a dot kernel
// follows); r -= alpha q with the partial sums of r.r; and x += alpha p,
// p = r + beta p, whose last block to finish closes the step (the new r.r,
// the count, the stopping test).  Eight vector passes a step, none of them
// for p.q when the product forms it.
#include <cmath>
#include <cstring>
#include <vector>

#include "spmvc_internal.h"

namespace spmvc {
int api_ensure_device(spmv_mat_s* m);
bool api_valid(spmv_mat_t m);
int api_apply_xmax(spmv_mat_s* A, const double* x, double* y, const uint32_t* xmax_part, int xmax_n,
                   cudaStream_t s, double* dot_part, int* dot_n);
int api_apply_f32_dot(spmv_mat_s* A, const float* x, float* y, cudaStream_t s, double* dot_part, int* dot_n);
int api_prepare_f32(spmv_mat_s* m);
int api_spmm_xmax(spmv_mat_s* A, int32_t k, const double* X, int64_t ldx, double* Y, int64_t ldy, cudaStream_t s,
                  const uint32_t* xmax_part, int xmax_n);

namespace {

// Streaming kernels: grid-stride loops over a fixed grid that is one wave
// on 152 SMs (4 blocks of 256 an SM, so up to 64 registers a thread: the
// unrolled loops keep several 16-byte loads in flight without spilling).
// A grid larger than what the SMs hold at once would leave a second,
// partly empty wave at the end of every pass.
constexpr int kRedPerSm = 4;
constexpr int kRedBlocks = 152 * kRedPerSm;
constexpr int kRedThreads = 256;

struct CgState {
    double rr;          // inner r.r (IR)
    double rr2[2];      // r.r before the step of that parity (FP64 and binary32 loops)
    double rr0;         // inner: initial r.r
    double bnorm;
    double tol;
    double alpha;       // the step's alpha (block 0 of the r update writes it)
    int32_t it;         // steps taken
    int32_t max_it;
    int32_t done;
    uint32_t closed;    // blocks of the step's last kernel that have finished
};

// Sum of the kRedBlocks partials by one warp in a fixed order.
__device__ __forceinline__ double sum_partials(const double* __restrict__ p) {
    double s = 0.0;
    for (int i = threadIdx.x & 31; i < kRedBlocks; i += 32) s += p[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    return s;
}

__device__ __forceinline__ double block_sum(double v, double* sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    }
    return s;  // valid in thread 0
}

// Sum of `count` partials by the whole block in a fixed order, returned to
// every thread (sm: 33 doubles).
__device__ __forceinline__ double block_sum_partials(const double* __restrict__ p, int count, double* sm) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += p[i];
    s = block_sum(s, sm);
    if (threadIdx.x == 0) sm[32] = s;
    __syncthreads();
    return sm[32];
}

// True in thread 0 of the block that finishes the kernel last (the others'
// stores are then all issued); it resets the count for the next launch.
__device__ __forceinline__ bool last_block(CgState* st) {
    __syncthreads();
    if (threadIdx.x != 0) return false;
    __threadfence();
    const bool last = atomicAdd(&st->closed, 1u) == gridDim.x - 1;
    if (last) {
        __threadfence();
        st->closed = 0u;
    }
    return last;
}

// Per block, the largest high word of |v| over the values the block wrote
// (the next product's scale), into pmax[blockIdx.x].
__device__ __forceinline__ void block_hi_max(uint32_t mx, uint32_t* __restrict__ pmax) {
    __shared__ uint32_t s_mx[32];
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < (blockDim.x >> 5) ? s_mx[threadIdx.x] : 0u;
        v = __reduce_max_sync(0xFFFFFFFFu, v);
        if (threadIdx.x == 0) pmax[blockIdx.x] = v;
    }
}

__device__ __forceinline__ uint32_t hi_abs(double v) { return uint32_t(__double2hiint(v)) & 0x7FFFFFFFu; }

__global__ void __launch_bounds__(kRedThreads, kRedPerSm) dot_kernel(const double* __restrict__ a,
                                                                    const double* __restrict__ b, int64_t n,
                                                                    double* __restrict__ partial,
                                                                    const CgState* __restrict__ st) {
    if (st && st->done) return;
    __shared__ double sm[32];
    double s = 0.0, s2 = 0.0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u) == 0) {
        const int64_t n2 = n / 2;
        const double2* a2 = reinterpret_cast<const double2*>(a);
        const double2* b2 = reinterpret_cast<const double2*>(b);
        for (; i + 3 * stride < n2; i += 4 * stride) {
            double2 u[4], v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                u[k] = a2[i + k * stride];
                v[k] = b2[i + k * stride];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                s = fma(u[k].x, v[k].x, s);
                s2 = fma(u[k].y, v[k].y, s2);
            }
        }
        for (; i < n2; i += stride) {
            const double2 u = a2[i], v = b2[i];
            s = fma(u.x, v.x, s);
            s2 = fma(u.y, v.y, s2);
        }
        if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) s = fma(a[n - 1], b[n - 1], s);
    } else {
        for (; i < n; i += stride) s = fma(a[i], b[i], s);
    }
    s = block_sum(s + s2, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// alpha = rr / (p.q) (npq partial sums of p.q); r -= alpha q; partial sums
// of r.r.  par: the step's parity, which of st->rr2 holds its r.r.
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) update_r_kernel(double* __restrict__ r, const double* __restrict__ q,
                                                               int64_t n, const double* __restrict__ partial_pq,
                                                               int npq, double* __restrict__ partial_rr,
                                                               CgState* __restrict__ st, int par) {
    if (st->done) return;
    __shared__ double sm[33];
    const double alpha = st->rr2[par] / block_sum_partials(partial_pq, npq, sm);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->alpha = alpha;
    double s = 0.0, s2 = 0.0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    if (((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(q)) & 15u) == 0) {
        const int64_t n2 = n / 2;
        double2* r2 = reinterpret_cast<double2*>(r);
        const double2* q2 = reinterpret_cast<const double2*>(q);
        auto one = [&](double2 rv, const double2 qv, int64_t j) {
            rv.x = fma(-alpha, qv.x, rv.x);
            rv.y = fma(-alpha, qv.y, rv.y);
            r2[j] = rv;
            s = fma(rv.x, rv.x, s);
            s2 = fma(rv.y, rv.y, s2);
        };
        int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
        // four elements in flight a thread: loads first, then the updates
        for (; i + 3 * stride < n2; i += 4 * stride) {
            double2 rv[4], qv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                rv[k] = r2[i + k * stride];
                qv[k] = q2[i + k * stride];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) one(rv[k], qv[k], i + k * stride);
        }
        for (; i < n2; i += stride) one(r2[i], q2[i], i);
        if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
            const double ri = fma(-alpha, q[n - 1], r[n - 1]);
            r[n - 1] = ri;
            s = fma(ri, ri, s);
        }
    } else {
        for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += stride) {
            const double ri = fma(-alpha, q[i], r[i]);
            r[i] = ri;
            s = fma(ri, ri, s);
        }
    }
    s = block_sum(s + s2, sm);
    if (threadIdx.x == 0) partial_rr[blockIdx.x] = s;
}

// beta = rr_new / rr; x += alpha p; p = r + beta p; per block the largest
// high word of |p|.  The block that finishes last closes the step: the new
// r.r into the other parity's slot, the step count, the history and the
// convergence flag (every block has read the flag by then).
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) update_xp_kernel(double* __restrict__ x, double* __restrict__ p,
                                                                const double* __restrict__ r, int64_t n,
                                                                const double* __restrict__ partial_rr,
                                                                CgState* __restrict__ st, double* __restrict__ hist,
                                                                int par, uint32_t* __restrict__ pmax) {
    if (st->done) return;
    __shared__ double sm[33];
    const double rr_new = block_sum_partials(partial_rr, kRedBlocks, sm);
    const double alpha = st->alpha, beta = rr_new / st->rr2[par];
    uint32_t mx = 0u;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(r)) & 15u) ==
        0) {
        const int64_t n2 = n / 2;
        double2* x2 = reinterpret_cast<double2*>(x);
        double2* p2 = reinterpret_cast<double2*>(p);
        const double2* r2 = reinterpret_cast<const double2*>(r);
        auto one = [&](double2 xv, double2 pv, const double2 rv, int64_t j) {
            xv.x = fma(alpha, pv.x, xv.x);
            xv.y = fma(alpha, pv.y, xv.y);
            pv.x = fma(beta, pv.x, rv.x);
            pv.y = fma(beta, pv.y, rv.y);
            x2[j] = xv;
            p2[j] = pv;
            mx = max(mx, max(hi_abs(pv.x), hi_abs(pv.y)));
        };
        int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
        for (; i + 3 * stride < n2; i += 4 * stride) {
            double2 xv[4], pv[4], rv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                xv[k] = x2[i + k * stride];
                pv[k] = p2[i + k * stride];
                rv[k] = r2[i + k * stride];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) one(xv[k], pv[k], rv[k], i + k * stride);
        }
        for (; i < n2; i += stride) one(x2[i], p2[i], r2[i], i);
        if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
            const double po = p[n - 1];
            x[n - 1] = fma(alpha, po, x[n - 1]);
            const double pl = fma(beta, po, r[n - 1]);
            p[n - 1] = pl;
            mx = max(mx, hi_abs(pl));
        }
    } else {
        for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += stride) {
            const double po = p[i];
            x[i] = fma(alpha, po, x[i]);
            const double pl = fma(beta, po, r[i]);
            p[i] = pl;
            mx = max(mx, hi_abs(pl));
        }
    }
    block_hi_max(mx, pmax);
    if (last_block(st)) {
        st->rr2[par ^ 1] = rr_new;
        const int32_t it = st->it + 1;
        st->it = it;
        const double rel = sqrt(rr_new) / st->bnorm;
        hist[it] = rel;
        if (rel <= st->tol || it >= st->max_it) st->done = 1;
    }
}

// r = b - q, partial sums of r.r
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) residual_kernel(const double* __restrict__ b, const double* __restrict__ q,
                                                               double* __restrict__ r, int64_t n,
                                                               double* __restrict__ partial) {
    __shared__ double sm[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double ri = b[i] - q[i];
        r[i] = ri;
        s = fma(ri, ri, s);
    }
    s = block_sum(s, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// dst = src; pmax (optional): per block, the largest high word of |src|
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) copy_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                                           int64_t n, uint32_t* __restrict__ pmax) {
    uint32_t mx = 0u;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double v = src[i];
        dst[i] = v;
        mx = max(mx, hi_abs(v));
    }
    if (pmax) block_hi_max(mx, pmax);
}

// ---------------------------------------------------- binary32 inner CG ---
// chunks of 8 products summed in binary32, chunk sums accumulated in binary64
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) dot32_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                                            int64_t n, double* __restrict__ partial,
                                                            const CgState* __restrict__ st) {
    if (st->done) return;
    __shared__ double sm[32];
    double s = 0.0;
    // chunks of 8 products (two 16-byte loads per operand) summed in binary32
    const int64_t n8 = n / 8, stride = int64_t(gridDim.x) * blockDim.x;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    for (int64_t c8 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c8 < n8; c8 += stride) {
        const float4 u0 = a4[2 * c8], u1 = a4[2 * c8 + 1], v0 = b4[2 * c8], v1 = b4[2 * c8 + 1];
        float c = u0.x * v0.x;
        c = fmaf(u0.y, v0.y, c); c = fmaf(u0.z, v0.z, c); c = fmaf(u0.w, v0.w, c);
        c = fmaf(u1.x, v1.x, c); c = fmaf(u1.y, v1.y, c); c = fmaf(u1.z, v1.z, c); c = fmaf(u1.w, v1.w, c);
        s += double(c);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        float c = 0.0f;
        for (int64_t i = n8 * 8; i < n; ++i) c = fmaf(a[i], b[i], c);
        s += double(c);
    }
    s = block_sum(s, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// alpha = rr / (p.q) in binary32 (npq partial sums of p.q); r -= alpha q;
// partial sums of r.r (chunks of four in binary32)
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) update_r32_kernel(float* __restrict__ r, const float* __restrict__ q,
                                                                 int64_t n, const double* __restrict__ partial_pq,
                                                                 int npq, double* __restrict__ partial_rr,
                                                                 CgState* __restrict__ st, int par) {
    if (st->done) return;
    __shared__ double sm[33];
    const float alpha = float(st->rr2[par] / block_sum_partials(partial_pq, npq, sm));
    if (blockIdx.x == 0 && threadIdx.x == 0) st->alpha = alpha;
    double s = 0.0;
    const int64_t n4 = n / 4, stride = int64_t(gridDim.x) * blockDim.x;
    float4* r4 = reinterpret_cast<float4*>(r);
    const float4* q4 = reinterpret_cast<const float4*>(q);
    auto one = [&](float4 rv, const float4 qv, int64_t j) {
        rv.x = fmaf(-alpha, qv.x, rv.x); rv.y = fmaf(-alpha, qv.y, rv.y);
        rv.z = fmaf(-alpha, qv.z, rv.z); rv.w = fmaf(-alpha, qv.w, rv.w);
        r4[j] = rv;
        float c = rv.x * rv.x;
        c = fmaf(rv.y, rv.y, c); c = fmaf(rv.z, rv.z, c); c = fmaf(rv.w, rv.w, c);
        s += double(c);
    };
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    for (; i + 3 * stride < n4; i += 4 * stride) {
        float4 rv[4], qv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            rv[k] = r4[i + k * stride];
            qv[k] = q4[i + k * stride];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) one(rv[k], qv[k], i + k * stride);
    }
    for (; i < n4; i += stride) one(r4[i], q4[i], i);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        float c = 0.0f;
        for (int64_t i = n4 * 4; i < n; ++i) {
            const float ri = fmaf(-alpha, q[i], r[i]);
            r[i] = ri;
            c = fmaf(ri, ri, c);
        }
        s += double(c);
    }
    s = block_sum(s, sm);
    if (threadIdx.x == 0) partial_rr[blockIdx.x] = s;
}

// beta in binary32; d += alpha p; p = r + beta p.  The block that finishes
// last closes the inner step (r.r into the other parity's slot, the step
// count, the stopping test), as in the FP64 loop.
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) update_dp32_kernel(float* __restrict__ d, float* __restrict__ p,
                                                                  const float* __restrict__ r, int64_t n,
                                                                  const double* __restrict__ partial_rr,
                                                                  CgState* __restrict__ st, int par) {
    if (st->done) return;
    __shared__ double sm[33];
    const double rr_new = block_sum_partials(partial_rr, kRedBlocks, sm);
    const float alpha = float(st->alpha), beta = float(rr_new / st->rr2[par]);
    const int64_t n4 = n / 4, stride = int64_t(gridDim.x) * blockDim.x;
    float4* d4 = reinterpret_cast<float4*>(d);
    float4* p4 = reinterpret_cast<float4*>(p);
    const float4* r4 = reinterpret_cast<const float4*>(r);
    auto one = [&](float4 dv, float4 pv, const float4 rv, int64_t j) {
        dv.x = fmaf(alpha, pv.x, dv.x); dv.y = fmaf(alpha, pv.y, dv.y);
        dv.z = fmaf(alpha, pv.z, dv.z); dv.w = fmaf(alpha, pv.w, dv.w);
        pv.x = fmaf(beta, pv.x, rv.x); pv.y = fmaf(beta, pv.y, rv.y);
        pv.z = fmaf(beta, pv.z, rv.z); pv.w = fmaf(beta, pv.w, rv.w);
        d4[j] = dv;
        p4[j] = pv;
    };
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    for (; i + 3 * stride < n4; i += 4 * stride) {
        float4 dv[4], pv[4], rv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            dv[k] = d4[i + k * stride];
            pv[k] = p4[i + k * stride];
            rv[k] = r4[i + k * stride];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) one(dv[k], pv[k], rv[k], i + k * stride);
    }
    for (; i < n4; i += stride) one(d4[i], p4[i], r4[i], i);
    if (blockIdx.x == 0 && threadIdx.x < 4 && n4 * 4 + threadIdx.x < n) {
        const int64_t i = n4 * 4 + threadIdx.x;
        const float po = p[i];
        d[i] = fmaf(alpha, po, d[i]);
        p[i] = fmaf(beta, po, r[i]);
    }
    if (last_block(st)) {
        st->rr2[par ^ 1] = rr_new;
        const int32_t it = st->it + 1;
        st->it = it;
        if (sqrt(rr_new / st->rr0) <= st->tol || it >= st->max_it) st->done = 1;
    }
}

// inner start: r32 = r / |r|, p32 = r32, d32 = 0; partial sums of r32.r32
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) inner_start_kernel(const double* __restrict__ r, double inv_norm,
                                                                  float* __restrict__ r32, float* __restrict__ p32,
                                                                  float* __restrict__ d32, int64_t n,
                                                                  double* __restrict__ partial) {
    __shared__ double sm[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float v = float(r[i] * inv_norm);
        r32[i] = v;
        p32[i] = v;
        d32[i] = 0.0f;
        s += double(v) * double(v);
    }
    s = block_sum(s, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void inner_init_state_kernel(const double* __restrict__ partial, CgState* __restrict__ st, double inner_tol,
                                        int inner_max) {
    const double rr = sum_partials(partial);
    if (threadIdx.x == 0) {
        st->rr = rr;
        st->rr2[0] = rr;
        st->rr0 = rr;
        st->tol = inner_tol;
        st->it = 0;
        st->max_it = inner_max;
        st->done = rr > 0.0 ? 0 : 1;
        st->closed = 0u;
    }
}

// x += scale * d32 (binary64)
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) ir_update_kernel(double* __restrict__ x, const float* __restrict__ d32,
                                                                double scale, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x[i] = fma(scale, double(d32[i]), x[i]);
}

__global__ void sum_to_host_kernel(const double* __restrict__ partial, double* __restrict__ out) {
    const double s = sum_partials(partial);
    if (threadIdx.x == 0) *out = s;
}


// ------------------------------------------- k right-hand sides at once ---
// Vectors are n x k row-major; column j is an independent CG whose scalars
// live in ColState.  A column whose residual is exactly zero freezes
// (alpha = beta = 0).
constexpr int kMaxCols = 32;
struct ColState {
    double rr[kMaxCols], alpha[kMaxCols], beta[kMaxCols], bnorm[kMaxCols];
    double tol;
    int32_t k, it, max_it, done;
    int32_t live;   // the current step runs (set by the alpha kernel from done)
    int32_t pad;
};

// partial[b*k + j]: block b's sum over its rows of a[r,j]*b[r,j]
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) dot_cols_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                               int64_t n, int k, double* __restrict__ partial,
                                                               const ColState* __restrict__ st) {
    if (st && st->done) return;
    __shared__ double sm[kRedThreads];
    const int R = kRedThreads / k, j = threadIdx.x % k, sub = threadIdx.x / k;
    double s = 0.0;
    if (sub < R) {
        const int64_t rs = int64_t(gridDim.x) * R;
        int64_t r = blockIdx.x * int64_t(R) + sub;
        for (; r + 3 * rs < n; r += 4 * rs) {   // four rows in flight a thread
            double u[4], v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                u[c] = a[(r + c * rs) * k + j];
                v[c] = b[(r + c * rs) * k + j];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) s = fma(u[c], v[c], s);
        }
        for (; r < n; r += rs) s = fma(a[r * k + j], b[r * k + j], s);
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int i = 0; i < R; ++i) t += sm[i * k + threadIdx.x];
        partial[blockIdx.x * k + threadIdx.x] = t;
    }
}

// column j's partials (nb blocks) summed by one warp in a fixed order (valid
// in every lane)
__device__ __forceinline__ double sum_col_warp(const double* __restrict__ partial, int k, int j,
                                               int nb = kRedBlocks) {
    double s = 0.0;
    for (int b = threadIdx.x & 31; b < nb; b += 32) s += partial[b * k + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    return s;
}

// alpha_j = rr_j / (p_j . q_j), one warp per column; the step runs (live)
// exactly when the batch had not converged before it
__global__ void alpha_cols_kernel(const double* __restrict__ partial_pq, int npq, ColState* __restrict__ st) {
    if (st->done) {
        if (threadIdx.x == 0) st->live = 0;
        return;
    }
    if (threadIdx.x == 0) st->live = 1;
    const int j = threadIdx.x >> 5;
    if (j >= st->k) return;
    const double pq = sum_col_warp(partial_pq, st->k, j, npq);
    if ((threadIdx.x & 31) == 0) st->alpha[j] = (st->rr[j] > 0.0 && pq != 0.0) ? st->rr[j] / pq : 0.0;
}

// r -= alpha q; partial sums of r.r per column
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) update_r_cols_kernel(double* __restrict__ r,
                                                                     const double* __restrict__ q, int64_t n,
                                                                     double* __restrict__ partial_rr,
                                                                     const ColState* __restrict__ st) {
    if (st->done) return;
    __shared__ double sm[kRedThreads];
    const int k = st->k, R = kRedThreads / k, j = threadIdx.x % k, sub = threadIdx.x / k;
    const double alpha = st->alpha[j];
    double s = 0.0;
    if (sub < R) {
        const int64_t rs = int64_t(gridDim.x) * R;
        int64_t row = blockIdx.x * int64_t(R) + sub;
        for (; row + 3 * rs < n; row += 4 * rs) {
            double rv[4], qv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                rv[c] = r[(row + c * rs) * k + j];
                qv[c] = q[(row + c * rs) * k + j];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double ri = fma(-alpha, qv[c], rv[c]);
                r[(row + c * rs) * k + j] = ri;
                s = fma(ri, ri, s);
            }
        }
        for (; row < n; row += rs) {
            const int64_t i = row * k + j;
            const double ri = fma(-alpha, q[i], r[i]);
            r[i] = ri;
            s = fma(ri, ri, s);
        }
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int i = 0; i < R; ++i) t += sm[i * k + threadIdx.x];
        partial_rr[blockIdx.x * k + threadIdx.x] = t;
    }
}

// beta_j, rr_j, history (largest relative residual), convergence
__global__ void beta_cols_kernel(const double* __restrict__ partial_rr, ColState* __restrict__ st,
                                 double* __restrict__ hist) {
    if (st->done) return;
    __shared__ double rel[kMaxCols];
    const int j = threadIdx.x >> 5, k = st->k;
    if (j < k) {
        const double rr_new = sum_col_warp(partial_rr, k, j);
        if ((threadIdx.x & 31) == 0) {
            st->beta[j] = st->rr[j] > 0.0 ? rr_new / st->rr[j] : 0.0;
            st->rr[j] = rr_new;
            rel[j] = sqrt(rr_new) / st->bnorm[j];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int c = 0; c < k; ++c) m = fmax(m, rel[c]);
        st->it += 1;
        hist[st->it] = m;
        if (m <= st->tol || st->it >= st->max_it) st->done = 1;
    }
}

// Per column j, the largest high word of |v| this block's threads of that
// column saw (mx), into pmax[blockIdx.x * k + j] (the SpMM's scales).
__device__ __forceinline__ void block_col_hi_max(uint32_t mx, int k, uint32_t* __restrict__ pmax) {
    __shared__ uint32_t s_mx[kRedThreads];
    const int R = kRedThreads / k;
    s_mx[threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.x < k) {
        uint32_t m = 0u;
        for (int i = 0; i < R; ++i) m = max(m, s_mx[i * k + threadIdx.x]);
        pmax[blockIdx.x * k + threadIdx.x] = m;
    }
}

// x += alpha p; p = r + beta p (a step that ran: the beta kernel may have
// just set the convergence flag, and x still takes this step's update);
// per-block column maxima of |p| for the next SpMM
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) update_xp_cols_kernel(double* __restrict__ x,
                                                                     double* __restrict__ p,
                                                                     const double* __restrict__ r, int64_t n,
                                                                     const ColState* __restrict__ st,
                                                                     uint32_t* __restrict__ pmax) {
    if (!st->live) return;
    const int k = st->k, R = kRedThreads / k, j = threadIdx.x % k, sub = threadIdx.x / k;
    uint32_t mx = 0u;
    if (sub < R) {
        const double alpha = st->alpha[j], beta = st->beta[j];
        const int64_t rs = int64_t(gridDim.x) * R;
        int64_t row = blockIdx.x * int64_t(R) + sub;
        for (; row + 3 * rs < n; row += 4 * rs) {
            double xv[4], pv[4], rv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t i = (row + c * rs) * k + j;
                xv[c] = x[i];
                pv[c] = p[i];
                rv[c] = r[i];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t i = (row + c * rs) * k + j;
                x[i] = fma(alpha, pv[c], xv[c]);
                const double pn = fma(beta, pv[c], rv[c]);
                p[i] = pn;
                mx = max(mx, hi_abs(pn));
            }
        }
        for (; row < n; row += rs) {
            const int64_t i = row * k + j;
            const double po = p[i];
            x[i] = fma(alpha, po, x[i]);
            const double pn = fma(beta, po, r[i]);
            p[i] = pn;
            mx = max(mx, hi_abs(pn));
        }
    }
    block_col_hi_max(mx, k, pmax);
}

// dst = src (n x k) with per-block column maxima of |src| (the first SpMM's
// scales)
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) copy_cols_kernel(double* __restrict__ dst,
                                                                const double* __restrict__ src, int64_t n, int k,
                                                                uint32_t* __restrict__ pmax) {
    const int R = kRedThreads / k, j = threadIdx.x % k, sub = threadIdx.x / k;
    uint32_t mx = 0u;
    if (sub < R)
        for (int64_t row = blockIdx.x * int64_t(R) + sub; row < n; row += int64_t(gridDim.x) * R) {
            const double v = src[row * k + j];
            dst[row * k + j] = v;
            mx = max(mx, hi_abs(v));
        }
    block_col_hi_max(mx, k, pmax);
}

// r = b - q, partial sums of r.r per column
__global__ void __launch_bounds__(kRedThreads, kRedPerSm) residual_cols_kernel(const double* __restrict__ b,
                                                                    const double* __restrict__ q,
                                                                    double* __restrict__ r, int64_t n, int k,
                                                                    double* __restrict__ partial) {
    __shared__ double sm[kRedThreads];
    const int R = kRedThreads / k, j = threadIdx.x % k, sub = threadIdx.x / k;
    double s = 0.0;
    if (sub < R)
        for (int64_t row = blockIdx.x * int64_t(R) + sub; row < n; row += int64_t(gridDim.x) * R) {
            const int64_t i = row * k + j;
            const double ri = b[i] - q[i];
            r[i] = ri;
            s = fma(ri, ri, s);
        }
    sm[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int i = 0; i < R; ++i) t += sm[i * k + threadIdx.x];
        partial[blockIdx.x * k + threadIdx.x] = t;
    }
}

__global__ void col_sums_kernel(const double* __restrict__ partial, int k, double* __restrict__ out) {
    const int j = threadIdx.x >> 5;
    if (j >= k) return;
    const double s = sum_col_warp(partial, k, j);
    if ((threadIdx.x & 31) == 0) out[j] = s;
}

struct Workspace {
    std::vector<void*> allocs;
    ~Workspace() { for (void* p : allocs) cudaFree(p); }
    template <class T> T* get(size_t count) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(16, count * sizeof(T))) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        return static_cast<T*>(p);
    }
};

int cuda_err(cudaError_t e, const char* what) {
    return fail(SPMV_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CG_CUDA(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return cuda_err(e_, #call); } while (0)
#define CG_ST(call) do { int s_ = (call); if (s_) return s_; } while (0)

double read_scalar(const double* d, cudaStream_t s) {
    double h = 0.0;
    cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return h;
}

// Replays `body` (captured `chunk` times) until st->done.
template <class Body>
int run_until_done(cudaStream_t s, bool use_graph, int chunk, CgState* d_st, int max_replays, Body&& body) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (use_graph) {
        CG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int st = SPMV_OK;
        for (int k = 0; k < chunk && !st; ++k) st = body();
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return cuda_err(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&ge, g, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_err(e, "cudaGraphInstantiate"); }
    }
    int32_t done = 0;
    int rc = SPMV_OK;
    for (int rep = 0; rep < max_replays && !done; ++rep) {
        if (use_graph) {
            cudaError_t e = cudaGraphLaunch(ge, s);
            if (e != cudaSuccess) { rc = cuda_err(e, "cudaGraphLaunch"); break; }
        } else {
            for (int k = 0; k < chunk && !rc; ++k) rc = body();
            if (rc) break;
        }
        cudaError_t e = cudaMemcpyAsync(&done, &d_st->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_err(e, "convergence flag"); break; }
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    return rc;
}


// k right-hand sides at once (plain FP64 CG per column, products by SpMM)
int cg_solve_cols(spmv_mat_t A, const double* b, double* x, const spmv_cg_opts& o, spmv_cg_result* res) {
    const int64_t n = A->n;
    const int k = o.nrhs;
    cudaStream_t s;
    CG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard { cudaStream_t s; ~StreamGuard() { cudaStreamDestroy(s); } } guard{s};
    Workspace ws;
    double* r = ws.get<double>(n * k);
    double* q = ws.get<double>(n * k);
    double* p = ws.get<double>(n * k);
    double* part_a = ws.get<double>(size_t(kRedBlocks) * k);
    double* part_b = ws.get<double>(size_t(kRedBlocks) * k);
    double* d_sums = ws.get<double>(k);
    ColState* d_st = ws.get<ColState>(1);
    double* d_hist = ws.get<double>(o.max_iter + 2);
    uint32_t* pmax = ws.get<uint32_t>(size_t(kRedBlocks) * k);
    if (!r || !q || !p || !part_a || !part_b || !d_sums || !d_st || !d_hist || !pmax)
        return fail(SPMV_ENOMEM, "CG workspace");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    CG_CUDA(cudaEventRecord(e0, s));
    const unsigned G = kRedBlocks, T = kRedThreads;
    std::vector<double> h(k);
    auto col_norms2 = [&](const double* a) -> int {
        dot_cols_kernel<<<G, T, 0, s>>>(a, a, n, k, part_a, nullptr);
        col_sums_kernel<<<1, 32 * kMaxCols, 0, s>>>(part_a, k, d_sums);
        CG_CUDA(cudaMemcpyAsync(h.data(), d_sums, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
        CG_CUDA(cudaStreamSynchronize(s));
        return SPMV_OK;
    };
    auto residual = [&]() -> int {
        CG_ST(spmm_apply(A, k, x, k, q, k, s));
        residual_cols_kernel<<<G, T, 0, s>>>(b, q, r, n, k, part_a);
        col_sums_kernel<<<1, 32 * kMaxCols, 0, s>>>(part_a, k, d_sums);
        CG_CUDA(cudaMemcpyAsync(h.data(), d_sums, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
        CG_CUDA(cudaStreamSynchronize(s));
        return SPMV_OK;
    };
    CG_ST(col_norms2(b));
    ColState hs{};
    hs.k = k;
    hs.tol = o.tol;
    hs.max_it = o.max_iter;
    for (int j = 0; j < k; ++j) hs.bnorm[j] = std::sqrt(h[j]) > 0.0 ? std::sqrt(h[j]) : 1.0;
    CG_ST(residual());
    double rel0 = 0.0;
    for (int j = 0; j < k; ++j) {
        hs.rr[j] = h[j];
        rel0 = std::max(rel0, std::sqrt(h[j]) / hs.bnorm[j]);
    }
    hs.done = rel0 <= o.tol ? 1 : 0;
    CG_CUDA(cudaMemcpyAsync(d_st, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
    CG_CUDA(cudaMemcpyAsync(d_hist, &rel0, sizeof(double), cudaMemcpyHostToDevice, s));
    copy_cols_kernel<<<G, T, 0, s>>>(p, r, n, k, pmax);
    auto body = [&]() -> int {
        // p.q stays a pass of its own here: inside the SpMM its binary64
        // multiply a (row, column) would share the narrow FP64 pipe with
        // the rounding of every output
        CG_ST(api_spmm_xmax(A, k, p, k, q, k, s, pmax, int(G)));
        dot_cols_kernel<<<G, T, 0, s>>>(p, q, n, k, part_a, d_st);
        alpha_cols_kernel<<<1, 32 * kMaxCols, 0, s>>>(part_a, int(G), d_st);
        update_r_cols_kernel<<<G, T, 0, s>>>(r, q, n, part_b, d_st);
        beta_cols_kernel<<<1, 32 * kMaxCols, 0, s>>>(part_b, d_st, d_hist);
        update_xp_cols_kernel<<<G, T, 0, s>>>(x, p, r, n, d_st, pmax);
        CG_CUDA(cudaGetLastError());
        return SPMV_OK;
    };
    // the columns' loop replays its own graph and polls ColState's flag
    int32_t done = hs.done;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (o.use_graph) {
        CG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int st = SPMV_OK;
        for (int c = 0; c < o.check_every && !st; ++c) st = body();
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return cuda_err(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&ge, g, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_err(e, "cudaGraphInstantiate"); }
    }
    const int replays = (o.max_iter + o.check_every - 1) / o.check_every + 1;
    int rc = SPMV_OK;
    for (int rep = 0; rep < replays && !done && !rc; ++rep) {
        if (ge) {
            cudaError_t e = cudaGraphLaunch(ge, s);
            if (e != cudaSuccess) rc = cuda_err(e, "cudaGraphLaunch");
        } else {
            for (int c = 0; c < o.check_every && !rc; ++c) rc = body();
        }
        if (!rc) {
            cudaError_t e = cudaMemcpyAsync(&done, &d_st->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_err(e, "convergence flag");
        }
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
    CG_CUDA(cudaMemcpyAsync(&hs, d_st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    CG_CUDA(cudaStreamSynchronize(s));
    std::vector<double> history(hs.it + 1);
    CG_CUDA(cudaMemcpy(history.data(), d_hist, sizeof(double) * (hs.it + 1), cudaMemcpyDeviceToHost));
    CG_ST(residual());
    double rel = 0.0;
    for (int j = 0; j < k; ++j) rel = std::max(rel, std::sqrt(h[j]) / hs.bnorm[j]);
    CG_CUDA(cudaEventRecord(e1, s));
    CG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int status = (rel <= o.tol * 10.0 || history.back() <= o.tol) ? SPMV_OK : SPMV_ENOTCONVERGED;
    if (res) {
        res->status = status;
        res->iterations = hs.it;
        res->outer_iterations = 0;
        res->rel_residual = rel;
        res->seconds = ms * 1e-3;
        res->history_len = static_cast<int32_t>(history.size());
        res->history = static_cast<double*>(std::malloc(sizeof(double) * std::max<size_t>(1, history.size())));
        if (!res->history) return fail(SPMV_ENOMEM, "history allocation");
        std::memcpy(res->history, history.data(), sizeof(double) * history.size());
    }
    return status;
}

}  // namespace
}  // namespace spmvc

using namespace spmvc;

extern "C" int cg_solve(spmv_mat_t A, const double* b, double* x, const spmv_cg_opts* opts, spmv_cg_result* res) {
    if (!api_valid(A)) return fail(SPMV_EINVAL, "invalid matrix handle");
    spmv_cg_opts o{1e-10, 10000, SPMV_CG_FP64, 16, 60, 1e-5, 1, 1};
    if (opts) o = *opts;
    if (o.tol <= 0) o.tol = 1e-10;
    if (o.max_iter <= 0) o.max_iter = 10000;
    if (o.check_every <= 0) o.check_every = 16;
    if (o.inner_max_iter <= 0) o.inner_max_iter = 300;
    if (o.inner_tol <= 0) o.inner_tol = 1e-6;
    if (o.nrhs <= 0) o.nrhs = 1;
    if (o.nrhs < 1 || o.nrhs > kMaxCols) return fail(SPMV_EINVAL, "nrhs must be 1..32");
    if (o.nrhs > 1 && o.mode != SPMV_CG_FP64) return fail(SPMV_EUNSUPPORTED, "several right-hand sides: FP64 mode only");
    if (o.mode != SPMV_CG_FP64 && o.mode != SPMV_CG_IR_FP32) return fail(SPMV_EINVAL, "unknown CG mode");
    const int64_t n = A->n;
    if (n > 0 && (!b || !x)) return fail(SPMV_EINVAL, "null vector");
    if (res) std::memset(res, 0, sizeof(*res));
    CG_ST(api_ensure_device(A));
    if (o.nrhs > 1) return cg_solve_cols(A, b, x, o, res);
    cudaStream_t s;
    CG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard { cudaStream_t s; ~StreamGuard() { cudaStreamDestroy(s); } } guard{s};
    Workspace ws;
    double* r = ws.get<double>(n);
    double* q = ws.get<double>(n);
    double* p = ws.get<double>(n);
    double* part_a = ws.get<double>(kRedBlocks);
    double* part_b = ws.get<double>(kRedBlocks);
    double* d_scalar = ws.get<double>(1);
    CgState* d_st = ws.get<CgState>(1);
    const int hist_cap = o.max_iter + 2;
    double* d_hist = ws.get<double>(hist_cap);
    uint32_t* pmax = ws.get<uint32_t>(kRedBlocks);
    if (!r || !q || !p || !part_a || !part_b || !d_scalar || !d_st || !d_hist || !pmax)
        return fail(SPMV_ENOMEM, "CG workspace");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (o.mode != SPMV_CG_FP64) CG_ST(api_prepare_f32(A));   // row types built before the clock starts
    CG_CUDA(cudaEventRecord(e0, s));

    const unsigned G = kRedBlocks, T = kRedThreads;
    // b norm and the initial residual r = b - A x
    dot_kernel<<<G, T, 0, s>>>(b, b, n, part_a, nullptr);
    sum_to_host_kernel<<<1, 32, 0, s>>>(part_a, d_scalar);
    const double bnorm = std::sqrt(read_scalar(d_scalar, s));
    if (!(bnorm > 0.0)) {
        cudaMemsetAsync(x, 0, sizeof(double) * n, s);  // b == 0: x = 0 is the solution
        cudaStreamSynchronize(s);
        if (res) { res->status = SPMV_OK; }
        return SPMV_OK;
    }
    std::vector<double> history;
    int total_inner = 0, outer = 0;
    int status = SPMV_ENOTCONVERGED;
    double rel = 0.0;

    auto true_residual = [&]() -> int {
        CG_ST(spmv_apply(A, x, q, s));
        residual_kernel<<<G, T, 0, s>>>(b, q, r, n, part_a);
        sum_to_host_kernel<<<1, 32, 0, s>>>(part_a, d_scalar);
        CG_CUDA(cudaGetLastError());
        return SPMV_OK;
    };

    if (o.mode == SPMV_CG_FP64) {
        CG_ST(true_residual());
        const double rr0 = read_scalar(d_scalar, s);
        CgState h{rr0, {rr0, 0.0}, rr0, bnorm, o.tol, 0.0, 0, o.max_iter, 0, 0u};
        h.done = (std::sqrt(rr0) / bnorm <= o.tol) ? 1 : 0;
        CG_CUDA(cudaMemcpyAsync(d_st, &h, sizeof(h), cudaMemcpyHostToDevice, s));
        const double h0 = std::sqrt(rr0) / bnorm;
        CG_CUDA(cudaMemcpyAsync(d_hist, &h0, sizeof(double), cudaMemcpyHostToDevice, s));
        copy_kernel<<<G, T, 0, s>>>(p, r, n, pmax);
        // steps alternate which slot of rr2 they read: the body is called
        // once a step in order (captured or not), and an even chunk keeps a
        // replayed graph's parities those of the global step count
        int step = 0;
        auto body = [&]() -> int {
            const int par = step++ & 1;
            int npq = 0;   // partial sums of p.q the product wrote (0: a dot kernel forms them)
            CG_ST(api_apply_xmax(A, p, q, pmax, int(G), s, part_a, &npq));
            if (npq == 0) {
                dot_kernel<<<G, T, 0, s>>>(p, q, n, part_a, d_st);
                npq = int(G);
            }
            update_r_kernel<<<G, T, 0, s>>>(r, q, n, part_a, npq, part_b, d_st, par);
            update_xp_kernel<<<G, T, 0, s>>>(x, p, r, n, part_b, d_st, d_hist, par, pmax);
            CG_CUDA(cudaGetLastError());
            return SPMV_OK;
        };
        const int chunk = (o.check_every + 1) & ~1;
        const int replays = (o.max_iter + chunk - 1) / chunk + 1;
        CG_ST(run_until_done(s, o.use_graph != 0, chunk, d_st, replays, body));
        CG_CUDA(cudaMemcpyAsync(&h, d_st, sizeof(h), cudaMemcpyDeviceToHost, s));
        CG_CUDA(cudaStreamSynchronize(s));
        history.resize(h.it + 1);
        CG_CUDA(cudaMemcpy(history.data(), d_hist, sizeof(double) * (h.it + 1), cudaMemcpyDeviceToHost));
        total_inner = h.it;
        CG_ST(true_residual());
        rel = std::sqrt(read_scalar(d_scalar, s)) / bnorm;
        status = rel <= o.tol * 10.0 || history.back() <= o.tol ? SPMV_OK : SPMV_ENOTCONVERGED;
    } else {
        float* r32 = ws.get<float>(n);
        float* p32 = ws.get<float>(n);
        float* q32 = ws.get<float>(n);
        float* d32 = ws.get<float>(n);
        if (!r32 || !p32 || !q32 || !d32) return fail(SPMV_ENOMEM, "IR workspace");
        CG_CUDA(cudaMemsetAsync(p32, 0, sizeof(float) * n, s));
        CG_ST(spmv_apply_f32(A, p32, q32, s));  // first binary32 call may allocate: keep it out of capture
        for (;;) {
            CG_ST(true_residual());
            const double rr = read_scalar(d_scalar, s);
            rel = std::sqrt(rr) / bnorm;
            history.push_back(rel);
            if (rel <= o.tol) { status = SPMV_OK; break; }
            if (total_inner >= o.max_iter) break;
            const double rnorm = std::sqrt(rr);
            // the inner solve need not reduce its residual by more than a
            // quarter of what the outer target still asks (tol / rel): the
            // last one usually stops early
            const double inner_tol = std::max(o.inner_tol, 0.25 * o.tol / rel);
            inner_start_kernel<<<G, T, 0, s>>>(r, 1.0 / rnorm, r32, p32, d32, n, part_a);
            inner_init_state_kernel<<<1, 32, 0, s>>>(part_a, d_st, inner_tol,
                                                     std::min(o.inner_max_iter, o.max_iter - total_inner));
            int step = 0;   // parity of r.r's slot, as in the FP64 loop
            auto body = [&]() -> int {
                const int par = step++ & 1;
                int npq = 0;
                CG_ST(api_apply_f32_dot(A, p32, q32, s, part_a, &npq));
                if (npq == 0) {
                    dot32_kernel<<<G, T, 0, s>>>(p32, q32, n, part_a, d_st);
                    npq = int(G);
                }
                update_r32_kernel<<<G, T, 0, s>>>(r32, q32, n, part_a, npq, part_b, d_st, par);
                update_dp32_kernel<<<G, T, 0, s>>>(d32, p32, r32, n, part_b, d_st, par);
                CG_CUDA(cudaGetLastError());
                return SPMV_OK;
            };
            const int chunk = (o.check_every + 1) & ~1;
            const int replays = (o.inner_max_iter + chunk - 1) / chunk + 1;
            CG_ST(run_until_done(s, o.use_graph != 0, chunk, d_st, replays, body));
            CgState h;
            CG_CUDA(cudaMemcpyAsync(&h, d_st, sizeof(h), cudaMemcpyDeviceToHost, s));
            CG_CUDA(cudaStreamSynchronize(s));
            total_inner += h.it;
            ir_update_kernel<<<G, T, 0, s>>>(x, d32, rnorm, n);
            ++outer;
            if (h.it == 0) break;
        }
    }
    CG_CUDA(cudaEventRecord(e1, s));
    CG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (res) {
        res->status = status;
        res->iterations = total_inner;
        res->outer_iterations = outer;
        res->rel_residual = rel;
        res->seconds = ms * 1e-3;
        res->history_len = static_cast<int32_t>(history.size());
        res->history = static_cast<double*>(std::malloc(sizeof(double) * std::max<size_t>(1, history.size())));
        if (!res->history) return fail(SPMV_ENOMEM, "history allocation");
        std::memcpy(res->history, history.data(), sizeof(double) * history.size());
    }
    return status;
}

extern "C" int spmv_cg_result_free(spmv_cg_result* res) {
    if (!res) return SPMV_OK;
    std::free(res->history);
    res->history = nullptr;
    res->history_len = 0;
    return SPMV_OK;
}
