// Permutation passes around the product of a reordered matrix B = P A P^T
// (perm[new] = old): xp = P x before it, y = P^T yp after it.  Strided loops
// over a grid of whole waves; the permuted side is coalesced, the other side
// is a gather or a scatter.
#include <cstdint>

#include "spmvc_internal.h"

namespace spmvc {
namespace {

constexpr int kPermBlock = 256;

// Each thread moves kPermUnroll elements a pass, all their index loads
// first, so that several random accesses are in flight per thread.
constexpr int kPermUnroll = 8;

__global__ void __launch_bounds__(kPermBlock) gather_kernel(const int32_t* __restrict__ perm, int64_t n,
                                                           const double* __restrict__ x, double* __restrict__ xp) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i0 < n; i0 += kPermUnroll * stride) {
        int32_t p[kPermUnroll];
#pragma unroll
        for (int u = 0; u < kPermUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            p[u] = i < n ? __ldg(perm + i) : 0;
        }
        double v[kPermUnroll];
#pragma unroll
        for (int u = 0; u < kPermUnroll; ++u) v[u] = i0 + u * stride < n ? __ldg(x + p[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < kPermUnroll; ++u)
            if (i0 + u * stride < n) xp[i0 + u * stride] = v[u];
    }
}

__global__ void __launch_bounds__(kPermBlock) scatter_kernel(const int32_t* __restrict__ perm, int64_t n,
                                                            const double* __restrict__ yp, double* __restrict__ y) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i0 < n; i0 += kPermUnroll * stride) {
        int32_t p[kPermUnroll];
        double v[kPermUnroll];
#pragma unroll
        for (int u = 0; u < kPermUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            p[u] = i < n ? __ldg(perm + i) : 0;
            v[u] = i < n ? __ldg(yp + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kPermUnroll; ++u)
            if (i0 + u * stride < n) y[p[u]] = v[u];
    }
}

unsigned perm_grid(int64_t n) {
    const int64_t blocks = (n + kPermBlock - 1) / kPermBlock;
    return unsigned(blocks < 152 * 8 ? blocks : 152 * 8);
}

}  // namespace

cudaError_t launch_gather(const int32_t* perm, int64_t n, const double* x, double* xp, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    gather_kernel<<<perm_grid(n), kPermBlock, 0, s>>>(perm, n, x, xp);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const int32_t* perm, int64_t n, const double* yp, double* y, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    scatter_kernel<<<perm_grid(n), kPermBlock, 0, s>>>(perm, n, yp, y);
    return cudaGetLastError();
}

}  // namespace spmvc
