// Permutation passes around the product of a reordered matrix B = P A P^T
// (perm[new] = old): xp = P x before it, y = P^T yp after it.  One thread per
// element, 16-byte-friendly strided loops over a grid of whole waves; the
// permuted side is coalesced, the other side is a gather or a scatter.
#include <cstdint>

#include "spmvc_internal.h"

namespace spmvc {
namespace {

constexpr int kPermBlock = 256;

__global__ void __launch_bounds__(kPermBlock) gather_kernel(const int32_t* __restrict__ perm, int64_t n,
                                                           const double* __restrict__ x, double* __restrict__ xp) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        xp[i] = __ldg(x + __ldg(perm + i));
}

__global__ void __launch_bounds__(kPermBlock) scatter_kernel(const int32_t* __restrict__ perm, int64_t n,
                                                            const double* __restrict__ yp, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[__ldg(perm + i)] = __ldg(yp + i);
}

unsigned perm_grid(int64_t n) {
    const int64_t blocks = (n + kPermBlock - 1) / kPermBlock;
    return unsigned(blocks < 152 * 16 ? blocks : 152 * 16);
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
