// Result check used by the autotuner: a candidate FAST kernel's y must agree
// with the COLUMN-order product y_ref within the FAST error bound, element
// by element (non-finite entries must match exactly).  Also the largest
// |x_j| that scales the bound.
#include <cstdint>

#include "spmvc_internal.h"

namespace spmvc {
namespace {

constexpr int kCheckBlock = 256;

__global__ void __launch_bounds__(kCheckBlock) absmax_kernel(const double* __restrict__ x, int64_t n,
                                                            unsigned long long* __restrict__ out) {
    double m = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        m = fmax(m, fabs(__ldg(x + i)));
    // non-negative doubles order like their bit patterns
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(m));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, b, o);
        b = t > b ? t : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, b);
}

__global__ void __launch_bounds__(kCheckBlock) check_close_kernel(const double* __restrict__ y,
                                                                 const double* __restrict__ yref, int64_t n,
                                                                 double abs_tol, double rel_tol,
                                                                 unsigned long long* __restrict__ bad) {
    unsigned long long cnt = 0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double a = __ldg(y + i), b = __ldg(yref + i);
        bool ok;
        if (isfinite(b)) ok = isfinite(a) && fabs(a - b) <= abs_tol + rel_tol * fabs(b);
        else ok = (isnan(a) && isnan(b)) || a == b;
        cnt += ok ? 0 : 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(bad, cnt);
}

unsigned check_grid(int64_t n) {
    const int64_t b = (n + kCheckBlock - 1) / kCheckBlock;
    return unsigned(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

}  // namespace

cudaError_t launch_absmax(const double* x, int64_t n, unsigned long long* out, cudaStream_t s) {
    absmax_kernel<<<check_grid(n), kCheckBlock, 0, s>>>(x, n, out);
    return cudaGetLastError();
}

cudaError_t launch_check_close(const double* y, const double* yref, int64_t n, double abs_tol, double rel_tol,
                               unsigned long long* bad, cudaStream_t s) {
    check_close_kernel<<<check_grid(n), kCheckBlock, 0, s>>>(y, yref, n, abs_tol, rel_tol, bad);
    return cudaGetLastError();
}

}  // namespace spmvc
