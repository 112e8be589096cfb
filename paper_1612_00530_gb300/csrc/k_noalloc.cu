// spmm_apply_noalloc: the FAST-order multi-vector product Y = A X for
// callers that must not allocate device memory -- for instance code running
// inside a framework that owns every device allocation through its own
// pool, or a latency-critical loop where the implicit device
// synchronisation of cudaMalloc/cudaFree is not acceptable.  It runs the
// generic FAST SpMM path on the unconverted X: a column-maxima pass, then one
// thread per (row, column) converting X entries as it reads them.  It does
// not take spmm_apply's faster route for the full 27-point union (X
// converted once into a fixed-point copy, then the row-wise kernels), since
// that copy would need an allocation of n * k * 8 bytes; the two paths agree
// within FAST order's error bound, not bit for bit.  The scratch -- one
// maximum-exponent word per (block of the column-maxima pass, right-hand
// side) -- is a file-scope device array of fixed size, so every GPU that
// loads the library holds it (19.5 KB) until the process exits.
#include <mutex>

#include "spmvc_internal.h"

namespace spmvc {
bool api_valid(spmv_mat_t m);
}

namespace {

constexpr int kNoAllocMaxCols = 32;                    // widest X this entry point accepts
constexpr int kNoAllocWords = 152 * kNoAllocMaxCols;   // 152 partial maxima per column

// Shared by every call on a device: each call's column-maxima pass writes
// every word the following product reads, so nothing has to start at zero,
// but two calls whose kernels overlap on the GPU race on it.
static __device__ __align__(256) uint32_t g_noalloc_partials[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in, so the address is looked up once per device
// (with that device current) and cached.
int scratch_for_current_device(uint32_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return spmvc::fail(SPMV_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return spmvc::fail(SPMV_EUNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess)
            return spmvc::fail(SPMV_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch[dev];
    return SPMV_OK;
}

}  // namespace

extern "C" int spmm_apply_noalloc(spmv_mat_t A, int32_t k, const double* X, int64_t ldx, double* Y, int64_t ldy,
                                  spmv_stream_t stream) {
    if (!spmvc::api_valid(A)) return spmvc::fail(SPMV_EINVAL, "invalid matrix handle");
    if (k < 1 || k > kNoAllocMaxCols)
        return spmvc::fail(SPMV_EINVAL, "spmm_apply_noalloc takes 1 <= k <= 32 right-hand sides "
                                        "(the size of its static scratch)");
    if (ldx < k || ldy < k) return spmvc::fail(SPMV_EINVAL, "need ldx >= k and ldy >= k");
    if (A->n > 0 && (!X || !Y)) return spmvc::fail(SPMV_EINVAL, "null block");
    if (A->fmt != SPMV_FMT_PATTERN || A->order != SPMV_ORDER_FAST || !A->perm.empty())
        return spmvc::fail(SPMV_EUNSUPPORTED, "spmm_apply_noalloc needs a pattern-format matrix in FAST order, not reordered");
    int dev = 0;
    const cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return spmvc::fail(SPMV_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(de));
    if (A->device < 0 || A->device != dev)
        return spmvc::fail(SPMV_EINVAL, "the matrix is not on the current device yet: make one ordinary device call "
                                        "on it first (that call copies it and may allocate)");
    uint32_t* scratch = nullptr;
    int st = scratch_for_current_device(&scratch);
    if (st) return st;
    const cudaError_t e = spmvc::launch_pattern_spmm_fast(A->pat_view, k, X, ldx, Y, ldy, scratch,
                                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return spmvc::fail(SPMV_ECUDA, std::string("spmm_apply_noalloc launch: ") + cudaGetErrorString(e));
    return SPMV_OK;
}
