// PTX wrappers shared by the TMA-fed kernels: mbarriers (bounded waits),
// tensor and bulk copies into shared memory, the named barrier of the
// compute warps, and the split of (block, plane) work among persistent CTAs.
// Included inside each kernel file's anonymous namespace.
#pragma once

constexpr int32_t kErrWaitTimeout = 16;           // error-word bit: an mbarrier wait gave up
constexpr long long kWaitCycles = 2000000000LL;   // about one second at 2 GHz

__device__ __forceinline__ uint32_t saddr(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

// Waits until the phase of `bar` with the given parity has completed; false
// when that has not happened within kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = saddr(bar);
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    const long long t0 = clock64();
    do {
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(a), "r"(parity), "r"(20000u)
            : "memory");
        if (done) return true;
    } while (clock64() - t0 < kWaitCycles);
    return false;
}

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA, bulk copy) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(saddr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(saddr(bar))
        : "memory");
}

// Streams that are read once (the row records) are marked evict-first in L2
// so that x, read by neighbouring blocks too, stays there.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(saddr(dst)),
        "l"(src), "r"(bytes), "r"(saddr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

// Barrier 1 over the n compute threads only (the producer warp never joins).
__device__ __forceinline__ void compute_sync(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }

// The same barrier, returning whether any of the n threads passed true.
__device__ __forceinline__ bool compute_sync_or(int n, bool v) {
    uint32_t r;
    asm volatile(
        "{ .reg .pred pi, po; setp.ne.u32 pi, %1, 0; bar.red.or.pred po, 1, %2, pi; selp.u32 %0, 1, 0, po; }"
        : "=r"(r)
        : "r"(uint32_t(v)), "r"(n)
        : "memory");
    return r != 0;
}

// A CTA's share of the (block, plane) sequence, visited block-major, as
// runs of planes z0 .. z1-1 of one column block.  A run costs its planes
// plus about kRunCost steps of start-up, so each block counts kRunCost
// more units than it has planes (the start-up of the run that begins it)
// and the CTAs take equal ranges of those units: a CTA whose range crosses
// a block boundary gets fewer planes.
constexpr int kRunCost = 2;
struct Share {
    int64_t u, uend;      // units of this CTA still to visit: [u, uend)
    int nzr, z_lo;
    __device__ bool next(int& b, int& z0, int& z1) {
        const int per = nzr + kRunCost;
        while (u < uend) {
            b = int(u / per);
            const int o0 = int(u - int64_t(b) * per);
            const int o1 = int(min(uend - int64_t(b) * per, int64_t(per)));
            u = int64_t(b) * per + o1;
            // unit offsets 0 .. kRunCost-1 of a block stand for its start-up
            const int p0 = max(o0 - kRunCost, 0), p1 = max(o1 - kRunCost, 0);
            if (p1 > p0) {
                z0 = z_lo + p0;
                z1 = z_lo + p1;
                return true;
            }
        }
        return false;
    }
};

