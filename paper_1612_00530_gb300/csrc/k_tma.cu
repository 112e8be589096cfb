// FAST-order compressed SpMV, y = A x (Eq. 1 of arXiv:1612.00530), for the
// pattern format of a 27-point grid stencil (Sec. V: value codes plus a
// stencil-pattern number per row), fed by the Tensor Memory Accelerator.
//
// One persistent CTA an SM walks an equal share of the (column block, plane)
// sequence.  A column block is L whole grid lines of a plane (C = L*nx rows,
// a tile of TY lines by four columns a compute thread).  A producer warp keeps the copies
// going: lane 0 loads, for every plane z of the block, the x window W(z) --
// the box of nx+4 elements by L+2 lines at (ix = -2, iy = first line - 1, z),
// one TMA tensor copy that fills everything outside the grid with zeros
// (the 16-byte-aligned start at ix = -2 puts two zero columns on each side
// of a line) -- and lane 1 the block's row records of every plane (three
// planes of 16, 8 and 4 bytes a row, bulk copies), each into the next free
// stage of its ring (full/empty mbarrier pairs), so loads run up to two
// windows and three record planes ahead of the compute warps.  The compute
// warps, step by step:
//  - compare each row's record with the record its grid position implies
//    (the dominant codes at the in-grid slots, the absent code elsewhere,
//    the matching pattern number) and hand the record stage back;
//  - convert the newest window once into 53-bit fixed point (two int32
//    limbs) in a ring of four shared-memory slots, stored as four
//    sub-arrays by element index mod 4 so that the six consecutive elements
//    of a window line a tile reads are conflict-free 8-byte loads at
//    constant offsets, and hand the raw stage back;
//  - sum every row of the plane two windows back over all 27 window slots
//    with the dominant record's weights (an out-of-grid neighbour reads a
//    zero, which is what its absent slot contributes), round each exact
//    integer sum once and store the rows whose record was the expected one;
//    after the step's barrier the other rows are summed slot by slot from
//    their own record and global x.
// The scale exponent is the largest one the CTA has seen since its current
// run of planes began; a window that raises it is converted again (from x)
// and the two windows still in use are shifted down (exact: floor of floor).
// Every wait on an mbarrier is bounded: past about a second the kernel sets
// the handle's error word (bit 16), drains its copies in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "spmvc_internal.h"

namespace spmvc {

namespace {

#include "fast_fixed.cuh"
#include "tma_ptx.cuh"

constexpr int kRawStages = 2;
constexpr int kMaxBlockRows = 1536;             // C with one CTA an SM

// With MINB CTAs an SM (1 or 2) each holds at most kMaxBlockRows / MINB
// rows, a ring slot of slot_elems elements (16 KB, or 10 KB) and
// rec_stages record stages (three, or two), so that two CTAs' shared
// memory fits an SM.
__host__ __device__ constexpr int slot_elems(int minb) { return minb == 1 ? 2048 : 1280; }
__host__ __device__ constexpr int rec_stages(int minb) { return minb == 1 ? 3 : 2; }

// A compute thread sums a tile of TY grid lines by four columns (K = 4 TY
// rows).  A ring slot holds four sub-arrays, sub-array s the window elements
// e with e mod 4 = s at index e / 4: the six elements of a window line a
// tile reads (its four columns and one each side) are six conflict-free
// 8-byte loads at constant offsets.  Threads 0 .. C/K-1 compute; the last
// warp is the producer.  With DOT the kernel also forms x.y (the p.q of a
// CG step, Sec. II): every thread adds x[row]*y[row] of the rows it stores,
// in binary64 in its own order, and the CTA's sum of those goes to
// dot_part[blockIdx.x].
template <int TY, bool DOT, int MINB>
__global__ void __launch_bounds__(kMaxBlockRows / (4 * TY * MINB) + 32, MINB)
    pattern_fast_tma_kernel(const __grid_constant__ CUtensorMap xmap, const PatternView a, const TmaPlan tp,
                            const double* __restrict__ x, double* __restrict__ y,
                            const uint32_t* __restrict__ xmax_part, int xmax_n, double* __restrict__ dot_part) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int K = 4 * TY;                          // rows a compute thread
    constexpr int kSlotElems = slot_elems(MINB);
    constexpr int kRecStages = rec_stages(MINB);
    constexpr int SUB = kSlotElems / 4;
    constexpr uint32_t SUBB = uint32_t(SUB) * 8u;     // bytes of a sub-array
    constexpr uint32_t SLOTB = 4u * SUBB;              // bytes of a ring slot
    const int tid = threadIdx.x, lane = tid & 31;
    const int NC = tp.threads, C = tp.C, nx = tp.nx;   // compute threads, rows a block
    const int fw = C >> 5;                             // match words a plane
    unsigned char* const ring = smem;
    unsigned char* const raw = smem + tp.off_raw;
    unsigned char* const rec = smem + tp.off_rec;
    uint32_t* const sexp = reinterpret_cast<uint32_t*>(smem + tp.off_exp);
    uint32_t* const sflags = reinterpret_cast<uint32_t*>(smem + tp.off_flags);
    uint32_t* const swmax = reinterpret_cast<uint32_t*>(smem + tp.off_words);   // [4] largest hi word of a window
    uint32_t* const swexc = swmax + 4;                                           // [4] rows off their expected record
    volatile uint32_t* const sabort = swmax + 8;
    volatile uint32_t* const spdone = swmax + 9;       // producer lanes done (count)
    volatile uint32_t* const siss = swmax + 10;        // [2] windows / record planes issued
    uint64_t* const raw_full = reinterpret_cast<uint64_t*>(smem + tp.off_mbar);
    uint64_t* const raw_empty = raw_full + kRawStages;
    uint64_t* const rec_full = raw_empty + kRawStages;
    uint64_t* const rec_empty = rec_full + kRecStages;

    for (int i = tid; i < 64 * 8; i += blockDim.x) sexp[i] = __ldg(tp.expected + i);
    if (tid < 12) swmax[tid] = 0u;
    // a caller that knows max |x| (partial maxima of the high words) fixes
    // the scale for every run: no window ever raises it
    uint32_t E_given = 0u;
    if (xmax_part) {
        uint32_t m = 0u;
        for (int i = lane; i < xmax_n; i += 32) m = max(m, __ldg(xmax_part + i));
        E_given = __reduce_max_sync(0xFFFFFFFFu, m) >> 20;
    }
    if (tid == 0) {
        for (int i = 0; i < kRawStages; ++i) {
            mbar_init(raw_full + i, 1);
            mbar_init(raw_empty + i, NC / 32);   // one arrival a compute warp
        }
        for (int i = 0; i < kRecStages; ++i) {
            mbar_init(rec_full + i, 1);
            mbar_init(rec_empty + i, NC / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const int nzr = tp.z_hi - tp.z_lo;
    const int64_t units = int64_t(tp.nblk) * (nzr + kRunCost);
    Share share{units * blockIdx.x / gridDim.x, units * (blockIdx.x + 1) / gridDim.x, nzr, tp.z_lo};

    if (tid >= NC) {
        // ---- producer warp: lane 0 streams the x windows, lane 1 the row
        // records, each as far ahead as its free stages allow
        if (lane > 1) return;
        const uint64_t policy = evict_first_policy();
        uint32_t n = 0;
        int b, z0, z1;
        bool ok = true;
        while (ok && share.next(b, z0, z1)) {
            for (int w = z0 - 1; ok && w <= z1; ++w) {
                if (lane == 0) {
                    // W(w): consumed at step w
                    const uint32_t st = n % kRawStages, k = n / kRawStages;
                    if (k > 0 && !mbar_wait(raw_empty + st, (k - 1) & 1u)) ok = false;
                    if (ok && *sabort) ok = false;
                    if (!ok) break;
                    fence_proxy_async();
                    mbar_expect_tx(raw_full + st, uint32_t(tp.win_elems) * 8u);
                    tma_load_3d(raw + st * tp.raw_bytes, &xmap, -2, b * tp.L - 1, w, raw_full + st);
                    siss[0] = ++n;
                } else if (w >= z0 && w < z1) {
                    // records of plane w: checked at step w + 1
                    const uint32_t st = n % kRecStages, k = n / kRecStages;
                    if (k > 0 && !mbar_wait(rec_empty + st, (k - 1) & 1u)) ok = false;
                    if (ok && *sabort) ok = false;
                    if (!ok) break;
                    unsigned char* dst = rec + st * 28u * uint32_t(C);
                    const int64_t r0 = int64_t(w) * tp.S + int64_t(b) * C;
                    fence_proxy_async();
                    mbar_expect_tx(rec_full + st, 28u * uint32_t(C));
                    bulk_g2s(dst, a.p16a + r0, 16u * C, rec_full + st, policy);
                    bulk_g2s(dst + 16 * C, a.p8 + r0, 8u * C, rec_full + st, policy);
                    bulk_g2s(dst + 24 * C, a.p4 + r0, 4u * C, rec_full + st, policy);
                    siss[1] = ++n;
                }
            }
        }
        if (!ok && !*sabort) {
            atomicOr(reinterpret_cast<uint32_t*>(swmax + 8), 1u);
            raise_error(a.err, kErrWaitTimeout);
        }
        __threadfence_block();
        atomicAdd(reinterpret_cast<uint32_t*>(swmax + 9), 1u);
        return;
    }

    // ---- compute threads
    // summing: the tile of block lines TY*ctl .. TY*ctl+TY-1 and columns
    // cix .. cix+3 (four-column groups of a line: nx / 4)
    const int xgs = nx >> 2;
    const int ctl = tid / xgs, cix = 4 * (tid - ctl * xgs);
    // byte offset in a ring slot of the sub-array index of the first element
    // the tile reads in window line TY*ctl + l, l = 0 .. TY+1 (window line 0
    // is the line above the block): (TY*ctl + l) * pitch + cix + 1 = 4 q + 1
    uint32_t qoff[TY + 2];
#pragma unroll
    for (int l = 0; l < TY + 2; ++l) qoff[l] = uint32_t(((TY * ctl + l) * tp.pitch + cix) >> 2) * 8u;
    // checking: rows tid + k*NC of the block, one a lane, coalesced
    int ckx[K], ckl[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int rho = tid + k * NC;
        ckl[k] = rho / nx;
        const int ixk = rho - ckl[k] * nx;
        ckx[k] = (ixk > 0 ? 1 : 0) | (ixk < nx - 1 ? 2 : 0);
    }

    uint32_t nraw = 0, nrec = 0;   // windows / record planes consumed so far
    uint32_t it = 0;               // loop steps so far
    bool aborted = false;
    double dacc = 0.0;             // this thread's part of x.y (DOT)
    // this thread's rows of the plane checked last step / this step had a
    // record off its expected one
    bool exc_now = false, exc_next = false;
    int b, z0, z1;
    while (!aborted && share.next(b, z0, z1)) {
        const int64_t blk0 = int64_t(b) * C;    // the block's first row inside a plane
        int cxy[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int iy = b * tp.L + ckl[k];
            cxy[k] = ckx[k] | ((iy > 0 ? 1 : 0) | (iy < tp.ny - 1 ? 2 : 0)) << 2;
        }
        // the record of an interior row (class 63: every neighbour in the
        // grid), kept in registers; a warp with a boundary row reads its
        // rows' expected records from shared memory instead
        uint32_t exi[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) exi[i] = sexp[63 * 8 + i];
        uint32_t E_true = E_given;       // largest biased exponent seen in this run of planes
        uint32_t E_ring = max(E_given, 64u);   // scale of the converted windows: max(E_true, 64)

        auto store_limbs = [&](unsigned char* slot, int e, int2 v) {
            *reinterpret_cast<int2*>(slot + uint32_t(e & 3) * SUBB + uint32_t(e >> 2) * 8u) = v;
        };
        auto convert = [&](const unsigned char* rw, unsigned char* slot, uint32_t E) -> uint32_t {
            uint32_t mx = 0;
            const int npairs = tp.win_elems >> 1;
            for (int pi = tid; pi < npairs; pi += NC) {
                const uint4 v = *reinterpret_cast<const uint4*>(rw + 16 * pi);
                mx = max(mx, max(v.y & 0x7FFFFFFFu, v.w & 0x7FFFFFFFu));
                const int e = 2 * pi;   // elements e (an even sub-array) and e + 1 (the next one)
                unsigned char* d0 = slot + uint32_t(e & 3) * SUBB + uint32_t(e >> 2) * 8u;
                *reinterpret_cast<int2*>(d0) = fixed_limbs(v.x, v.y, E);
                *reinterpret_cast<int2*>(d0 + SUBB) = fixed_limbs(v.z, v.w, E);
            }
            return mx;
        };
        // the window W(w) again, from x itself (its raw stage is gone by then),
        // zero outside the grid as the TMA box is
        auto convert_global = [&](int w, unsigned char* slot, uint32_t E) {
            for (int e = tid; e < tp.win_elems; e += NC) {
                const int line = e / tp.pitch, ix = e - line * tp.pitch - 2, iy = b * tp.L - 1 + line;
                double v = 0.0;
                if (ix >= 0 && ix < nx && iy >= 0 && iy < tp.ny && w >= 0 && w < tp.nz)
                    v = __ldg(x + (int64_t(w) * tp.ny + iy) * nx + ix);
                store_limbs(slot, e, fixed_limbs(uint32_t(__double2loint(v)), uint32_t(__double2hiint(v)), E));
            }
        };
        auto rescale = [&](unsigned char* slot, uint32_t d) {
            for (int e = tid; e < tp.win_elems; e += NC) {
                int2* pv = reinterpret_cast<int2*>(slot + uint32_t(e & 3) * SUBB + uint32_t(e >> 2) * 8u);
                const int2 v = *pv;
                const int64_t X = int64_t(v.y) * (int64_t(1) << 26) + v.x;
                const uint64_t mag = X < 0 ? uint64_t(0) - uint64_t(X) : uint64_t(X);
                const uint64_t m2 = d >= 64u ? 0u : (mag >> d);
                const int32_t s1 = X < 0 ? -1 : 1;
                *pv = make_int2(int32_t(uint32_t(m2) & 0x3FFFFFFu) * s1, int32_t(uint32_t(m2 >> 26)) * s1);
            }
        };

        for (int w = z0 - 1; w <= z1 + 1; ++w, ++it) {
            const int j = w - z0 + 1;   // index of W(w) within this run: ring slot j & 3
            bool wait_ok = true;
            bool raises = false;        // this thread's part of W(w) raises the scale
            const int q = w - 2;        // the plane summed this step
            const bool have_q = q >= z0 && q < z1;
            // x at the tile's rows of plane q, loaded now for x.y at the
            // step's end (the window holds them in fixed point only)
            double2 pv[TY][2];
            if constexpr (DOT) {
                if (have_q) {
                    const double2* xr = reinterpret_cast<const double2*>(x + int64_t(q) * tp.S + blk0 +
                                                                         int64_t(TY * ctl) * nx + cix);
#pragma unroll
                    for (int ry = 0; ry < TY; ++ry) {
                        pv[ry][0] = __ldg(xr + int64_t(ry) * (nx >> 1));
                        pv[ry][1] = __ldg(xr + int64_t(ry) * (nx >> 1) + 1);
                    }
                }
            }
            exc_now = exc_next;
            exc_next = false;
            if (tid == 0) {
                swmax[(it + 2) & 3] = 0u;   // the word of step it - 2 (read before step it - 1's barrier)
                swexc[(it + 1) & 3] = 0u;   // the word of step it - 3
            }
            // ---- check the records of plane w-1 against their grid position,
            // then hand the record stage back to the producer
            if (w - 1 >= z0 && w - 1 < z1) {
                const int p = w - 1;
                const uint32_t st = nrec % kRecStages;
                if (!mbar_wait(rec_full + st, (nrec / kRecStages) & 1u)) wait_ok = false;
                const int cz = (p > 0 ? 1 : 0) | (p < tp.nz - 1 ? 2 : 0);
                const unsigned char* rs = rec + st * 28u * uint32_t(C);
                uint32_t nbad = 0;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int rho = tid + k * NC;
                    const uint4 v16 = *reinterpret_cast<const uint4*>(rs + 16 * rho);
                    const uint2 v8 = *reinterpret_cast<const uint2*>(rs + 16 * C + 8 * rho);
                    const uint32_t v4 = *reinterpret_cast<const uint32_t*>(rs + 24 * C + 4 * rho);
                    const int cls = cxy[k] | (cz << 4);
                    uint32_t ex[7];
                    if (__any_sync(0xFFFFFFFFu, cls != 63)) {
#pragma unroll
                        for (int i = 0; i < 7; ++i) ex[i] = sexp[cls * 8 + i];
                    } else {
#pragma unroll
                        for (int i = 0; i < 7; ++i) ex[i] = exi[i];
                    }
                    const uint32_t diff = (v16.x ^ ex[0]) | (v16.y ^ ex[1]) | (v16.z ^ ex[2]) | (v16.w ^ ex[3]) |
                                          (v8.x ^ ex[4]) | (v8.y ^ ex[5]) | (v4 ^ ex[6]);
                    const uint32_t match = __ballot_sync(0xFFFFFFFFu, diff == 0u);
                    if (lane == 0) sflags[(it % 3) * fw + (tid >> 5) + k * (NC >> 5)] = match;
                    nbad += 32u - __popc(match);
                    if (diff) exc_next = true;
                }
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(rec_empty + st);
                    if (nbad) atomicAdd(swexc + (it & 3), nbad);
                }
                ++nrec;
            }
            // ---- convert W(w) into ring slot j & 3 at the current scale, then
            // hand the raw stage back
            if (w <= z1) {
                const uint32_t st = nraw % kRawStages;
                uint32_t mx = 0;
                if (mbar_wait(raw_full + st, (nraw / kRawStages) & 1u))
                    mx = convert(raw + st * tp.raw_bytes, ring + uint32_t(j & 3) * SLOTB, E_ring);
                else
                    wait_ok = false;
                raises = (mx >> 20) > E_true;
                mx = __reduce_max_sync(0xFFFFFFFFu, mx);
                if (lane == 0) {
                    mbar_arrive(raw_empty + st);
                    atomicMax(swmax + (it & 3), mx);
                }
                ++nraw;
            }
            // ---- sum the rows of plane q = w-2 and store those whose record
            // is the expected one
            const bool fast_q = E_true >= 64u && E_true < 2047u;
            if (have_q) {
                const int64_t trow0 = int64_t(q) * tp.S + blk0 + int64_t(TY * ctl) * nx + cix;   // tile's first row
                if (fast_q) {
                    const unsigned char* slots[3] = {ring + uint32_t((j - 3) & 3) * SLOTB,   // W(q-1)
                                                     ring + uint32_t((j - 2) & 3) * SLOTB,   // W(q)
                                                     ring + uint32_t((j - 1) & 3) * SLOTB};  // W(q+1)
                    // per row: high limbs in two sums of at most 14 terms
                    // (|xh| < 2^27), low limbs in one of 26 (|xl| < 2^26): no
                    // int32 overflow; the centre apart
                    int32_t A[TY][4], B[TY][4], SL[TY][4], CH[TY][4], CL[TY][4];
#pragma unroll
                    for (int ry = 0; ry < TY; ++ry)
#pragma unroll
                        for (int rx = 0; rx < 4; ++rx) A[ry][rx] = B[ry][rx] = SL[ry][rx] = 0;
#pragma unroll
                    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                        for (int l = 0; l < TY + 2; ++l) {
                            const unsigned char* base = slots[dz] + qoff[l];
                            // element c of the window line: sub-array (1 + c) mod 4, index q + (1 + c) / 4
                            int2 e[6];
#pragma unroll
                            for (int c = 0; c < 6; ++c)
                                e[c] = *reinterpret_cast<const int2*>(base + uint32_t((1 + c) & 3) * SUBB +
                                                                      uint32_t((1 + c) >> 2) * 8u);
#pragma unroll
                            for (int ry = 0; ry < TY; ++ry) {
                                const int dy = l - 1 - ry;   // the line's offset from tile line ry
                                if (dy < -1 || dy > 1) continue;
#pragma unroll
                                for (int rx = 0; rx < 4; ++rx) {
                                    if (dz == 1 && dy == 0) {
                                        CH[ry][rx] = e[rx + 1].y;
                                        CL[ry][rx] = e[rx + 1].x;
                                        B[ry][rx] += e[rx].y + e[rx + 2].y;
                                        SL[ry][rx] += e[rx].x + e[rx + 2].x;
                                    } else if (dz == 0 || (dz == 1 && dy == -1)) {
                                        A[ry][rx] += e[rx].y + e[rx + 1].y + e[rx + 2].y;
                                        SL[ry][rx] += e[rx].x + e[rx + 1].x + e[rx + 2].x;
                                    } else {
                                        B[ry][rx] += e[rx].y + e[rx + 1].y + e[rx + 2].y;
                                        SL[ry][rx] += e[rx].x + e[rx + 1].x + e[rx + 2].x;
                                    }
                                }
                            }
                        }
                    const int S = int(E_ring) - 1075 + a.mult_exp;
                    const uint32_t* flq = sflags + ((it - 1) % 3) * fw;   // the check of plane q, one step ago
#pragma unroll
                    for (int ry = 0; ry < TY; ++ry) {
                        double o[4];
#pragma unroll
                        for (int rx = 0; rx < 4; ++rx) {
                            const int64_t ah = int64_t(a.dom_mo) * A[ry][rx] + int64_t(a.dom_mo) * B[ry][rx] +
                                               int64_t(a.dom_mc) * CH[ry][rx];
                            const int64_t al = int64_t(a.dom_mo) * SL[ry][rx] + int64_t(a.dom_mc) * CL[ry][rx];
                            o[rx] = fixed_to_double(ah * (int64_t(1) << 26) + al, S);
                        }
                        // store the rows whose record was the expected one
                        const int rho = (TY * ctl + ry) * nx + cix;
                        const uint32_t mbits = (flq[rho >> 5] >> (rho & 31)) & 15u;
                        double* yr = y + trow0 + int64_t(ry) * nx;
                        if (mbits == 15u) {
                            reinterpret_cast<double2*>(yr)[0] = make_double2(o[0], o[1]);
                            reinterpret_cast<double2*>(yr)[1] = make_double2(o[2], o[3]);
                            if constexpr (DOT) {
                                dacc = fma(pv[ry][0].x, o[0], dacc);
                                dacc = fma(pv[ry][0].y, o[1], dacc);
                                dacc = fma(pv[ry][1].x, o[2], dacc);
                                dacc = fma(pv[ry][1].y, o[3], dacc);
                            }
                        } else {
#pragma unroll
                            for (int rx = 0; rx < 4; ++rx)
                                if ((mbits >> rx) & 1u) {
                                    yr[rx] = o[rx];
                                    if constexpr (DOT) {
                                        const double2 h = pv[ry][rx >> 1];
                                        dacc = fma((rx & 1) ? h.y : h.x, o[rx], dacc);
                                    }
                                }
                        }
                    }
                } else {
                    // zero/subnormal-only or non-finite x in play: the COLUMN order
                    for (int r = 0; r < K; ++r) {
                        const int64_t row = trow0 + int64_t(r >> 2) * nx + (r & 3);
                        uint32_t w7[kMaxRecordWords];
                        load_record<7>(a, row, w7);
                        const uint32_t pat = byte_of(w7, 27);
                        if (pat >= uint32_t(a.npat)) raise_error(a.err, 1);
                        const uint32_t mask = pat < uint32_t(a.npat) ? __ldg(a.pmask_dev + pat) : 0u;
                        double acc = 0.0;
#pragma unroll
                        for (int uu = 0; uu < 27; ++uu)
                            if ((mask >> uu) & 1u)
                                acc = fma(__ldg(a.dict + (byte_of(w7, uu) & 7)), __ldg(x + row + a.uoff[uu]), acc);
                        y[row] = acc;
                        if constexpr (DOT) dacc = fma(__ldg(x + row), acc, dacc);
                    }
                }
            }
            if (!wait_ok) {
                atomicOr(reinterpret_cast<uint32_t*>(swmax + 8), 1u);
                raise_error(a.err, kErrWaitTimeout);
            }
            // the step's barrier also tells every thread whether anything needs
            // a look after it (a raised scale, rows off their expected record,
            // an abort): in the common case no shared word is read here
            if (!compute_sync_or(NC, raises || exc_now || !wait_ok)) continue;
            if (*sabort) {
                aborted = true;
                break;
            }
            // ---- rows of plane q off their expected record: slot by slot
            if (have_q && fast_q && swexc[(it - 1) & 3] != 0u) {
                const uint32_t* fl = sflags + ((it - 1) % 3) * fw;
                const int S = int(E_ring) - 1075 + a.mult_exp;
                for (int i = tid >> 5; i < fw; i += NC >> 5) {
                    const uint32_t m = fl[i];
                    if (m == 0xFFFFFFFFu || ((m >> lane) & 1u)) continue;
                    const int64_t row = int64_t(q) * tp.S + blk0 + 32 * i + lane;
                    uint32_t w7[kMaxRecordWords];
                    load_record<7>(a, row, w7);
                    const uint32_t pat = byte_of(w7, 27);
                    if (pat >= uint32_t(a.npat)) raise_error(a.err, 1);
                    const uint32_t mask = pat < uint32_t(a.npat) ? __ldg(a.pmask_dev + pat) : 0u;
                    int64_t ah = 0, al = 0;
#pragma unroll
                    for (int uu = 0; uu < 27; ++uu)
                        if ((mask >> uu) & 1u) {
                            const int32_t m8 = mult_of(a.mult_lo, a.mult_hi, byte_of(w7, uu));
                            int32_t xh, xl;
                            to_fixed(__ldg(x + row + a.uoff[uu]), int(E_ring), xh, xl);
                            ah += int64_t(m8) * xh;
                            al += int64_t(m8) * xl;
                        }
                    const double yv = fixed_to_double(ah * (int64_t(1) << 26) + al, S);
                    y[row] = yv;
                    if constexpr (DOT) dacc = fma(__ldg(x + row), yv, dacc);
                }
            }
            // ---- the scale after W(w): a larger exponent re-converts W(w)
            // and shifts the two windows that plane w-1 still reads
            if (w <= z1) {
                const uint32_t Mw = swmax[it & 3] >> 20;
                if (Mw > E_true) {
                    const uint32_t Rn = max(Mw, 64u);
                    if (Mw < 2047u && Rn > E_ring) {
                        if (j >= 2) rescale(ring + uint32_t((j - 2) & 3) * SLOTB, Rn - E_ring);
                        if (j >= 1) rescale(ring + uint32_t((j - 1) & 3) * SLOTB, Rn - E_ring);
                        convert_global(w, ring + uint32_t(j & 3) * SLOTB, Rn);
                        E_ring = Rn;
                        compute_sync(NC);
                    }
                    E_true = Mw;
                }
            }
        }
    }
    if (aborted && tid == 0) {
        // wait (bounded) for the producer lanes to stop, then for the latest
        // copy into every stage, which may still be in flight
        const long long t0 = clock64();
        while (*spdone < 2u && clock64() - t0 < kWaitCycles) {
        }
        const uint32_t iw = siss[0], ir = siss[1];
        for (uint32_t i = iw > kRawStages ? iw - kRawStages : 0; i < iw; ++i)
            mbar_wait(raw_full + i % kRawStages, (i / kRawStages) & 1u);
        for (uint32_t i = ir > kRecStages ? ir - kRecStages : 0; i < ir; ++i)
            mbar_wait(rec_full + i % kRecStages, (i / kRecStages) & 1u);
    }
    if constexpr (DOT) {
        // the CTA's x.y: warp sums, then the warps in order (the expected-record
        // table is no longer read and holds them)
        for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xFFFFFFFFu, dacc, o);
        compute_sync(NC);
        double* const sred = reinterpret_cast<double*>(sexp);
        if (lane == 0) sred[tid >> 5] = dacc;
        compute_sync(NC);
        if (tid == 0) {
            double s = 0.0;
            for (int i = 0; i < (NC >> 5); ++i) s += sred[i];
            dot_part[blockIdx.x] = s;
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// The record each boundary class of grid position implies (64 classes: two
// bits a dimension, bit 0 set when the lower neighbour is inside the grid,
// bit 1 the upper): the dominant record's codes at the in-grid slots, the
// absent code elsewhere, and the pattern number of that slot set; all ones
// (never a record) for a class no row has.
void expected_records(const PatternFormat& p, const PatternView& v, std::vector<uint32_t>* out) {
    std::vector<uint32_t> tab(64 * 8, 0xFFFFFFFFu);
    const uint32_t absent = uint32_t(p.dict.size());
    for (int cls = 0; cls < 64; ++cls) {
        const int c[3] = {cls & 3, (cls >> 2) & 3, (cls >> 4) & 3};   // x, y, z
        uint32_t mask = 0;
        for (int u = 0; u < 27; ++u) {
            const int d[3] = {u % 3 - 1, (u / 3) % 3 - 1, u / 9 - 1};
            bool present = true;
            for (int k = 0; k < 3; ++k)
                if ((d[k] == -1 && !(c[k] & 1)) || (d[k] == 1 && !(c[k] & 2))) present = false;
            if (present) mask |= 1u << u;
        }
        int pn = -1;
        for (size_t i = 0; i < p.pmask.size(); ++i)
            if (p.pmask[i] == mask) pn = int(i);
        if (pn < 0) continue;   // no row of this class exists: the table entry never matches
        uint8_t bytes[32] = {};
        for (int u = 0; u < 27; ++u)
            bytes[u] = (mask >> u) & 1u ? uint8_t((v.dom_w[u >> 2] >> (8 * (u & 3))) & 0xFFu) : uint8_t(absent);
        bytes[27] = uint8_t(pn);
        for (int k = 0; k < 8; ++k)
            tab[cls * 8 + k] = uint32_t(bytes[4 * k]) | uint32_t(bytes[4 * k + 1]) << 8 |
                               uint32_t(bytes[4 * k + 2]) << 16 | uint32_t(bytes[4 * k + 3]) << 24;
    }
    *out = std::move(tab);
}

bool make_tma_plan(const PatternFormat& p, const PatternView& v, int64_t n, int num_sms, int ty, int ctas,
                   TmaPlan* out, std::vector<uint32_t>* expected) {
    if (ty != 1 && ty != 2) return false;
    if (ctas != 1 && ctas != 2) return false;
    const int kSlotElems = slot_elems(ctas), kRecStages = rec_stages(ctas);
    if (!p.fast_ok || v.nu != 27 || v.words != 7 || v.run_len != 3 || !v.dom_ok || !v.dom_uni) return false;
    const std::vector<int32_t>& U = p.uoff;
    if (U.size() != 27) return false;
    const int64_t nx = U[16], S = U[22];
    if (nx < 3 || S <= 2 * nx + 2) return false;
    for (int u = 0; u < 27; ++u) {
        const int64_t dz = u / 9 - 1, dy = (u / 3) % 3 - 1, dx = u % 3 - 1;
        if (U[u] != dz * S + dy * nx + dx) return false;   // the 27-point box of an nx-wide grid
    }
    if (S % nx != 0 || n % S != 0) return false;
    const int64_t ny = S / nx, nz = n / S;
    if (nx % 4 != 0 || nx + 4 > 256 || nz < 1) return false;
    // the most lines a block (whole warps of ty-by-4 tiles) whose window fits
    // a ring slot
    int L = 0;
    for (int64_t l = ty; l <= ny && l * nx <= kMaxBlockRows / ctas; l += ty)
        if (ny % l == 0 && (l * nx) % (128 * ty) == 0 && (l + 2) * (nx + 4) <= kSlotElems) L = int(l);
    if (L == 0) return false;
    TmaPlan t{};
    t.nx = int32_t(nx);
    t.ny = int32_t(ny);
    t.nz = int32_t(nz);
    t.L = L;
    t.C = int32_t(L * nx);
    t.ty = ty;
    t.threads = t.C / (4 * ty);
    t.pitch = t.nx + 4;
    t.win_elems = (L + 2) * t.pitch;
    t.nblk = int32_t(ny / L);
    t.S = S;
    t.grid = std::max(num_sms, 1) * ctas;
    t.ctas = ctas;
    t.z_lo = 0;
    t.z_hi = t.nz;
    auto up = [](int64_t v_, int64_t a_) { return (v_ + a_ - 1) / a_ * a_; };
    t.raw_bytes = int32_t(up(int64_t(t.win_elems) * 8, 128));
    t.off_raw = 4 * kSlotElems * 8;
    t.off_rec = t.off_raw + kRawStages * t.raw_bytes;
    t.off_exp = t.off_rec + kRecStages * 28 * t.C;
    t.off_flags = t.off_exp + 64 * 8 * 4;
    t.off_words = t.off_flags + int32_t(up(3 * (t.C / 32) * 4, 16));
    t.off_mbar = t.off_words + 64;
    t.smem_bytes = int32_t(up(t.off_mbar + 8 * 2 * (kRawStages + kRecStages), 128));
    if (t.smem_bytes > (ctas == 1 ? 227 * 1024 : 227 * 1024 / ctas - 1024)) return false;
    std::vector<uint32_t> tab;
    expected_records(p, v, &tab);
    *out = t;
    *expected = std::move(tab);
    return true;
}

cudaError_t launch_pattern_fast_tma(const PatternView& a, const TmaPlan& tp, const double* x, double* y,
                                    cudaStream_t s, const uint32_t* xmax_part, int xmax_n, double* dot_part,
                                    int* dot_n) {
    if (dot_n) *dot_n = 0;
    if (a.n == 0 || tp.z_hi <= tp.z_lo) return cudaSuccess;
    if (dot_part && (tp.z_lo != 0 || tp.z_hi != tp.nz)) return cudaErrorNotSupported;   // x.y of the whole vector
    if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) != 0) return cudaErrorNotSupported;
    if (tp.z_lo < 0 || tp.z_hi > tp.nz) return cudaErrorInvalidValue;
    const int64_t units = int64_t(tp.nblk) * (tp.z_hi - tp.z_lo);
    const unsigned grid = unsigned(std::min<int64_t>(units, tp.grid));
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc || !tp.expected) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[3] = {cuuint64_t(tp.nx), cuuint64_t(tp.ny), cuuint64_t(tp.nz)};
    const cuuint64_t strides[2] = {cuuint64_t(tp.nx) * 8u, cuuint64_t(tp.S) * 8u};
    const cuuint32_t box[3] = {cuuint32_t(tp.pitch), cuuint32_t(tp.L + 2), 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double*>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    if (tp.ctas != 1 && tp.ctas != 2) return cudaErrorInvalidValue;
    using Kernel = void (*)(CUtensorMap, PatternView, TmaPlan, const double*, double*, const uint32_t*, int, double*);
    static const Kernel kernels[2][2][2] = {   // [ctas - 1][dot][ty - 1]
        {{pattern_fast_tma_kernel<1, false, 1>, pattern_fast_tma_kernel<2, false, 1>},
         {pattern_fast_tma_kernel<1, true, 1>, pattern_fast_tma_kernel<2, true, 1>}},
        {{pattern_fast_tma_kernel<1, false, 2>, pattern_fast_tma_kernel<2, false, 2>},
         {pattern_fast_tma_kernel<1, true, 2>, pattern_fast_tma_kernel<2, true, 2>}}};
    const int ci = tp.ctas - 1, di = dot_part ? 1 : 0, ti = tp.ty == 2 ? 1 : 0;
    const Kernel kernel = kernels[ci][di][ti];
    {
        static std::mutex mu;
        static bool set[64][2][2][2] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> g(mu);
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!set[dev][ci][di][ti]) {
            e = cudaFuncSetAttribute(reinterpret_cast<const void*>(kernel),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     tp.ctas == 1 ? 227 * 1024 : 227 * 1024 / tp.ctas - 1024);
            if (e != cudaSuccess) return e;
            set[dev][ci][di][ti] = true;
        }
    }
    kernel<<<grid, tp.threads + 32, tp.smem_bytes, s>>>(map, a, tp, x, y, xmax_part, xmax_n, dot_part);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && dot_n) *dot_n = int(grid);
    return e;
}

}  // namespace spmvc
