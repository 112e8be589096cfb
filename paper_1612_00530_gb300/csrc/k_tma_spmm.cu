// FAST-order compressed SpMM, Y = A X for k right-hand sides (Eq. 1 of
// arXiv:1612.00530 for every column of a row-major n x k block), for the
// pattern format of a 27-point grid stencil (Sec. V), fed by the Tensor
// Memory Accelerator.  The matrix is read once for KC columns (Sec. I's
// argument for reusing what is loaded: here the row records and the x
// windows).
//
// One persistent CTA an SM walks an equal share of the (block, plane)
// sequence.  A block is L lines by W columns of a plane (C = L*W rows); a
// pass covers KC consecutive columns of X.  A compute thread owns a tile of
// four consecutive rows of a line for one column.  A producer warp keeps the
// copies going: lane 0 loads, for every plane z of the block, the window
// W(z) -- KC columns by W+4 elements by L+2 lines at (c0, x0-2, y0-1, z) of
// the 4-D view (column, ix, iy, iz) of X, one tensor copy that fills
// everything outside the grid with zeros -- and lane 1 the block's row
// records of every plane (three bulk copies a line segment), each into the
// next free stage of its ring (full/empty mbarrier pairs).  The compute
// warps, step by step:
//  - compare each row's record with the record its grid position implies,
//    and hand the record stage back;
//  - convert the newest window once into 53-bit fixed point (two int32
//    limbs) at each column's scale, into per-column sub-arrays of a
//    two-slot ring (element e at sub-array e mod 4, index e / 4), and hand
//    the raw stage back;
//  - form the tile's 3x3 (x-y) box sums of the window converted one step
//    earlier; with the box sums of the two planes before, kept in
//    registers, a row holding its expected record sums to
//    m_o * (box sum over 3x3x3) + (m_c - m_o) * (centre), exact in integers
//    and rounded once; a row off its expected record is summed slot by slot
//    from its own record and X.
// Each column has its own scale: the largest exponent its windows have shown
// since the run of planes began (per column, as spmv_apply's rule asks of
// each column of Y).  A window that raises a column's scale is converted
// again from X for that column, and the box sums still in use are formed
// again from X.  Zero/subnormal-only or non-finite columns take the COLUMN
// order.  Every mbarrier wait is bounded (error word bit 16, then a drain
// of the copies in flight).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "spmvc_internal.h"

namespace spmvc {

namespace {

#include "fast_fixed.cuh"
#include "tma_ptx.cuh"

constexpr int kSpRawStages = 2;
constexpr int kSpRecStages = 3;
constexpr int kSpMaxOutputs = 1536;   // rows x columns of a block step with one CTA an SM, at most

// MINB CTAs an SM: each computes at most kSpMaxOutputs / MINB outputs a step,
// so that the steps (and barriers) of several CTAs overlap on an SM
template <int KC, int MINB>
__global__ void __launch_bounds__(kSpMaxOutputs / (4 * MINB) + 32, MINB)
    pattern_spmm_tma_kernel(const __grid_constant__ CUtensorMap xmap, const PatternView a, const TmaSpmmPlan tp,
                            const double* __restrict__ X, int64_t ldx, double* __restrict__ Y, int64_t ldy,
                            int c_base, int kcols, const uint32_t* __restrict__ xmax_part, int xmax_n,
                            int xmax_ld) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int KP = KC / 2;                          // column pairs a window element
    const int tid = threadIdx.x, lane = tid & 31;
    const int NC = tp.threads, C = tp.C, W = tp.W, nx = tp.nx;
    const int fw = C >> 5;                              // match words a plane
    const uint32_t SUBB = uint32_t(tp.sub) * 8u;        // bytes of a sub-array
    const uint32_t CB = uint32_t(tp.col_bytes);         // bytes of a column's four sub-arrays (padded)
    const uint32_t SLOTB = uint32_t(KC) * CB;
    unsigned char* const ring = smem;
    unsigned char* const raw = smem + tp.off_raw;
    unsigned char* const rec = smem + tp.off_rec;
    uint32_t* const sexp = reinterpret_cast<uint32_t*>(smem + tp.off_exp);
    uint32_t* const sflags = reinterpret_cast<uint32_t*>(smem + tp.off_flags);
    uint32_t* const swmax = reinterpret_cast<uint32_t*>(smem + tp.off_words);   // [4][KC] largest hi word
    volatile uint32_t* const sabort = swmax + 4 * KC;
    volatile uint32_t* const spdone = swmax + 4 * KC + 1;
    volatile uint32_t* const siss = swmax + 4 * KC + 2;                          // [2] issued
    uint64_t* const raw_full = reinterpret_cast<uint64_t*>(smem + tp.off_mbar);
    uint64_t* const raw_empty = raw_full + kSpRawStages;
    uint64_t* const rec_full = raw_empty + kSpRawStages;
    uint64_t* const rec_empty = rec_full + kSpRecStages;
    const int ncheck = C >> 5;                          // warps that check records (rows 0 .. C-1)

    for (int i = tid; i < 64 * 8; i += blockDim.x) sexp[i] = __ldg(tp.expected + i);
    for (int i = tid; i < 5 * KC + 4; i += blockDim.x) swmax[i] = 0u;
    // a caller that knows each column's largest |x| (partial maxima of the
    // high words, xmax_part[b * xmax_ld + column], sign cleared) fixes the
    // columns' scales for every run: no window ever raises them
    uint32_t* const sgiven = swmax + 4 * KC + 4;        // [KC]
    __syncthreads();
    if (xmax_part) {
        uint32_t m = 0u;
        for (int i = tid; i < xmax_n * KC; i += blockDim.x)   // blockDim.x is a multiple of KC
            if (i % KC < kcols) m = max(m, __ldg(xmax_part + int64_t(i / KC) * xmax_ld + c_base + i % KC));
#pragma unroll
        for (int o = KC; o < 32; o <<= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        if (lane < KC) atomicMax(sgiven + lane, m);
    }
    if (tid == 0) {
        for (int i = 0; i < kSpRawStages; ++i) {
            mbar_init(raw_full + i, 1);
            mbar_init(raw_empty + i, NC / 32);
        }
        for (int i = 0; i < kSpRecStages; ++i) {
            mbar_init(rec_full + i, 1);
            mbar_init(rec_empty + i, ncheck);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const int64_t units = int64_t(tp.nblk) * (tp.nz + kRunCost);
    Share share{units * blockIdx.x / gridDim.x, units * (blockIdx.x + 1) / gridDim.x, tp.nz, 0};

    if (tid >= NC) {
        // ---- producer warp
        if (lane > 1) return;
        const uint64_t policy = evict_first_policy();
        uint32_t n = 0;
        int b, z0, z1;
        bool ok = true;
        while (ok && share.next(b, z0, z1)) {
            const int y0 = (b / tp.nbx) * tp.L, x0 = (b % tp.nbx) * W;
            for (int w = z0 - 1; ok && w <= z1; ++w) {
                if (lane == 0) {
                    const uint32_t st = n % kSpRawStages, k = n / kSpRawStages;
                    if (k > 0 && !mbar_wait(raw_empty + st, (k - 1) & 1u)) ok = false;
                    if (ok && *sabort) ok = false;
                    if (!ok) break;
                    fence_proxy_async();
                    mbar_expect_tx(raw_full + st, uint32_t(tp.win_elems) * KC * 8u);
                    tma_load_4d(raw + st * tp.raw_bytes, &xmap, c_base, x0 - 2, y0 - 1, w, raw_full + st);
                    siss[0] = ++n;
                } else if (w >= z0 && w < z1) {
                    const uint32_t st = n % kSpRecStages, k = n / kSpRecStages;
                    if (k > 0 && !mbar_wait(rec_empty + st, (k - 1) & 1u)) ok = false;
                    if (ok && *sabort) ok = false;
                    if (!ok) break;
                    unsigned char* dst = rec + st * 28u * uint32_t(C);
                    fence_proxy_async();
                    mbar_expect_tx(rec_full + st, 28u * uint32_t(C));
                    for (int l = 0; l < tp.L; ++l) {
                        const int64_t r0 = int64_t(w) * tp.S + int64_t(y0 + l) * nx + x0;
                        const uint32_t o = uint32_t(l * W);
                        bulk_g2s(dst + 16u * o, a.p16a + r0, 16u * W, rec_full + st, policy);
                        bulk_g2s(dst + 16u * C + 8u * o, a.p8 + r0, 8u * W, rec_full + st, policy);
                        bulk_g2s(dst + 24u * C + 4u * o, a.p4 + r0, 4u * W, rec_full + st, policy);
                    }
                    siss[1] = ++n;
                }
            }
        }
        if (!ok && !*sabort) {
            atomicOr(reinterpret_cast<uint32_t*>(swmax + 4 * KC), 1u);
            raise_error(a.err, kErrWaitTimeout);
        }
        __threadfence_block();
        atomicAdd(reinterpret_cast<uint32_t*>(swmax + 4 * KC + 1), 1u);
        return;
    }

    // ---- compute threads: tile t (line lt of the block, columns 4*gx ..
    // 4*gx+3) for column c of the pass
    const int c = tid % KC, t = tid / KC;
    const int tpl = W >> 2;                             // tiles a line
    const int lt = t / tpl, gx = t - lt * tpl;
    const int cp = tid % KP;                            // the column pair this thread converts
    const bool col_ok = c < kcols;
    uint32_t qoff[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) qoff[l] = uint32_t(((lt + l) * tp.pitch + 4 * gx) >> 2) * 8u;
    const int pitch = tp.pitch;

    uint32_t nraw = 0, nrec = 0, it = 0;
    bool aborted = false;
    int b, z0, z1;
    while (!aborted && share.next(b, z0, z1)) {
        const int y0 = (b / tp.nbx) * tp.L, x0 = (b % tp.nbx) * W;
        const int64_t xrow0 = int64_t(y0) * nx + x0;    // the block's first row inside a plane
        // the record check: row tid of the block (threads 0 .. C-1)
        int cxy = 0;
        if (tid < C) {
            const int lr = tid / W, xr = tid - lr * W;
            const int ix = x0 + xr, iy = y0 + lr;
            cxy = ((ix > 0 ? 1 : 0) | (ix < nx - 1 ? 2 : 0)) | ((iy > 0 ? 1 : 0) | (iy < tp.ny - 1 ? 2 : 0)) << 2;
        }
        int cz_cached = -1;
        uint32_t ex[7];
        // scales: own column (sums) and the two converted columns
        const uint32_t G = sgiven[c] >> 20, G0 = sgiven[2 * cp] >> 20, G1 = sgiven[2 * cp + 1] >> 20;
        uint32_t Et = G, Er = max(G, 64u), Et0 = G0, Er0 = max(G0, 64u), Et1 = G1, Er1 = max(G1, 64u);
        // box sums: after step w, B2(w-2) in p2*, B2(w-1) in p1*, centres of
        // plane w-1 in c1* (|sum| < 9 * 2^27 fits int32)
        int32_t p2h[4], p2l[4], p1h[4], p1l[4], c1h[4], c1l[4];
#pragma unroll
        for (int rx = 0; rx < 4; ++rx) p2h[rx] = p2l[rx] = p1h[rx] = p1l[rx] = c1h[rx] = c1l[rx] = 0;

        // the tile's 3x3 box sums and centre values of one plane from its
        // six elements in each of three window lines (wrapping adds: a window
        // outside the scale, which only the exact path follows, must not be UB)
        auto box_lines = [&](auto&& line_elems, int32_t (&sh)[4], int32_t (&sl)[4], int32_t (&ch)[4],
                             int32_t (&cl)[4]) {
#pragma unroll
            for (int rx = 0; rx < 4; ++rx) sh[rx] = sl[rx] = 0;
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                int2 e[6];
                line_elems(l, e);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t hh = uint32_t(e[k].y) + uint32_t(e[k + 1].y) + uint32_t(e[k + 2].y);
                    const uint32_t hl = uint32_t(e[k].x) + uint32_t(e[k + 1].x) + uint32_t(e[k + 2].x);
                    sh[k] = int32_t(uint32_t(sh[k]) + hh);
                    sl[k] = int32_t(uint32_t(sl[k]) + hl);
                    if (l == 1) {
                        ch[k] = e[k + 1].y;
                        cl[k] = e[k + 1].x;
                    }
                }
            }
        };
        // X at (plane p, grid line iy, column ix) of this thread's column, 0 outside
        auto xval = [&](int p, int iy, int ix) -> double {
            if (ix < 0 || ix >= nx || iy < 0 || iy >= tp.ny || p < 0 || p >= tp.nz || !col_ok) return 0.0;
            return __ldg(X + ((int64_t(p) * tp.ny + iy) * nx + ix) * ldx + c_base + c);
        };
        auto box_global = [&](int p, uint32_t E, int32_t (&sh)[4], int32_t (&sl)[4], int32_t (&ch)[4],
                              int32_t (&cl)[4]) {
            box_lines([&](int l, int2 (&e)[6]) {
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const double v = xval(p, y0 - 1 + lt + l, x0 - 1 + 4 * gx + k);
                    e[k] = fixed_limbs(uint32_t(__double2loint(v)), uint32_t(__double2hiint(v)), E);
                }
            }, sh, sl, ch, cl);
        };
        // one row of this thread's column from its own record and X: exact
        // fixed-point sum (fast) or the COLUMN order's fma chain
        auto row_from_record = [&](int64_t row, bool fast, uint32_t E) -> double {
            uint32_t w7[kMaxRecordWords];
            load_record<7>(a, row, w7);
            const uint32_t pat = byte_of(w7, 27);
            if (pat >= uint32_t(a.npat)) raise_error(a.err, 1);
            const uint32_t mask = pat < uint32_t(a.npat) ? __ldg(a.pmask_dev + pat) : 0u;
            const double* xc = X + c_base + c;
            if (fast) {
                int64_t ah = 0, al = 0;
#pragma unroll
                for (int uu = 0; uu < 27; ++uu)
                    if ((mask >> uu) & 1u) {
                        const int32_t m8 = mult_of(a.mult_lo, a.mult_hi, byte_of(w7, uu));
                        int32_t xh, xl;
                        to_fixed(__ldg(xc + (row + a.uoff[uu]) * ldx), int(E), xh, xl);
                        ah += int64_t(m8) * xh;
                        al += int64_t(m8) * xl;
                    }
                return fixed_to_double(ah * (int64_t(1) << 26) + al, int(E) - 1075 + a.mult_exp);
            }
            double acc = 0.0;
#pragma unroll
            for (int uu = 0; uu < 27; ++uu)
                if ((mask >> uu) & 1u)
                    acc = fma(__ldg(a.dict + (byte_of(w7, uu) & 7)), __ldg(xc + (row + a.uoff[uu]) * ldx), acc);
            return acc;
        };

        for (int w = z0 - 1; w <= z1 + 1; ++w, ++it) {
            const int j = w - z0 + 1;
            bool wait_ok = true, raises = false;
            if (tid < KC) swmax[((it + 2) & 3) * KC + tid] = 0u;   // the words of step it - 2
            // ---- records of plane w-1 against their grid position
            if (w - 1 >= z0 && w - 1 < z1 && tid < C) {
                const int p = w - 1;
                const uint32_t st = nrec % kSpRecStages;
                if (!mbar_wait(rec_full + st, (nrec / kSpRecStages) & 1u)) wait_ok = false;
                const int cz = (p > 0 ? 1 : 0) | (p < tp.nz - 1 ? 2 : 0);
                if (cz != cz_cached) {
#pragma unroll
                    for (int i = 0; i < 7; ++i) ex[i] = sexp[(cxy | (cz << 4)) * 8 + i];
                    cz_cached = cz;
                }
                const unsigned char* rs = rec + st * 28u * uint32_t(C);
                const uint4 v16 = *reinterpret_cast<const uint4*>(rs + 16 * tid);
                const uint2 v8 = *reinterpret_cast<const uint2*>(rs + 16 * C + 8 * tid);
                const uint32_t v4 = *reinterpret_cast<const uint32_t*>(rs + 24 * C + 4 * tid);
                const uint32_t diff = (v16.x ^ ex[0]) | (v16.y ^ ex[1]) | (v16.z ^ ex[2]) | (v16.w ^ ex[3]) |
                                      (v8.x ^ ex[4]) | (v8.y ^ ex[5]) | (v4 ^ ex[6]);
                const uint32_t match = __ballot_sync(0xFFFFFFFFu, diff == 0u);
                __syncwarp();
                if (lane == 0) {
                    sflags[(it % 3) * fw + (tid >> 5)] = match;
                    mbar_arrive(rec_empty + st);
                }
                ++nrec;
            } else if (w - 1 >= z0 && w - 1 < z1) {
                ++nrec;
            }
            // ---- convert W(w) into ring slot j & 1 at each column's scale
            if (w <= z1) {
                const uint32_t st = nraw % kSpRawStages;
                uint32_t m0 = 0, m1 = 0;
                if (mbar_wait(raw_full + st, (nraw / kSpRawStages) & 1u)) {
                    const unsigned char* rw = raw + st * tp.raw_bytes;
                    unsigned char* slot = ring + uint32_t(j & 1) * SLOTB;
                    const int npairs = tp.win_elems * KP;
                    for (int pi = tid; pi < npairs; pi += NC) {
                        const int e = pi / KP;   // pi % KP == cp
                        const uint4 v = *reinterpret_cast<const uint4*>(rw + 16 * pi);
                        m0 = max(m0, v.y & 0x7FFFFFFFu);
                        m1 = max(m1, v.w & 0x7FFFFFFFu);
                        const uint32_t off = uint32_t(e & 3) * SUBB + uint32_t(e >> 2) * 8u;
                        *reinterpret_cast<int2*>(slot + uint32_t(2 * cp) * CB + off) = fixed_limbs(v.x, v.y, Er0);
                        *reinterpret_cast<int2*>(slot + uint32_t(2 * cp + 1) * CB + off) = fixed_limbs(v.z, v.w, Er1);
                    }
                } else {
                    wait_ok = false;
                }
                raises = (m0 >> 20) > Et0 || (m1 >> 20) > Et1;
                // the maxima of each column over the warp's lanes that hold it
#pragma unroll
                for (int o = KP; o < 32; o <<= 1) {
                    m0 = max(m0, __shfl_xor_sync(0xFFFFFFFFu, m0, o));
                    m1 = max(m1, __shfl_xor_sync(0xFFFFFFFFu, m1, o));
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(raw_empty + st);
                if (lane < KP) {
                    atomicMax(swmax + (it & 3) * KC + 2 * lane, m0);
                    atomicMax(swmax + (it & 3) * KC + 2 * lane + 1, m1);
                }
                ++nraw;
            }
            // ---- box sums of W(w-1), then plane q = w-2
            int32_t nh[4], nl[4], mh[4], ml[4];
            if (w >= z0) {
                const unsigned char* sw = ring + uint32_t((j - 1) & 1) * SLOTB + uint32_t(c) * CB;
                box_lines([&](int l, int2 (&e)[6]) {
                    const unsigned char* base = sw + qoff[l];
#pragma unroll
                    for (int k = 0; k < 6; ++k)
                        e[k] = *reinterpret_cast<const int2*>(base + uint32_t((1 + k) & 3) * SUBB +
                                                              uint32_t((1 + k) >> 2) * 8u);
                }, nh, nl, mh, ml);
            }
            const int q = w - 2;
            if (q >= z0 && q < z1 && col_ok) {
                const bool fast = Et >= 64u && Et < 2047u;
                const int64_t row0 = int64_t(q) * tp.S + xrow0 + int64_t(lt) * nx + 4 * gx;
                const uint32_t* flq = sflags + ((it - 1) % 3) * fw;
                const int rho = lt * W + 4 * gx;
                const uint32_t mbits = (flq[rho >> 5] >> (rho & 31)) & 15u;
                const int S = int(Er) - 1075 + a.mult_exp;
                double* yr = Y + row0 * ldy + c_base + c;
#pragma unroll
                for (int rx = 0; rx < 4; ++rx) {
                    double o;
                    if (fast && ((mbits >> rx) & 1u)) {
                        // high limbs widened plane by plane (two of them could
                        // leave int32); low limbs: 27 * 2^26 fits int32
                        const int32_t mo = a.dom_mo, mcmo = a.dom_mc - a.dom_mo;
                        const int64_t ah = int64_t(mo) * p2h[rx] + int64_t(mo) * p1h[rx] + int64_t(mo) * nh[rx] +
                                           int64_t(mcmo) * c1h[rx];
                        const int32_t boxl = p2l[rx] + p1l[rx] + nl[rx];
                        const int64_t al = int64_t(mo) * boxl + int64_t(mcmo) * c1l[rx];
                        o = fixed_to_double(ah * (int64_t(1) << 26) + al, S);
                    } else {
                        o = row_from_record(row0 + rx, fast, Er);
                    }
                    yr[int64_t(rx) * ldy] = o;
                }
            }
            if (w >= z0) {
#pragma unroll
                for (int rx = 0; rx < 4; ++rx) {
                    p2h[rx] = p1h[rx];
                    p2l[rx] = p1l[rx];
                    p1h[rx] = nh[rx];
                    p1l[rx] = nl[rx];
                    c1h[rx] = mh[rx];
                    c1l[rx] = ml[rx];
                }
            }
            if (!wait_ok) {
                atomicOr(reinterpret_cast<uint32_t*>(swmax + 4 * KC), 1u);
                raise_error(a.err, kErrWaitTimeout);
            }
            if (!compute_sync_or(NC, raises || !wait_ok)) continue;
            if (*sabort) {
                aborted = true;
                break;
            }
            // ---- a column whose window W(w) raised its scale: every thread
            // moves its copies of that column's scale the same way; the
            // threads of the column form their box sums again and convert
            // their share of W(w) again, from X
            if (w <= z1) {
                const uint32_t* mw = swmax + (it & 3) * KC;
                auto step_scale = [&](uint32_t M, uint32_t& Etx, uint32_t& Erx) -> bool {
                    bool re = false;
                    if (M > Etx) {
                        const uint32_t Rn = max(M, 64u);
                        if (M < 2047u && Rn > Erx) {
                            Erx = Rn;
                            re = true;
                        }
                        Etx = M;
                    }
                    return re;
                };
                step_scale(mw[2 * cp] >> 20, Et0, Er0);
                step_scale(mw[2 * cp + 1] >> 20, Et1, Er1);
                if (step_scale(mw[c] >> 20, Et, Er)) {
                    int32_t th[4], tl[4];
                    box_global(w - 2, Er, p2h, p2l, th, tl);
                    box_global(w - 1, Er, p1h, p1l, c1h, c1l);
                    unsigned char* slot = ring + uint32_t(j & 1) * SLOTB + uint32_t(c) * CB;
                    for (int e = t; e < tp.win_elems; e += NC / KC) {
                        const int l = e / pitch, xw = e - l * pitch;
                        const double v = xval(w, y0 - 1 + l, x0 - 2 + xw);
                        *reinterpret_cast<int2*>(slot + uint32_t(e & 3) * SUBB + uint32_t(e >> 2) * 8u) =
                            fixed_limbs(uint32_t(__double2loint(v)), uint32_t(__double2hiint(v)), Er);
                    }
                }
                compute_sync(NC);
            }
        }
    }
    if (aborted && tid == 0) {
        const long long t0 = clock64();
        while (*spdone < 2u && clock64() - t0 < kWaitCycles) {
        }
        const uint32_t iw = siss[0], ir = siss[1];
        for (uint32_t i = iw > kSpRawStages ? iw - kSpRawStages : 0; i < iw; ++i)
            mbar_wait(raw_full + i % kSpRawStages, (i / kSpRawStages) & 1u);
        for (uint32_t i = ir > kSpRecStages ? ir - kSpRecStages : 0; i < ir; ++i)
            mbar_wait(rec_full + i % kSpRecStages, (i / kSpRecStages) & 1u);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn_spmm() {
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

bool make_tma_spmm_plan(const PatternFormat& p, const PatternView& v, int64_t n, int num_sms, int kc, int ctas,
                        TmaSpmmPlan* out) {
    if (kc != 4 && kc != 8) return false;
    if (ctas < 1 || ctas > 3) return false;
    const int64_t max_out = kSpMaxOutputs / ctas;
    if (!p.fast_ok || v.nu != 27 || v.words != 7 || v.run_len != 3 || !v.dom_ok || !v.dom_uni) return false;
    const std::vector<int32_t>& U = p.uoff;
    if (U.size() != 27) return false;
    const int64_t nx = U[16], S = U[22];
    if (nx < 3 || S <= 2 * nx + 2) return false;
    for (int u = 0; u < 27; ++u) {
        const int64_t dz = u / 9 - 1, dy = (u / 3) % 3 - 1, dx = u % 3 - 1;
        if (U[u] != dz * S + dy * nx + dx) return false;
    }
    if (S % nx != 0 || n % S != 0) return false;
    const int64_t ny = S / nx, nz = n / S;
    if (nx % 4 != 0 || nz < 1) return false;
    // the block (L lines by W columns) with the least window overhead
    // (L+2)(W+4)/(L W) among those whose rows fill whole warps, whose step
    // has at most max_out outputs and whose window a TMA box can hold
    auto up = [](int64_t v_, int64_t a_) { return (v_ + a_ - 1) / a_ * a_; };
    int bestL = 0, bestW = 0;
    double best = 1e30;
    for (int64_t W = 4; W <= nx && W + 4 <= 256; W += 4) {
        if (nx % W) continue;
        for (int64_t L = 1; L <= ny && L + 2 <= 256; ++L) {
            if (ny % L) continue;
            const int64_t C = L * W;
            if (C % 32 || C * kc > max_out) continue;
            const double ov = double((L + 2) * (W + 4)) / double(C);
            if (ov < best - 1e-9 || (ov < best + 1e-9 && C > int64_t(bestL) * bestW)) {
                best = ov;
                bestL = int(L);
                bestW = int(W);
            }
        }
    }
    if (bestL == 0) return false;
    TmaSpmmPlan t{};
    t.nx = int32_t(nx);
    t.ny = int32_t(ny);
    t.nz = int32_t(nz);
    t.L = bestL;
    t.W = bestW;
    t.C = bestL * bestW;
    t.kc = kc;
    t.threads = t.C / 4 * kc;
    t.pitch = bestW + 4;
    t.win_elems = (bestL + 2) * t.pitch;
    t.nbx = int32_t(nx / bestW);
    t.nby = int32_t(ny / bestL);
    t.nblk = t.nbx * t.nby;
    t.S = S;
    t.ctas = ctas;
    t.grid = std::max(num_sms, 1) * ctas;
    t.sub = (t.win_elems + 3) / 4;
    // a column's four sub-arrays, padded so that successive columns start
    // 8*(32/kc) bytes apart modulo 128: the 32/kc tiles of one column a warp
    // reads then fill distinct banks beside the other columns' tiles
    const int64_t tiles_a_warp = 32 / kc;
    int64_t cb = up(int64_t(t.sub) * 4 * 8, 8);
    while (cb % 128 != (8 * tiles_a_warp) % 128) cb += 8;
    t.col_bytes = int32_t(cb);
    const int64_t slot = cb * kc;
    t.raw_bytes = int32_t(up(int64_t(t.win_elems) * kc * 8, 128));
    t.off_raw = int32_t(up(2 * slot, 128));
    t.off_rec = t.off_raw + kSpRawStages * t.raw_bytes;
    t.off_exp = t.off_rec + kSpRecStages * 28 * t.C;
    t.off_flags = t.off_exp + 64 * 8 * 4;
    t.off_words = t.off_flags + int32_t(up(3 * (t.C / 32) * 4, 16));
    t.off_mbar = t.off_words + int32_t(up((5 * kc + 4) * 4, 16));
    t.smem_bytes = int32_t(up(t.off_mbar + 8 * 2 * (kSpRawStages + kSpRecStages), 128));
    if (t.smem_bytes > 227 * 1024 / ctas - 1024) return false;
    *out = t;
    return true;
}

cudaError_t launch_pattern_spmm_tma(const PatternView& a, const TmaSpmmPlan& tp, int k, const double* X, int64_t ldx,
                                    double* Y, int64_t ldy, cudaStream_t s, const uint32_t* xmax_part, int xmax_n) {
    if (a.n == 0) return cudaSuccess;
    // the 4-D view needs 16-byte aligned rows of X; Y is written by element
    if ((reinterpret_cast<uintptr_t>(X) & 15u) != 0 || (ldx & 1) != 0 || k < tp.kc || k > ldx || k > ldy)
        return cudaErrorNotSupported;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn_spmm();
    if (!enc || !tp.expected) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[4] = {cuuint64_t(k), cuuint64_t(tp.nx), cuuint64_t(tp.ny), cuuint64_t(tp.nz)};
    const cuuint64_t strides[3] = {cuuint64_t(ldx) * 8u, cuuint64_t(ldx) * 8u * cuuint64_t(tp.nx),
                                   cuuint64_t(ldx) * 8u * cuuint64_t(tp.S)};
    const cuuint32_t box[4] = {cuuint32_t(tp.kc), cuuint32_t(tp.pitch), cuuint32_t(tp.L + 2), 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<double*>(X), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    using Kernel = void (*)(CUtensorMap, PatternView, TmaSpmmPlan, const double*, int64_t, double*, int64_t, int, int,
                            const uint32_t*, int, int);
    static const Kernel kernels[2][3] = {
        {pattern_spmm_tma_kernel<4, 1>, pattern_spmm_tma_kernel<4, 2>, pattern_spmm_tma_kernel<4, 3>},
        {pattern_spmm_tma_kernel<8, 1>, pattern_spmm_tma_kernel<8, 2>, pattern_spmm_tma_kernel<8, 3>}};
    if (tp.ctas < 1 || tp.ctas > 3 || tp.threads > kSpMaxOutputs / (4 * tp.ctas)) return cudaErrorInvalidValue;
    const int ki = tp.kc == 8 ? 1 : 0;
    const Kernel kernel = kernels[ki][tp.ctas - 1];
    {
        static std::mutex mu;
        static bool set[64][2][3] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> g(mu);
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!set[dev][ki][tp.ctas - 1]) {
            e = cudaFuncSetAttribute(reinterpret_cast<const void*>(kernel),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 / tp.ctas - 1024);
            if (e != cudaSuccess) return e;
            set[dev][ki][tp.ctas - 1] = true;
        }
    }
    const int64_t units = int64_t(tp.nblk) * tp.nz;
    const unsigned grid = unsigned(std::min<int64_t>(units, tp.grid));
    // one pass a group of kc columns; the last may be partial (its columns
    // past k read zeros from the box and store nothing)
    for (int c0 = 0; c0 < k; c0 += tp.kc) {
        kernel<<<grid, tp.threads + 32, tp.smem_bytes, s>>>(map, a, tp, X, ldx, Y, ldy, c0, std::min(tp.kc, k - c0),
                                                            xmax_part, xmax_part ? xmax_n : 0, k);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace spmvc
