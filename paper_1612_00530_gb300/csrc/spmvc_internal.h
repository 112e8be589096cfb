// Internal declarations shared by the library's translation units: host-side
// formats (generation, compression, decompression), device views of each
// format, and the kernel launchers.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "spmvc.h"

namespace spmvc {

constexpr int kSliceRows = 32;      // rows per slice (one warp)
constexpr int kMaxUnion = 31;       // union of displacements, pattern format
constexpr int kMaxPatterns = 32;    // 5-bit pattern numbers
constexpr int kMaxRecordWords = 8;  // 32-byte row records at most
constexpr int kMaxFastDict = 7;     // codes 0..6 plus the absent-slot code

void set_error(const std::string& msg);
int fail(int status, const std::string& msg);

// ---------------------------------------------------------------- CSR ----
struct Csr {
    int64_t n = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
    std::vector<double> val;
    int64_t nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
};

// Generators (Sec. III-A and its irregular variant).
int generate_hpcg(int nx, int ny, int nz, Csr* out);
int generate_irregular(const spmv_gen_desc& d, Csr* out);
// Structural validation of caller CSR.
int validate_csr(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val);

// ---------------------------------------------------------------- ELL ----
// Slices of 32 rows, slot-major inside a slice: entry t of row 32s+l is at
// slice_off[s] + 32*t + l.  Padding slots hold column -1.
struct EllFormat {
    int64_t nslices = 0;
    std::vector<int64_t> slice_off;  // nslices + 1, in entries
    std::vector<int32_t> slice_w;    // slots per row in the slice
    std::vector<double> val;
    std::vector<int32_t> col;
};
int pack_ell(const Csr& a, EllFormat* out);

// ------------------------------------------------------------ pattern ----
// One record of `words` 32-bit words per row: byte u (u < nu) is the value
// code of union slot u (code = dict index; dict.size() marks an absent
// slot), byte nu is the row's pattern number, the rest is zero.
struct PatternFormat {
    std::vector<double> dict;       // value table, ascending
    std::vector<int32_t> uoff;      // union displacements, ascending
    std::vector<uint32_t> pmask;    // per pattern: bit u set if slot u present
    int words = 0;
    std::vector<uint32_t> rec;      // n * words
    // exact fixed-point order: dict[v] = mult[v] * 2^mult_exp
    bool fast_ok = false;
    int mult_exp = 0;
    std::vector<int32_t> mult;
    int64_t max_row_abs = 0;        // max over rows of sum |mult|
    // values registered in the pattern (Sec. V): the distinct records as row
    // types, built on demand; empty when there are more than 256
    std::vector<uint8_t> rtype;     // n
    std::vector<uint32_t> rtypes;   // ntypes x 8 words
};
// Builds p->rtype / p->rtypes from the records; false (and both left empty)
// when the records take more than 256 distinct values or words != 7.
bool build_row_types(int64_t n, PatternFormat* p);
int compress_pattern(const Csr& a, int max_dict, PatternFormat* out);
void derive_fast_order(int64_t n, PatternFormat* p);

// -------------------------------------------------------------- delta ----
// Per slice, one column encoding (int16 delta col-row by default, 24-bit
// delta, or raw int32 column) and one value encoding (uint8 code into the
// global table by default; codes into the global table and, from its size
// up, into a table of the slice's own values; or raw double).
enum : uint32_t { kSliceValRaw = 1u, kSliceColRaw = 2u, kSliceCol24 = 4u, kSliceValLocal = 8u };
struct DeltaSlice {                 // 16 bytes, one per 32-row slice
    uint64_t off;                   // byte offset of the slice payload
    uint32_t w;                     // slots per row
    uint32_t flags;                 // kSlice* bits
};
// Slice payload, each part 16-byte aligned:
//   row lengths uint8[32];
//   columns [w][32]: int16 delta (col - row), or int32 column (ColRaw), or
//     (Col24) the low 16 bits of a 24-bit delta as int16 followed by an
//     int8 plane [w][32] of its high bits: delta = hi * 65536 + (uint16)lo;
//   values [w][32]: uint8 codes, or doubles (ValRaw); with ValLocal a code
//     c >= |global table| names entry c - |global table| of the slice's own
//     table: a uint32 count (padded to 16 bytes), then that many doubles.
struct DeltaParts {
    uint64_t cols, hi, vals, local;   // byte offsets inside the slice payload
};
__host__ __device__ inline uint64_t delta_up16(uint64_t v) { return (v + 15) & ~uint64_t(15); }
__host__ __device__ inline DeltaParts delta_parts(uint32_t w, uint32_t flags) {
    const uint64_t slots = uint64_t(w) * 32;
    DeltaParts p;
    p.cols = 32;
    uint64_t o = delta_up16(32 + slots * ((flags & kSliceColRaw) ? 4 : 2));
    p.hi = o;
    if (flags & kSliceCol24) o = delta_up16(o + slots);
    p.vals = o;
    p.local = delta_up16(o + slots * ((flags & kSliceValRaw) ? 8 : 1));
    return p;
}
struct DeltaFormat {
    std::vector<double> dict;
    int64_t nslices = 0;
    std::vector<DeltaSlice> hdr;
    std::vector<uint8_t> payload;
};
int compress_delta(const Csr& a, int max_dict, int min_count, DeltaFormat* out);
void delta_dictionary(const std::vector<double>& val, int max_dict, int min_count, std::vector<double>* dict);

// Locality reordering (host_reorder.cpp): reverse Cuthill-McKee over the
// matrix graph, then inside each breadth-first level the rows whose values
// all sit in the value table ahead of the others, so that table-coded slices
// and raw-value slices cluster.  perm[new] = old.
int reorder_rcm(const Csr& a, const std::vector<double>& dict, std::vector<int32_t>* perm);
void permute_csr(const Csr& a, const std::vector<int32_t>& perm, Csr* out);      // P A P^T
void unpermute_csr(const Csr& b, const std::vector<int32_t>& perm, Csr* out);    // P^T B P

// The "Data+Index Table" of Sec. V as Listing 1 reads it: the value table V;
// for every row its type, the number of a registered list of column
// displacements in value-grouped order (groups by ascending value, columns
// ascending inside a group), and the exclusive end of each value group in
// that list.  Types are uint8 (at most 256), ends uint8 (rows of at most 255
// entries) stored value-major so that a warp reads them coalesced.
struct DitFormat {
    std::vector<double> dict;
    int32_t maxlen = 0;
    std::vector<int32_t> disp;      // ntypes x maxlen, unused tail zero
    std::vector<int32_t> tlen;      // entries of each type
    std::vector<uint8_t> type;      // n
    std::vector<uint8_t> ends;      // nv x n
};
int compress_dit(const Csr& a, DitFormat* out);

// The "Data Table" of Sec. V (Fig. 2): the value table V; for every row its
// columns sorted by value, S_i (ties in ascending column order), and the
// exclusive end of each value group in S_i (T_i + 1; T_i is the last
// position of the group).  Rows in 32-row slices, S as int32 slot-major
// [w][32] per slice (w its longest row, padding -1), ends uint8 value-major
// [nv][n]; rows of at most 255 entries, at most 255 values.
struct DataTableFormat {
    std::vector<double> dict;
    int64_t nslices = 0;
    std::vector<int64_t> slice_off;   // nslices + 1, in S entries
    std::vector<uint8_t> slice_w;     // slots a row of the slice
    std::vector<int32_t> S;
    std::vector<uint8_t> ends;        // nv x n
};
int compress_data_table(const Csr& a, DataTableFormat* out);

// --------------------------------------------------------- device views --
struct EllView {
    int64_t n, nslices;
    const int64_t* slice_off;
    const int32_t* slice_w;
    const double* val;
    const float* val32;
    const int32_t* col;
};

struct PatternView {
    int64_t n;
    int32_t nu, words, dict_size, npat;
    int32_t uoff[32];
    uint32_t pmask[32];
    const uint4* p16a;              // words 0..3
    const uint4* p16b;              // words 4..7 (words == 8)
    const uint2* p8;                // words 4..5 (words 6,7)
    const uint32_t* p4;             // last odd word
    const uint32_t* pmask_dev;      // device copy of pmask
    const double* dict;             // device copy of the value table
    const float* dict32;
    uint32_t mult_lo, mult_hi;      // fast order: int8 multipliers, absent -> 0
    int32_t mult_exp;
    int32_t run_len;                // the union is nu/run_len runs of run_len consecutive
                                    // displacements (0 when it is not so split)
    // the most frequent row record, when it has no absent slot: a warp whose
    // rows all carry it takes multipliers / values from these parameters
    int32_t dom_ok;
    uint32_t dom_w[kMaxRecordWords];
    int32_t dom_m[32];              // FAST order: int8 multipliers of its slots
    float dom_v32[32];              // binary32: its slot values
    // FAST order, full 27-slot union: the dominant record's multipliers are
    // dom_mc at the middle slot (displacement 0) and one value dom_mo at all
    // 26 others (a stencil with uniform neighbour weights)
    int32_t dom_uni, dom_mo, dom_mc;
    // values registered in the pattern (Sec. V): a one-byte type per row
    // indexing the table of distinct records (8 words a type, 7 used)
    const uint8_t* rtype;
    const uint32_t* rtypes;
    int32_t ntypes;
    int32_t dom_type;               // the type number of the dominant record (-1: none)
    int32_t* err;                   // sticky device error word
};

struct DitView {
    int64_t n;
    int32_t nv, ntypes, maxlen;
    const uint8_t* type;
    const uint8_t* ends;            // nv x n
    const int32_t* disp;            // ntypes x maxlen
    const double* dict;
    int32_t* err;
};

struct DataTableView {
    int64_t n, nslices;
    int32_t nv;
    const int64_t* slice_off;
    const uint8_t* slice_w;
    const int32_t* S;
    const uint8_t* ends;            // nv x n
    const double* dict;
    int32_t* err;
};

struct DeltaView {
    int64_t n, nslices;
    const DeltaSlice* hdr;
    const uint8_t* payload;
    const double* dict;
    const float* dict32;
    int32_t dict_size;
    int32_t* err;
};

// Shared-memory staging plan of the FAST kernel for tiles of `rows` rows:
// the union displacements are merged into segments whose x windows
// [r0 + seg_min, r0 + rows - 1 + seg_min + seg_span] overlap; segment s
// starts at element seg_base[s] of the tile's staged copy, and slot u of
// row r reads element (r - r0) + soff[u].  Built from the pattern table
// alone (interval merging), no grid geometry involved.
constexpr int kMaxSegments = 8;
struct StagePlan {
    int32_t rows;                   // tile rows (block threads * rows per thread)
    int32_t rows_per_thread;
    int32_t nseg;
    int32_t elems;                  // staged elements per tile
    int32_t seg_min[kMaxSegments];
    int32_t seg_span[kMaxSegments];
    int32_t seg_base[kMaxSegments];
    int32_t soff[32];
    // layout for 16-byte copies of an int2 array (seg_min - seg_pad even)
    int32_t seg_pad[kMaxSegments];
    int32_t seg_pbase[kMaxSegments];
    int32_t soff_padded[32];
    int32_t elems_padded;
    // tiles covered by a launch: tile0, tile0 + 1, ... (ntiles of them; 0 =
    // through the last row).  make_stage_plan: all tiles.
    int64_t tile0;
    int64_t ntiles;
};
// z-marching plan of the full 27-point union: its tile windows are three
// copies of one window shape spaced by the plane stride S (the displacement
// between consecutive segments).  A CTA owns a column block of `rows`
// consecutive rows inside a plane and walks planes z0 .. z0+zc-1: plane z
// needs the windows W(z-1), W(z), W(z+1), so each step loads one new window
// into a ring of three shared-memory slots.
struct ZPlan {
    int32_t rows, rows_per_thread, threads;
    int32_t pairs;                  // 16-byte pairs per window (covers an odd start)
    int32_t slot;                   // int2 entries per ring slot (2 * pairs)
    int32_t nblk, zc, nchunks;      // column blocks per plane, planes per CTA, CTAs per block column
    int32_t chunk0;                 // z-block kernel: first chunk of zc planes this launch computes
    int32_t m1;                     // first displacement of the middle segment
    int32_t rel[27];                // slot u: displacement minus its segment's first one
    int64_t S, nplanes;
};
bool make_zplan(const std::vector<int32_t>& uoff, int64_t n, int rows_per_thread, int threads, int num_sms,
                ZPlan* out);
bool zmarch_supported(const ZPlan& zp);  // shapes with a compiled z-marching kernel
// z-block plan: 512-row column blocks of `planes` (3 or 4) consecutive planes
// a CTA, 256 threads (two rows a thread per plane); false where no compiled
// kernel fits (the z-marching plan's conditions: three equal segments spaced
// by the plane stride, which must be a multiple of 512)
bool make_zblock_plan(const std::vector<int32_t>& uoff, int64_t n, int planes, int threads, ZPlan* out);
bool zblock_supported(const ZPlan& zp);
bool make_stage_plan(const std::vector<int32_t>& uoff, int rows_per_thread, int threads, int max_elems,
                     StagePlan* out);

// TMA z-marching plan (FAST variant 11, k_tma.cu) for a pattern-format
// matrix whose union is the full 27-point box {dz*S + dy*nx + dx} of an
// nx*ny*nz grid (n = nx*ny*nz, S = nx*ny) and whose dominant record has
// uniform neighbour weights.  A column block is L whole grid lines
// (C = L*nx rows of a plane, a tile of ty lines by four columns a compute
// thread, and a producer warp that keeps the copies going); persistent CTAs (one an SM)
// walk equal shares of the (block, plane) sequence, block-major.  The x window of a block in
// plane z is the box [nx+4 elements, L+2 lines] at (ix = -2, iy = b*L - 1,
// z), loaded by TMA with zero fill outside the grid.  Each row's record is
// compared with the record its grid position implies (expected[class],
// class = 2 bits a dimension: bit 0 a lower neighbour exists, bit 1 an
// upper one): a row that matches sums all 27 window slots with the dominant
// weights (out-of-grid slots read zero); any other row is summed slot by
// slot from its own record and global x.
struct TmaPlan {
    int32_t nx, ny, nz;
    int32_t L, C, ty, threads;      // lines a block, rows a block (L*nx), lines a compute thread's tile (1 or 2,
                                    // four columns wide), C/(4*ty) compute threads
    int32_t pitch;                  // nx + 4: elements of a window line
    int32_t win_elems;              // (L + 2) * pitch
    int32_t nblk;                   // column blocks a plane (ny / L)
    int32_t grid;                   // persistent CTAs at most (the SM count times ctas)
    int32_t ctas;                   // CTAs an SM: 1, or 2 (half the rows a block, smaller ring and record stages)
    int32_t z_lo, z_hi;             // planes a launch computes (0 and nz: all)
    int64_t S;                      // plane stride nx*ny
    // dynamic shared memory: ring of 4 converted windows at 0, then
    int32_t off_raw, raw_bytes;     // 2 raw window stages
    int32_t off_rec;                // 3 record stages of 28*C bytes (2 with two CTAs an SM)
    int32_t off_exp;                // 64 expected records x 8 words
    int32_t off_flags;              // 3 x C/32 words of per-row match bits
    int32_t off_words;              // exponent words, mismatch counts, abort and producer words
    int32_t off_mbar;               // full and empty mbarriers of the raw and record stages
    int32_t smem_bytes;
    const uint32_t* expected;       // device copy of the 64 x 8-word table
};
// FAST-order SpMM fed by TMA (k_tma_spmm.cu): blocks of L lines by W
// columns of a plane, kc right-hand sides a pass, a compute thread a tile of
// four rows of a line for one column.
struct TmaSpmmPlan {
    int32_t nx, ny, nz;
    int32_t L, W, C, kc, threads;   // block lines and columns, rows (L*W), columns a pass, C/4*kc threads
    int32_t pitch, win_elems;       // W + 4, (L + 2) * pitch
    int32_t nbx, nby, nblk;         // blocks across a line, down a plane, in a plane
    int32_t ctas;                   // CTAs an SM (1 to 3; a step has at most 1536 / ctas outputs)
    int32_t grid;                   // persistent CTAs at most (the SM count times ctas)
    int64_t S;                      // plane stride nx*ny
    int32_t sub, col_bytes;         // converted window: a column's 4 sub-arrays of `sub` int2 (padded)
    // dynamic shared memory: 2 converted windows (kc columns each) at 0, then
    int32_t off_raw, raw_bytes;     // 2 raw window stages
    int32_t off_rec;                // 3 record stages of 28*C bytes
    int32_t off_exp;                // 64 expected records x 8 words
    int32_t off_flags;              // 3 x C/32 words of per-row match bits
    int32_t off_words;              // per-column exponent words, abort and producer words, given scales
    int32_t off_mbar;
    int32_t smem_bytes;
    const uint32_t* expected;       // device copy of the 64 x 8-word table
};
bool make_tma_spmm_plan(const PatternFormat& p, const PatternView& v, int64_t n, int num_sms, int kc, int ctas,
                        TmaSpmmPlan* out);
// Y = A X with the plan's kernel, ceil(k / kc) passes; cudaErrorNotSupported
// (nothing launched) when X is not 16-byte aligned, ldx is odd (the 4-D
// tensor view needs both) or k < kc.
// xmax_part (optional): xmax_n rows of k words, the partial maxima of the
// high words of |X| by column (b * k + j); they fix each column's scale.
cudaError_t launch_pattern_spmm_tma(const PatternView& a, const TmaSpmmPlan& tp, int k, const double* X, int64_t ldx,
                                    double* Y, int64_t ldy, cudaStream_t s, const uint32_t* xmax_part = nullptr,
                                    int xmax_n = 0);

// Binary32 product fed by TMA (k_tma_f32.cu): blocks of L lines (a multiple
// of four), a compute thread four vertically consecutive rows of a column,
// the rows' one-byte types copied beside the x windows.
struct TmaF32Plan {
    int32_t nx, ny, nz;
    int32_t L, C, threads;          // block lines, rows (L*nx), compute threads (C/4)
    int32_t pitch, win_floats;      // nx + 8, (L + 2) * pitch
    int32_t raw_stride;             // floats between window stages (128-byte multiple)
    int32_t nblk, grid;             // column blocks a plane, persistent CTAs at most
    int64_t S;                      // plane stride nx*ny
    int32_t off_raw, off_types, off_tab, off_tmask, off_dict, off_words, off_mbar, smem_bytes;
    int16_t exp_type[64];           // the row type whose record a row of each boundary class holds (-1: none)
};
bool make_tma_f32_plan(const PatternFormat& p, const PatternView& v, int64_t n, int num_sms, TmaF32Plan* out);
// cudaErrorNotSupported (nothing launched) without row types or when x is
// not 16-byte aligned.
// dot_part / dot_n as for launch_pattern_fast_tma (a thread's four rows of
// a step summed in binary32, those chunks summed in binary64).
cudaError_t launch_pattern_f32_tma(const PatternView& a, const TmaF32Plan& tp, const float* x, float* y,
                                   cudaStream_t s, double* dot_part = nullptr, int* dot_n = nullptr);

// The record each boundary class of grid position implies, 64 classes x 8
// words (the TMA-fed kernels compare every row's record with it).
void expected_records(const PatternFormat& p, const PatternView& v, std::vector<uint32_t>* out);
// Builds the plan and the expected-record table (64 classes x 8 words);
// false when the matrix or its grid has no compiled shape for variant 11.
bool make_tma_plan(const PatternFormat& p, const PatternView& v, int64_t n, int num_sms, int ty, int ctas,
                   TmaPlan* out, std::vector<uint32_t>* expected);
// Launches variant 11; returns cudaErrorNotSupported (nothing launched)
// when x or y is not 16-byte aligned (the TMA box and the vector stores
// need it).  xmax_part (optional): xmax_n words whose maximum is the largest
// high word of |x_j| (sign cleared); the product then scales every run by
// that exponent (the whole vector's) instead of the largest one it has met.
// With dot_part (a whole-grid plan only) the kernel also writes, for each of
// its CTAs, the binary64 sum of x[i]*y[i] over the rows that CTA stored into
// dot_part[cta]; *dot_n receives the number of CTAs (0 when nothing ran).
cudaError_t launch_pattern_fast_tma(const PatternView& a, const TmaPlan& tp, const double* x, double* y,
                                    cudaStream_t s, const uint32_t* xmax_part = nullptr, int xmax_n = 0,
                                    double* dot_part = nullptr, int* dot_n = nullptr);
bool stage_supported(int nu);  // union sizes with a compiled staged kernel
bool rstage_supported(const StagePlan& sp);  // plans the register-staged kernel takes

// Kernel launchers (k_spmv.cu).
cudaError_t launch_ell_f64(const EllView& a, const double* x, double* y, cudaStream_t s);
cudaError_t launch_ell_f32(const EllView& a, const float* x, float* y, cudaStream_t s);
cudaError_t launch_pattern_col_f64(const PatternView& a, const double* x, double* y, cudaStream_t s);
cudaError_t launch_pattern_col_f32(const PatternView& a, const float* x, float* y, cudaStream_t s);
cudaError_t launch_pattern_fast_f64(const PatternView& a, const double* x, double* y,
                                    uint32_t* xmax_word, cudaStream_t s);
cudaError_t launch_pattern_fast_staged(const PatternView& a, const StagePlan& sp, const double* x, double* y,
                                       cudaStream_t s);
// recs: 0 records from global memory (register prefetch), 1 record planes
// staged in shared memory, 2 one-byte row types (a.rtype, a.rtypes)
cudaError_t launch_pattern_fast_rstaged(const PatternView& a, const StagePlan& sp, const double* x, double* y,
                                        int recs, cudaStream_t s);
cudaError_t launch_pattern_fast_zmarch(const PatternView& a, const ZPlan& zp, const double* x, double* y,
                                       uint32_t* partial, cudaStream_t s);
cudaError_t launch_pattern_fast_zblock(const PatternView& a, const ZPlan& zp, const double* x, double* y,
                                       uint32_t* partial, cudaStream_t s);
cudaError_t launch_pattern_fast_xstaged(const PatternView& a, const StagePlan& sp, const double* x, double* y,
                                        uint32_t* partial, int2* X_guarded, int64_t guard, cudaStream_t s);
cudaError_t launch_pattern_fast_async(const PatternView& a, const StagePlan& sp, const double* x, double* y,
                                      int num_sms, cudaStream_t s);
cudaError_t launch_pattern_fast_async_x(const PatternView& a, const StagePlan& sp, const double* x, double* y,
                                        uint32_t* partial, int2* X_guarded, int64_t guard, int num_sms,
                                        cudaStream_t s);
cudaError_t launch_pattern_fast_x(const PatternView& a, const double* x, double* y, uint32_t* partial,
                                  int2* X_guarded, int64_t guard, cudaStream_t s);
cudaError_t launch_delta_f64(const DeltaView& a, const double* x, double* y, cudaStream_t s);
// the same writing y[perm[r]] (a reordered handle's product and scatter in one pass)
cudaError_t launch_delta_f64_scatter(const DeltaView& a, const double* x, double* y, const int32_t* perm,
                                     cudaStream_t s);
cudaError_t launch_dit_f64(const DitView& a, const double* x, double* y, cudaStream_t s);
// binary32 product from the one-byte row types (pattern format, 7-word records)
cudaError_t launch_pattern_types_f32(const PatternView& a, const float* x, float* y, cudaStream_t s);
cudaError_t launch_data_table_f64(const DataTableView& a, const double* x, double* y, cudaStream_t s);
// k_check.cu: *out = max |x_j| as bits (atomicMax; *out zeroed by the
// caller); *bad += count of i with |y_i - yref_i| > abs_tol + rel_tol |yref_i|
// (non-finite entries must match)
cudaError_t launch_absmax(const double* x, int64_t n, unsigned long long* out, cudaStream_t s);
cudaError_t launch_check_close(const double* y, const double* yref, int64_t n, double abs_tol, double rel_tol,
                               unsigned long long* bad, cudaStream_t s);
// k_perm.cu: xp[i] = x[perm[i]] and y[perm[i]] = yp[i]
cudaError_t launch_gather(const int32_t* perm, int64_t n, const double* x, double* xp, cudaStream_t s);
cudaError_t launch_scatter(const int32_t* perm, int64_t n, const double* yp, double* y, cudaStream_t s);
cudaError_t launch_delta_f32(const DeltaView& a, const float* x, float* y, cudaStream_t s);
// SpMM (k right-hand sides, row-major).
cudaError_t launch_pattern_spmm_col(const PatternView& a, int k, const double* X, int64_t ldx,
                                    double* Y, int64_t ldy, cudaStream_t s);
cudaError_t launch_pattern_spmm_fast(const PatternView& a, int k, const double* X, int64_t ldx,
                                     double* Y, int64_t ldy, uint32_t* xmax_words, cudaStream_t s);
cudaError_t launch_pattern_spmm_fast_x(const PatternView& a, int k, const double* X, int64_t ldx, double* Y,
                                       int64_t ldy, uint32_t* partial, int2* Xf_guarded, int64_t guard_rows,
                                       cudaStream_t s);
cudaError_t launch_ell_spmm(const EllView& a, int k, const double* X, int64_t ldx, double* Y,
                            int64_t ldy, cudaStream_t s);
cudaError_t launch_delta_spmm(const DeltaView& a, int k, const double* X, int64_t ldx, double* Y,
                              int64_t ldy, cudaStream_t s);

// Ragged batch (k_batch.cu): one work item = rows [r0, r1) of matrix m.
struct BatchItem {
    int32_t m;
    int32_t pad;
    int64_t r0, r1;
};
cudaError_t launch_pattern_batch(const PatternView* mats_dev, const double* const* xs_dev,
                                 double* const* ys_dev, const BatchItem* items, int64_t nitems,
                                 uint32_t* counter, int words, int grid, cudaStream_t s);
// FAST order: zeroes the counter and the count exponent words, runs the
// exponent pass, then the batch kernel.
cudaError_t launch_pattern_batch_fast(const PatternView* mats_dev, const double* const* xs_dev,
                                      double* const* ys_dev, const BatchItem* items, int64_t nitems,
                                      uint32_t* counter, uint32_t* mat_max, int count, int words, int grid,
                                      cudaStream_t s);

// Utility kernels.
cudaError_t launch_fill_u32(uint32_t* p, uint32_t v, int64_t n, cudaStream_t s);

}  // namespace spmvc

// ------------------------------------------------------------ the handle --
struct spmv_mat_s {
    uint32_t magic = 0;
    int32_t fmt = 0;
    int32_t order = SPMV_ORDER_COLUMN;
    int64_t n = 0, nnz = 0;
    int32_t max_row_nnz = 0;
    int64_t bandwidth = 0;              // max |column - row| of the stored matrix
    spmvc::Csr csr;                     // plain handles keep the CSR
    // locality reordering: the stored matrix is P A P^T with perm[new] = old
    // (empty: not reordered); products gather x and scatter y around it
    std::vector<int32_t> perm;
    int32_t* d_perm = nullptr;
    double* d_xp = nullptr;
    double* d_yp = nullptr;
    spmvc::EllFormat ell;
    spmvc::PatternFormat pat;
    spmvc::DeltaFormat dlt;
    spmvc::DitFormat dit;
    spmvc::DataTableFormat dt;
    uint64_t checksum = 0;

    // device side (allocated on first use)
    int device = -1;
    std::vector<void*> dev_allocs;
    spmvc::EllView ell_view{};
    spmvc::PatternView pat_view{};
    spmvc::DeltaView dlt_view{};
    spmvc::DitView dit_view{};
    spmvc::DataTableView dt_view{};
    int32_t* d_err = nullptr;
    spmvc::StagePlan stage{};          // FAST order: shared-memory staging plan
    bool stage_ok = false;
    spmvc::ZPlan zplan{};              // FAST order, z-marching kernel
    bool zplan_ok = false;
    spmvc::ZPlan zbplan{};             // FAST order, z-block kernel (set on request or by the autotuner)
    bool zbplan_ok = false;
    spmvc::TmaPlan tplan{};            // FAST order, TMA z-marching kernel (variant 11)
    bool tplan_ok = false;
    spmvc::TmaPlan tplan_cg{};         // the CG product (with p.q): tiles of one line, two CTAs an SM
    bool tplan_cg_ok = false;
    // FAST order, TMA SpMM: [4 or 8 columns a pass][1 to 3 CTAs an SM]
    spmvc::TmaSpmmPlan splan[2][3]{};
    bool splan_ok[2][3] = {};
    int32_t spmm_kind = 3;             // 0 per-(row, column) kernel, 1 to 3: TMA kernel, CTAs an SM
    int32_t f32_kind = 2;              // binary32 kernel: 0 records, 1 row types, 2 TMA-fed with row types
    spmvc::TmaF32Plan f32plan{};
    bool f32plan_ok = false;
    bool types_failed = false;         // more than 256 distinct records: no row types
    spmvc::StagePlan async_plan{};     // FAST order, persistent double-buffered kernel (1024-row tiles)
    bool async_ok = false;
    int32_t num_sms = 0;
    int32_t fast_variant = 0;          // 0 direct, 1 staged, 2 pre-converted, 3 staged pre-converted,
                                       // 4 persistent double-buffered, 5 the same from the pre-converted copy
    int2* d_xfixed = nullptr;          // FAST order: fixed-point copy of x with guard zones
    int64_t xfixed_guard = 0;
    int2* d_xfixed_block = nullptr;    // FAST SpMM: fixed-point copy of X (guard rows), k_cap columns
    int32_t xfixed_block_cols = 0;
    uint32_t* d_scratch_words = nullptr; // fast order: per-column max |x| words
    int64_t scratch_words = 0;
    // spmv_apply_host staging
    double* d_hx = nullptr;
    double* d_hy = nullptr;
    cudaStream_t own_stream = nullptr;
    // spmv_apply_host's pipeline: x chunks in on one stream, y chunks out on
    // another, the product's row ranges on own_stream
    cudaStream_t h2d_stream = nullptr;
    cudaStream_t d2h_stream = nullptr;
    std::vector<cudaEvent_t> host_events;
    float* d_ell_val32 = nullptr;
};
