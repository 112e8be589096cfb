/*
 * spmvc.h -- C ABI of a compressed-matrix SpMV library for one NVIDIA GB300
 * (sm_103a), after Yoshifuji, Sakamoto, Nitadori and Makino, "Implementation
 * and evaluation of data-compression algorithms for irregular-grid iterative
 * methods on the PEZY-SC processor" (arXiv:1612.00530).
 *
 * The library computes y = A x (Eq. 1) with A held in device memory either
 * as plain sliced ELL (the "Original" row of Table II) or in a compressed
 * form decoded on the fly (Sec. V): matrix values become small indices into
 * a per-matrix value table V (sorted ascending, Fig. 2), and column indices
 * become stencil-pattern numbers (displacements relative to the diagonal,
 * registered in a pattern table, Sec. V) or narrow deltas, with a raw
 * per-slice fallback.  Compression and decompression are the "data
 * compression/decompression subroutines" the abstract adds to an otherwise
 * unchanged program; the Krylov solver built on top is the CG iteration of
 * Table I without the preconditioner.
 *
 * Conventions for every function below:
 *  - Every function returns an int status (SPMV_OK or an SPMV_E* code) and
 *    never throws; spmv_strerror() names a code and spmv_last_error() gives
 *    the calling thread's last detailed message.
 *  - Invalid arguments are reported as SPMV_EINVAL before any device work.
 *  - "device pointer" means memory on the current CUDA device, owned by the
 *    caller; "host pointer" means ordinary (pageable or pinned) host memory,
 *    owned by the caller.  The library never frees caller memory.
 *  - A spmv_mat_t owns all memory it allocates (host and device) until
 *    spmv_free().  Device copies are made on the first call that needs them,
 *    on the device current at that call; later calls must use that device.
 *  - spmv_stream_t is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Functions taking a stream enqueue their work on it and
 *    return without waiting, unless documented otherwise.
 *  - Input and output vectors must not overlap.
 *  - Kernel-side checks (bounds of decoded indices) never trap: they set a
 *    sticky per-matrix error word that spmv_device_error() reads.
 */
#ifndef SPMVC_H
#define SPMVC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SPMV_OK 0
#define SPMV_EINVAL 1          /* bad argument (null pointer, size, handle) */
#define SPMV_ENOMEM 2          /* host or device allocation failed */
#define SPMV_ECUDA 3           /* a CUDA runtime call failed */
#define SPMV_ECORRUPT 4        /* compressed stream fails its checksum/bounds check */
#define SPMV_EUNSUPPORTED 5    /* matrix does not fit the requested format */
#define SPMV_ENOTCONVERGED 6   /* cg_solve hit max_iter before the tolerance */
#define SPMV_ETIMEOUT 7        /* reserved, never returned as a status: a
                                  TMA-fed kernel whose bounded wait for its
                                  copies gives up (about a second) sets 16 in
                                  the matrix's device error word instead */
#define SPMV_EDEVICE 8         /* a kernel reported a decoding error */

typedef struct spmv_mat_s *spmv_mat_t;
typedef void *spmv_stream_t;

/* ---- formats and summation orders ------------------------------------ */
#define SPMV_FMT_AUTO 0        /* compress: pattern format if it fits, else delta */
#define SPMV_FMT_ELL 1         /* plain sliced ELL, FP64 value + int32 column */
#define SPMV_FMT_PATTERN 2     /* uint8 value codes + stencil-pattern number per row */
#define SPMV_FMT_DELTA 3       /* per 32-row slice: int16 delta, 24-bit delta
                                  (int16 + int8 planes) or int32 column; uint8
                                  code, uint8 code with per-entry escapes to
                                  FP64 (a 32-bit mask a slot locates them), or
                                  FP64 value -- the narrowest that holds the
                                  slice */
#define SPMV_FMT_DIT 4         /* Sec. V "Data+Index Table": per row a type (a
                                  registered value-grouped displacement list)
                                  and its value-group ends; Listing 1 decode */
#define SPMV_FMT_DATA_TABLE 5  /* Sec. V "Data Table" (Fig. 2): per row its
                                  columns sorted by value, S_i (int32, columns
                                  ascending inside a value; 32-row slices,
                                  slot-major), and the exclusive end of each
                                  value group, T_i + 1 (uint8, value-major);
                                  4 B a nonzero + 1 B a value a row, where the
                                  paper counts (27 + 2) * 4 = 116 B a row.
                                  Decoded like Listing 1: value groups
                                  ascending, one fma per entry.  At most 255
                                  distinct values and 255 entries a row. */

#define SPMV_ORDER_COLUMN 0    /* y_i = fma chain over ascending columns from 0:
                                  bit-identical to the plain CSR product (the
                                  Data+Index Table and Data Table formats:
                                  Listing 1's chain, value groups ascending,
                                  columns ascending inside a group) */
#define SPMV_ORDER_FAST 1      /* pattern format only: exact fixed-point sums,
                                  one rounding per row (error bound below) */

/* ---- matrix construction (host side; nothing is sent to the GPU yet) -- */
#define SPMV_GEN_HPCG 0
#define SPMV_GEN_IRREGULAR 1

typedef struct {
    int32_t kind;          /* SPMV_GEN_HPCG or SPMV_GEN_IRREGULAR */
    int32_t nx, ny, nz;    /* grid edges, each >= 1; nx*ny*nz < 2^31 */
    uint64_t seed;         /* irregular only */
    double drop_prob;      /* irregular: probability a stencil link is removed (0.10) */
    double special_frac;   /* irregular: fraction of rows with unique values (0.05) */
    int32_t diag_rule;     /* irregular: 0 = diagonal 26 on ordinary rows,
                              1 = max(26, 1.05 * off-diagonal row sum) */
    int32_t permute;       /* irregular: 1 = random symmetric renumbering */
} spmv_gen_desc;

/* Builds a plain matrix from a generator.
 * HPCG (Sec. III-A): the 27-point stencil on an nx*ny*nz grid, node
 * i = ix + nx*(iy + ny*iz), diagonal 26 and -1 for every neighbour inside
 * the grid (Fig. 2 values).
 * IRREGULAR (the paper motivates irregular grids without fixing one; this
 * is the library's construction).  Random numbers come from SplitMix64: the
 * stream for a purpose starts from the first output of a SplitMix64 seeded
 * with seed XOR the purpose name's ASCII bytes read little-endian; a draw is
 * u = (next >> 11) * 2^-53, and an index below m is min(floor(u m), m - 1).
 * Steps:
 *  1. "special": floor(special_frac * n) special nodes, the first picks of
 *     a partial Fisher-Yates shuffle of 0..n-1 (slot t, from 0 up, swaps
 *     with slot t + (an index below n - t));
 *  2. links: every stencil pair i < j, i ascending, then j ascending; one
 *     "drop" draw a link removes it (both a_ij and a_ji) when
 *     u < drop_prob; a kept link then takes one "val" draw: -2 + 1.9 u (in
 *     [-2, -0.1)) when either end is special, else the level -1.5 + k/15
 *     with k an index below 16; a_ji = a_ij;
 *  3. diagonal: 1.05 * s on special rows, s = sum_j |a_ij| added left to
 *     right in ascending column order; on the others 26 (diag_rule 0) or
 *     max(26, 1.05 * s) (diag_rule 1);
 *  4. "perm" (permute = 1): a full Fisher-Yates shuffle p of 0..n-1 (slot t,
 *     from n-1 down to 1, swaps with an index below t + 1), old node k
 *     becoming node p[k]; the stored matrix is P A P^T, columns ascending.
 * *out receives a new handle of format SPMV_FMT_ELL. */
int spmv_build(const spmv_gen_desc *desc, spmv_mat_t *out);

/* Builds a plain matrix from host CSR arrays (copied; the caller keeps
 * ownership).  rowptr: n+1 entries, rowptr[0] = 0, nondecreasing; col:
 * rowptr[n] column indices in [0, n), strictly ascending inside each row;
 * val: rowptr[n] FP64 values.  Errors: SPMV_EINVAL for any violation. */
int spmv_build_csr(int64_t n, const int64_t *rowptr, const int32_t *col,
                   const double *val, spmv_mat_t *out);

/* ---- compression (Sec. V) -------------------------------------------- */
typedef struct {
    int32_t format;        /* SPMV_FMT_AUTO, SPMV_FMT_PATTERN, SPMV_FMT_DELTA or
                              SPMV_FMT_DIT or SPMV_FMT_DATA_TABLE (neither
                              chosen by AUTO; no stream form, no binary32
                              product, no SpMM, COLUMN order only) */
    int32_t order;         /* SPMV_ORDER_COLUMN or SPMV_ORDER_FAST */
    int32_t max_dict;      /* largest value table, 1..254 (default 254 when 0) */
    int32_t min_count;     /* delta format: a value enters the table only if it
                              occurs at least this often (default 64 when 0) */
    int32_t reorder;       /* 0: keep the numbering; 1: locality reordering
                              (reverse Cuthill-McKee, table-coded rows ahead of
                              the others inside each level), stored as
                              B = P A P^T, products gather x and scatter y */
} spmv_opts;

/* Compresses plain matrix A into a new handle *out (A is unchanged and stays
 * valid).  The value table V lists the matrix values in ascending order
 * (Sec. V, Fig. 2).  Pattern format: each row's column displacements from
 * the diagonal form a pattern registered in a table of at most 32 entries
 * (Sec. V), the union of all displacements has at most 31 entries, and
 * every value is in V; each row is stored as one uint8 code per union slot
 * plus its 5-bit pattern number.  Delta format: rows in slices of 32, each
 * slice storing int16 column deltas (or raw int32 columns) and uint8 codes
 * (or raw FP64 values).  Data+Index Table (Sec. V, Fig. 2, Listing 1): each
 * row's entries sorted by value (columns ascending inside a value), made
 * relative to the row and registered as one of at most 256 types; the row
 * keeps a uint8 type and one uint8 group end per value (at most 255 values
 * and 255 entries a row).  It serves spmv_apply, spmv_apply_host,
 * spmv_decompress and FP64 cg_solve; other calls return SPMV_EUNSUPPORTED.
 * opts may be NULL (AUTO, COLUMN).  Errors: SPMV_EUNSUPPORTED when the
 * requested format cannot hold A. */
int spmv_compress(spmv_mat_t A, const spmv_opts *opts, spmv_mat_t *out);

/* The permutation of a handle compressed with reorder = 1: perm[new] = old
 * for n entries (caller-owned host buffer).  The handle stores B = P A P^T;
 * spmv_apply, spmv_apply_host, spmv_decompress and FP64 cg_solve still take
 * and return A's numbering (a gather of x and a scatter of y around the
 * product, two extra passes of 20 bytes a row); its products sum each row in
 * B's column order.  SPMV_EINVAL when A is not reordered.  Reordered handles
 * serve no binary32, SpMM, batch or stream call (SPMV_EUNSUPPORTED). */
int spmv_permutation(spmv_mat_t A, int32_t *perm);

/* Selects the summation order used by later spmv_apply/spmm_apply calls on a
 * pattern-format handle.  SPMV_ORDER_FAST needs every value to be a small
 * integer multiple (|m| <= 127) of one power of two and at most 7 values;
 * otherwise SPMV_EUNSUPPORTED.  Other formats accept SPMV_ORDER_COLUMN only. */
int spmv_set_order(spmv_mat_t A, int32_t order);

typedef struct {
    int64_t n;                  /* rows (= columns) */
    int64_t nnz;                /* stored nonzeros */
    int32_t format;             /* SPMV_FMT_* */
    int32_t order;              /* SPMV_ORDER_* */
    int32_t dict_size;          /* |V| (0 for ELL) */
    int32_t n_patterns;         /* pattern format: registered patterns */
    int32_t union_size;         /* pattern format: union of displacements */
    int32_t record_bytes;       /* pattern format: bytes per row record */
    int32_t max_row_nnz;
    int32_t fast_eligible;      /* 1 if SPMV_ORDER_FAST is available */
    int64_t n_slices;           /* ELL / delta: 32-row slices */
    int64_t slices_value_raw;   /* delta: slices storing raw FP64 values */
    int64_t slices_col_raw;     /* delta: slices storing raw int32 columns */
    int64_t device_bytes;       /* matrix bytes held in device memory */
    int64_t format_bytes;       /* matrix bytes one product reads (incl. padding) */
    int64_t padding_bytes;      /* of format_bytes: padding slots and records */
    uint64_t checksum;          /* FNV-1a of the compressed stream */
    int32_t fast_tile_rows;     /* FAST order: rows per shared-memory tile of the
                                   staged kernel (z-block kernel: rows a CTA
                                   computes, 512 per plane; 0 = no staged
                                   kernel for A) */
    int32_t fast_variant;       /* FAST kernel in use: 0 direct, 1 staged tiles,
                                   2 pre-converted fixed-point copy of x, 3 staged
                                   tiles of that copy, 4 persistent double-buffered
                                   tiles, 5 the same from the copy, 6 register-
                                   staged tiles, 7 z-marching tiles, 8 register-
                                   staged with records in shared memory, 9 the
                                   same reading row types, 10 z-block tiles;
                                   -1 before A's first device call */
    int32_t fast_block_threads; /* FAST order: threads per block of the staged
                                   kernel (512 or 256; 0 = no staged kernel) */
    int32_t row_types;          /* pattern format: distinct row records held as
                                   one-byte row types (variant 9), else 0 */
    int32_t reordered;          /* 1 if compressed with reorder = 1 */
    int32_t slices_col24;       /* delta: slices storing 24-bit column deltas */
    int64_t bandwidth;          /* max |column - row| of the stored matrix */
} spmv_info_t;

/* Fills *out with the sizes and statistics of A (host only). */
int spmv_info(spmv_mat_t A, spmv_info_t *out);

/* Rebuilds host CSR arrays from A's stored form, bit-exact (integer and
 * bitwise work only; values are copied, never recomputed).  Buffers are
 * caller-owned host memory of n+1, nnz and nnz entries (sizes from
 * spmv_info).  Works for every format. */
int spmv_decompress(spmv_mat_t A, int64_t *rowptr, int32_t *col, double *val);

/* Serialises A's compressed stream (header, tables, checksum, payload) to a
 * caller buffer.  With buf == NULL only *len is set to the size needed. */
int spmv_export(spmv_mat_t A, void *buf, size_t *len);

/* Rebuilds a handle from spmv_export() output.  The stream's checksum, its
 * sizes and every table entry are checked on the host before anything is
 * kept: SPMV_ECORRUPT on any mismatch, and no kernel ever sees it. */
int spmv_import(const void *buf, size_t len, spmv_mat_t *out);

/* ---- products (Eq. 1) -------------------------------------------------- */

/* y = A x.  x and y: device pointers to n doubles.  Enqueued on stream.
 * COLUMN order gives exactly the plain CSR fma chain.  FAST order (pattern
 * format) converts x to 53-bit fixed point scaled by the largest exponent
 * among the x entries a CTA reads (never above that of max_j |x_j|), sums
 * each row exactly in integers and rounds once, so for every row
 *   |y_i - (A x)_i| <= sum_j |a_ij| * ulp(max_j |x_j|) + ulp(y_i)/2.
 * Componentwise accuracy is therefore relative to the largest |x_j|, not to
 * the row's own terms: |y_i - (A x)_i| <= 1e-14 * sum_j |a_ij x_j| holds on
 * every row with
 *   sum_j |a_ij x_j| >= C * sum_j |a_ij| * max_j |x_j|,
 *   C = 2^-52 / (1e-14 - 2^-53), about 0.0225,
 * i.e. rows whose |a|-weighted mean |x_j| is at least 2.25 % of max |x|
 * (every row, in practice, of x drawn uniformly from [-1, 1)); a row of
 * tiny entries next to a huge one elsewhere gets only the first bound.
 * Zero/subnormal-only or non-finite x falls back to the COLUMN order on the
 * device (per CTA for the tiled kernels). */
int spmv_apply(spmv_mat_t A, const double *x, double *y, spmv_stream_t stream);

/* y = A x with x and y in host memory: copies x to the device, runs
 * spmv_apply on the library's own streams, copies y back and waits.
 * Uses library-owned device buffers kept with the handle.  For the tiled
 * FAST kernels (variants 1, 6, 8, 9, and 10 in whole plane groups) the call
 * is pipelined in 8 row chunks of whole tiles: x chunks go in on one
 * stream, a chunk's tiles run once every x chunk up to its last row plus
 * the largest displacement plus two is in (a tile's last 16-byte pair may
 * reach one element further, and it enters the tile's exponent), and its y
 * goes out on another stream while later x chunks still come in (the same
 * tiles, so the same result bits as spmv_apply).  Pinned host buffers let
 * the copies overlap; pageable ones work but serialise. */
int spmv_apply_host(spmv_mat_t A, const double *x, double *y);

/* y = A x in binary32: x and y device pointers to n floats; values are the
 * table entries rounded to float; y_i = fmaf chain over ascending columns
 * (bit-identical to the binary32 CSR product).  Pattern and delta formats,
 * and ELL (a float copy of the values is made on first use). */
int spmv_apply_f32(spmv_mat_t A, const float *x, float *y, spmv_stream_t stream);

/* Y = A X for k right-hand sides, X (n x k, leading dimension ldx >= k) and
 * Y (n x k, ldy >= k) row-major device arrays of doubles, 1 <= k <= 64.
 * Each column of Y obeys spmv_apply's rule for the handle's order.  FAST
 * order keeps per-column exponent words and a fixed-point copy of X with
 * the handle: calls on one handle whose kernels can overlap on the GPU
 * (different streams without ordering) race on them. */
int spmm_apply(spmv_mat_t A, int32_t k, const double *X, int64_t ldx, double *Y,
               int64_t ldy, spmv_stream_t stream);

/* Autotuner: times the kernel configurations available to A (FAST order:
 * the pre-converted-x kernels, the persistent kernels, the shared-memory
 * staged kernel with tiles of 512, 1024 and 2048 rows of 512 or 256
 * threads, the register-staged kernels with records from global or shared
 * memory, the z-marching kernel and the z-block kernel of 3 and 4 planes;
 * not the row types of variant 9, a
 * different stored form) on the caller's device vectors
 * x and y (n doubles each; y is overwritten), keeps the fastest for later
 * calls on A, and remembers it for matrices with the same signature (device
 * name, n, nnz, union size) uploaded later in this process.  reps: timed
 * launches per candidate (default 10 when <= 0).  *choice (may be NULL)
 * receives the chosen tile rows for a tiled kernel (variants 1, 3, 6, 7, 8;
 * for 10 the rows a CTA computes), 1
 * for the pre-converted kernel, 4 or 5 for the persistent kernels, 0 when
 * A has nothing to tune.  Each candidate's y is first compared with the
 * COLUMN-order product on the same x (|difference| <= R max|x| 2^-46 +
 * 2^-50 |y|, R the largest absolute row sum; non-finite entries equal): a
 * candidate that disagrees is never chosen, and SPMV_EDEVICE is returned if
 * none agrees.  Allocates two scratch buffers (n doubles, 16 bytes) for the
 * duration of the call.  Synchronous, uses the legacy default stream: call
 * it outside any stream capture. */
int spmv_autotune(spmv_mat_t A, const double *x, double *y, int32_t reps, int32_t *choice);

/* Selects A's FAST kernel by hand (what spmv_autotune chooses): variant 0
 * direct, 1 staged tiles of tile_rows rows (512, 1024 or 2048), 2
 * pre-converted copy of x, 3 staged tiles of that copy, 4 persistent
 * double-buffered tiles, 5 the same fed from the copy, 6 register-staged
 * tiles (full 27-point union; tile_rows 1024 with spmv_set_tile's 512 or
 * 256 threads, or 512 with 256 threads), 7 z-marching tiles (full 27-point
 * union whose plane stride is a multiple of tile_rows; same shapes as 6),
 * 8 register-staged tiles whose row records are copied to shared memory by
 * cp.async (shapes as 6), 9 register-staged tiles reading one-byte row
 * types instead of records -- the values registered in the pattern that
 * Sec. V proposes; the first selection builds the types (at most 256
 * distinct records) and copies them to the device (shapes as 6), 10
 * z-block tiles: a CTA owns a 512-row column block of tile_rows/512 (3 or
 * 4) consecutive planes, loads and converts the planes' tile_rows/512 + 2
 * x windows once and sums all its rows from shared memory, each x element
 * converted (planes + 2)/planes times instead of three (full 27-point union
 * whose plane stride is a multiple of 512; 256 threads only, so through
 * spmv_set_tile); tile_rows is ignored for 0, 2, 4, 5.  SPMV_EUNSUPPORTED
 * when A has no such kernel.
 * Copies A to the device if it is not there yet. */
int spmv_set_variant(spmv_mat_t A, int32_t variant, int32_t tile_rows);

/* As spmv_set_variant with 512-thread blocks, but also sets the block size
 * of the staged kernels: block_threads 512 (tile_rows 512, 1024 or 2048) or,
 * for variants 1, 6, 7, 8 and 9 on the full 27-slot union of a 3-D
 * 27-point stencil, 256 (tile_rows 512, 1024 or 2048: two, four or eight
 * rows per thread); variant 10 takes 256 with tile_rows 1536 or 2048.
 * Variant 11 (the TMA-fed kernel) takes tile_rows 1 or 2 (grid lines of a
 * thread's tile; 0 keeps the current plan) and block_threads 2 for two
 * CTAs an SM (column blocks of at most 768 rows, two record stages), any
 * other value for one (at most 1536 rows).
 * Ignored for variants 0, 2, 4, 5.  SPMV_EINVAL for other block sizes,
 * SPMV_EUNSUPPORTED for shapes A has no kernel for. */
int spmv_set_tile(spmv_mat_t A, int32_t variant, int32_t tile_rows, int32_t block_threads);

/* The FAST-order SpMM kernel of a pattern-format handle.  kind 1, 2 or 3
 * (3 is the default): for k >= 4 on a 27-point grid stencil with uniform
 * neighbour weights, the TMA-fed z-marching kernel (blocks of L lines by W
 * columns, 4 or 8 right-hand sides a pass, each row record read once a
 * pass, every window converted once a column) with `kind` CTAs an SM, each
 * taking blocks of at most 1536 / kind (row, column) outputs; X must then be
 * 16-byte aligned with an even ldx, else the call takes kind 0.  kind 0: one
 * thread a (row, column) pair.  All follow spmv_apply's FAST rule for every
 * column, with the scale taken per column (the largest exponent a CTA has
 * met in that column since its current run of planes began).  SPMV_EINVAL
 * for another kind. */
int spmv_set_spmm_kernel(spmv_mat_t A, int32_t kind);

/* The binary32 product kernel of a pattern-format handle.  kind 2 (the
 * default): for a 27-point grid stencil, the TMA-fed kernel that sums each
 * row from shared-memory windows of x and reads the one-byte row types
 * (values registered in the pattern, Sec. V); x must be 16-byte aligned,
 * else the call takes kind 1.  kind 1: the row types with x read through
 * L1.  kind 0: the row records.  Row types are built on the first binary32
 * call, when the matrix has at most 256 distinct records (else kind 0
 * runs).  All compute the same fmaf chain.  SPMV_EINVAL for another kind. */
int spmv_set_f32_kernel(spmv_mat_t A, int32_t kind);

/* Y = A X like spmm_apply, for callers that cannot allocate device memory
 * (a framework that routes every device allocation through its own pool, a
 * latency-critical loop that cannot afford the implicit synchronisation of
 * cudaMalloc/cudaFree).  This call allocates nothing: its only scratch (the
 * per-column maximum exponents of X, 152 words per column) is a fixed
 * device array inside the library, present on every GPU that loads it.
 * The paper has no counterpart; it is an interface convenience.
 * Limits and rules:
 *  - pattern-format A in SPMV_ORDER_FAST, already on the current device (an
 *    earlier ordinary device call on A copies it there; this call never
 *    does) -- otherwise SPMV_EUNSUPPORTED / SPMV_EINVAL;
 *  - 1 <= k <= 32 (the scratch's size), ldx >= k, ldy >= k, else SPMV_EINVAL;
 *  - the first call on each device looks up the scratch's device address
 *    (no allocation); make that first call before any stream capture;
 *  - all calls on a device share the one scratch array: calls whose
 *    kernels can overlap on the GPU race and give wrong results. */
int spmm_apply_noalloc(spmv_mat_t A, int32_t k, const double *X, int64_t ldx, double *Y,
                       int64_t ldy, spmv_stream_t stream);

/* ---- ragged batches: one persistent launch over many matrices --------- */
typedef struct spmv_batch_s *spmv_batch_t;

/* Plans y_b = A_b x_b for count pattern-format matrices of any sizes (their
 * records must have equal record_bytes).  xs/ys: host arrays of count device
 * pointers, fixed for the plan's lifetime.  The work list (matrix, row range
 * of 256 rows) is uploaded once and the launch is captured in a CUDA graph.
 * Order: when every matrix is in FAST order (spmv_set_order), each row is
 * the exact fixed-point sum rounded once, at the scale of the largest
 * exponent of its x_b (a pass over the x_b inside the same graph; a
 * matrix whose x is zero/subnormal only or not finite takes the COLUMN
 * order); otherwise every row is the COLUMN order's fma chain (bit-exact
 * with the CSR product). */
int spmv_batch_create(int32_t count, const spmv_mat_t *mats, const double *const *xs,
                      double *const *ys, spmv_batch_t *out);
/* Times the plan with work items of 64, 128, 256, 512 and 1024 rows (reps
 * graph launches each, default 10 when <= 0; this writes the plan's ys),
 * keeps the fastest and re-captures the plan's graph with it; *item_rows
 * (may be NULL) receives it.  Synchronous. */
int spmv_batch_autotune(spmv_batch_t plan, int32_t reps, int32_t *item_rows);
/* Replays the plan's graph on stream (one persistent kernel launch).  Each
 * replay resets and then draws from the plan's one work counter, so two
 * launches of the same plan must not overlap on the GPU. */
int spmv_batch_launch(spmv_batch_t plan, spmv_stream_t stream);
int spmv_batch_free(spmv_batch_t plan);
/* create + launch + wait + free, for one-off use. */
int spmv_apply_batched(int32_t count, const spmv_mat_t *mats, const double *const *xs,
                       double *const *ys, spmv_stream_t stream);

/* ---- conjugate gradients (Table I's CG iteration, no preconditioner) -- */
#define SPMV_CG_FP64 0         /* plain CG, all vectors and products in FP64 */
#define SPMV_CG_IR_FP32 1      /* iterative refinement: FP64 residual b - A x,
                                  norms and solution update; inner CG with the
                                  binary32 product and binary32 vectors */

typedef struct {
    double tol;            /* stop when |b - A x|_2 / |b|_2 <= tol (default 1e-10) */
    int32_t max_iter;      /* cap on (inner) CG steps (default 10000) */
    int32_t mode;          /* SPMV_CG_FP64 or SPMV_CG_IR_FP32 */
    int32_t check_every;   /* host reads the device convergence flag every
                              this many steps (default 16) */
    int32_t inner_max_iter;/* IR: cap per inner solve (default 300) */
    double inner_tol;      /* IR: inner relative reduction (default 1e-6); an
                              inner solve stops at the larger of this and
                              tol / (4 x the current relative residual) */
    int32_t nrhs;          /* right-hand sides solved together (1..32, default 1):
                              b and x are n x nrhs row-major */
    int32_t use_graph;     /* 1 (default): replay captured CUDA graphs */
} spmv_cg_opts;

typedef struct {
    int32_t status;        /* SPMV_OK or SPMV_ENOTCONVERGED */
    int32_t iterations;    /* CG steps (IR: total inner steps) */
    int32_t outer_iterations;  /* IR refinement steps (FP64: 0) */
    int32_t history_len;   /* entries in history */
    double rel_residual;   /* final true relative residual (max over columns) */
    double seconds;        /* device time of the solve (CUDA events) */
    double *history;       /* |r_k|/|b| per step (column 0), library-owned
                              until spmv_cg_result_free() */
} spmv_cg_result;

/* Solves A x = b (device pointers, n x nrhs doubles each; x holds the
 * initial guess).  Synchronous: returns when done.  res may be NULL. */
int cg_solve(spmv_mat_t A, const double *b, double *x, const spmv_cg_opts *opts,
             spmv_cg_result *res);
int spmv_cg_result_free(spmv_cg_result *res);

/* ---- lifetime and diagnostics ---------------------------------------- */
int spmv_free(spmv_mat_t A);
const char *spmv_strerror(int status);
/* The calling thread's last detailed error message ("" if none). */
const char *spmv_last_error(void);
/* Reads and clears A's sticky device error word (0 = none; an OR of 1: a
 * pattern number out of range, 2: a decoded column or value code out of
 * range, 4: a delta slice longer than its width, 16: a TMA-fed kernel's
 * bounded wait for its copies gave up and the kernel stopped early); waits
 * for the device. */
int spmv_device_error(spmv_mat_t A, int32_t *code);
/* Library version string. */
const char *spmv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPMVC_H */
