/*
 * damn.h -- C ABI of the GB300 (sm_103a) DA-CSR sparse matrix library.
 *
 * Diagonally-addressed CSR (DA-CSR) stores, for every stored entry of row r
 * with column c, the offset c - r instead of c (Saak & Schulze,
 * "Diagonally-Addressed Matrix Nicknack", arXiv 2307.06305, Section 2).  When
 * every offset fits a signed 16-bit integer the index stream shrinks from 4 to
 * 2 bytes per entry, and a memory-bound SpMV streams fewer bytes (Eq. (1),
 * Eq. (3), Fig. 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers are DEVICE pointers unless their name starts with h_ (host).
 *   The caller owns every buffer; the library never frees caller memory.
 * - Scratch memory comes from a caller-provided device workspace whose size
 *   is given by the matching *_workspace_size() query (16-byte aligned).
 *   Only plan handles (*_plan_create) allocate device memory of their own.
 * - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *   stream.  Calls are asynchronous on stream unless documented as
 *   synchronising.
 * - Every function returns a status code (DAMN_OK = 0 or a negative
 *   DAMN_ERR_*); damn_last_error() returns a message for the calling thread.
 *   No exception crosses the ABI and nothing aborts the process.
 * - Matrices use CSR arrays: rowptr int32[nrows+1] (rowptr[0] = 0,
 *   rowptr[nrows] = nnz, non-decreasing) and per entry a column index
 *   col int32[nnz] (CSR-32) or a diagonal offset off int16[nnz] (DA-CSR-16),
 *   plus values val[nnz].  Argument checks are O(1) host checks (sizes,
 *   null pointers, alignment, dtype); damn_validate_csr() checks the arrays.
 * - dtype selects the value type: DAMN_F64 (values, x and y FP64, FP64
 *   accumulation), DAMN_F32 or DAMN_BF16 (values FP32 / BF16; x and y FP32;
 *   FP32 accumulation).  The SpMV entry points (CSR-32, DA-CSR-16, DA-CSR-8)
 *   also take DAMN_F8E4M3: FP8 E4M3 values (1 sign, 4 exponent bits with
 *   bias 7, 3 significand bits, largest finite 448, no infinity), decoded
 *   exactly to FP32, x and y FP32, FP32 accumulation -- the float8 value
 *   column of the traffic lattice of Section 2, Fig. 3.  val, x, y, col and off must be 16-byte aligned
 *   (torch allocations are); misaligned pointers are rejected with
 *   DAMN_ERR_INVALID_ARG.
 */
#ifndef DAMN_H
#define DAMN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* Status codes, types, diagnostics                                          */
/* ------------------------------------------------------------------------ */
#define DAMN_OK                  0
#define DAMN_ERR_INVALID_ARG    -1 /* bad size, pointer, alignment or dtype      */
#define DAMN_ERR_NOFIT          -2 /* an offset c - r lies outside int16 range  */
#define DAMN_ERR_CUDA           -3 /* a CUDA runtime call failed                  */
#define DAMN_ERR_NOT_CONVERGED  -4 /* an iterative solver hit its iteration cap  */
#define DAMN_ERR_TIMEOUT        -5 /* a bounded device-side wait gave up          */
#define DAMN_ERR_UNSUPPORTED    -6 /* valid request the library does not handle   */

#define DAMN_F64   0
#define DAMN_F32   1
#define DAMN_BF16  2
#define DAMN_F8E4M3 3  /* FP8 E4M3 values (SpMV only; x and y FP32) */

#define DAMN_FMT_CSR32   0
#define DAMN_FMT_DACSR16 1
#define DAMN_FMT_DACSR8  2

/* Message describing the last error reported to the calling host thread. */
const char *damn_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int damn_version(void);

/* Reads the library's device status word for the current device into
 * *h_status and clears it when reset != 0: DAMN_OK, DAMN_ERR_TIMEOUT after a
 * bounded wait inside a kernel gave up, or DAMN_ERR_INVALID_ARG after
 * damn_permute_sym found that perm is not a permutation or a column of A out
 * of range.  The first error is kept until reset.  Synchronises stream. */
int damn_device_status(int32_t *h_status, int reset, void *stream);

/* Failure-detection self test: launches one kernel that waits on a device
 * barrier which nothing ever completes, with a wait limit of timeout_ns
 * nanoseconds (1e3 .. 1e10).  The kernel records DAMN_ERR_TIMEOUT in the
 * device status word and returns; the call synchronises and returns
 * DAMN_ERR_TIMEOUT when the bounded wait worked as designed (the device status
 * word is cleared afterwards).  No fault, trap or hang is involved. */
int damn_selftest_wait_timeout(int64_t timeout_ns, void *stream);

/* ------------------------------------------------------------------------ */
/* a1: CSR -> DA-CSR-16 translation and fit check (Section 2, Example 1,     */
/*     Eq. (2); fit reading: every c - r in [-32768, 32767])                 */
/* ------------------------------------------------------------------------ */
/* min_off and max_off saturate at the int32 limits; only columns outside
 * [0, ncols) can reach them (then n_bad > 0 and fits == 0). */
typedef struct {
  int32_t min_off;  /* smallest c - r over stored entries (0 if nnz == 0)      */
  int32_t max_off;  /* largest c - r (0 if nnz == 0)                            */
  int64_t w;        /* Eq. (2) bandwidth max |c - r|                           */
  int64_t n_fit;    /* entries with c - r in [-32768, 32767]                    */
  int64_t n_bad;    /* entries whose column lies outside [0, ncols)             */
  int32_t fits;     /* 1 iff n_fit == nnz and n_bad == 0                         */
  int32_t reserved;
} damn_fit_info;

/* Workspace bytes needed by damn_csr_to_dacsr. */
size_t damn_csr_to_dacsr_workspace_size(void);

/* off_out[i] = col[i] - r_i (narrowed to int16) for every stored entry i of
 * row r_i; entry order and values are unchanged (values are not touched).
 * Also computes the fit information into *h_info (always filled).
 * Synchronises stream.  Returns DAMN_ERR_NOFIT when some offset does not fit
 * int16 or a column is out of range; off_out is then unspecified.
 * rowptr and col are device arrays; nrows, ncols >= 0; nnz < 2^31. */
int damn_csr_to_dacsr(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                      const int32_t *col, int16_t *off_out, damn_fit_info *h_info,
                      void *workspace, size_t ws_bytes, void *stream);

/* Same with 8-bit offsets (DA-CSR-8; the int8 index width of the traffic
 * lattice of Section 2, Fig. 3): off_out[i] = col[i] - r_i narrowed to
 * int8, fits iff every offset lies in [-128, 127] (h_info->n_fit counts the
 * entries in that range).  Same workspace and errors as damn_csr_to_dacsr. */
int damn_csr_to_dacsr8(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                       const int32_t *col, int8_t *off_out, damn_fit_info *h_info,
                       void *workspace, size_t ws_bytes, void *stream);

/* Allocation-free variant of damn_csr_to_dacsr (the paper has no counterpart
 * to this entry point).  For callers that cannot allocate device memory: an
 * application or framework that owns every device allocation through its own
 * pool, or a latency-critical loop where cudaMalloc (which can synchronise
 * the whole device) is not acceptable.  Same arguments and results as
 * damn_csr_to_dacsr minus the workspace: its scratch is a static array inside
 * the library (about 64 KiB on every device that loads the library, held until
 * the process exits), which limits nrows to DAMN_NOALLOC_MAX_ROWS; larger
 * matrices are rejected with DAMN_ERR_INVALID_ARG.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress), so make that
 * first call before any stream capture; the lookup is repeated once after a
 * device reset, which gives the device a new context.  Every call uses the
 * same array and leaves its last contents there (each call overwrites every
 * record it reads): calls that overlap on the GPU (other streams or host
 * threads without ordering between them) race.  The call waits for stream to
 * finish (it reads the fit result back to *h_info); it calls no allocator. */
#define DAMN_NOALLOC_MAX_ROWS 1048576
int damn_csr_to_dacsr_noalloc(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                              const int32_t *col, int16_t *off_out, damn_fit_info *h_info,
                              void *stream);

/* Workspace bytes needed by damn_validate_csr. */
size_t damn_validate_csr_workspace_size(void);

/* Checks rowptr[0] == 0, rowptr[nrows] == nnz, rowptr non-decreasing and
 * every col in [0, ncols).  *h_bad_rows receives the number of r with
 * rowptr[r] > rowptr[r+1] (plus 1 when an end point is wrong), *h_bad_cols
 * the number of out-of-range columns.  Synchronises stream.  Returns
 * DAMN_ERR_INVALID_ARG when either count is non-zero. */
int damn_validate_csr(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                      const int32_t *col, int64_t *h_bad_rows, int64_t *h_bad_cols,
                      void *workspace, size_t ws_bytes, void *stream);

/* The same checks for a DA-CSR matrix (off int16 when off_bits == 16, int8
 * when 8): rowptr[0] == 0, rowptr[nrows] == nnz, rowptr non-decreasing, and
 * every stored entry of row r addresses a column r + off inside [0, ncols)
 * (the shifted view of Listing 2 is only dereferenced in range: Section 4,
 * Remark 3).  The SpMV kernels clamp their x accesses to [0, ncols) instead
 * of checking, so a matrix that fails here gives wrong results, not memory
 * faults.  *h_bad_rows / *h_bad_cols as for damn_validate_csr (h_bad_cols
 * counts entries whose r + off is out of range).  Uses the workspace of
 * damn_validate_csr_workspace_size().  Synchronises stream.  Returns
 * DAMN_ERR_INVALID_ARG when either count is non-zero. */
int damn_validate_dacsr(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                        const void *off, int32_t off_bits, int64_t *h_bad_rows,
                        int64_t *h_bad_cols, void *workspace, size_t ws_bytes, void *stream);

/* Round-to-nearest-even conversion of n values: FP64 -> FP32, BF16 or FP8
 * E4M3 (one rounding step, no double rounding through FP32), or FP32 -> BF16
 * or E4M3.  E4M3 has no infinity: a value beyond 464 (rounding past the
 * largest finite 448), an infinity or a NaN becomes NaN.  Used to make the
 * reduced-precision copy of a matrix's values. */
int damn_cast_values(int64_t n, const void *src, int src_dtype, void *dst, int dst_dtype,
                     void *stream);

/* ------------------------------------------------------------------------ */
/* a2: reverse Cuthill-McKee ordering and symmetric permutation             */
/*     (Section 2, Example 2; Section 3)                                     */
/* ------------------------------------------------------------------------ */

/* Host-side RCM ordering of a square pattern (host arrays).  Graph: pattern of
 * A + A^T without self loops; components by smallest vertex; George-Liu
 * pseudo-peripheral start from the component's minimum-degree vertex;
 * neighbours appended by (degree, index); the concatenation reversed.
 * h_perm[new] = old.  Optionally returns the bandwidth before / after.
 * Runs on the calling host thread; no device work. */
int damn_rcm_order(int32_t n, int64_t nnz, const int32_t *h_rowptr, const int32_t *h_col,
                   int32_t *h_perm, int64_t *h_w_before, int64_t *h_w_after);

/* Workspace bytes needed by damn_permute_sym for an n x n matrix. */
size_t damn_permute_sym_workspace_size(int32_t n);

/* B = P A P^T on the device: row i of B is row perm[i] of A, every column c
 * becomes iperm[c], and each row is sorted by new column (entries with equal
 * columns keep their stored order).  val/val_out have type dtype (F64, F32,
 * BF16; val may be NULL to permute the pattern only).  All pointers except
 * the workspace are device arrays owned by the caller: rowptr[n+1], col[nnz],
 * perm[n] (new -> old), rowptr_out[n+1], col_out[nnz], val_out[nnz].
 * rowptr must be a valid CSR row pointer with rowptr[n] == nnz <= INT32_MAX.
 * workspace: device, 16-byte aligned, >= damn_permute_sym_workspace_size(n)
 * bytes, no initial contents.  Asynchronous.  If perm is not a permutation
 * of 0..n-1 (checked on the device) nothing is written to col_out/val_out
 * and the device status word reports DAMN_ERR_INVALID_ARG; a column outside
 * 0..n-1 is reported the same way and stored as INT32_MAX.  Cost: one warp
 * per row, O(len^2 / 32) comparisons for a row of len entries. */
int damn_permute_sym(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                     const void *val, int dtype, const int32_t *perm, int32_t *rowptr_out,
                     int32_t *col_out, void *val_out, void *workspace, size_t ws_bytes,
                     void *stream);

typedef struct {
  int64_t w_before;  /* Eq. (2) bandwidth of A          */
  int64_t w_after;   /* Eq. (2) bandwidth of P A P^T    */
} damn_bw_info;

/* Convenience: copies the pattern to the host, runs damn_rcm_order, copies
 * perm to perm_out (device) and runs damn_permute_sym.  Synchronises. */
int damn_rcm_permute(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                     const void *val, int dtype, int32_t *perm_out, int32_t *rowptr_out,
                     int32_t *col_out, void *val_out, damn_bw_info *h_info, void *workspace,
                     size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* a3/a4/a5/a8: SpMV y <- alpha A x + beta y (Section 4, Listing 2)           */
/* ------------------------------------------------------------------------ */
typedef struct damn_plan damn_plan;

typedef struct {
  int32_t mode;          /* 0 = row tiles (ROWS, ROWS_LONG), 1 = balanced entry slices */
  int32_t tile_items;    /* rows per tile, or rows+entries budget of a balanced tile */
  int32_t ntiles;
  int32_t grid;          /* persistent CTAs of the last launch                 */
  int32_t stages;        /* shared-memory ring depth of the last launch        */
  int32_t threads;       /* consumer threads per CTA                           */
  double row_efficiency; /* nnz / (32 * sum over 32-row groups of max row len) */
  int32_t max_row;       /* longest row                                        */
  int32_t dtype;
  int32_t tiling;        /* DAMN_TILING_*                                      */
  int32_t x_staged_tiles;/* tiles whose x window is staged in shared memory
                           (x windows of <= 4 segments; 0 for DAMN_TILING_BAND,
                           whose ring is filled as the kernel runs)           */
  int32_t stages_requested; /* ring depth set by damn_plan_set_stages or the
                           autotuner (0: automatic)                           */
  int32_t x_staging;     /* rows tilings: 1 = x windows staged in shared
                           memory, 0 = x read from global memory (L1 / L2)    */
} damn_plan_desc;

/* Tilings (see damn_plan_set_tiling). */
#define DAMN_TILING_SLICES        0
#define DAMN_TILING_ROWS          1
#define DAMN_TILING_ROWS_LONG     2
#define DAMN_TILING_BAND          3
#define DAMN_TILING_ROWS_LANES4   4
#define DAMN_TILING_ROWS_LANES8   5
#define DAMN_TILING_ROWS_LANES16  6
#define DAMN_TILING_ROWS_LANES32  7
#define DAMN_TILING_SORTED_ROWS   8
#define DAMN_TILING_ROWS_X2       9

/* Builds a plan for one matrix and value dtype: the partition of the rows
 * into tiles and the compute mode (the tiling), chosen from the row-length
 * statistics: rows of uniform length inside 32-row groups (row_efficiency
 * >= 0.85) get a rows tiling with the fewest lanes per row (1, 2, 4, 8, 16
 * or 32) that keeps a row's entries in registers and a tile in a stage;
 * ragged rows get DAMN_TILING_BAND.  When idx (col for DAMN_FMT_CSR32, off
 * for DAMN_FMT_DACSR16 / DAMN_FMT_DACSR8) is given, the plan also prepares
 * how the SpMV kernels stage x in shared memory (the band-window staging of
 * DA-CSR: row r reads x only in [r - w, r + w], Eq. (2)): for rows and
 * slices tilings the x window of every tile -- its sorted distinct columns
 * cut into at most 4 contiguous segments (gaps of up to 32 columns merged);
 * for the band tiling the column range of every tile.  Tiles whose x cannot
 * be staged gather it from global memory.  idx may be NULL (no staging).
 * Reads rowptr/idx on the device; synchronises.  rowptr and idx must stay
 * valid while the plan is used, and an SpMV given this plan must pass these
 * same rowptr and (for the plan's own format) idx arrays; another index
 * format's copy of the same matrix is accepted.  The plan owns device
 * memory until damn_plan_destroy.  One plan serves the CSR-32, DA-CSR-16
 * and DA-CSR-8 copies of the same matrix, giving bitwise equal results. */
int damn_plan_create(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                     int format, const void *idx, int dtype, void *stream, damn_plan **out);

/* Autotuner: times every tiling on the given operands (format DAMN_FMT_*;
 * idx is col or off) -- rows with 1 and 2 lanes per row, rows with twice
 * the rows per thread, balanced slices, band, sorted rows, and rows with
 * 4 / 8 / 16 / 32 lanes per row where an average row has
 * at least two entries per lane -- keeps the fastest, then times ring depths
 * of 2 to 6 stages for it and keeps one only when it is at least 3 % faster
 * than the automatic depth, then (rows tilings) times x read from global
 * memory instead of staged, kept on the same 3 % rule.  y is overwritten.
 * Synchronises stream. */
int damn_plan_autotune(damn_plan *plan, int format, const void *idx, const void *val,
                       const void *x, void *y, void *stream);

/* Pins the plan's tiling:
 *  DAMN_TILING_ROWS: tiles of 256 rows with FP64 values, one row per
 *    thread, or 512 rows with FP32 / BF16 values, two rows per thread;
 *  DAMN_TILING_ROWS_X2: as DAMN_TILING_ROWS with twice the rows per thread
 *    (FP64 values: 512-row tiles, two rows per thread; FP32 / BF16 / FP8
 *    values: 1024-row tiles, four rows per thread);
 *  DAMN_TILING_ROWS_LONG: 128-row tiles, two lanes per row;
 *  DAMN_TILING_ROWS_LANES4 / 8 / 16 / 32: tiles of 64 / 32 / 16 / 8 rows,
 *    4 / 8 / 16 / 32 lanes per row (lane i takes entries i, i + E, ...; the
 *    lanes' partial sums are added by a butterfly);
 *  DAMN_TILING_SLICES: tiles balanced on rows + entries, each thread one
 *    contiguous slice of entries, x windows of up to 4 segments;
 *  DAMN_TILING_BAND: the same balanced tiles and slices, each CTA walking a
 *    contiguous run of tiles with x in a shared-memory ring (column c in slot
 *    c mod W, W = 8192 for FP64 x, 16384 for FP32 x); a tile whose columns
 *    the ring cannot hold reads x from global memory;
 *  DAMN_TILING_SORTED_ROWS: tiles of 192 rows, each CTA walking a contiguous
 *    run of tiles with x in a ring (W = 4096 for FP64 x, 8192 for FP32 x);
 *    one row per thread, the tile's rows dealt to threads in order of
 *    decreasing length (a permutation the plan computes), so a warp's rows
 *    have similar lengths; rows longer than 128 entries are summed by a
 *    whole warp (lane-strided partial sums added by a butterfly).
 * Recomputes the staging data; synchronises the legacy default stream. */
int damn_plan_set_tiling(damn_plan *plan, int tiling);

/* Ring depth (shared-memory stages per CTA) of the plan's SpMV launches:
 * 0 = automatic (the deepest ring that keeps the kernel's CTAs per SM), or
 * 2 .. 8; a depth that does not fit the kernel's shared memory falls back to
 * automatic.  The band and sorted-rows tilings run several consumer groups
 * that take turns on the tiles; their depth is rounded down to a multiple of
 * the number of groups (4 and 2).  No device work. */
int damn_plan_set_stages(damn_plan *plan, int32_t stages);

/* Rows tilings (DAMN_TILING_ROWS*, ROWS_LONG, ROWS_LANES*): on != 0 (the
 * default) stages each tile's x window in shared memory; on == 0 reads x
 * from global memory (L1 / L2) instead, with the same register-batched row
 * loop -- cheaper per entry when a warp's rows read consecutive x entries at
 * each offset (stencil-like patterns).  DAMN_TILING_BAND: on == 0 launches
 * without the x ring (every tile gathers x from L1 / L2), leaving the ring's
 * 64 KB of shared memory to the L1 cache -- for bands too wide for the ring.
 * Results are bitwise the same either way.  No device work.  The autotuner
 * tries both for rows and band tilings. */
int damn_plan_set_x_staging(damn_plan *plan, int32_t on);

int damn_plan_describe(const damn_plan *plan, damn_plan_desc *h_desc);
int damn_plan_destroy(damn_plan *plan);

/* y <- alpha A x + beta y with A in CSR-32 (col = absolute column indices).
 * x has ncols entries, y nrows.  beta == 0: y is output only (never read).
 * plan may be NULL (fixed row tiles, balanced slices).  For a given plan the
 * result is bitwise identical to damn_spmv_dacsr16 on the same matrix. */
int damn_spmv_csr32(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                    const int32_t *col, const void *val, int dtype, const void *x, void *y,
                    double alpha, double beta, const damn_plan *plan, void *stream);

/* Same with A in DA-CSR-16: entry i of row r multiplies x[r + off[i]]
 * (Listing 2's shifted view of x; Remark 3 for nrows != ncols). */
int damn_spmv_dacsr16(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                      const int16_t *off, const void *val, int dtype, const void *x, void *y,
                      double alpha, double beta, const damn_plan *plan, void *stream);

/* Same with A in DA-CSR-8 (int8 offsets, from damn_csr_to_dacsr8); for a
 * given plan bitwise identical to damn_spmv_dacsr16 and damn_spmv_csr32. */
int damn_spmv_dacsr8(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                     const int8_t *off, const void *val, int dtype, const void *x, void *y,
                     double alpha, double beta, const damn_plan *plan, void *stream);

/* ------------------------------------------------------------------------ */
/* DA-BSR: diagonal addressing of block CSR (the technique applied to BSR,   */
/* Section 1)                                                                */
/* ------------------------------------------------------------------------ */
/* y <- alpha A x + beta y with A in block CSR: nbr x nbc blocks of b x b
 * (b in {1, 2, 3, 4, 6, 8}), browptr int32[nbr+1] over the nblk stored
 * blocks, per block its column (bsr32: absolute block column, int32) or its
 * offset from the block diagonal (dabsr16 / dabsr8: C - R as int16 / int8,
 * produced by damn_csr_to_dacsr / damn_csr_to_dacsr8 applied to the block
 * pattern (nbr, nbc, nblk, browptr, bcol)), and b*b values per block,
 * row-major inside the block (val[nblk][b][b]).  x has nbc*b entries, y
 * nbr*b.  Scalar row R*b + i accumulates, over the row's blocks in stored
 * order and j = 0..b-1, val[k][i][j] * x[C_k*b + j] with FMA; the three
 * variants give bitwise equal results.  dtype as for damn_spmv_dacsr16.
 * beta == 0: y is output only.  Asynchronous. */
int damn_spmv_bsr32(int32_t nbr, int32_t nbc, int64_t nblk, int32_t b, const int32_t *browptr,
                    const int32_t *bcol, const void *val, int dtype, const void *x, void *y,
                    double alpha, double beta, void *stream);
int damn_spmv_dabsr16(int32_t nbr, int32_t nbc, int64_t nblk, int32_t b, const int32_t *browptr,
                      const int16_t *boff, const void *val, int dtype, const void *x, void *y,
                      double alpha, double beta, void *stream);
int damn_spmv_dabsr8(int32_t nbr, int32_t nbc, int64_t nblk, int32_t b, const int32_t *browptr,
                     const int8_t *boff, const void *val, int dtype, const void *x, void *y,
                     double alpha, double beta, void *stream);

/* ------------------------------------------------------------------------ */
/* DA-COO: diagonal addressing of the column vector of COO storage           */
/* (Section 1)                                                               */
/* ------------------------------------------------------------------------ */
/* Workspace bytes for the COO SpMVs below (two partial sums per tile of 2048
 * entries). */
size_t damn_coo_workspace_size(int64_t nnz, int dtype);

/* y <- alpha A x + beta y with A in COO sorted by row: row int32[nnz] and per
 * entry its column (coo32: col int32) or its offset from the diagonal
 * (dacoo16: c - r as int16, e.g. from damn_csr_to_dacsr on the same entries),
 * values val[nnz] of dtype (as for damn_spmv_dacsr16).  Entries of a row in
 * stored order are summed with FMA in chunks of 8 consecutive entries (chunk
 * j = entries 8j .. 8j+7); a row crossing chunks adds its chunk sums left to
 * right.  y[r] = alpha * sum + beta * y[r], y not read when beta == 0.
 * Deterministic (no atomics); coo32 and dacoo16 give bitwise equal results.
 * Rows without entries get beta y (0 when beta == 0).  Row indices outside
 * [0, nrows) are never written.  16-byte aligned row, idx and val arrays are
 * read with 16-byte loads.  workspace: device, 16-byte aligned,
 * >= damn_coo_workspace_size(nnz, dtype) bytes.  Two launches, asynchronous. */
int damn_spmv_coo32(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *row,
                    const int32_t *col, const void *val, int dtype, const void *x, void *y,
                    double alpha, double beta, void *workspace, size_t ws_bytes, void *stream);
int damn_spmv_dacoo16(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *row,
                      const int16_t *off, const void *val, int dtype, const void *x, void *y,
                      double alpha, double beta, void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* a6: CG (FP64) and mixed-precision CG with iterative refinement            */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t iterations;   /* CG steps (inner steps summed for CG-IR)           */
  int32_t outer;        /* refinement steps (CG-IR), 0 for CG                */
  int32_t converged;
  int32_t reserved;
  double relres;        /* last ||r|| / ||b|| (recurrence for CG, true for IR) */
  double true_relres;   /* ||b - A x|| / ||b|| recomputed in FP64 at exit     */
} damn_cg_result;

size_t damn_cg_workspace_size(int32_t n);

/* FP64 conjugate gradients on an SPD matrix in DA-CSR-16 with FP64 values:
 * x (in: x0, out: solution), stop when ||r|| <= rtol ||b|| or after
 * max_iter steps.  Synchronises; returns DAMN_ERR_NOT_CONVERGED at the cap. */
int damn_cg(int32_t n, int64_t nnz, const int32_t *rowptr, const int16_t *off,
            const double *val, const double *b, double *x, double rtol, int32_t max_iter,
            const damn_plan *plan, damn_cg_result *h_res, void *workspace, size_t ws_bytes,
            void *stream);

size_t damn_cg_ir_workspace_size(int32_t n);

/* Mixed-precision refinement: outer residual r = b - A x with the FP64
 * values (FP64 accumulation), inner CG on A_low d = r/||r|| with val_low of
 * type low_dtype (DAMN_F32 or DAMN_BF16), FP32 vectors, FP32 accumulation and
 * FP64 dot products, to inner_rtol or max_inner steps; x += ||r|| d in FP64.
 * plan64 / plan_low may be NULL.  Synchronises. */
int damn_cg_ir(int32_t n, int64_t nnz, const int32_t *rowptr, const int16_t *off,
               const double *val, const void *val_low, int low_dtype, const double *b,
               double *x, double rtol, double inner_rtol, int32_t max_inner, int32_t max_outer,
               const damn_plan *plan64, const damn_plan *plan_low, damn_cg_result *h_res,
               void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* a7: multi-RHS SpMM and the batched persistent launch                      */
/* ------------------------------------------------------------------------ */

/* Y = A X for one DA-CSR-16 matrix, X row-major ncols x k, Y row-major
 * nrows x k (1 <= k <= 64).  dtype F64 (X, Y FP64) or F32 (X, Y FP32).
 * Each row's entries are split over E lanes (E chosen from nnz / nrows, about
 * four entries per lane and pass) whose partial sums are added in a fixed
 * butterfly order; results depend only on (k, E).  nnz at most 2^31 - 65
 * per matrix; nnz > 0 needs ncols >= 1;
 * an entry whose column r + off lies outside [0, ncols) (invalid input, which
 * damn_validate_dacsr reports) reads row ncols - 1 of X instead of memory
 * outside X.  The same holds for the batched launches. */
int damn_spmm_dacsr16(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                      const int16_t *off, const void *val, int dtype, int32_t k, const void *X,
                      void *Y, void *stream);

typedef struct {
  int32_t nrows, ncols;
  int64_t nnz;
  const int32_t *rowptr;   /* device */
  const int16_t *off;      /* device */
  const void *val;         /* device, dtype of the batch */
  const void *X;           /* device, row-major ncols x k */
  void *Y;                 /* device, row-major nrows x k */
} damn_mat_desc;

typedef struct damn_batch_plan damn_batch_plan;

typedef struct {
  int32_t count, k, dtype, ntiles, grid, threads, tile_items, graph_ready;
  int32_t entry_lanes;     /* E: lanes splitting each row's entries */
  int32_t streamed;        /* 1: row groups take the next row as they finish */
  double tune_ms;          /* best time measured by the autotuner (0 if none) */
} damn_batch_desc;

/* Builds the work list of a batch of independent DA-CSR-16 products
 * Y_m = A_m X_m (host descriptors, device data): items of rows_per_item
 * consecutive rows of one matrix, one warp per item.  Each row is computed by
 * a row group of L * E lanes (L = the largest power of two <= min(k, 32)
 * column lanes, E entry lanes; Section 4's shifted-x row loop applied to
 * every column of X; the E partial sums added by a fixed butterfly), so
 * results depend only on (k, E).  Two schedules of the row groups:
 *   fixed passes: the warp's 32 / (L E) groups take 32 / (L E) consecutive
 *     rows at a time and the pass lasts as long as its longest row;
 *   streamed: a group that has finished its row takes the item's next row at
 *     once (rows dealt in order), so the warp's steps stay nearly full.
 * Every row is computed and written exactly once; an empty row gets 0.
 * autotune != 0 times the candidate shapes (E, schedule, rows per item,
 * threads) on the real operands (Y is overwritten) and keeps the fastest; the
 * default is fixed passes with E from nnz / nrows and items of 256 rows.  Then
 * the persistent launch is captured in a CUDA graph.  Synchronises stream.
 * The plan owns device memory until destroyed. */
int damn_batch_plan_create(int32_t count, const damn_mat_desc *h_descs, int32_t k, int dtype,
                           int autotune, void *stream, damn_batch_plan **out);
int damn_batch_plan_describe(const damn_batch_plan *plan, damn_batch_desc *h_desc);

/* Sets the launch shape of a batch plan and captures its graph again:
 * streamed != 0 for streamed rows, else fixed passes; entry_lanes E a power
 * of two <= 8 with L * E <= 32; rows_per_item in [1, 1024]; threads per block
 * 32, 64, 128 or 256.  DAMN_ERR_INVALID_ARG for anything else (the plan is
 * then unchanged).  Synchronises stream before the change. */
int damn_batch_plan_set_shape(damn_batch_plan *plan, int32_t streamed, int32_t rows_per_item,
                              int32_t entry_lanes, int32_t threads, void *stream);
int damn_batch_plan_destroy(damn_batch_plan *plan);

/* One persistent launch computing every Y_m of the batch. */
int damn_spmm_dacsr16_batched(const damn_batch_plan *plan, void *stream);

/* Replays the CUDA graph captured by damn_batch_plan_create on stream. */
int damn_batch_graph_launch(damn_batch_plan *plan, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DAMN_H */
