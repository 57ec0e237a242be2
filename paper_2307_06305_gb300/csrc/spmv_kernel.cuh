// Device side of the SpMV engine: y <- alpha A x + beta y for CSR-32,
// DA-CSR-16 and DA-CSR-8 (Section 4, Listing 2) with FP64 values, or FP32 /
// BF16 values with FP32 vectors and FP32 accumulation.  Included by spmv.cu
// only.
//
// Design (GB300, sm_103a)
// -----------------------
// The rows are cut into tiles (fixed row blocks, or blocks balanced on
// rows + entries).  A persistent grid of CTAs walks the tiles round-robin.
// Each CTA has one producer warp and NT consumer threads:
//
//  * the producer stages, per tile, the row pointers, values and indices and
//    the tile's x window -- the few contiguous x segments the tile's columns
//    fall into, found at plan time -- into a ring of shared-memory stages with
//    bulk asynchronous copies (cp.async.bulk, evict-first for the matrix)
//    completing on an mbarrier.  Lane i of the producer prepares tile i
//    (copy ranges, stage header) 32 tiles at a time; the serial per-tile work
//    is the stage wait, the header stores, the byte count and the copies
//    (each copy costs its issuing thread ~170 cycles on this part);
//  * the consumers compute the tile entirely from shared memory: DA-CSR reads
//    x at row + off (the shifted view of Listing 2), CSR at col, through a
//    branch-free map from the tile-local column to its slot in the staged
//    window.  Tiles whose window does not fit a stage gather x from global
//    memory instead.
//
// Staging x is what lets the FP64 FMAs overlap the matrix stream: on this part
// a DFMA warp instruction occupies an SM sub-partition's FP64 unit for ~67
// cycles whatever the active lanes, so the FMA chains must never wait for
// ~1 us L2 gathers.
//
// Compute modes (chosen per plan from the row-length statistics):
//
//  rows (mode 0): E lanes per row (E = 1 for short rows, 2 for rows of a few
//    dozen entries), each lane running its share of the row's FMA chain in
//    stored order (E = 2: entries e, e + 2, ... per lane, then one shuffle
//    add).  A warp loads its rows' values and x into registers, hands the
//    stage back at once, then runs the FMAs; warps never wait for each other.
//    FP64 short rows: 8 consumer warps per CTA and three CTAs per SM, six
//    consumer warps per sub-partition to hide the shared-memory latency;
//    FP32 / BF16 short rows: two rows per thread.
//  slices (mode 1): the tile's m entries are cut into NT contiguous slices
//    of ceil(m/NT); every thread runs exactly its slice's FMAs, writing
//    finished rows to shared memory and the partial sum of a row that
//    continues into the next slice to carry[i].  After a barrier, the thread
//    that finishes a row begun in an earlier slice adds the carries of the
//    slices the row spans, left to right.  For irregular rows.
//
// Summation order depends only on the plan (tile partition, mode, NT, E), so
// for one plan CSR-32, DA-CSR-16 and DA-CSR-8 give bitwise equal results.
// Tiles whose entries do not fit a stage are computed from global memory.
//
// Every mbarrier wait is bounded (global timer); a wait that gives up records
// DAMN_ERR_TIMEOUT in the library status word, and the CTA drains its own
// copies (bounded) and returns.
#pragma once

#include <climits>

#include "damn_common.cuh"

namespace damn {
namespace spmvk {

constexpr int kXSegMax = 4;        // x segments per tile
constexpr int kMaxStages = 8;

// x window of one tile, computed at plan time: segments of x that start at
// columns lo[i] (ascending, disjoint); nseg == 0: the tile gathers x from
// global memory.  Segment i is bulk-copied from element src[i] (its 16-byte
// aligned start) for cnt[i] elements to the shared slots starting at
// pos[i] - (lo[i] - src[i]), so that column lo[i] lands at slot pos[i].
// Windows that would need a partial 16-byte block at the end of x are not
// staged.
struct __align__(16) XSeg {
  int nseg;
  int pad[3];
  int lo[kXSegMax];
  int pos[kXSegMax];
  int src[kXSegMax];
  int cnt[kXSegMax];
};

// Per-stage tile header written by the producer.  The x-window map is stored
// ready to use, in tile-local columns cl = c - r0 (see XMap).
constexpr int kTileDirect = 1;   // entries not staged: read from global memory
constexpr int kTileStaged = 2;   // x window staged in shared memory

struct __align__(16) TileHdr {
  int r0, nr, k0, flags;
  int rp_sh, v_sh, i_sh, d0;
  int lo1, lo2, lo3, dd1;
  int dd2, dd3, m, nseg;
};

struct SpmvParams {
  int nrows, ncols;
  long long nnz;
  const int *rowptr;
  const void *idx;
  const void *val;
  const void *x;
  const void *y0;
  void *y;
  double alpha, beta;
  int ab_mode;         // 0: y = acc, 1: y = alpha acc, 2: y = alpha acc + beta y0
  int mode;            // 0 one row per thread, 1 balanced slices
  int ntiles;
  int rows_per_tile;   // > 0: fixed row tiles; 0: tile bounds from `bounds`
  const int2 *bounds;  // {first row, rowptr[first row]} per tile, ntiles + 1 entries
  const XSeg *xseg;    // per tile x window (NULL: gather everything)
  const void *dot_w;
  int dot_self;
  double *dot_partials;
  int stages;          // depth of the shared-memory ring (<= kMaxStages)
  int stages_req;      // requested depth (0: the deepest that keeps MINB CTAs per SM)
  int max_nseg;        // most x segments of any tile's window
  const int2 *colrange;  // band mode: {min, max} column of every tile (NULL: none)
  const uint16_t *perm;  // sorted-rows mode: tile-local rows by decreasing length
  int *status;
  unsigned long long timeout_ns;
};

// NT consumer threads; rows mode: tiles of TILE_ROWS = RPT * NT / E rows,
// E lanes sharing each row (entries e, e + E, ... per lane, partial sums
// added by a butterfly), each lane group computing RPT rows.  CAP_NZ / CAP_ROWS / XCAP: capacity of one
// stage (entries, rows, staged x elements).  MINB CTAs of NT + 32 threads are
// meant to share an SM.
template <int NT_, int CAP_NZ_, int CAP_ROWS_, int XCAP_, int MINB_, int RPT_ = 1, int E_ = 1>
struct KCfg {
  static constexpr int NT = NT_, CAP_NZ = CAP_NZ_, CAP_ROWS = CAP_ROWS_, XCAP = XCAP_;
  static constexpr int MINB = MINB_, RPT = RPT_;
  static constexpr int E = E_;                       // lanes sharing one row (rows mode)
  static constexpr int TILE_ROWS = NT * RPT / E;
  static_assert(E == 1 || E == 2 || E == 4 || E == 8 || E == 16 || E == 32,
                "a power of two from 1 to 32 lanes per row");
};

// Rows mode, short rows, FP64 values: 256 consumers (8 warps: two on each SM
// sub-partition, so the FP64 units of all four carry the same load) + the
// producer warp, three CTAs per SM (at most 72 registers per thread) so that
// six consumer warps per sub-partition keep its FP64 unit fed while the
// others wait on shared-memory loads.  Tiles of 256 rows, two stages of up
// to 1792 entries: rows of up to 7 entries stay in registers.
// Rows mode, short rows, FP32 / BF16 values: the same CTAs with tiles of 512
// rows, two rows per thread loaded together (their FP32 operands fit the
// registers), so each warp pays the shared-memory latency chain once per two
// rows and the producer -- whose bulk copies cost a fixed ~170 cycles each to
// issue -- starts half as many tiles per row.
// Rows mode, long rows: 256 consumers, two lanes per row (each keeping up
// to 14 of the row's entries in registers, so eight consumer warps fit the
// registers of two CTAs per SM), tiles of 128 rows, stages of 3584 entries:
// rows of up to 28 entries stay in registers.
// Slices mode: 256 consumers, two CTAs per SM, balanced tiles of up to 2048
// entries and 512 rows.
// Rows mode, E = 4, 8, 16, 32 lanes per row (rows of dozens to hundreds of
// entries): the long-rows stages with tiles of 64, 32, 16 or 8 rows; each
// lane keeps 14 of its row's entries in registers.
using CfgShort = KCfg<256, 1792, 256, 1280, 3, 1>;
using CfgShortNarrow = KCfg<256, 3584, 512, 2560, 3, 2>;
using CfgLong = KCfg<256, 3584, 128, 1536, 2, 1, 2>;
// Rows mode, long rows, FP32 / BF16 / FP8 values: the same tiles with three
// CTAs per SM (the narrow stages leave the shared memory for it; at most 72
// registers per thread), so that more warps hide the shared-memory latency
// of the narrow kernels, which issue more instructions per byte.
using CfgLongNarrow = KCfg<256, 3584, 128, 1536, 3, 1, 2>;
using CfgSlices = KCfg<256, 2048, 512, 1280, 2, 1>;
// Rows mode with twice the rows per thread of CfgShort / CfgShortNarrow:
// FP64 values two rows per thread (two independent FMA chains), FP32 / BF16
// / FP8 values four; tiles of 512 / 1024 rows, two CTAs per SM.
using CfgShortX2 = KCfg<256, 3584, 512, 2048, 2, 2>;
using CfgShortNarrowX2 = KCfg<256, 7168, 1024, 4096, 2, 4>;
using CfgLanes4 = KCfg<256, 3584, 64, 1536, 2, 1, 4>;
using CfgLanes8 = KCfg<256, 3584, 32, 1536, 2, 1, 8>;
using CfgLanes16 = KCfg<256, 3584, 16, 1536, 2, 1, 16>;
using CfgLanes32 = KCfg<256, 3584, 8, 1536, 2, 1, 32>;

// Plan shapes (kernel configurations); cfg_geom in spmv.cu gives their geometry.
enum Shape {
  kShapeShort = 0,   // rows, one lane per row (CfgShort / CfgShortNarrow)
  kShapeLong = 1,    // rows, two lanes per row
  kShapeSlices = 2,  // balanced tiles, entry slices, x windows of <= 4 segments
  kShapeBand = 3,    // balanced tiles, entry slices, x ring (band mode)
  kShapeLanes4 = 4,
  kShapeLanes8 = 5,
  kShapeLanes16 = 6,
  kShapeLanes32 = 7,
  kShapeSorted = 8,  // row tiles sorted by length, one row per thread, x ring
  kShapeShortX2 = 9, // rows, one lane per row, twice the rows per thread of kShapeShort
};

constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared memory: [stage 0 .. stage S-1][control][mode-1 buffers]
template <typename V, typename I, class C>
struct Layout {
  using A = typename AccOf<V>::type;
  static constexpr int EV = 16 / (int)sizeof(V), EI = 16 / (int)sizeof(I), EX = 16 / (int)sizeof(A);
  static constexpr int XCAP = C::XCAP;  // staged x elements per tile
  static constexpr size_t RP_BYTES = align_up((C::CAP_ROWS + 1 + 8) * 4, 128);
  static constexpr size_t V_BYTES = align_up((C::CAP_NZ + 2 * EV) * sizeof(V), 128);
  static constexpr size_t I_BYTES = align_up((C::CAP_NZ + 2 * EI) * sizeof(I), 128);
  static constexpr size_t X_BYTES = align_up((XCAP + 2 * kXSegMax * EX) * sizeof(A), 128);
  static constexpr int X_ELEMS = static_cast<int>(X_BYTES / sizeof(A));  // slots of the x buffer
  static constexpr size_t OFF_V = RP_BYTES, OFF_I = RP_BYTES + V_BYTES,
                          OFF_X = RP_BYTES + V_BYTES + I_BYTES;
  static constexpr size_t STAGE = OFF_X + X_BYTES;
  static constexpr size_t C_FULL = 0;
  static constexpr size_t C_EMPTY = kMaxStages * 8;
  static constexpr size_t C_HDR = 2 * kMaxStages * 8;
  static constexpr size_t C_RED = align_up(C_HDR + kMaxStages * sizeof(TileHdr), 16);
  static constexpr size_t CTRL = align_up(C_RED + (C::NT / 32) * sizeof(double), 128);
  static constexpr size_t M1_CARRY = 0;
  static constexpr size_t M1_ROWSUM = 2 * C::NT * sizeof(A);
  static constexpr size_t M1_BYTES = M1_ROWSUM + 2 * C::CAP_ROWS * sizeof(A);
  static size_t total(int stages, int mode) {
    return stages * STAGE + CTRL + (mode == 1 ? M1_BYTES : 0);
  }
};

// Position in the ring of shared-memory stages: the stage of a tile and the
// phase parity of that stage's pass, advanced by additions instead of the
// division tile / stages (a run-time 32- or 64-bit division costs dozens to
// hundreds of instructions per tile).
struct RingPos {
  int s = 0;        // stage
  uint32_t ph = 0;  // parity of the current pass over the ring
  __device__ __forceinline__ void advance(int by, int stages) {  // by <= stages
    s += by;
    if (s >= stages) { s -= stages; ph ^= 1u; }
  }
};

// Element range [first, first+count) of an array of len elements, split into a
// 16-byte aligned bulk part [a0, b1) and a plainly loaded tail [tb, first+count)
// beyond the array's last full 16-byte block.
struct Range {
  long long a0, tb;
  uint32_t bulk_bytes;
};

template <int ESZ>
__device__ __forceinline__ Range split_range(long long first, long long count, long long len) {
  constexpr long long E = 16 / ESZ;
  Range r;
  r.a0 = first & ~(E - 1);
  const long long a1 = (first + count + E - 1) & ~(E - 1);
  const long long full_end = len & ~(E - 1);
  const long long b1 = a1 < full_end ? a1 : full_end;
  r.bulk_bytes = b1 > r.a0 ? static_cast<uint32_t>((b1 - r.a0) * ESZ) : 0u;
  r.tb = b1 > r.a0 ? b1 : r.a0;
  return r;
}

// ----------------------------------------------------------------------------
// Producer
// ----------------------------------------------------------------------------

// What a producer lane prefetches for one tile.
struct TileMeta {
  int r0, r1, k0, k1, nseg;
  int lo[kXSegMax], pos[kXSegMax], src[kXSegMax], cnt[kXSegMax];
};

template <class C>
__device__ __forceinline__ void load_meta(const SpmvParams &p, long long t, TileMeta &mt) {
  if (p.rows_per_tile > 0) {
    mt.r0 = static_cast<int>(t * p.rows_per_tile);
    mt.r1 = min(mt.r0 + p.rows_per_tile, p.nrows);
    mt.k0 = __ldg(p.rowptr + mt.r0);
    mt.k1 = __ldg(p.rowptr + mt.r1);
  } else {
    const int2 b0 = __ldg(p.bounds + t), b1 = __ldg(p.bounds + t + 1);
    mt.r0 = b0.x; mt.k0 = b0.y; mt.r1 = b1.x; mt.k1 = b1.y;
  }
  mt.nseg = 0;
  if (p.xseg && mt.k1 - mt.k0 <= C::CAP_NZ) {
    const XSeg *xs = p.xseg + t;
    mt.nseg = __ldg(&xs->nseg);
    const int4 lo = __ldg(reinterpret_cast<const int4 *>(xs->lo));
    const int4 pos = __ldg(reinterpret_cast<const int4 *>(xs->pos));
    const int4 src = __ldg(reinterpret_cast<const int4 *>(xs->src));
    const int4 cnt = __ldg(reinterpret_cast<const int4 *>(xs->cnt));
    mt.lo[0] = lo.x; mt.lo[1] = lo.y; mt.lo[2] = lo.z; mt.lo[3] = lo.w;
    mt.pos[0] = pos.x; mt.pos[1] = pos.y; mt.pos[2] = pos.z; mt.pos[3] = pos.w;
    mt.src[0] = src.x; mt.src[1] = src.y; mt.src[2] = src.z; mt.src[3] = src.w;
    mt.cnt[0] = cnt.x; mt.cnt[1] = cnt.y; mt.cnt[2] = cnt.z; mt.cnt[3] = cnt.w;
  }
}

template <typename T>
__device__ __forceinline__ void load_tail(T *dst, const T *src, long long a0, long long tb,
                                          long long end) {
  for (long long e = tb; e < end; ++e) dst[e - a0] = src[e];
}

// Everything the producer needs to issue one tile, computed ahead (by the
// lane that will issue it, 32 tiles at a time in parallel): the stage
// header, the 16-byte aligned bulk ranges of row pointers / values /
// indices, the x segments, and whether a partial block at the very end of an
// array has to be loaded with plain loads.
struct TileIssue {
  int4 h0, h1, h2, h3;       // stage header (TileHdr layout)
  long long rp_a0, v_a0, i_a0;
  uint32_t rp_bytes, v_bytes, i_bytes, tx_bytes;
  int xsrc[kXSegMax], xdst[kXSegMax], xcnt[kXSegMax];
  int tails;                 // a plain-loaded tail exists (last tiles only)
};

template <typename V, typename I, class C>
__device__ __forceinline__ void prepare_tile(const SpmvParams &p, long long t, TileIssue &ti) {
  using A = typename AccOf<V>::type;
  TileMeta mt;
  load_meta<C>(p, t, mt);
  const int nr = mt.r1 - mt.r0, m = mt.k1 - mt.k0;
  const int direct = m > C::CAP_NZ ? 1 : 0;
  const int nseg = direct ? 0 : mt.nseg;
  const Range rr = split_range<4>(mt.r0, nr + 1, (long long)p.nrows + 1);
  Range rv{mt.k0, mt.k0, 0u}, ri{mt.k0, mt.k0, 0u};
  if (!direct && m > 0) {
    rv = split_range<(int)sizeof(V)>(mt.k0, m, p.nnz);
    ri = split_range<(int)sizeof(I)>(mt.k0, m, p.nnz);
  }
  ti.tails = (rr.tb < mt.r1 + 1) || (!direct && m > 0 && (rv.tb < mt.k1 || ri.tb < mt.k1));
  // x-window map in tile-local columns: segment q starts at column lo_q - r0
  // and its slot displacement is e_q = pos_q - (lo_q - r0); unused segments
  // repeat the last displacement and never match (lo = INT_MAX).
  int e[kXSegMax];
#pragma unroll
  for (int q = 0; q < kXSegMax; ++q)
    e[q] = q < nseg ? mt.pos[q] - (mt.lo[q] - mt.r0) : (q > 0 ? e[q - 1] : 0);
  ti.h0 = make_int4(mt.r0, nr, mt.k0, (direct ? kTileDirect : 0) | (nseg > 0 ? kTileStaged : 0));
  ti.h1 = make_int4(static_cast<int>(mt.r0 - rr.a0), static_cast<int>(mt.k0 - rv.a0),
                    static_cast<int>(mt.k0 - ri.a0), e[0]);
  ti.h2 = make_int4(nseg > 1 ? mt.lo[1] - mt.r0 : INT_MAX, nseg > 2 ? mt.lo[2] - mt.r0 : INT_MAX,
                    nseg > 3 ? mt.lo[3] - mt.r0 : INT_MAX, e[1] - e[0]);
  ti.h3 = make_int4(e[2] - e[1], e[3] - e[2], m, nseg);
  ti.rp_a0 = rr.a0; ti.rp_bytes = rr.bulk_bytes;
  ti.v_a0 = rv.a0; ti.v_bytes = rv.bulk_bytes;
  ti.i_a0 = ri.a0; ti.i_bytes = ri.bulk_bytes;
  uint32_t bytes = rr.bulk_bytes + rv.bulk_bytes + ri.bulk_bytes;
#pragma unroll
  for (int q = 0; q < kXSegMax; ++q) {
    const bool on = q < nseg && mt.cnt[q] > 0;
    ti.xsrc[q] = mt.src[q];
    ti.xdst[q] = mt.pos[q] - (mt.lo[q] - mt.src[q]);
    ti.xcnt[q] = on ? mt.cnt[q] : 0;
    bytes += static_cast<uint32_t>(ti.xcnt[q]) * sizeof(A);
  }
  ti.tx_bytes = bytes;
}

// Issues tile j (prepared in ti) into stage j % stages (one lane): wait for
// the stage, write its header, post the byte count, start the bulk copies.
// Returns false when the wait for a free stage gave up.
template <typename V, typename I, class C>
__device__ __forceinline__ bool issue_tile(const SpmvParams &p, unsigned char *smem, uint64_t *full,
                                           uint64_t *empty, TileHdr *hdr, const TileIssue &ti,
                                           int j, RingPos rp, uint64_t pol) {
  using L = Layout<V, I, C>;
  using A = typename L::A;
  const int S = p.stages;
  const int s = rp.s;
  // the stage's previous pass (tile j - S) must have been consumed
  if (j >= S && !mbar_wait_bounded(&empty[s], rp.ph ^ 1u, p.status, p.timeout_ns))
    return false;
  unsigned char *st = smem + (size_t)s * L::STAGE;
  int *rp_s = reinterpret_cast<int *>(st);
  V *v_s = reinterpret_cast<V *>(st + L::OFF_V);
  I *i_s = reinterpret_cast<I *>(st + L::OFF_I);
  A *x_s = reinterpret_cast<A *>(st + L::OFF_X);
  const V *val = static_cast<const V *>(p.val);
  const I *idx = static_cast<const I *>(p.idx);
  const A *x = static_cast<const A *>(p.x);
  if (ti.tails) {  // partial 16-byte blocks at the very end of an array
    const int r0 = ti.h0.x, nr = ti.h0.y, k0 = ti.h0.z, m = ti.h3.z;
    const long long rtb = ti.rp_a0 + ti.rp_bytes / 4;
    if (rtb < r0 + nr + 1) load_tail(rp_s, p.rowptr, ti.rp_a0, rtb, (long long)r0 + nr + 1);
    if (!(ti.h0.w & kTileDirect) && m > 0) {
      const long long vtb = ti.v_a0 + ti.v_bytes / sizeof(V);
      const long long itb = ti.i_a0 + ti.i_bytes / sizeof(I);
      if (vtb < k0 + m) load_tail(v_s, val, ti.v_a0, vtb, (long long)k0 + m);
      if (itb < k0 + m) load_tail(i_s, idx, ti.i_a0, itb, (long long)k0 + m);
    }
  }
  int4 *hv = reinterpret_cast<int4 *>(&hdr[s]);
  hv[0] = ti.h0; hv[1] = ti.h1; hv[2] = ti.h2; hv[3] = ti.h3;
  // No proxy fence: the async copies write only bytes that no generic store
  // of this tile writes, and the consumers' reads of the stage's previous
  // tile are ordered before these copies by the empty barrier.
  mbar_arrive_expect_tx(&full[s], ti.tx_bytes);
  if (ti.rp_bytes) bulk_copy_g2s(rp_s, p.rowptr + ti.rp_a0, ti.rp_bytes, &full[s], pol);
  if (ti.v_bytes) bulk_copy_g2s(v_s, val + ti.v_a0, ti.v_bytes, &full[s], pol);
  if (ti.i_bytes) bulk_copy_g2s(i_s, idx + ti.i_a0, ti.i_bytes, &full[s], pol);
#pragma unroll
  for (int q = 0; q < kXSegMax; ++q)
    if (ti.xcnt[q] > 0)
      bulk_copy_g2s_nohint(x_s + ti.xdst[q], x + ti.xsrc[q],
                           static_cast<uint32_t>(ti.xcnt[q]) * sizeof(A), &full[s]);
  return true;
}

// Producer warp: for each group of 32 consecutive tiles of this CTA, lane i
// prepares tile i (bounds, staging descriptors, copy ranges, header: one
// round of memory latency and the arithmetic for 32 tiles, all lanes in
// parallel); then lane i issues tile i, in tile order.
template <typename V, typename I, class C>
__device__ __forceinline__ void produce(const SpmvParams &p, unsigned char *smem, uint64_t *full,
                                        uint64_t *empty, TileHdr *hdr) {
  const int lane = threadIdx.x & 31;
  const uint64_t pol = l2_policy_evict_first();
  int j = 0;
  RingPos rpos;  // ring position of tile j (the same in every lane)
  bool stop = false;
  while (!stop) {
    const long long tl = (long long)blockIdx.x + (long long)(j + lane) * gridDim.x;
    TileIssue ti;
    if (tl < p.ntiles) prepare_tile<V, I, C>(p, tl, ti);
    for (int i = 0; i < 32; ++i) {
      const long long t = (long long)blockIdx.x + (long long)j * gridDim.x;
      if (t >= p.ntiles) { stop = true; break; }
      int ok = 1;
      if (lane == i) ok = issue_tile<V, I, C>(p, smem, full, empty, hdr, ti, j, rpos, pol) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, i);
      if (!ok) { stop = true; break; }
      ++j;
      rpos.advance(1, p.stages);
    }
  }
  // Do not leave copies in flight: wait (bounded) for the last issued stages.
  const int S = p.stages;
  if (lane == 0)
    for (int q = (j > S ? j - S : 0); q < j; ++q)
      mbar_wait_bounded(&full[q % S], (q / S) & 1, p.status, p.timeout_ns);
}

// ----------------------------------------------------------------------------
// Consumers
// ----------------------------------------------------------------------------

// Tile-local column cl = c - r0 -> shared-memory slot of the staged x window:
// with the (at most four) segments sorted by first column and e_i their
// displacements,
//   slot(cl) = cl + e_0 + [cl >= lo_1] (e_1 - e_0) + [cl >= lo_2] (e_2 - e_1) + ...
// Unused segments have lo = INT_MAX: no branch and no indexing by a runtime
// segment number.  For DA-CSR the tile-local column of row r0 + i is simply
// i + off.  The slot is clamped (one unsigned min) to the x buffer of XL
// elements, so that a column the plan did not see (a call whose pattern is
// not the plan's) reads a wrong value inside the stage instead of shared
// memory outside it.
template <int XL>
struct XMap {
  int d0, lo1, lo2, lo3, dd1, dd2, dd3;
  __device__ __forceinline__ void load(const TileHdr &h) {
    const int4 *hv = reinterpret_cast<const int4 *>(&h);
    const int4 b = hv[1], c = hv[2], d = hv[3];
    d0 = b.w; lo1 = c.x; lo2 = c.y; lo3 = c.z; dd1 = c.w; dd2 = d.x; dd3 = d.y;
  }
  __device__ __forceinline__ int slot(int cl) const { return slot_n<kXSegMax>(cl); }
  // the same when the window has at most NS segments
  template <int NS>
  __device__ __forceinline__ int slot_n(int cl) const {
    int r = cl + d0;
    if (NS > 1) r += cl >= lo1 ? dd1 : 0;
    if (NS > 2) r += cl >= lo2 ? dd2 : 0;
    if (NS > 3) r += cl >= lo3 ? dd3 : 0;
    return static_cast<int>(min(static_cast<unsigned>(r), static_cast<unsigned>(XL - 1)));
  }
};

// y[row] <- alpha acc + beta y0[row] (+ optional fused dot).  PLAIN is the
// common y = A x case: no floating-point operation in the epilogue.
template <bool PLAIN, typename A>
__device__ __forceinline__ void store_row(const SpmvParams &p, int row, A acc, DotAcc<A> &dsum) {
  if (PLAIN) {
    static_cast<A *>(p.y)[row] = acc;
    return;
  }
  A out;
  if (p.ab_mode == 0) {
    out = acc;
  } else if (p.ab_mode == 1) {
    out = static_cast<A>(p.alpha) * acc;
  } else {
    out = fma_acc(static_cast<A>(p.beta), static_cast<const A *>(p.y0)[row],
                  static_cast<A>(p.alpha) * acc);
  }
  static_cast<A *>(p.y)[row] = out;
  if (p.dot_w)
    dsum.add(static_cast<const A *>(p.dot_w)[row], out);
  else if (p.dot_self)
    dsum.add(out, out);
}

// Pointers of a tile's values / indices / staged x (element 0 = entry k0).
template <typename V, typename I, class C>
struct TileView {
  using A = typename AccOf<V>::type;
  const int *rp;  // rp[lr] = rowptr[r0 + lr]
  const V *vs;
  const I *is;
  const A *xs;    // staged x window (valid when nseg > 0)
  __device__ __forceinline__ void init(const SpmvParams &p, unsigned char *smem, const TileHdr &h,
                                       int s) {
    using L = Layout<V, I, C>;
    unsigned char *st = smem + (size_t)s * L::STAGE;
    rp = reinterpret_cast<const int *>(st) + h.rp_sh;
    const bool direct = (h.flags & kTileDirect) != 0;
    vs = direct ? static_cast<const V *>(p.val) + h.k0 : reinterpret_cast<const V *>(st + L::OFF_V) + h.v_sh;
    is = direct ? static_cast<const I *>(p.idx) + h.k0 : reinterpret_cast<const I *>(st + L::OFF_I) + h.i_sh;
    xs = reinterpret_cast<const A *>(st + L::OFF_X);
  }
};

// x[c] read from global memory with c clamped into [0, ncols): a column
// outside x (invalid input, e.g. offsets that did not fit their type) reads
// a wrong entry of x instead of memory outside it.  One unsigned min.
template <typename A>
__device__ __forceinline__ A x_global(const A *xg, int c, int ncols) {
  return ldg(xg + min(static_cast<unsigned>(c), static_cast<unsigned>(ncols - 1)));
}

// x value of column c of a tile starting at row r0: from the staged window or
// gathered from global memory.
template <typename A, class XM>
__device__ __forceinline__ A x_at(const A *xg, const A *xs, const XM &xm, bool staged, int c,
                                  int r0, int ncols) {
  return staged ? xs[xm.slot(c - r0)] : x_global(xg, c, ncols);
}

// Mode 0 -------------------------------------------------------------------
// A tile that is not fully staged (entries too many for a stage, or no x
// window): thread i computes rows i, i + NT, ... of the tile, reading what is
// not in shared memory from global memory.
template <bool PLAIN, typename V, typename I, class C>
__device__ __noinline__ void rows_general(const SpmvParams &p, unsigned char *smem,
                                          const TileHdr &h, int s, int ctid, DotAcc<typename AccOf<V>::type> &dsum) {
  using A = typename AccOf<V>::type;
  constexpr bool DA = sizeof(I) < 4;  // int16 / int8 offsets
  TileView<V, I, C> tv;
  tv.init(p, smem, h, s);
  XMap<Layout<V, I, C>::X_ELEMS> xm;
  const bool staged = (h.flags & kTileStaged) != 0;
  if (staged) xm.load(h);
  const A *xg = static_cast<const A *>(p.x);
  for (int lr = ctid; lr < h.nr; lr += C::NT) {
    const int row = h.r0 + lr;
    A acc = 0;
    for (int q = tv.rp[lr] - h.k0; q < tv.rp[lr + 1] - h.k0; ++q)
      acc = fma_acc(to_acc(tv.vs[q]),
                    x_at(xg, tv.xs, xm, staged, static_cast<int>(tv.is[q]) + (DA ? row : 0), h.r0,
                         p.ncols),
                    acc);
    store_row<PLAIN>(p, row, acc, dsum);
  }
}

// One row per thread.  For a fully staged tile (the common case) every
// operand comes from shared memory through shared-memory pointers: the warp
// loads its rows' values and x into registers, hands the stage back, then
// runs the FMA chains, so the warps of a CTA do not wait for each other.
// Rows longer than U entries finish from the stage before it is released.
// NS = 0: the plan stages no x window; x is read from global memory (L1 /
// L2) in the same register-batched way -- for stencil-like rows the lanes of
// a warp read consecutive x entries at each offset, and no column -> slot
// map is computed per entry.
template <bool PLAIN, typename V, typename I, class C, int NS>
__device__ __forceinline__ void consume_rows(const SpmvParams &p, unsigned char *smem,
                                             uint64_t *full, uint64_t *empty, const TileHdr *hdr,
                                             int ctid, DotAcc<typename AccOf<V>::type> &dsum) {
  using L = Layout<V, I, C>;
  using A = typename AccOf<V>::type;
  constexpr bool DA = sizeof(I) < 4;  // int16 / int8 offsets
  constexpr int U = C::CAP_NZ / C::TILE_ROWS;
  const int lane = threadIdx.x & 31;
  RingPos rpos;
  for (long long t = blockIdx.x; t < p.ntiles; t += gridDim.x, rpos.advance(1, p.stages)) {
    const int s = rpos.s;
    if (!mbar_wait_bounded(&full[s], rpos.ph, p.status, p.timeout_ns)) return;
    const int4 *hv = reinterpret_cast<const int4 *>(&hdr[s]);
    const int4 h0 = hv[0];  // r0, nr, k0, flags
    if (NS > 0 ? h0.w != kTileStaged : (h0.w & kTileDirect) != 0) {
      rows_general<PLAIN, V, I, C>(p, smem, hdr[s], s, ctid, dsum);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      continue;
    }
    const int4 h1 = hv[1];  // rp_sh, v_sh, i_sh, d0
    XMap<L::X_ELEMS> xm;
    if (NS > 0) xm.load(hdr[s]);
    unsigned char *st = smem + (size_t)s * L::STAGE;
    const int *rp = reinterpret_cast<const int *>(st) + h1.x;
    const V *vs = reinterpret_cast<const V *>(st + L::OFF_V) + h1.y;
    const I *is = reinterpret_cast<const I *>(st + L::OFF_I) + h1.z;
    const A *xs = reinterpret_cast<const A *>(st + L::OFF_X);
    const A *xg = static_cast<const A *>(p.x);
    const int r0 = h0.x, nr = h0.y, k0 = h0.z;
    auto xval = [&](int cl) -> A {
      if constexpr (NS == 0) return x_global(xg, r0 + cl, p.ncols);
      else return xs[xm.template slot_n<NS>(cl)];
    };
    // lane ei of the E lanes of a row takes the row's entries ei, ei + E, ...
    constexpr int E = C::E;
    constexpr int UL = U / E;  // entries per lane kept in registers
    const int ei = ctid % E;
    // the thread's RPT rows: operands of all of them into registers first
    A av[C::RPT][UL], xv[C::RPT][UL];
    int b[C::RPT], cnt[C::RPT];
    bool fits = true;
#pragma unroll
    for (int rr = 0; rr < C::RPT; ++rr) {
      const int lr = ctid / E + rr * (C::NT / E);
      b[rr] = 0;
      cnt[rr] = 0;
      if (lr < nr) {
        b[rr] = rp[lr] - k0;
        cnt[rr] = rp[lr + 1] - k0 - b[rr];
      }
#pragma unroll
      for (int u = 0; u < UL; ++u) {
        const int q = ei + u * E;
        if (q < cnt[rr]) {
          const int cl = DA ? lr + static_cast<int>(is[b[rr] + q])
                            : static_cast<int>(is[b[rr] + q]) - r0;
          av[rr][u] = to_acc(vs[b[rr] + q]);
          xv[rr][u] = xval(cl);
        }
      }
      fits = fits && cnt[rr] <= U;
    }
    // every row of this warp in registers: hand the stage back at once
    fits = __all_sync(0xffffffffu, fits);
    if (fits) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
#pragma unroll
    for (int rr = 0; rr < C::RPT; ++rr) {
      const int lr = ctid / E + rr * (C::NT / E);
      A acc = 0;
#pragma unroll
      for (int u = 0; u < UL; ++u)
        if (ei + u * E < cnt[rr]) acc = fma_acc(av[rr][u], xv[rr][u], acc);
      for (int q = ei + UL * E; q < cnt[rr]; q += E) {  // rows longer than U
        const int cl = DA ? lr + static_cast<int>(is[b[rr] + q])
                          : static_cast<int>(is[b[rr] + q]) - r0;
        acc = fma_acc(to_acc(vs[b[rr] + q]), xval(cl), acc);
      }
#pragma unroll
      for (int o = 1; o < E; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lr < nr && ei == 0) store_row<PLAIN>(p, r0 + lr, acc, dsum);
    }
    if (!fits) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
}

// Mode 1 -------------------------------------------------------------------
template <bool PLAIN, typename V, typename I, class C>
__device__ __forceinline__ void tile_slices(const SpmvParams &p, const TileHdr &h,
                                            const TileView<V, I, C> &tv, int ctid,
                                            typename AccOf<V>::type *carry,
                                            typename AccOf<V>::type *rowsum, DotAcc<typename AccOf<V>::type> &dsum) {
  using A = typename AccOf<V>::type;
  constexpr bool DA = sizeof(I) < 4;  // int16 / int8 offsets
  constexpr int G = 8;
  const A *xg = static_cast<const A *>(p.x);
  const int *rp = tv.rp;
  const int nr = h.nr, m = h.m, k0 = h.k0;
  const bool staged = (h.flags & kTileStaged) != 0;
  XMap<Layout<V, I, C>::X_ELEMS> xm;
  if (staged) xm.load(h);
  const int K = m > 0 ? (m + C::NT - 1) / C::NT : 0;
  const int s = ctid * K;
  const int e = min(s + K, m);
  const bool has = s < m;
  const int last = m > 0 ? (m - 1) / K : 0;
  int pend_row = -1;
  A pend_acc = 0;
  if (has || ctid == last) {
    int lo = 0, hi = nr;  // first row whose start is >= s
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (rp[mid] - k0 >= s) hi = mid; else lo = mid + 1;
    }
    bool cont = (s > 0) && (lo == nr || rp[lo] - k0 > s);
    int cr = cont ? lo - 1 : lo;
    int cend = (cr < nr) ? rp[cr + 1] - k0 : m;
    A acc = 0;
    for (int q = s; q < e; q += G) {
      A av[G], xv[G];
      int tcr = cr, tend = cend;
#pragma unroll
      for (int u = 0; u < G; ++u) {
        if (q + u < e) {
          while (tend <= q + u) { ++tcr; tend = rp[tcr + 1] - k0; }
          const int c = static_cast<int>(tv.is[q + u]) + (DA ? h.r0 + tcr : 0);
          av[u] = to_acc(tv.vs[q + u]);
          xv[u] = x_at(xg, tv.xs, xm, staged, c, h.r0, p.ncols);
        }
      }
#pragma unroll
      for (int u = 0; u < G; ++u) {
        if (q + u < e) {
          while (cend <= q + u) {
            if (cont) { pend_row = cr; pend_acc = acc; } else { rowsum[cr] = acc; }
            acc = 0; cont = false; ++cr; cend = rp[cr + 1] - k0;
          }
          acc = fma_acc(av[u], xv[u], acc);
        }
      }
    }
    if (has) {
      if (cend == e) {
        if (cont) { pend_row = cr; pend_acc = acc; } else { rowsum[cr] = acc; }
        ++cr;
        if (e == m)
          for (; cr < nr; ++cr) rowsum[cr] = 0;  // empty rows at the tile end
      } else {
        carry[ctid] = acc;
      }
    } else {
      for (int r = 0; r < nr; ++r) rowsum[r] = 0;  // tile without entries
    }
  }
  named_bar_sync(1, C::NT);
  if (pend_row >= 0) {
    const int a = (rp[pend_row] - k0) / K;
    A tot = carry[a];
    for (int jj = a + 1; jj < ctid; ++jj) tot += carry[jj];
    rowsum[pend_row] = tot + pend_acc;
  }
  named_bar_sync(1, C::NT);
  for (int lr = ctid; lr < nr; lr += C::NT) store_row<PLAIN>(p, h.r0 + lr, rowsum[lr], dsum);
}

// ----------------------------------------------------------------------------
// Kernel
// ----------------------------------------------------------------------------
template <bool PLAIN, typename V, typename I, class C, int NS>
__global__ void __launch_bounds__(C::NT + 32, C::MINB) k_spmv(const SpmvParams p) {
  using A = typename AccOf<V>::type;
  using L = Layout<V, I, C>;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *ctrl = smem + (size_t)p.stages * L::STAGE;
  uint64_t *full = reinterpret_cast<uint64_t *>(ctrl + L::C_FULL);
  uint64_t *empty = reinterpret_cast<uint64_t *>(ctrl + L::C_EMPTY);
  TileHdr *hdr = reinterpret_cast<TileHdr *>(ctrl + L::C_HDR);
  double *red = reinterpret_cast<double *>(ctrl + L::C_RED);
  A *carry = reinterpret_cast<A *>(ctrl + L::CTRL + L::M1_CARRY);
  A *rowsum = reinterpret_cast<A *>(ctrl + L::CTRL + L::M1_ROWSUM);
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::NT / 32);
    }
    fence_mbar_init();
  }
  __syncthreads();
  // shared-memory set-up above overlaps the previous kernel of the stream;
  // global memory only after it has completed
  grid_dependency_wait();
  grid_launch_dependents();
  if (tid < 32) {
    produce<V, I, C>(p, smem, full, empty, hdr);
    return;
  }
  const int ctid = tid - 32;
  DotAcc<A> dacc;
  if (p.mode == 0) {
    consume_rows<PLAIN, V, I, C, NS>(p, smem, full, empty, hdr, ctid, dacc);
  } else {
    RingPos rpos;
    int j = 0;  // tile count: the slice scratch is double-buffered by its parity
    for (long long t = blockIdx.x; t < p.ntiles;
         t += gridDim.x, rpos.advance(1, p.stages), ++j) {
      const int s = rpos.s;
      const bool got = mbar_wait_bounded(&full[s], rpos.ph, p.status, p.timeout_ns);
      // the consumers synchronise inside a tile, so they give up together
      if (named_bar_or(2, C::NT, !got)) break;
      const TileHdr &h = hdr[s];
      TileView<V, I, C> tv;
      tv.init(p, smem, h, s);
      tile_slices<PLAIN, V, I, C>(p, h, tv, ctid, carry + (j & 1) * C::NT,
                                  rowsum + (j & 1) * C::CAP_ROWS, dacc);
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(&empty[s]);
    }
  }
  if (p.dot_partials) {
    double dsum = dacc.value();
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if ((ctid & 31) == 0) red[ctid >> 5] = dsum;
    named_bar_sync(3, C::NT);
    if (ctid == 0) {
      double tot = 0.0;
      for (int w = 0; w < C::NT / 32; ++w) tot += red[w];
      p.dot_partials[blockIdx.x] = tot;
    }
  }
}

}  // namespace spmvk
}  // namespace damn
