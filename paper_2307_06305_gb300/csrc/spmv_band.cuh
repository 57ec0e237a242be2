// Band mode of the SpMV engine (Section 4, Listing 2 for banded matrices):
// y <- alpha A x + beta y with x streamed through a shared-memory ring.
// Included by the SpMV instantiation units only.
//
// In DA-CSR an entry of row r reads x[r + off] with |off| <= w (the
// bandwidth of Eq. (2)), so consecutive rows read overlapping windows of x.
// Band mode exploits this directly:
//
//  * every persistent CTA owns a contiguous chunk of the plan's balanced
//    tiles (rows + entries), so its tiles walk down the band in order;
//  * x lives in a ring of W elements in shared memory, column c in slot
//    c mod W.  For each tile the producer warp copies only the columns beyond
//    the ring's current end (cp.async.bulk, like the matrix streams), so each
//    element of x crosses from L2 into the SM about once per CTA instead of
//    once per stored entry;
//  * a tile whose columns are not all present in the ring (a band wider than
//    the ring allows, an outlier entry far from the diagonal) reads x from
//    global memory instead, with all of a thread's gathers issued together.
//
// The consumers are G groups of NT threads; group g computes the chunk's
// tiles g, g + G, ... so that the groups drift apart in phase and one
// group's FMAs overlap the other's loads and barriers.  Inside a tile every
// thread takes a contiguous slice of ceil(m / NT) entries (so every warp-wide
// FMA carries a full warp of entries whatever the row lengths), accumulates
// each row's part of its slice in stored order with FMA, and a row crossing
// slices is finished by the thread holding its last entry, adding the
// earlier slices' partial sums left to right.  Summation order depends only
// on the tile partition and NT, so CSR-32, DA-CSR-16 and DA-CSR-8 give
// bitwise equal results under one plan.
//
// Ring validity.  The producer keeps [vrun, F): the columns present in the
// ring (a contiguous run, F its end).  Tile j needs [lo_j, hi_j].  Loading
// [max(F, lo_j), hi_j + 1) overwrites the slots of columns below
// F' - W (F' the new end); that is allowed only when no tile still in flight
// -- the S - 1 tiles issued before j -- needs them, and tile j's own columns
// must lie in [max(vrun', F' - W), F').  Otherwise tile j gathers x and the
// ring is left as it was.  Every wait is bounded as in the other modes.
#pragma once

#include "spmv_kernel.cuh"

namespace damn {
namespace spmvk {

constexpr int kBandRing = 4;  // tile flag: x read from the ring

// G consumer groups of NT threads; a stage holds up to CAP_NZ entries and
// CAP_ROWS rows; the x ring has W elements (a power of two).
template <int NT_, int G_, int CAP_NZ_, int CAP_ROWS_, int W_>
struct BCfg {
  static constexpr int NT = NT_, G = G_, CAP_NZ = CAP_NZ_, CAP_ROWS = CAP_ROWS_, W = W_;
  static constexpr bool PERM = false;  // no row permutation in the stages
  static constexpr int CH = 8;  // entries of a slice handled per unrolled step
  static_assert((W & (W - 1)) == 0, "ring size must be a power of two");
  static_assert(G * NT / 32 <= 32, "too many consumer warps");
  static_assert(2 * G <= 8, "two named barriers per group, ids 1 .. 2G, below the dot barrier");
};

// Four groups of 128 threads (a slice of about 13 entries per thread for
// rows of a dozen entries, so that a row rarely spans more than two slices
// and the FP64 adds of slice carries stay few), 2048-entry stages; FP64: an
// 8192-element ring (64 KB, bands up to a few thousand columns each side);
// FP32 / BF16 values (FP32 x): a 16384-element ring (64 KB).  (Stages of 2560
// entries, tried: no faster for bands up to 1000 wide and much slower for
// wide bands whose x is gathered from global memory.)
using CfgBand64 = BCfg<128, 4, 2048, 512, 8192>;
using CfgBand32 = BCfg<128, 4, 2048, 512, 16384>;

// Sorted-rows band mode: tiles of NT rows, one row per consumer thread, the
// tile's rows taken in order of decreasing length (a permutation computed by
// the plan), x through the same ring; G groups of NT threads take turns on
// the tiles, as in band mode.  Tiles of 192 rows in stages of up to 3584
// entries (four or more stages in flight); FP64: a 4096-element ring, FP32
// x: 8192 elements (32 KB each).
template <int NT_, int G_, int CAP_NZ_, int W_>
struct RCfg {
  static constexpr int NT = NT_, G = G_, CAP_NZ = CAP_NZ_, CAP_ROWS = NT_, W = W_;
  static constexpr bool PERM = true;  // the tile's row permutation in each stage
  static constexpr int CH = 16;     // entries loaded ahead per row (even)
  static constexpr int LONG = 128;  // rows longer than this are shared by a warp
  static_assert((W & (W - 1)) == 0, "ring size must be a power of two");
  static_assert(NT % 32 == 0 && NT <= 1024, "whole warps, at most 1024 rows per tile");
};
using CfgSorted64 = RCfg<192, 2, 3584, 4096>;
using CfgSorted32 = RCfg<192, 2, 3584, 8192>;

struct __align__(16) BandHdr {
  int r0, nr, k0, m;
  int flags, rp_sh, v_sh, i_sh;
  int kd;          // entries per consumer slice: ceil(m / NT), made odd
  unsigned kdm;    // ceil(2^32 / kd): a / kd as a multiply-high (DivK)
  int pad[2];
};

template <typename V, typename I, class C>
struct BandLayout {
  using A = typename AccOf<V>::type;
  static constexpr int EV = 16 / (int)sizeof(V), EI = 16 / (int)sizeof(I), EX = 16 / (int)sizeof(A);
  static constexpr size_t RP_BYTES = align_up((C::CAP_ROWS + 1 + 8) * 4, 128);
  static constexpr size_t V_BYTES = align_up((C::CAP_NZ + 2 * EV) * sizeof(V), 128);
  static constexpr size_t I_BYTES = align_up((C::CAP_NZ + 2 * EI) * sizeof(I), 128);
  // row permutation of a sorted-rows tile (uint16 per row)
  static constexpr size_t P_BYTES = C::PERM ? align_up((C::CAP_ROWS + 8) * 2, 128) : 0;
  static constexpr size_t OFF_V = RP_BYTES, OFF_I = RP_BYTES + V_BYTES,
                          OFF_P = RP_BYTES + V_BYTES + I_BYTES;
  static constexpr size_t STAGE = RP_BYTES + V_BYTES + I_BYTES + P_BYTES;
  static constexpr size_t RING_BYTES = (size_t)C::W * sizeof(A);
  static constexpr size_t C_FULL = 0;
  static constexpr size_t C_EMPTY = kMaxStages * 8;
  static constexpr size_t C_HDR = 2 * kMaxStages * 8;
  static constexpr size_t C_RED = align_up(C_HDR + kMaxStages * sizeof(BandHdr), 16);
  static constexpr size_t CTRL = align_up(C_RED + (C::G * C::NT / 32) * sizeof(double), 128);
  // per consumer group: start rows of the slices, slice carries, row sums
  static constexpr size_t G_SROW = 0;
  static constexpr size_t G_CARRY = align_up((C::NT + 1) * 4, 16);
  static constexpr size_t G_ROWSUM = align_up(G_CARRY + C::NT * sizeof(A), 16);
  static constexpr size_t G_BYTES = align_up(G_ROWSUM + C::CAP_ROWS * sizeof(A), 128);
  static size_t total(int stages) {
    return stages * STAGE + RING_BYTES + CTRL + C::G * G_BYTES;
  }
};

// Tiles [t0, t1) of the chunk of CTA b out of nb (balanced: the plan's tiles
// are balanced on rows + entries).
__device__ __forceinline__ void band_chunk(long long ntiles, int b, int nb, long long &t0,
                                           long long &t1) {
  t0 = ntiles * b / nb;
  t1 = ntiles * (b + 1) / nb;
}

// ----------------------------------------------------------------------------
// Producer
// ----------------------------------------------------------------------------
struct BandIssue {
  int4 h0;                 // r0, nr, k0, m
  int4 h1;                 // flags (entries direct), rp_sh, v_sh, i_sh
  int4 h2;                 // kd, kdm (for consumer groups of NT threads)
  long long rp_a0, v_a0, i_a0;
  uint32_t rp_bytes, v_bytes, i_bytes, p_bytes;
  int lo, hi;              // the tile's column range (lo > hi: none known)
  int minlo;               // smallest lo of the tiles issued just before (in flight)
  int tails;
};

template <typename V, typename I, class C>
__device__ __forceinline__ void band_prepare(const SpmvParams &p, long long t, long long t0,
                                             BandIssue &bi) {
  const int2 b0 = __ldg(p.bounds + t), b1 = __ldg(p.bounds + t + 1);
  const int r0 = b0.x, k0 = b0.y, r1 = b1.x, k1 = b1.y;
  const int nr = r1 - r0, m = k1 - k0;
  const int direct = (m > C::CAP_NZ) ? 1 : 0;
  const Range rr = split_range<4>(r0, nr + 1, (long long)p.nrows + 1);
  Range rv{k0, k0, 0u}, ri{k0, k0, 0u};
  if (!direct && m > 0) {
    rv = split_range<(int)sizeof(V)>(k0, m, p.nnz);
    ri = split_range<(int)sizeof(I)>(k0, m, p.nnz);
  }
  bi.tails = (rr.tb < r1 + 1) || (!direct && m > 0 && (rv.tb < k1 || ri.tb < k1));
  bi.h0 = make_int4(r0, nr, k0, m);
  {
    // an odd slice length: thread t's loads of entry t kd + u then fall in
    // distinct shared-memory banks for 8-, 4- and 2-byte elements (an even
    // kd, 16 say, would put every thread of a warp on one bank)
    const int kd = m > 0 ? ((m + C::NT - 1) / C::NT) | 1 : 1;
    bi.h2 = make_int4(kd, static_cast<int>(0xFFFFFFFFu / static_cast<unsigned>(kd) + 1u), 0, 0);
  }
  bi.h1 = make_int4(direct ? kTileDirect : 0, static_cast<int>(r0 - rr.a0),
                    static_cast<int>(k0 - rv.a0), static_cast<int>(k0 - ri.a0));
  bi.rp_a0 = rr.a0; bi.rp_bytes = rr.bulk_bytes;
  bi.v_a0 = rv.a0; bi.v_bytes = rv.bulk_bytes;
  bi.i_a0 = ri.a0; bi.i_bytes = ri.bulk_bytes;
  // the permutation array is padded to whole tiles: copy whole 16-byte blocks
  // (stages of a layout without a permutation buffer never receive one)
  bi.p_bytes = (C::PERM && p.perm) ? static_cast<uint32_t>(((nr + 7) & ~7) * 2) : 0u;
  bi.lo = INT_MAX; bi.hi = INT_MIN; bi.minlo = INT_MAX;
  if (p.colrange && !direct && m > 0) {
    const int2 cr = __ldg(p.colrange + t);
    bi.lo = cr.x; bi.hi = cr.y;
    for (int k = 1; k < p.stages; ++k)
      if (t - k >= t0) bi.minlo = min(bi.minlo, __ldg(&p.colrange[t - k].x));
  }
}

// Issues one tile (the calling lane only); F / vrun: the ring's run, updated
// when the tile's x comes from the ring.  Returns false when the wait for a
// free stage gave up.
template <typename V, typename I, class C>
__device__ __forceinline__ bool band_issue(const SpmvParams &p, unsigned char *smem,
                                           typename AccOf<V>::type *ring, uint64_t *full,
                                           uint64_t *empty, BandHdr *hdr, const BandIssue &bi,
                                           long long j, RingPos rp, uint64_t pol, int &F,
                                           int &vrun) {
  using L = BandLayout<V, I, C>;
  using A = typename L::A;
  constexpr int EX = L::EX;
  const int S = p.stages;
  const int s = rp.s;
  // the stage's previous pass (tile j - S) must have been consumed
  if (j >= S && !mbar_wait_bounded(&empty[s], rp.ph ^ 1u, p.status, p.timeout_ns)) return false;
  unsigned char *st = smem + (size_t)s * L::STAGE;
  int *rp_s = reinterpret_cast<int *>(st);
  V *v_s = reinterpret_cast<V *>(st + L::OFF_V);
  I *i_s = reinterpret_cast<I *>(st + L::OFF_I);
  const V *val = static_cast<const V *>(p.val);
  const I *idx = static_cast<const I *>(p.idx);
  const A *x = static_cast<const A *>(p.x);
  const int r0 = bi.h0.x, nr = bi.h0.y, k0 = bi.h0.z, m = bi.h0.w;
  if (bi.tails) {
    const long long rtb = bi.rp_a0 + bi.rp_bytes / 4;
    if (rtb < r0 + nr + 1) load_tail(rp_s, p.rowptr, bi.rp_a0, rtb, (long long)r0 + nr + 1);
    if (!(bi.h1.x & kTileDirect) && m > 0) {
      const long long vtb = bi.v_a0 + bi.v_bytes / sizeof(V);
      const long long itb = bi.i_a0 + bi.i_bytes / sizeof(I);
      if (vtb < k0 + m) load_tail(v_s, val, bi.v_a0, vtb, (long long)k0 + m);
      if (itb < k0 + m) load_tail(i_s, idx, bi.i_a0, itb, (long long)k0 + m);
    }
  }
  // x: extend the ring's run to cover [lo, hi] if that keeps every column
  // of the tiles in flight
  const int x_full = p.ncols & ~(EX - 1);  // columns in whole 16-byte blocks
  int flags = bi.h1.x;
  int xl = 0, xn = 0;
  if (bi.lo <= bi.hi && bi.lo >= 0 && bi.hi < x_full) {
    const int lo_a = bi.lo & ~(EX - 1);
    const int hi_a = (bi.hi + EX) & ~(EX - 1);  // end of the aligned block holding hi
    int start, vn;
    if (F < 0 || lo_a >= F) { start = lo_a; vn = lo_a; } else { start = F; vn = vrun; }
    const int fn = max(F, hi_a);
    if (bi.lo >= max(vn, fn - C::W) && bi.minlo >= fn - C::W) {
      flags |= kBandRing;
      xl = start;
      xn = fn - start;
      F = fn;
      vrun = vn;
    }
  }
  int4 *hv = reinterpret_cast<int4 *>(&hdr[s]);
  hv[0] = bi.h0;
  hv[1] = make_int4(flags, bi.h1.y, bi.h1.z, bi.h1.w);
  hv[2] = bi.h2;
  const uint32_t tx =
      bi.rp_bytes + bi.v_bytes + bi.i_bytes + bi.p_bytes + static_cast<uint32_t>(xn) * sizeof(A);
  mbar_arrive_expect_tx(&full[s], tx);
  if (bi.p_bytes)
    bulk_copy_g2s(st + L::OFF_P, p.perm + r0, bi.p_bytes, &full[s], pol);
  if (bi.rp_bytes) bulk_copy_g2s(rp_s, p.rowptr + bi.rp_a0, bi.rp_bytes, &full[s], pol);
  if (bi.v_bytes) bulk_copy_g2s(v_s, val + bi.v_a0, bi.v_bytes, &full[s], pol);
  if (bi.i_bytes) bulk_copy_g2s(i_s, idx + bi.i_a0, bi.i_bytes, &full[s], pol);
  if (xn > 0) {
    const int slot = xl & (C::W - 1);
    const int n1 = min(xn, C::W - slot);
    bulk_copy_g2s_nohint(ring + slot, x + xl, static_cast<uint32_t>(n1) * sizeof(A), &full[s]);
    if (xn > n1)
      bulk_copy_g2s_nohint(ring, x + xl + n1, static_cast<uint32_t>(xn - n1) * sizeof(A), &full[s]);
  }
  return true;
}

// Producer warp: lane i prepares tile i of each group of 32 (in parallel),
// then the lanes issue in tile order, handing the ring state on by shuffle.
template <typename V, typename I, class C>
__device__ __forceinline__ void band_produce(const SpmvParams &p, unsigned char *smem,
                                             typename AccOf<V>::type *ring, uint64_t *full,
                                             uint64_t *empty, BandHdr *hdr, long long t0,
                                             long long t1) {
  const int lane = threadIdx.x & 31;
  const uint64_t pol = l2_policy_evict_first();
  int F = -1, vrun = 0;
  long long j = 0;
  RingPos rpos;  // ring position of tile j (the same in every lane)
  bool stop = false;
  while (!stop && t0 + j < t1) {
    BandIssue bi;
    if (t0 + j + lane < t1) band_prepare<V, I, C>(p, t0 + j + lane, t0, bi);
    for (int i = 0; i < 32; ++i) {
      if (t0 + j >= t1) { stop = true; break; }
      int ok = 1;
      if (lane == i)
        ok = band_issue<V, I, C>(p, smem, ring, full, empty, hdr, bi, j, rpos, pol, F, vrun);
      ok = __shfl_sync(0xffffffffu, ok, i);
      F = __shfl_sync(0xffffffffu, F, i);
      vrun = __shfl_sync(0xffffffffu, vrun, i);
      if (!ok) { stop = true; break; }
      ++j;
      rpos.advance(1, p.stages);
    }
  }
  // no copies left in flight: wait (bounded) for the last issued stages
  const int S = p.stages;
  if (lane == 0)
    for (long long q = (j > S ? j - S : 0); q < j; ++q)
      mbar_wait_bounded(&full[q % S], static_cast<uint32_t>((q / S) & 1), p.status, p.timeout_ns);
}

// ----------------------------------------------------------------------------
// Consumers
// ----------------------------------------------------------------------------

// v, or +0 when z: a bit mask, so that no branch separates the lanes.
__device__ __forceinline__ double zero_if(bool z, double v) {
  return __longlong_as_double(__double_as_longlong(v) & (z ? 0ll : -1ll));
}
__device__ __forceinline__ float zero_if(bool z, float v) {
  return __int_as_float(__float_as_int(v) & (z ? 0 : -1));
}

// Division by the tile's slice length Kd (tile-uniform): a / Kd as a
// multiply-high by M = ceil(2^32 / Kd).  The error a (M Kd - 2^32) / (Kd 2^32)
// is below a / 2^32, so the quotient is exact while a * Kd < 2^32 -- always
// for tiles of fewer than 2^20 entries (Kd < 2^12); larger tiles divide.
struct DivK {
  int d;
  unsigned m;
  bool fast;
  __device__ __forceinline__ void init(int d_, int tile_m) {
    d = d_;
    m = 0xFFFFFFFFu / static_cast<unsigned>(d_) + 1u;
    fast = tile_m < (1 << 20);
  }
  // from the tile header (the producer did the division)
  __device__ __forceinline__ void init(const BandHdr &h) {
    d = h.kd;
    m = h.kdm;
    fast = h.m < (1 << 20);
  }
  __device__ __forceinline__ int div(int a) const {
    if (d == 1) return a;
    return fast ? static_cast<int>(__umulhi(static_cast<unsigned>(a), m)) : a / d;
  }
};

// Step 1 of a tile: the row holding the first entry of every thread's slice
// (srow[t], written by the thread of that row), and the results of empty
// rows.  Kd = ceil(m / NT) entries per slice.
template <bool PLAIN, class C, typename A>
__device__ __forceinline__ void band_start_rows(const SpmvParams &p, const BandHdr &h,
                                                const int *rp, int *srow, A *rowsum, int gtid,
                                                DotAcc<A> &dsum) {
  const int nr = h.nr, k0 = h.k0;
  const int Kd = h.kd;
  DivK dk;
  dk.init(h);
  for (int lr = gtid; lr < nr; lr += C::NT) {
    const int b = rp[lr] - k0, e = rp[lr + 1] - k0;
    if (e > b) {
      for (int t = dk.div(b + Kd - 1); t * Kd < e; ++t) srow[t] = lr;
    } else {
      rowsum[lr] = A(0);
    }
  }
}

// Steps 2 and 3 of a tile: the thread's slice, then (after the group
// barrier) the rows it finishes from earlier slices' carries.
//
// The row of each entry comes from the ends of the next NB rows, preloaded
// once: row(q) = row + #{i : q >= end_i}, compares and adds without a
// branch.  A slice chunk that holds more than NB - 1 row ends (rows of one
// or two entries) takes a loop instead.  Rows finished inside the slice are
// stored by predicated stores; the first row of the slice, if it began in an
// earlier slice, is finished after the barrier from the carries.
template <bool PLAIN, typename V, typename I, class C>
__device__ __forceinline__ void band_tile(const SpmvParams &p, const BandHdr &h, const int *rp,
                                          const V *vs, const I *is,
                                          const typename AccOf<V>::type *ring, const int *srow,
                                          typename AccOf<V>::type *carry,
                                          typename AccOf<V>::type *rowsum, int gtid, int bar,
                                          uint64_t *empty_s,
                                          DotAcc<typename AccOf<V>::type> &dsum) {
  using A = typename AccOf<V>::type;
  constexpr bool DA = sizeof(I) < 4;  // int16 / int8 offsets
  constexpr int CH = C::CH;
  constexpr int NB = 4;
  const A *xg = static_cast<const A *>(p.x);
  const int r0 = h.r0, m = h.m, k0 = h.k0, nr = h.nr;
  const bool from_ring = (h.flags & kBandRing) != 0;
  const int Kd = h.kd;
  const int s0 = gtid * Kd, e0 = min(s0 + Kd, m);
  int pend_row = -1, pend_b = 0;
  A pend_acc = 0;
  if (s0 < e0) {
    int row = srow[gtid];
    const int rb = rp[row] - k0;
    const bool open = rb < s0;  // the row began in an earlier slice
    bool first = true;
    A acc = 0;
    int eb[NB];  // ends of rows row, row + 1, ...
#pragma unroll
    for (int i = 0; i < NB; ++i) eb[i] = row + 1 + i <= nr ? rp[row + 1 + i] - k0 : INT_MAX;
    for (int q = s0; q < e0; q += CH) {
      const int qe = min(q + CH, e0);
      int lrow[CH];
      if (qe - 1 < eb[NB - 1]) {
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          int d = 0;
#pragma unroll
          for (int i = 0; i < NB - 1; ++i) d += (q + u >= eb[i]) ? 1 : 0;
          lrow[u] = row + d;
        }
      } else {  // many short rows in this chunk
        int rr = row, re = eb[0];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          if (q + u < qe) {
            // (rr + 1 < nr: a non-monotone rowptr cannot walk out of the stage)
            while (q + u >= re && rr + 1 < nr) { ++rr; re = rp[rr + 1] - k0; }
          }
          lrow[u] = rr;
        }
      }
      A av[CH], xv[CH];
      // one loop per x source (the choice is the tile's): a per-entry select
      // would issue both loads under predicates
      if (from_ring) {
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          if (q + u < qe) {
            const int c = DA ? r0 + lrow[u] + static_cast<int>(is[q + u]) : static_cast<int>(is[q + u]);
            av[u] = to_acc(vs[q + u]);
            xv[u] = ring[c & (C::W - 1)];
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          if (q + u < qe) {
            const int c = DA ? r0 + lrow[u] + static_cast<int>(is[q + u]) : static_cast<int>(is[q + u]);
            av[u] = to_acc(vs[q + u]);
            xv[u] = x_global(xg, c, p.ncols);
          }
        }
      }
      // The FMA first, for every lane at once (the accumulator reset by a
      // mask, not a branch); a row that ended just before this entry goes to
      // the tile's row sums by a predicated shared-memory store (the first
      // row of the slice, when it began in an earlier slice, is finished
      // after the barrier; its partial sum is kept in a register).
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (q + u < qe) {
          const int prev = row;
          const bool nb = lrow[u] != prev;
          const A done = acc;
          acc = fma_acc(av[u], xv[u], zero_if(nb, acc));
          row = lrow[u];
          const bool pend_now = nb && first && open;
          pend_acc = pend_now ? done : pend_acc;
          if (nb && !pend_now) rowsum[prev] = done;
          first = first && !nb;
        }
      }
      if (qe < e0) {  // another chunk: row ends from the current row on
#pragma unroll
        for (int i = 0; i < NB; ++i) eb[i] = row + 1 + i <= nr ? rp[row + 1 + i] - k0 : INT_MAX;
      }
    }
    const int rend = rp[row + 1] - k0;
    if (rend == e0) {  // the slice's last row ends with the slice
      if (first && open) pend_acc = acc;
      else rowsum[row] = acc;
    } else {
      carry[gtid] = acc;  // continues into the next slice
    }
    if (open && (rend == e0 || !first)) { pend_row = srow[gtid]; pend_b = rb; }
  }
  // every read of the stage and of the ring for this tile is done
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(empty_s);
  named_bar_sync(bar, C::NT);
  if (pend_row >= 0) {
    DivK dk;
    dk.init(h);
    const int a = dk.div(pend_b);  // the slice where the row began
    A tot = carry[a];
    for (int t = a + 1; t < gtid; ++t) tot += carry[t];
    rowsum[pend_row] = tot + pend_acc;
  }
  // y for the tile's rows in one coalesced pass (alpha, beta and the fused
  // dot, if any, with all lanes)
  named_bar_sync(bar, C::NT);
  for (int lr = gtid; lr < nr; lr += C::NT) store_row<PLAIN>(p, r0 + lr, rowsum[lr], dsum);
}

// ----------------------------------------------------------------------------
// Kernel
// ----------------------------------------------------------------------------
template <bool PLAIN, typename V, typename I, class C>
__global__ void __launch_bounds__(C::G * C::NT + 32, 1) k_spmv_band(const SpmvParams p) {
  using A = typename AccOf<V>::type;
  using L = BandLayout<V, I, C>;
  extern __shared__ __align__(128) unsigned char smem[];
  // without column ranges no tile reads x through the ring, and the launch
  // leaves out its shared memory (the L1 cache gets it)
  A *ring = reinterpret_cast<A *>(smem + (size_t)p.stages * L::STAGE);
  unsigned char *ctrl =
      smem + (size_t)p.stages * L::STAGE + (p.colrange ? L::RING_BYTES : size_t(0));
  uint64_t *full = reinterpret_cast<uint64_t *>(ctrl + L::C_FULL);
  uint64_t *empty = reinterpret_cast<uint64_t *>(ctrl + L::C_EMPTY);
  BandHdr *hdr = reinterpret_cast<BandHdr *>(ctrl + L::C_HDR);
  double *red = reinterpret_cast<double *>(ctrl + L::C_RED);
  unsigned char *gsc = ctrl + L::CTRL;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::NT / 32);  // one group consumes each stage
    }
    fence_mbar_init();
  }
  __syncthreads();
  grid_dependency_wait();  // global memory only after the previous kernel
  grid_launch_dependents();
  long long t0, t1;
  band_chunk(p.ntiles, blockIdx.x, gridDim.x, t0, t1);
  if (tid < 32) {
    band_produce<V, I, C>(p, smem, ring, full, empty, hdr, t0, t1);
    return;
  }
  const int ctid = tid - 32, g = ctid / C::NT, gtid = ctid % C::NT;
  int *srow = reinterpret_cast<int *>(gsc + g * L::G_BYTES + L::G_SROW);
  A *carry = reinterpret_cast<A *>(gsc + g * L::G_BYTES + L::G_CARRY);
  A *rowsum = reinterpret_cast<A *>(gsc + g * L::G_BYTES + L::G_ROWSUM);
  const int bar_a = 1 + 2 * g, bar_b = 2 + 2 * g;
  DotAcc<A> dsum;
  RingPos rpos;
  rpos.s = g;  // tile g: the depth is a multiple of G, so g < stages and parity 0
  for (long long j = g; t0 + j < t1; j += C::G, rpos.advance(C::G, p.stages)) {
    const int s = rpos.s;
    const bool got = mbar_wait_bounded(&full[s], rpos.ph, p.status, p.timeout_ns);
    const BandHdr &h = hdr[s];
    unsigned char *st = smem + (size_t)s * L::STAGE;
    const int *rp = reinterpret_cast<const int *>(st) + h.rp_sh;
    if (got) band_start_rows<PLAIN, C>(p, h, rp, srow, rowsum, gtid, dsum);
    // slice start rows ready; the group gives up together after a timeout
    if (named_bar_or(bar_a, C::NT, !got)) break;
    const bool direct = (h.flags & kTileDirect) != 0;
    const V *vs = direct ? static_cast<const V *>(p.val) + h.k0
                         : reinterpret_cast<const V *>(st + L::OFF_V) + h.v_sh;
    const I *is = direct ? static_cast<const I *>(p.idx) + h.k0
                         : reinterpret_cast<const I *>(st + L::OFF_I) + h.i_sh;
    band_tile<PLAIN, V, I, C>(p, h, rp, vs, is, ring, srow, carry, rowsum, gtid, bar_b, &empty[s],
                              dsum);
  }
  if (p.dot_partials) {
    double dv = dsum.value();
    for (int o = 16; o > 0; o >>= 1) dv += __shfl_xor_sync(0xffffffffu, dv, o);
    if ((ctid & 31) == 0) red[ctid >> 5] = dv;
    named_bar_sync(15, C::G * C::NT);
    if (ctid == 0) {
      double tot = 0.0;
      for (int w = 0; w < C::G * C::NT / 32; ++w) tot += red[w];
      p.dot_partials[blockIdx.x] = tot;
    }
  }
}

// ----------------------------------------------------------------------------
// Sorted-rows band mode
// ----------------------------------------------------------------------------

// One tile: consumer thread ctid takes the tile's ctid-th longest row (the
// plan's permutation), so the rows of a warp have similar lengths and the
// warp's FMA steps carry nearly full lanes.  Each row is summed by its
// thread as two interleaved chains in stored order (even and odd entries),
// added at the end.  Rows longer than C::LONG (a warp would otherwise step
// through them with one lane) are summed by the whole warp instead: lane i
// takes entries i, i + 32, ... and the 32 partial sums are added by a
// butterfly.
template <bool PLAIN, typename V, typename I, class C>
__device__ __forceinline__ void sorted_tile(const SpmvParams &p, const BandHdr &h, const int *rp,
                                            const uint16_t *perm, const V *vs, const I *is,
                                            const typename AccOf<V>::type *ring, int ctid,
                                            DotAcc<typename AccOf<V>::type> &dsum) {
  using A = typename AccOf<V>::type;
  constexpr bool DA = sizeof(I) < 4;  // int16 / int8 offsets
  constexpr int CH = C::CH;
  const A *xg = static_cast<const A *>(p.x);
  const int r0 = h.r0, nr = h.nr, k0 = h.k0;
  const bool from_ring = (h.flags & kBandRing) != 0;
  const int lane = threadIdx.x & 31;
  auto xval = [&](int c) -> A {
    return from_ring ? ring[c & (C::W - 1)] : x_global(xg, c, p.ncols);
  };
  const int lr = ctid < nr ? static_cast<int>(perm[ctid]) : -1;
  int b = 0, len = 0;
  if (lr >= 0) {
    b = rp[lr] - k0;
    len = rp[lr + 1] - k0 - b;
  }
  A res = 0;
  // long rows: the whole warp, one row at a time
  unsigned longs = __ballot_sync(0xffffffffu, len > C::LONG);
  while (longs) {
    const int src = __ffs(longs) - 1;
    longs &= longs - 1;
    const int lb = __shfl_sync(0xffffffffu, b, src), ll = __shfl_sync(0xffffffffu, len, src);
    const int lrow = __shfl_sync(0xffffffffu, lr, src);
    A acc = 0;
    for (int q = lane; q < ll; q += 32) {
      const int c = DA ? r0 + lrow + static_cast<int>(is[lb + q]) : static_cast<int>(is[lb + q]);
      acc = fma_acc(to_acc(vs[lb + q]), xval(c), acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == src) res = acc;
  }
  // the other rows: one per lane, CH entries loaded ahead; lanes past the
  // end of their row multiply zeros (adding +0 leaves a sum unchanged: a sum
  // started at +0 is never -0)
  const int mylen = len > C::LONG ? 0 : len;
  int maxlen = mylen;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
  if (maxlen > 0) {
    // two FMA chains per row (entries 0, 2, 4, ... and 1, 3, 5, ...), added
    // at the end, so that a warp keeps two independent FMAs in flight
    A acc0 = 0, acc1 = 0;
    for (int q = 0; q < maxlen; q += CH) {
      A av[CH], xv[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        av[u] = 0;
        xv[u] = 0;
        if (q + u < mylen) {
          const int c = DA ? r0 + lr + static_cast<int>(is[b + q + u])
                           : static_cast<int>(is[b + q + u]);
          av[u] = to_acc(vs[b + q + u]);
          xv[u] = xval(c);
        }
      }
#pragma unroll
      for (int u = 0; u < CH; u += 2) {
        if (q + u < maxlen) acc0 = fma_acc(av[u], xv[u], acc0);
        if (q + u + 1 < maxlen) acc1 = fma_acc(av[u + 1], xv[u + 1], acc1);
      }
    }
    if (len <= C::LONG) res = acc0 + acc1;
  }
  if (lr >= 0) store_row<PLAIN>(p, r0 + lr, res, dsum);
}

template <bool PLAIN, typename V, typename I, class C>
__global__ void __launch_bounds__(C::G * C::NT + 32, 1) k_spmv_sorted(const SpmvParams p) {
  using A = typename AccOf<V>::type;
  using L = BandLayout<V, I, C>;
  extern __shared__ __align__(128) unsigned char smem[];
  A *ring = reinterpret_cast<A *>(smem + (size_t)p.stages * L::STAGE);
  unsigned char *ctrl = smem + (size_t)p.stages * L::STAGE + L::RING_BYTES;
  uint64_t *full = reinterpret_cast<uint64_t *>(ctrl + L::C_FULL);
  uint64_t *empty = reinterpret_cast<uint64_t *>(ctrl + L::C_EMPTY);
  BandHdr *hdr = reinterpret_cast<BandHdr *>(ctrl + L::C_HDR);
  double *red = reinterpret_cast<double *>(ctrl + L::C_RED);
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::NT / 32);
    }
    fence_mbar_init();
  }
  __syncthreads();
  grid_dependency_wait();  // global memory only after the previous kernel
  grid_launch_dependents();
  long long t0, t1;
  band_chunk(p.ntiles, blockIdx.x, gridDim.x, t0, t1);
  if (tid < 32) {
    band_produce<V, I, C>(p, smem, ring, full, empty, hdr, t0, t1);
    return;
  }
  const int ctid = tid - 32, g = ctid / C::NT, gtid = ctid % C::NT;
  DotAcc<A> dsum;
  // warps work independently: a warp whose bounded wait gives up stops
  RingPos rpos;
  rpos.s = g;  // tile g: the depth is a multiple of G, so g < stages and parity 0
  for (long long j = g; t0 + j < t1; j += C::G, rpos.advance(C::G, p.stages)) {
    const int s = rpos.s;
    if (!mbar_wait_bounded(&full[s], rpos.ph, p.status, p.timeout_ns)) break;
    const BandHdr &h = hdr[s];
    unsigned char *st = smem + (size_t)s * L::STAGE;
    const int *rp = reinterpret_cast<const int *>(st) + h.rp_sh;
    const uint16_t *perm = reinterpret_cast<const uint16_t *>(st + L::OFF_P);
    // one call per kind of tile, so that each sees plain shared-memory (or
    // global) pointers and the loads need no generic addressing
    if (h.flags & kTileDirect)
      sorted_tile<PLAIN, V, I, C>(p, h, rp, perm, static_cast<const V *>(p.val) + h.k0,
                                  static_cast<const I *>(p.idx) + h.k0, ring, gtid, dsum);
    else
      sorted_tile<PLAIN, V, I, C>(p, h, rp, perm,
                                  reinterpret_cast<const V *>(st + L::OFF_V) + h.v_sh,
                                  reinterpret_cast<const I *>(st + L::OFF_I) + h.i_sh, ring, gtid,
                                  dsum);
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(&empty[s]);
  }
  if (p.dot_partials) {
    double dv = dsum.value();
    for (int o = 16; o > 0; o >>= 1) dv += __shfl_xor_sync(0xffffffffu, dv, o);
    if ((ctid & 31) == 0) red[ctid >> 5] = dv;
    named_bar_sync(15, C::G * C::NT);
    if (ctid == 0) {
      double tot = 0.0;
      for (int w = 0; w < C::G * C::NT / 32; ++w) tot += red[w];
      p.dot_partials[blockIdx.x] = tot;
    }
  }
}

}  // namespace spmvk
}  // namespace damn
