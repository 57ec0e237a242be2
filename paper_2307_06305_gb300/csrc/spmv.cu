// SpMV entry points, plans and launch plumbing.  The kernels are in
// spmv_kernel.cuh; see there for the design.
//
// A plan fixes, for one matrix: the tile partition (fixed row blocks, or
// blocks balanced on rows + entries), the compute mode (one row per thread or
// balanced slices), and, when the column indices are given, the x window of
// every tile -- the sorted distinct columns of the tile clustered into at most
// four contiguous segments (gaps of up to kXGap columns merged, then the
// closest segments merged until four remain) that the
// producer stages into shared memory with the matrix data.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "damn_common.cuh"
#include "spmv_band.cuh"
#include "spmv_internal.h"
#include "spmv_kernel.cuh"

using namespace damn::spmvk;

namespace damn {
namespace {

constexpr int kRowWeight = 4;       // merge-path weight of a row against an entry
constexpr int kBalancedItems = 2048;
constexpr int kXGap = 32;           // columns: smaller gaps are staged, not split
static_assert(kBalancedItems / kRowWeight <= CfgSlices::CAP_ROWS, "balanced tiles too tall");
static_assert(CfgShort::TILE_ROWS <= CfgShort::CAP_ROWS &&
                  CfgShortNarrow::TILE_ROWS <= CfgShortNarrow::CAP_ROWS &&
                  CfgLong::TILE_ROWS <= CfgLong::CAP_ROWS && 256 <= CfgSlices::CAP_ROWS &&
                  CfgLongNarrow::TILE_ROWS <= CfgLongNarrow::CAP_ROWS &&
                  CfgShortX2::TILE_ROWS <= CfgShortX2::CAP_ROWS &&
                  CfgShortNarrowX2::TILE_ROWS <= CfgShortNarrowX2::CAP_ROWS,
              "row tiles too tall");
static_assert(kBalancedItems <= CfgBand64::CAP_NZ && kBalancedItems / kRowWeight <= CfgBand64::CAP_ROWS &&
                  kBalancedItems <= CfgBand32::CAP_NZ &&
                  kBalancedItems / kRowWeight <= CfgBand32::CAP_ROWS,
              "balanced tiles exceed a band stage");

// ----------------------------------------------------------------------------
// Launch: one launcher per (index format, value type), in spmv_inst_*.cu
// ----------------------------------------------------------------------------
}  // namespace
#define DAMN_DECL_LAUNCH(NAME) int NAME(const SpmvParams &, int, cudaStream_t, int *);
DAMN_DECL_LAUNCH(spmv_launch_csr32_f64)
DAMN_DECL_LAUNCH(spmv_launch_csr32_f32)
DAMN_DECL_LAUNCH(spmv_launch_csr32_bf16)
DAMN_DECL_LAUNCH(spmv_launch_dacsr16_f64)
DAMN_DECL_LAUNCH(spmv_launch_dacsr16_f32)
DAMN_DECL_LAUNCH(spmv_launch_dacsr16_bf16)
DAMN_DECL_LAUNCH(spmv_launch_dacsr8_f64)
DAMN_DECL_LAUNCH(spmv_launch_dacsr8_f32)
DAMN_DECL_LAUNCH(spmv_launch_dacsr8_bf16)
DAMN_DECL_LAUNCH(spmv_launch_csr32_f8)
DAMN_DECL_LAUNCH(spmv_launch_dacsr16_f8)
DAMN_DECL_LAUNCH(spmv_launch_dacsr8_f8)
#undef DAMN_DECL_LAUNCH
namespace {

int launch_any(const SpmvParams &p, int dtype, int fmt, int shape, cudaStream_t s, int *gs) {
  if (fmt == DAMN_FMT_DACSR16) {
    if (dtype == DAMN_F64) return spmv_launch_dacsr16_f64(p, shape, s, gs);
    if (dtype == DAMN_F32) return spmv_launch_dacsr16_f32(p, shape, s, gs);
    if (dtype == DAMN_F8E4M3) return spmv_launch_dacsr16_f8(p, shape, s, gs);
    return spmv_launch_dacsr16_bf16(p, shape, s, gs);
  }
  if (fmt == DAMN_FMT_DACSR8) {
    if (dtype == DAMN_F64) return spmv_launch_dacsr8_f64(p, shape, s, gs);
    if (dtype == DAMN_F32) return spmv_launch_dacsr8_f32(p, shape, s, gs);
    if (dtype == DAMN_F8E4M3) return spmv_launch_dacsr8_f8(p, shape, s, gs);
    return spmv_launch_dacsr8_bf16(p, shape, s, gs);
  }
  if (dtype == DAMN_F64) return spmv_launch_csr32_f64(p, shape, s, gs);
  if (dtype == DAMN_F32) return spmv_launch_csr32_f32(p, shape, s, gs);
  if (dtype == DAMN_F8E4M3) return spmv_launch_csr32_f8(p, shape, s, gs);
  return spmv_launch_csr32_bf16(p, shape, s, gs);
}

// ----------------------------------------------------------------------------
// Plan kernels
// ----------------------------------------------------------------------------

// Tile t starts at the first row r with kRowWeight * r + rowptr[r] >= t * D.
__global__ void k_plan_bounds(int nrows, const int *__restrict__ rowptr, long long D, int ntiles,
                              int2 *bounds) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > ntiles) return;
  int r;
  if (t == ntiles) {
    r = nrows;
  } else {
    const long long target = (long long)t * D;
    int lo = 0, hi = nrows;
    while (lo < hi) {
      const int mid = lo + ((hi - lo) >> 1);
      if ((long long)kRowWeight * mid + rowptr[mid] >= target) hi = mid; else lo = mid + 1;
    }
    r = lo;
  }
  bounds[t] = make_int2(r, rowptr[r]);
}

struct PlanStats {
  unsigned long long sum_group_max;  // sum over 32-row groups of the longest row
  int max_row;
  int max_tile_short;                // most entries in a short-rows tile
  int max_tile_long;                 // most entries in a long-rows tile
  int pad;
};

__global__ void k_plan_stats(int nrows, const int *__restrict__ rowptr, int tile_short,
                             int tile_long, PlanStats *st) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int len = 0;
  if (i < nrows) len = rowptr[i + 1] - rowptr[i];
  int gmax = len;
  for (int o = 16; o > 0; o >>= 1) gmax = max(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&st->sum_group_max, (unsigned long long)gmax);
    atomicMax(&st->max_row, gmax);
  }
  if (i < nrows && i % tile_short == 0) {
    const int r1 = (int)min((long long)nrows, i + tile_short);
    atomicMax(&st->max_tile_short, rowptr[r1] - rowptr[i]);
  }
  if (i < nrows && i % tile_long == 0) {
    const int r1 = (int)min((long long)nrows, i + tile_long);
    atomicMax(&st->max_tile_long, rowptr[r1] - rowptr[i]);
  }
}

constexpr int kXSortCap = 8192;  // >= every CAP_NZ
constexpr int kXRowsCap = 1025;  // >= every CAP_ROWS + 1
static_assert(CfgShortNarrowX2::CAP_NZ <= kXSortCap && CfgShortNarrowX2::CAP_ROWS + 1 <= kXRowsCap,
              "x-window plan kernel too small for a stage");
constexpr int kXStartCap = 64;   // segment starts considered for merging

// x window of every tile: columns of the tile's entries, sorted (bitonic, in
// shared memory), cut where consecutive columns differ by more than kXGap.
// A tile gets a window when it has at most kXSegMax segments whose 16-byte
// aligned lengths (ex elements per 16 bytes) add up to at most xcap elements;
// otherwise nseg = 0 and the kernel gathers x from global memory.
__global__ void __launch_bounds__(256)
k_plan_xseg(int nrows, int ncols, const int *__restrict__ rowptr, const void *idx, int fmt,
            int ntiles, int rows_per_tile, const int2 *__restrict__ bounds, int cap_nz, int xcap,
            int ex, XSeg *out) {
  __shared__ int keys[kXSortCap];
  __shared__ int rps[kXRowsCap];
  __shared__ int bpos[kXStartCap];
  __shared__ int nb;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int r0, r1, k0, k1;
    if (rows_per_tile > 0) {
      r0 = t * rows_per_tile;
      r1 = min(r0 + rows_per_tile, nrows);
      k0 = rowptr[r0];
      k1 = rowptr[r1];
    } else {
      const int2 b0 = bounds[t], b1 = bounds[t + 1];
      r0 = b0.x; k0 = b0.y; r1 = b1.x; k1 = b1.y;
    }
    const int m = k1 - k0, nr = r1 - r0;
    if (m == 0 || m > cap_nz || m > kXSortCap || nr + 1 > kXRowsCap) {
      if (threadIdx.x == 0) out[t].nseg = 0;
      continue;  // uniform across the block
    }
    for (int i = threadIdx.x; i <= nr; i += blockDim.x) rps[i] = rowptr[r0 + i];
    if (threadIdx.x == 0) nb = 0;
    __syncthreads();
    int P = 1;
    while (P < m) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      int c = INT_MAX;
      if (i < m) {
        const int k = k0 + i;
        if (fmt == DAMN_FMT_CSR32) {
          c = static_cast<const int *>(idx)[k];
        } else {
          int lo = 0, hi = nr - 1;  // last local row with rps[row] <= k
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rps[mid] <= k) lo = mid; else hi = mid - 1;
          }
          c = r0 + lo + (fmt == DAMN_FMT_DACSR8
                             ? static_cast<int>(static_cast<const int8_t *>(idx)[k])
                             : static_cast<int>(static_cast<const int16_t *>(idx)[k]));
        }
      }
      keys[i] = c;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          const int jx = i ^ stride;
          if (jx > i) {
            const bool up = (i & size) == 0;
            const int a = keys[i], b = keys[jx];
            if ((a > b) == up) { keys[i] = b; keys[jx] = a; }
          }
        }
        __syncthreads();
      }
    }
    // Runs of columns separated by more than kXGap start a new segment; while
    // there are more than kXSegMax segments, the two neighbours with the
    // smallest gap are merged (thread 0; the starts are few).
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      if (i == 0 || keys[i] - keys[i - 1] > kXGap) {
        const int slot = atomicAdd(&nb, 1);
        if (slot < kXStartCap) bpos[slot] = i;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int n = nb;
      XSeg seg;
      seg.nseg = 0;
      if (n <= kXStartCap) {
        for (int a = 1; a < n; ++a) {  // insertion sort of the starts
          const int v = bpos[a];
          int b = a - 1;
          while (b >= 0 && bpos[b] > v) { bpos[b + 1] = bpos[b]; --b; }
          bpos[b + 1] = v;
        }
        while (n > kXSegMax) {  // merge across the smallest gap
          int best = 1, bg = INT_MAX;
          for (int a = 1; a < n; ++a) {
            const int g = keys[bpos[a]] - keys[bpos[a] - 1];
            if (g < bg) { bg = g; best = a; }
          }
          for (int a = best; a + 1 < n; ++a) bpos[a] = bpos[a + 1];
          --n;
        }
        // staging layout: segment a is copied from its 16-byte aligned start
        // src to slot dst (running sum of aligned lengths); x must hold every
        // copied element (no partial block at the end of x).
        long long total = 0;
        bool fits = true;
        const long long x_full = (long long)ncols & ~(long long)(ex - 1);
        for (int a = 0; a < n; ++a) {
          const int first = bpos[a];
          const int lastpos = (a + 1 < n ? bpos[a + 1] : m) - 1;
          const int lo = keys[first], hi = keys[lastpos] + 1;
          const long long a0 = lo & ~(long long)(ex - 1);
          const long long a1 = ((long long)hi + ex - 1) & ~(long long)(ex - 1);
          if (a1 > x_full) fits = false;
          seg.lo[a] = lo;
          seg.src[a] = static_cast<int>(a0);
          seg.cnt[a] = static_cast<int>(a1 - a0);
          seg.pos[a] = static_cast<int>(total + (lo - a0));
          total += a1 - a0;
        }
        if (fits && total <= xcap) seg.nseg = n;
      }
      for (int a = seg.nseg; a < kXSegMax; ++a) {
        seg.lo[a] = 0; seg.pos[a] = 0; seg.src[a] = 0; seg.cnt[a] = 0;
      }
      seg.pad[0] = seg.pad[1] = seg.pad[2] = 0;
      out[t] = seg;
    }
    __syncthreads();
  }
}

// count[0]: tiles with a staged x window; count[1]: most segments of a window
__global__ void k_count_staged(const XSeg *xs, int ntiles, int *count) {
  int c = 0, mx = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
    c += xs[t].nseg > 0 ? 1 : 0;
    mx = max(mx, xs[t].nseg);
  }
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (c) atomicAdd(count, c);
    atomicMax(count + 1, mx);
  }
}

// {min, max} column of the entries of every balanced tile (one block per
// tile, a thread per row); {INT_MAX, INT_MIN} for a tile without entries.
__global__ void __launch_bounds__(256)
k_plan_colrange(const int *__restrict__ rowptr, const void *idx, int fmt, int ntiles,
                const int2 *__restrict__ bounds, int2 *out) {
  __shared__ int s_lo[8], s_hi[8];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 b0 = bounds[t], b1 = bounds[t + 1];
    int lo = INT_MAX, hi = INT_MIN;
    for (int r = b0.x + threadIdx.x; r < b1.x; r += blockDim.x) {
      for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
        int c;
        if (fmt == DAMN_FMT_CSR32) c = static_cast<const int *>(idx)[k];
        else if (fmt == DAMN_FMT_DACSR8) c = r + static_cast<const int8_t *>(idx)[k];
        else c = r + static_cast<const int16_t *>(idx)[k];
        lo = min(lo, c);
        hi = max(hi, c);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) { s_lo[threadIdx.x >> 5] = lo; s_hi[threadIdx.x >> 5] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { lo = min(lo, s_lo[w]); hi = max(hi, s_hi[w]); }
      out[t] = make_int2(lo, hi);
    }
    __syncthreads();
  }
}

// Bounds of fixed tiles of tile_rows rows: {first row, rowptr[first row]}.
__global__ void k_plan_fixed_bounds(int nrows, const int *__restrict__ rowptr, int tile_rows,
                                    int ntiles, int2 *bounds) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > ntiles) return;
  const int r = (int)min((long long)t * tile_rows, (long long)nrows);
  bounds[t] = make_int2(r, rowptr[r]);
}

// Rows of every tile of tile_rows (<= 1024) rows in order of decreasing
// length, equal lengths by increasing index (a bitonic sort of 1024 keys per
// block): perm[t * tile_rows + i] = tile-local index of the i-th longest row.
__global__ void __launch_bounds__(512)
k_plan_sortrows(int nrows, const int *__restrict__ rowptr, int tile_rows, int ntiles,
                uint16_t *perm) {
  __shared__ unsigned keys[1024];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r0 = t * tile_rows;
    const int nr = min(tile_rows, nrows - r0);
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
      unsigned k = 0;  // padding sorts last
      if (i < nr) {
        const unsigned len = (unsigned)min(rowptr[r0 + i + 1] - rowptr[r0 + i], (1 << 21) - 1);
        k = (len << 10) | (1023u - (unsigned)i);
      }
      keys[i] = k;
    }
    __syncthreads();
    for (int size = 2; size <= 1024; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
          const int jx = i ^ stride;
          if (jx > i) {
            const bool down = (i & size) == 0;  // descending overall
            const unsigned a = keys[i], b = keys[jx];
            if ((a < b) == down) { keys[i] = b; keys[jx] = a; }
          }
        }
        __syncthreads();
      }
    }
    for (int i = threadIdx.x; i < tile_rows; i += blockDim.x)
      perm[(long long)t * tile_rows + i] =
          i < nr ? (uint16_t)(1023u - (keys[i] & 1023u)) : (uint16_t)0;
    __syncthreads();
  }
}

// Most entries of any tile of tile_rows consecutive rows (*out, atomicMax).
__global__ void k_plan_max_tile(int nrows, const int *__restrict__ rowptr, int tile_rows, int *out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long r0 = t * tile_rows;
  if (r0 >= nrows) return;
  const int r1 = (int)min((long long)nrows, r0 + tile_rows);
  atomicMax(out, rowptr[r1] - rowptr[r0]);
}

}  // namespace
}  // namespace damn

struct damn_plan {
  int nrows, ncols;
  long long nnz;
  int dtype;
  const int32_t *rowptr;  // caller's arrays (kept for the autotuner and the x windows)
  const void *idx;        // column indices (may be NULL: no x windows)
  int fmt;
  int mode;               // 0 rows, 1 balanced slices, 2 band, 3 sorted rows
  int shape;              // kernel configuration (spmvk::Shape)
  int rows_per_tile;      // > 0 fixed row tiles, 0 bounds
  int ntiles;
  int2 *d_bounds;         // bounds of the current tiling (NULL for fixed rows)
  int2 *d_bounds_balanced;
  int ntiles_balanced;
  XSeg *d_xseg;           // x windows of the current tiling (NULL: none)
  int xseg_cap;
  int2 *d_colrange;       // band mode: column range of every balanced tile (NULL: none)
  int ntiles_sorted;      // sorted-rows tiling: fixed tiles, their bounds, column
  int2 *d_bounds_sorted;  // ranges and row permutation (built on first use)
  int2 *d_colrange_sorted;
  uint16_t *d_perm;
  int staged_tiles;
  int max_nseg;           // most x segments of a tile's window (rows mode kernel variant)
  int max_row;
  double row_eff;
  int max_tile_short, max_tile_long;
  int stages_req;         // requested ring depth (0: automatic)
  int no_xstage;          // rows tilings: stage no x window; band: no x ring (x from L1 / L2)
  int grid, stages;       // geometry of the last launch
};

namespace damn {

int spmv_max_grid() { return 8 * sm_count(); }

// Tile height, stage entry capacity and staged-x capacity of the kernel
// configuration a plan shape uses for a value type (must match launch_types).
struct CfgGeom {
  int tile_rows, cap_nz, xcap, threads;
};
static CfgGeom cfg_geom(int shape, int dtype) {
  switch (shape) {
    case kShapeLong:
      if (dtype != DAMN_F64)
        return {CfgLongNarrow::TILE_ROWS, CfgLongNarrow::CAP_NZ, CfgLongNarrow::XCAP,
                CfgLongNarrow::NT};
      return {CfgLong::TILE_ROWS, CfgLong::CAP_NZ, CfgLong::XCAP, CfgLong::NT};
    case kShapeSlices: return {0, CfgSlices::CAP_NZ, CfgSlices::XCAP, CfgSlices::NT};
    case kShapeBand:
      return {0, CfgBand64::CAP_NZ, dtype == DAMN_F64 ? CfgBand64::W : CfgBand32::W,
              CfgBand64::G * CfgBand64::NT};
    case kShapeLanes4: return {CfgLanes4::TILE_ROWS, CfgLanes4::CAP_NZ, CfgLanes4::XCAP, 256};
    case kShapeLanes8: return {CfgLanes8::TILE_ROWS, CfgLanes8::CAP_NZ, CfgLanes8::XCAP, 256};
    case kShapeLanes16: return {CfgLanes16::TILE_ROWS, CfgLanes16::CAP_NZ, CfgLanes16::XCAP, 256};
    case kShapeLanes32: return {CfgLanes32::TILE_ROWS, CfgLanes32::CAP_NZ, CfgLanes32::XCAP, 256};
    case kShapeShortX2:
      if (dtype != DAMN_F64)
        return {CfgShortNarrowX2::TILE_ROWS, CfgShortNarrowX2::CAP_NZ, CfgShortNarrowX2::XCAP, 256};
      return {CfgShortX2::TILE_ROWS, CfgShortX2::CAP_NZ, CfgShortX2::XCAP, 256};
    case kShapeSorted:
      return {CfgSorted64::NT, CfgSorted64::CAP_NZ,
              dtype == DAMN_F64 ? CfgSorted64::W : CfgSorted32::W,
              CfgSorted64::G * CfgSorted64::NT};
    default: break;
  }
  if (dtype != DAMN_F64)
    return {CfgShortNarrow::TILE_ROWS, CfgShortNarrow::CAP_NZ, CfgShortNarrow::XCAP, 256};
  return {CfgShort::TILE_ROWS, CfgShort::CAP_NZ, CfgShort::XCAP, 256};
}

// Public tiling <-> kernel shape.
static int shape_of_tiling(int tiling) {
  switch (tiling) {
    case DAMN_TILING_SLICES: return kShapeSlices;
    case DAMN_TILING_ROWS: return kShapeShort;
    case DAMN_TILING_ROWS_LONG: return kShapeLong;
    case DAMN_TILING_BAND: return kShapeBand;
    case DAMN_TILING_ROWS_LANES4: return kShapeLanes4;
    case DAMN_TILING_ROWS_LANES8: return kShapeLanes8;
    case DAMN_TILING_ROWS_LANES16: return kShapeLanes16;
    case DAMN_TILING_ROWS_LANES32: return kShapeLanes32;
    case DAMN_TILING_SORTED_ROWS: return kShapeSorted;
    case DAMN_TILING_ROWS_X2: return kShapeShortX2;
    default: return -1;
  }
}
static int tiling_of_shape(int shape) {
  switch (shape) {
    case kShapeSlices: return DAMN_TILING_SLICES;
    case kShapeLong: return DAMN_TILING_ROWS_LONG;
    case kShapeBand: return DAMN_TILING_BAND;
    case kShapeLanes4: return DAMN_TILING_ROWS_LANES4;
    case kShapeLanes8: return DAMN_TILING_ROWS_LANES8;
    case kShapeLanes16: return DAMN_TILING_ROWS_LANES16;
    case kShapeLanes32: return DAMN_TILING_ROWS_LANES32;
    case kShapeSorted: return DAMN_TILING_SORTED_ROWS;
    case kShapeShortX2: return DAMN_TILING_ROWS_X2;
    default: return DAMN_TILING_ROWS;
  }
}

static int make_params(const SpmvCall &c, const damn_plan *plan, SpmvParams &p, int &shape) {
  std::memset(&p, 0, sizeof(p));
  p.nrows = c.nrows;
  p.ncols = c.ncols;
  p.nnz = c.nnz;
  p.rowptr = c.rowptr;
  p.idx = c.idx;
  p.val = c.val;
  p.x = c.x;
  p.y0 = c.y0 ? c.y0 : c.y;
  p.y = c.y;
  p.alpha = c.alpha;
  p.beta = c.beta;
  p.ab_mode = (c.beta != 0.0) ? 2 : (c.alpha == 1.0 ? 0 : 1);
  p.dot_w = c.dot_w;
  p.dot_self = c.dot_self;
  p.dot_partials = c.dot_partials;
  p.status = device_status_ptr();
  p.timeout_ns = kWaitTimeoutNs;
  if (!p.status) return set_error(DAMN_ERR_CUDA, "no device status word");
  if (plan) {
    p.mode = plan->mode;
    p.rows_per_tile = plan->rows_per_tile;
    p.ntiles = plan->ntiles;
    p.bounds = plan->d_bounds;
    p.xseg = (plan->mode >= 2 || (plan->mode == 0 && plan->no_xstage)) ? nullptr : plan->d_xseg;
    p.colrange = plan->mode == 2 ? (plan->no_xstage ? nullptr : plan->d_colrange)
                 : plan->mode == 3 ? plan->d_colrange_sorted : nullptr;
    p.perm = plan->mode == 3 ? plan->d_perm : nullptr;
    p.stages_req = plan->stages_req;
    p.max_nseg = p.xseg ? plan->max_nseg : kXSegMax;
    shape = plan->shape;
  } else {
    p.mode = 1;
    p.rows_per_tile = 256;
    p.ntiles = (c.nrows + 255) / 256;
    p.bounds = nullptr;
    p.xseg = nullptr;
    p.max_nseg = kXSegMax;
    shape = 2;
  }
  return DAMN_OK;
}

int spmv_launch(const SpmvCall &c, const damn_plan *plan, cudaStream_t s, int *grid_out) {
  SpmvParams p;
  int shape = 0;
  int rc = make_params(c, plan, p, shape);
  if (rc) return rc;
  int gs[2] = {0, 0};
  rc = launch_any(p, c.dtype, c.fmt, shape, s, gs);
  if (grid_out) *grid_out = gs[0];
  if (plan && rc == DAMN_OK) {
    // launch geometry is reported by damn_plan_describe
    const_cast<damn_plan *>(plan)->grid = gs[0];
    const_cast<damn_plan *>(plan)->stages = gs[1];
  }
  return rc;
}

int plan_check(const char *fn, const damn_plan *plan, int fmt, int32_t nrows, int32_t ncols,
               int64_t nnz, const int32_t *rowptr, const void *idx, int dtype) {
  if (!plan) return DAMN_OK;
  if (plan->nrows != nrows || plan->ncols != ncols || plan->nnz != nnz || plan->dtype != dtype)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: plan was built for another matrix or dtype", fn);
  // The plan's tiles and x windows were computed from its own rowptr and
  // index array: a call with other arrays of the same sizes would read rows
  // and x slots the plan never prepared.  The same matrix in another index
  // format (CSR-32 col for a plan built from DA-CSR offsets, or the reverse)
  // is the documented exception.
  if (nrows > 0 && plan->rowptr != rowptr)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: rowptr is not the array the plan was built from", fn);
  if (plan->idx && plan->fmt == fmt && plan->idx != idx)
    return set_error(DAMN_ERR_INVALID_ARG,
                     "%s: index array is not the one the plan was built from", fn);
  return DAMN_OK;
}

}  // namespace damn

using namespace damn;

static int check_spmv_args(const char *fn, int fmt, int32_t nrows, int32_t ncols, int64_t nnz,
                           const int32_t *rowptr, const void *idx, const void *val, int dtype,
                           const void *x, void *y, const damn_plan *plan) {
  if (nrows < 0 || ncols < 0 || nnz < 0 || nnz > INT_MAX)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: bad sizes", fn);
  if (dtype != DAMN_F64 && dtype != DAMN_F32 && dtype != DAMN_BF16 && dtype != DAMN_F8E4M3)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: bad dtype %d", fn, dtype);
  if (nrows > 0 && (!rowptr || !y)) return set_error(DAMN_ERR_INVALID_ARG, "%s: NULL pointer", fn);
  if (nnz > 0 && (!idx || !val || !x)) return set_error(DAMN_ERR_INVALID_ARG, "%s: NULL pointer", fn);
  if (nnz > 0 && ncols == 0)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: entries but no columns (ncols == 0)", fn);
  if (!aligned16(rowptr) || !aligned16(idx) || !aligned16(val) || !aligned16(x) || !aligned16(y))
    return set_error(DAMN_ERR_INVALID_ARG, "%s: pointers must be 16-byte aligned", fn);
  return plan_check(fn, plan, fmt, nrows, ncols, nnz, rowptr, idx, dtype);
}

static int spmv_entry(const char *fn, int fmt, int32_t nrows, int32_t ncols, int64_t nnz,
                      const int32_t *rowptr, const void *idx, const void *val, int dtype,
                      const void *x, void *y, double alpha, double beta, const damn_plan *plan,
                      void *stream) {
  int rc = check_spmv_args(fn, fmt, nrows, ncols, nnz, rowptr, idx, val, dtype, x, y, plan);
  if (rc) return rc;
  if (nrows == 0) return DAMN_OK;
  SpmvCall c;
  c.nrows = nrows; c.ncols = ncols; c.nnz = nnz; c.rowptr = rowptr; c.idx = idx; c.fmt = fmt;
  c.val = val; c.dtype = dtype; c.x = x; c.y0 = y; c.y = y; c.alpha = alpha; c.beta = beta;
  return spmv_launch(c, plan, static_cast<cudaStream_t>(stream), nullptr);
}

extern "C" int damn_spmv_csr32(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                               const int32_t *col, const void *val, int dtype, const void *x,
                               void *y, double alpha, double beta, const damn_plan *plan,
                               void *stream) {
  return spmv_entry("damn_spmv_csr32", DAMN_FMT_CSR32, nrows, ncols, nnz, rowptr, col, val, dtype,
                    x, y, alpha, beta, plan, stream);
}

extern "C" int damn_spmv_dacsr16(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                                 const int16_t *off, const void *val, int dtype, const void *x,
                                 void *y, double alpha, double beta, const damn_plan *plan,
                                 void *stream) {
  return spmv_entry("damn_spmv_dacsr16", DAMN_FMT_DACSR16, nrows, ncols, nnz, rowptr, off, val,
                    dtype, x, y, alpha, beta, plan, stream);
}

extern "C" int damn_spmv_dacsr8(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                                const int8_t *off, const void *val, int dtype, const void *x,
                                void *y, double alpha, double beta, const damn_plan *plan,
                                void *stream) {
  return spmv_entry("damn_spmv_dacsr8", DAMN_FMT_DACSR8, nrows, ncols, nnz, rowptr, off, val, dtype,
                    x, y, alpha, beta, plan, stream);
}

// ----------------------------------------------------------------------------
// Plans
// ----------------------------------------------------------------------------
static void plan_free_device(damn_plan *pl) {
  if (pl->d_bounds_balanced) cudaFree(pl->d_bounds_balanced);
  if (pl->d_xseg) cudaFree(pl->d_xseg);
  if (pl->d_colrange) cudaFree(pl->d_colrange);
  if (pl->d_bounds_sorted) cudaFree(pl->d_bounds_sorted);
  if (pl->d_colrange_sorted) cudaFree(pl->d_colrange_sorted);
  if (pl->d_perm) cudaFree(pl->d_perm);
  pl->d_bounds_sorted = nullptr;
  pl->d_colrange_sorted = nullptr;
  pl->d_perm = nullptr;
  pl->d_bounds_balanced = nullptr;
  pl->d_xseg = nullptr;
  pl->d_colrange = nullptr;
  pl->d_bounds = nullptr;
}

static int plan_xwindows(damn_plan *pl, cudaStream_t s) {
  pl->staged_tiles = 0;
  pl->max_nseg = kXSegMax;
  if (!pl->idx || pl->ntiles == 0 || pl->nrows == 0) return DAMN_OK;
  if (pl->xseg_cap < pl->ntiles) {
    if (pl->d_xseg) cudaFree(pl->d_xseg);
    pl->d_xseg = nullptr;
    pl->xseg_cap = 0;
    DAMN_CUDA(cudaMalloc(&pl->d_xseg, sizeof(XSeg) * (size_t)pl->ntiles));
    pl->xseg_cap = pl->ntiles;
  }
  const int asz = pl->dtype == DAMN_F64 ? 8 : 4;
  const CfgGeom geo = cfg_geom(pl->shape, pl->dtype);
  const int cap_nz = geo.cap_nz;
  const int xcap = geo.xcap;
  const int blocks = std::min(pl->ntiles, 16 * sm_count());
  k_plan_xseg<<<blocks, 256, 0, s>>>(pl->nrows, pl->ncols, pl->rowptr, pl->idx, pl->fmt, pl->ntiles,
                                     pl->rows_per_tile, pl->d_bounds, cap_nz, xcap,
                                     16 / asz, pl->d_xseg);
  DAMN_CHECK_LAUNCH("k_plan_xseg");
  int *d_cnt = nullptr;
  DAMN_CUDA(cudaMallocAsync(&d_cnt, 2 * sizeof(int), s));
  DAMN_CUDA(cudaMemsetAsync(d_cnt, 0, 2 * sizeof(int), s));
  k_count_staged<<<std::min(1024, (pl->ntiles + 255) / 256), 256, 0, s>>>(pl->d_xseg, pl->ntiles,
                                                                          d_cnt);
  int h[2] = {0, 0};
  DAMN_CUDA(cudaMemcpyAsync(h, d_cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaFreeAsync(d_cnt, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  pl->staged_tiles = h[0];
  pl->max_nseg = h[1];
  return DAMN_OK;
}

// Column range of every balanced tile, for band mode (once per plan).
static int plan_colrange(damn_plan *pl, cudaStream_t s) {
  if (pl->d_colrange || !pl->idx || pl->ntiles_balanced == 0) return DAMN_OK;
  DAMN_CUDA(cudaMalloc(&pl->d_colrange, sizeof(int2) * (size_t)pl->ntiles_balanced));
  const int blocks = std::min(pl->ntiles_balanced, 16 * sm_count());
  k_plan_colrange<<<blocks, 256, 0, s>>>(pl->rowptr, pl->idx, pl->fmt, pl->ntiles_balanced,
                                         pl->d_bounds_balanced, pl->d_colrange);
  DAMN_CHECK_LAUNCH("k_plan_colrange");
  DAMN_CUDA(cudaStreamSynchronize(s));
  return DAMN_OK;
}

// Fixed tiles (CfgSorted64::NT rows), their column ranges and row permutations, for the
// sorted-rows tiling (once per plan; synchronises).
static int plan_sorted(damn_plan *pl, cudaStream_t s) {
  if (pl->d_perm || pl->nrows == 0) return DAMN_OK;
  const int tr = CfgSorted64::NT;
  const int nt = (pl->nrows + tr - 1) / tr;
  DAMN_CUDA(cudaMalloc(&pl->d_bounds_sorted, sizeof(int2) * (size_t)(nt + 1)));
  DAMN_CUDA(cudaMalloc(&pl->d_perm, sizeof(uint16_t) * (size_t)nt * tr));
  k_plan_fixed_bounds<<<(nt + 1 + 255) / 256, 256, 0, s>>>(pl->nrows, pl->rowptr, tr, nt,
                                                            pl->d_bounds_sorted);
  k_plan_sortrows<<<std::min(nt, 16 * sm_count()), 512, 0, s>>>(pl->nrows, pl->rowptr, tr, nt,
                                                                pl->d_perm);
  DAMN_CHECK_LAUNCH("k_plan_sortrows");
  if (pl->idx) {
    DAMN_CUDA(cudaMalloc(&pl->d_colrange_sorted, sizeof(int2) * (size_t)nt));
    k_plan_colrange<<<std::min(nt, 16 * sm_count()), 256, 0, s>>>(
        pl->rowptr, pl->idx, pl->fmt, nt, pl->d_bounds_sorted, pl->d_colrange_sorted);
    DAMN_CHECK_LAUNCH("k_plan_colrange");
  }
  pl->ntiles_sorted = nt;
  DAMN_CUDA(cudaStreamSynchronize(s));
  return DAMN_OK;
}

static int plan_use(damn_plan *pl, int tiling, cudaStream_t s) {
  const int shape = shape_of_tiling(tiling);
  pl->shape = shape;
  if (shape == kShapeSorted) {
    int rc = plan_sorted(pl, s);
    if (rc) return rc;
    pl->mode = 3;
    pl->rows_per_tile = 0;
    pl->ntiles = pl->ntiles_sorted;
    pl->d_bounds = pl->d_bounds_sorted;
    pl->staged_tiles = 0;
    pl->max_nseg = kXSegMax;
    return DAMN_OK;
  }
  if (shape == kShapeSlices || shape == kShapeBand) {
    pl->mode = shape == kShapeBand ? 2 : 1;
    pl->rows_per_tile = 0;
    pl->ntiles = pl->ntiles_balanced;
    pl->d_bounds = pl->d_bounds_balanced;
  } else {
    pl->mode = 0;
    pl->rows_per_tile = cfg_geom(shape, pl->dtype).tile_rows;
    pl->ntiles = (pl->nrows + pl->rows_per_tile - 1) / pl->rows_per_tile;
    pl->d_bounds = nullptr;
  }
  if (shape == kShapeBand) {
    pl->staged_tiles = 0;
    pl->max_nseg = kXSegMax;
    return plan_colrange(pl, s);
  }
  return plan_xwindows(pl, s);
}

static int plan_tiling_of(const damn_plan *pl) { return tiling_of_shape(pl->shape); }

// Most entries of a tile of tile_rows consecutive rows (synchronises).
static int plan_max_tile(const damn_plan *pl, int tile_rows, cudaStream_t s, int *out) {
  *out = 0;
  if (pl->nrows == 0) return DAMN_OK;
  int *d = nullptr;
  DAMN_CUDA(cudaMallocAsync(&d, sizeof(int), s));
  DAMN_CUDA(cudaMemsetAsync(d, 0, sizeof(int), s));
  const long long nt = (pl->nrows + (long long)tile_rows - 1) / tile_rows;
  k_plan_max_tile<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(pl->nrows, pl->rowptr, tile_rows, d);
  DAMN_CHECK_LAUNCH("k_plan_max_tile");
  DAMN_CUDA(cudaMemcpyAsync(out, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaFreeAsync(d, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  return DAMN_OK;
}

// Rows-mode tiling for uniform rows of mean length `mean`: the fewest lanes
// per row that keep at most 7 (one lane) or 14 (more lanes) of a row's
// entries per lane, among the tilings whose tiles fit a stage.
static int uniform_rows_tiling(const damn_plan *pl, double mean, cudaStream_t s, int *tiling) {
  *tiling = -1;
  const int cands[6] = {DAMN_TILING_ROWS, DAMN_TILING_ROWS_LONG, DAMN_TILING_ROWS_LANES4,
                        DAMN_TILING_ROWS_LANES8, DAMN_TILING_ROWS_LANES16, DAMN_TILING_ROWS_LANES32};
  const int lanes[6] = {1, 2, 4, 8, 16, 32};
  for (int i = 0; i < 6; ++i) {
    const CfgGeom g = cfg_geom(shape_of_tiling(cands[i]), pl->dtype);
    const double per_lane = mean / lanes[i];
    if (i < 5 && per_lane > (i == 0 ? 7.0 : 14.0)) continue;
    int mt = 0;
    if (i == 0) mt = pl->max_tile_short;
    else if (i == 1) mt = pl->max_tile_long;
    else {
      int rc = plan_max_tile(pl, g.tile_rows, s, &mt);
      if (rc) return rc;
    }
    if (mt <= g.cap_nz) { *tiling = cands[i]; return DAMN_OK; }
  }
  return DAMN_OK;
}

extern "C" int damn_plan_create(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                                int format, const void *idx, int dtype, void *stream,
                                damn_plan **out) {
  if (!out) return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_create: out is NULL");
  *out = nullptr;
  if (nrows < 0 || ncols < 0 || nnz < 0 || nnz > INT_MAX || (nrows > 0 && !rowptr))
    return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_create: bad arguments");
  if (dtype != DAMN_F64 && dtype != DAMN_F32 && dtype != DAMN_BF16 && dtype != DAMN_F8E4M3)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_create: bad dtype");
  if (idx && format != DAMN_FMT_CSR32 && format != DAMN_FMT_DACSR16 && format != DAMN_FMT_DACSR8)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_create: bad format");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  damn_plan *pl = new damn_plan();
  std::memset(pl, 0, sizeof(*pl));
  pl->nrows = nrows; pl->ncols = ncols; pl->nnz = nnz; pl->dtype = dtype;
  pl->rowptr = rowptr;
  pl->idx = nnz > 0 ? idx : nullptr;
  pl->fmt = format;
  const long long items = (long long)kRowWeight * nrows + nnz;
  const long long D = kBalancedItems;
  pl->ntiles_balanced = (int)((items + D - 1) / D);
  cudaError_t e = cudaMalloc(&pl->d_bounds_balanced, sizeof(int2) * (pl->ntiles_balanced + 1));
  if (e != cudaSuccess) { delete pl; return cuda_error(e, "damn_plan_create: cudaMalloc"); }
  PlanStats *d_st = nullptr;
  e = cudaMallocAsync(&d_st, sizeof(PlanStats), s);
  if (e != cudaSuccess) { plan_free_device(pl); delete pl; return cuda_error(e, "cudaMallocAsync"); }
  cudaMemsetAsync(d_st, 0, sizeof(PlanStats), s);
  if (nrows > 0) {
    k_plan_bounds<<<(pl->ntiles_balanced + 1 + 255) / 256, 256, 0, s>>>(
        nrows, rowptr, D, pl->ntiles_balanced, pl->d_bounds_balanced);
    k_plan_stats<<<(nrows + 255) / 256, 256, 0, s>>>(nrows, rowptr,
                                                     cfg_geom(0, dtype).tile_rows,
                                                     cfg_geom(1, dtype).tile_rows, d_st);
  }
  PlanStats h{};
  cudaMemcpyAsync(&h, d_st, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d_st, s);
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) { plan_free_device(pl); delete pl; return cuda_error(e, "damn_plan_create"); }
  pl->max_row = h.max_row;
  pl->max_tile_short = h.max_tile_short;
  pl->max_tile_long = h.max_tile_long;
  pl->row_eff = h.sum_group_max ? (double)nnz / (32.0 * (double)h.sum_group_max) : 1.0;
  // Heuristic choice.  Rows of uniform length inside 32-row groups: rows
  // mode with the fewest lanes per row that keep a row's entries in
  // registers.  Ragged rows: the sorted-rows tiling -- rows dealt to the
  // threads of a tile by decreasing length, so a warp's FMA steps carry
  // nearly full lanes, x through the ring when the band is narrow enough and
  // gathered otherwise.
  int tiling = DAMN_TILING_SORTED_ROWS;
  int rc = DAMN_OK;
  if (pl->row_eff >= 0.85) {
    int t = -1;
    rc = uniform_rows_tiling(pl, nrows > 0 ? (double)nnz / nrows : 0.0, s, &t);
    if (t >= 0) tiling = t;
  }
  if (!rc) rc = plan_use(pl, tiling, s);
  if (rc) { plan_free_device(pl); delete pl; return rc; }
  *out = pl;
  return DAMN_OK;
}

extern "C" int damn_plan_autotune(damn_plan *plan, int format, const void *idx, const void *val,
                                  const void *x, void *y, void *stream) {
  if (!plan) return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_autotune: plan is NULL");
  if (format != DAMN_FMT_CSR32 && format != DAMN_FMT_DACSR16 && format != DAMN_FMT_DACSR8)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_autotune: bad format");
  int rc = check_spmv_args("damn_plan_autotune", format, plan->nrows, plan->ncols, plan->nnz,
                           plan->rowptr, idx, val, plan->dtype, x, y, plan);
  if (rc) return rc;
  if (plan->nrows == 0) return DAMN_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SpmvCall c;
  c.nrows = plan->nrows; c.ncols = plan->ncols; c.nnz = plan->nnz; c.rowptr = plan->rowptr;
  c.idx = idx; c.fmt = format; c.val = val; c.dtype = plan->dtype; c.x = x; c.y0 = y; c.y = y;
  cudaEvent_t e0, e1;
  DAMN_CUDA(cudaEventCreate(&e0));
  DAMN_CUDA(cudaEventCreate(&e1));
  // best of 5 launches after 2 warm-up launches, in ms
  auto time_plan = [&](float *out) {
    int r2 = DAMN_OK;
    for (int w = 0; w < 2 && r2 == DAMN_OK; ++w) r2 = spmv_launch(c, plan, s, nullptr);
    float tmin = 1e30f;
    for (int r = 0; r < 5 && r2 == DAMN_OK; ++r) {
      cudaEventRecord(e0, s);
      r2 = spmv_launch(c, plan, s, nullptr);
      cudaEventRecord(e1, s);
      cudaError_t ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) { r2 = cuda_error(ce, "damn_plan_autotune"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      tmin = std::min(tmin, ms);
    }
    *out = tmin;
    return r2;
  };
  // 1. tilings: the fixed shapes, and the lanes-per-row tilings whose lanes
  //    would each hold at least two entries of an average row
  const double mean = (double)plan->nnz / plan->nrows;
  int cands[10], nc = 0;
  cands[nc++] = DAMN_TILING_ROWS;
  cands[nc++] = DAMN_TILING_ROWS_X2;
  cands[nc++] = DAMN_TILING_ROWS_LONG;
  cands[nc++] = DAMN_TILING_SLICES;
  cands[nc++] = DAMN_TILING_BAND;
  cands[nc++] = DAMN_TILING_SORTED_ROWS;
  const int lane_t[4] = {DAMN_TILING_ROWS_LANES4, DAMN_TILING_ROWS_LANES8, DAMN_TILING_ROWS_LANES16,
                         DAMN_TILING_ROWS_LANES32};
  for (int i = 0; i < 4; ++i)
    if (mean >= 2.0 * (4 << i)) cands[nc++] = lane_t[i];
  const int keep_stages = plan->stages_req;
  plan->stages_req = 0;
  plan->no_xstage = 0;
  float best_ms = 1e30f;
  int best = plan_tiling_of(plan);
  for (int ci = 0; ci < nc && rc == DAMN_OK; ++ci) {
    rc = plan_use(plan, cands[ci], s);
    float t = 1e30f;
    if (!rc) rc = time_plan(&t);
    if (t < best_ms) { best_ms = t; best = cands[ci]; }
  }
  // 2. ring depth for the best tiling: automatic, or 2 .. 6 stages
  int best_st = 0;
  if (!rc) rc = plan_use(plan, best, s);
  for (int st = 2; st <= 6 && rc == DAMN_OK; ++st) {
    plan->stages_req = st;
    float t = 1e30f;
    rc = time_plan(&t);
    if (plan->stages != st) continue;  // that depth does not fit this kernel
    if (t < 0.97f * best_ms) { best_ms = t; best_st = st; }
  }
  plan->stages_req = rc ? keep_stages : best_st;
  // 3. rows tilings: x staged in shared memory, or read from L1 / L2; band
  //    tiling: x through the ring, or gathered from L1 / L2 with the ring's
  //    shared memory left to the L1 cache
  if (!rc && ((plan->mode == 0 && plan->d_xseg) || (plan->mode == 2 && plan->d_colrange))) {
    plan->no_xstage = 1;
    float t = 1e30f;
    rc = time_plan(&t);
    if (rc || !(t < 0.97f * best_ms)) plan->no_xstage = 0;
    else best_ms = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

extern "C" int damn_plan_set_tiling(damn_plan *plan, int tiling) {
  if (!plan) return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_set_tiling: plan is NULL");
  if (shape_of_tiling(tiling) < 0)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_set_tiling: bad tiling %d", tiling);
  return plan_use(plan, tiling, nullptr);
}

extern "C" int damn_plan_set_x_staging(damn_plan *plan, int32_t on) {
  if (!plan) return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_set_x_staging: plan is NULL");
  plan->no_xstage = on ? 0 : 1;
  return DAMN_OK;
}

extern "C" int damn_plan_set_stages(damn_plan *plan, int32_t stages) {
  if (!plan) return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_set_stages: plan is NULL");
  if (stages != 0 && (stages < 2 || stages > kMaxStages))
    return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_set_stages: stages must be 0 or 2..%d",
                     kMaxStages);
  plan->stages_req = stages;
  return DAMN_OK;
}

extern "C" int damn_plan_describe(const damn_plan *plan, damn_plan_desc *h_desc) {
  if (!plan || !h_desc) return set_error(DAMN_ERR_INVALID_ARG, "damn_plan_describe: NULL");
  h_desc->mode = plan->mode;
  h_desc->tile_items = plan->rows_per_tile > 0    ? plan->rows_per_tile
                       : plan->shape == kShapeSorted ? CfgSorted64::NT
                                                     : kBalancedItems;
  h_desc->ntiles = plan->ntiles;
  h_desc->grid = plan->grid;
  h_desc->stages = plan->stages;
  h_desc->threads = cfg_geom(plan->shape, plan->dtype).threads;
  h_desc->row_efficiency = plan->row_eff;
  h_desc->max_row = plan->max_row;
  h_desc->dtype = plan->dtype;
  h_desc->tiling = plan_tiling_of(plan);
  h_desc->x_staged_tiles = plan->staged_tiles;
  h_desc->stages_requested = plan->stages_req;
  h_desc->x_staging = plan->no_xstage ? 0 : 1;
  return DAMN_OK;
}

extern "C" int damn_plan_destroy(damn_plan *plan) {
  if (!plan) return DAMN_OK;
  plan_free_device(plan);
  delete plan;
  return DAMN_OK;
}
