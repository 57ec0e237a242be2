// Multi-right-hand-side products Y = A X for DA-CSR-16 matrices, singly and
// for a whole batch of independent matrices in one persistent launch.
//
// For each matrix, X is row-major ncols x k and Y row-major nrows x k; entry
// i of row r multiplies row r + off[i] of X (the shifted view of Listing 2,
// Section 4, applied to each column of X).
//
// Work decomposition: a row group of L * E lanes computes one row, L = the
// largest power of two <= min(k, 32): column lane l owns the right-hand-side
// columns l, l + L (at most two), so the X loads of a row group are
// contiguous; entry lane e walks the row's entries e, e + E, ... (E = 1:
// Listing 2 order per column), four steps at a time so that several loads
// are in flight, and the E partial sums are added by a butterfly.  A warp
// takes 32 / (L * E) rows per pass.
//
// Batched launch: the host builds a list of (matrix, first row) work items
// of rows_per_item rows each; persistent warps take items round-robin.  A
// warp's row groups either take the item's rows in fixed passes (a pass
// lasts as long as its longest row) or are streamed rows (a group whose row
// ended takes the item's next row at once); both sum a row the same way.
// The plan's autotuner times the (schedule, rows_per_item, E, threads)
// shapes on the real operands and keeps the fastest; the launch is captured
// in a CUDA graph.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "damn_common.cuh"

namespace damn {
namespace {

struct DevDesc {  // device copy of damn_mat_desc
  int nrows, ncols;
  long long nnz;
  const int *rowptr;
  const int16_t *off;
  const void *val;
  const void *X;
  void *Y;
};

// One row group of G = L * E lanes computes y[row, :]: column lane li owns
// the right-hand-side columns li, li + L (at most J of them), entry lane ei
// takes the row's entries ei, ei + E, ... in stored order; the E partial sums
// of a column are then added by a butterfly over the entry lanes (a fixed
// order, so results depend only on (L, J, E)).  All lanes of the warp call
// this together (valid == false for a lane whose row does not exist).
template <typename T, int L, int J, int E>
__device__ __forceinline__ void spmm_row(const DevDesc &d, int row, bool valid, int k, int li,
                                         int ei) {
  const T *val = static_cast<const T *>(d.val);
  const T *X = static_cast<const T *>(d.X);
  T *Y = static_cast<T *>(d.Y);
  int b = 0, e = 0;
  if (valid) {
    b = __ldg(d.rowptr + row);
    e = __ldg(d.rowptr + row + 1);
  }
  T acc[J];
#pragma unroll
  for (int jj = 0; jj < J; ++jj) acc[jj] = T(0);
  constexpr int U = 4;
  const unsigned ncols = static_cast<unsigned>(d.ncols);
  for (int q0 = b + ei; q0 < e; q0 += U * E) {
    T v[U];
    unsigned c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u * E;
      v[u] = T(0);
      c[u] = 0;
      if (q < e) {
        v[u] = __ldg(val + q);
        // a column outside [0, ncols) (an invalid offset) reads a valid row
        c[u] = min(static_cast<unsigned>(row + static_cast<int>(__ldg(d.off + q))), ncols - 1u);
      }
    }
    T xv[U][J];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int jj = 0; jj < J; ++jj) {
        const int j = li + jj * L;
        xv[u][jj] = (q0 + u * E < e && j < k) ? __ldg(X + (size_t)c[u] * k + j) : T(0);
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q0 + u * E < e)
#pragma unroll
        for (int jj = 0; jj < J; ++jj) acc[jj] = fma_acc(v[u], xv[u][jj], acc[jj]);
  }
#pragma unroll
  for (int o = L; o < L * E; o <<= 1)
#pragma unroll
    for (int jj = 0; jj < J; ++jj) acc[jj] += __shfl_xor_sync(0xffffffffu, acc[jj], o);
  if (valid && ei == 0) {
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
      const int j = li + jj * L;
      if (j < k) Y[(size_t)row * k + j] = acc[jj];
    }
  }
}

// Batched: items[i] = {matrix, first row}; rows_per_item rows per item.
template <typename T, int L, int J, int E>
__global__ void k_spmm_batched(const DevDesc *descs, const int2 *items, int nitems, int k,
                               int rows_per_item) {
  constexpr int G = L * E, R = 32 / G;
  const int lane = threadIdx.x & 31, grp = lane / G, li = lane % L, ei = (lane % G) / L;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long it = warp; it < nitems; it += nwarps) {
    const int2 item = items[it];
    const DevDesc d = descs[item.x];
    const int rend = min(item.y + rows_per_item, d.nrows);
    for (int base = item.y; base < rend; base += R)  // warp-uniform bound: shuffles
      spmm_row<T, L, J, E>(d, base + grp, base + grp < rend, k, li, ei);
  }
}

// One matrix: the rows are the work, no descriptor array.
template <typename T, int L, int J, int E>
__global__ void k_spmm_single(DevDesc d, int k) {
  constexpr int G = L * E, R = 32 / G;
  const int lane = threadIdx.x & 31, grp = lane / G, li = lane % L, ei = (lane % G) / L;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * R; base < d.nrows; base += nwarps * R)
    spmm_row<T, L, J, E>(d, static_cast<int>(base + grp), base + grp < d.nrows, k, li, ei);
}

// Row-streaming batched kernel: the same row groups and the same per-row
// arithmetic as k_spmm_batched (so the same bits for the same (k, E)), but a
// group that has finished its row takes the item's next row at once instead
// of waiting for the longest row of the warp's pass.  The warp steps U
// entries per entry lane at a time; after each step the groups whose row
// ended add their entry lanes' sums (butterfly), write the row and are dealt
// the next rows in order (a ballot over the finished groups).  So a warp's
// FMA steps stay nearly full whatever the mix of row lengths; an empty row
// costs one step.  Groups of one or two lanes step 8 entries per lane (more
// loads in flight per lane, where each lane gathers from its own row), wider
// groups 4.
template <typename T, int L, int J, int E>
__global__ void k_spmm_streamed(const DevDesc *descs, const int2 *items, int nitems, int k,
                                int rows_per_item) {
  constexpr int G = L * E, R = 32 / G, U = G <= 2 ? 8 : 4;
  const int lane = threadIdx.x & 31, grp = lane / G, li = lane % L, ei = (lane % G) / L;
  const bool leader = (lane % G) == 0;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long it = warp; it < nitems; it += nwarps) {
    const int2 item = items[it];
    const DevDesc d = descs[item.x];
    const int r0 = item.y, nr = min(rows_per_item, d.nrows - r0);
    const T *val = static_cast<const T *>(d.val);
    const T *X = static_cast<const T *>(d.X);
    T *Y = static_cast<T *>(d.Y);
    const unsigned ncols = static_cast<unsigned>(d.ncols);
    int row = grp, next = R, pos = 0, end = 0;
    if (row < nr) {
      pos = __ldg(d.rowptr + r0 + row);
      end = __ldg(d.rowptr + r0 + row + 1);
    }
    T acc[J];
#pragma unroll
    for (int jj = 0; jj < J; ++jj) acc[jj] = T(0);
    while (__any_sync(0xffffffffu, row < nr)) {
      const bool active = row < nr;
      T v[U];
      unsigned c[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = pos + ei + u * E;
        v[u] = T(0);
        c[u] = 0;
        if (active && q < end) {
          v[u] = __ldg(val + q);
          // a column outside [0, ncols) (an invalid offset) reads a valid row
          c[u] = min(static_cast<unsigned>(r0 + row + static_cast<int>(__ldg(d.off + q))),
                     ncols - 1u);
        }
      }
      T xv[U][J];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
          const int j = li + jj * L;
          xv[u][jj] = (active && pos + ei + u * E < end && j < k) ? __ldg(X + (size_t)c[u] * k + j)
                                                                  : T(0);
        }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (active && pos + ei + u * E < end)
#pragma unroll
          for (int jj = 0; jj < J; ++jj) acc[jj] = fma_acc(v[u], xv[u][jj], acc[jj]);
      pos += U * E;
      const bool done = active && pos >= end;
      if (__any_sync(0xffffffffu, done)) {
        T tot[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) tot[jj] = acc[jj];
#pragma unroll
        for (int o = L; o < G; o <<= 1)
#pragma unroll
          for (int jj = 0; jj < J; ++jj) tot[jj] += __shfl_xor_sync(0xffffffffu, tot[jj], o);
        const unsigned dm = __ballot_sync(0xffffffffu, done && leader);
        if (done) {
          if (ei == 0) {
#pragma unroll
            for (int jj = 0; jj < J; ++jj) {
              const int j = li + jj * L;
              if (j < k) Y[(size_t)(r0 + row) * k + j] = tot[jj];
            }
          }
#pragma unroll
          for (int jj = 0; jj < J; ++jj) acc[jj] = T(0);
          // this group's rank among the finished groups (its leader's bit)
          row = next + __popc(dm & ((1u << (grp * G)) - 1u));
          if (row < nr) {
            pos = __ldg(d.rowptr + r0 + row);
            end = __ldg(d.rowptr + r0 + row + 1);
          }
        }
        next += __popc(dm);
      }
    }
  }
}

int lanes_for(int k) {
  int L = 1;
  while (L * 2 <= std::min(k, 32)) L *= 2;
  return L;
}

// Entry lanes for one matrix without timing: about four entries per lane
// and pass, at most 32 / L.
int entry_lanes_for(const DevDesc &d, int L) {
  const double avg = d.nrows > 0 ? (double)d.nnz / d.nrows : 0.0;
  int E = 1;
  while (E * 2 * L <= 32 && E * 2 * 4 <= avg) E *= 2;
  return E;
}

template <typename T, int L, int E>
int launch_single_le(const DevDesc &d, int k, cudaStream_t s) {
  constexpr int R = 32 / (L * E);
  const long long warps_needed = (d.nrows + R - 1) / R;
  const int threads = 256;
  const int blocks = (int)std::max(1LL, std::min<long long>(8LL * sm_count(),
                                                            (warps_needed * 32 + threads - 1) / threads));
  if ((k + L - 1) / L <= 1)
    k_spmm_single<T, L, 1, E><<<blocks, threads, 0, s>>>(d, k);
  else
    k_spmm_single<T, L, 2, E><<<blocks, threads, 0, s>>>(d, k);
  DAMN_CHECK_LAUNCH("k_spmm_single");
  return DAMN_OK;
}

template <typename T, int L>
int launch_single_l(const DevDesc &d, int k, int E, cudaStream_t s) {
  if constexpr (L <= 16)
    if (E >= 2) {
      if constexpr (L <= 4)
        if (E >= 8) return launch_single_le<T, L, 8>(d, k, s);
      if constexpr (L <= 8)
        if (E >= 4) return launch_single_le<T, L, 4>(d, k, s);
      return launch_single_le<T, L, 2>(d, k, s);
    }
  return launch_single_le<T, L, 1>(d, k, s);
}

template <typename T>
int launch_single(const DevDesc &d, int k, int E, cudaStream_t s) {
  switch (lanes_for(k)) {
    case 1: return launch_single_l<T, 1>(d, k, E, s);
    case 2: return launch_single_l<T, 2>(d, k, E, s);
    case 4: return launch_single_l<T, 4>(d, k, E, s);
    case 8: return launch_single_l<T, 8>(d, k, E, s);
    case 16: return launch_single_l<T, 16>(d, k, E, s);
    default: return launch_single_l<T, 32>(d, k, E, s);
  }
}

template <typename T, int L, int E>
int launch_batched_le(const DevDesc *descs, const int2 *items, int nitems, int k, int rpi,
                      int blocks, int threads, cudaStream_t s) {
  if ((k + L - 1) / L <= 1)
    k_spmm_batched<T, L, 1, E><<<blocks, threads, 0, s>>>(descs, items, nitems, k, rpi);
  else
    k_spmm_batched<T, L, 2, E><<<blocks, threads, 0, s>>>(descs, items, nitems, k, rpi);
  DAMN_CHECK_LAUNCH("k_spmm_batched");
  return DAMN_OK;
}

template <typename T, int L>
int launch_batched_l(const DevDesc *descs, const int2 *items, int nitems, int k, int rpi, int E,
                     int blocks, int threads, cudaStream_t s) {
  if constexpr (L <= 16)
    if (E >= 2) {
      if constexpr (L <= 4)
        if (E >= 8) return launch_batched_le<T, L, 8>(descs, items, nitems, k, rpi, blocks, threads, s);
      if constexpr (L <= 8)
        if (E >= 4) return launch_batched_le<T, L, 4>(descs, items, nitems, k, rpi, blocks, threads, s);
      return launch_batched_le<T, L, 2>(descs, items, nitems, k, rpi, blocks, threads, s);
    }
  return launch_batched_le<T, L, 1>(descs, items, nitems, k, rpi, blocks, threads, s);
}

template <typename T>
int launch_batched(const DevDesc *descs, const int2 *items, int nitems, int k, int rpi, int E,
                   int blocks, int threads, cudaStream_t s) {
  switch (lanes_for(k)) {
    case 1: return launch_batched_l<T, 1>(descs, items, nitems, k, rpi, E, blocks, threads, s);
    case 2: return launch_batched_l<T, 2>(descs, items, nitems, k, rpi, E, blocks, threads, s);
    case 4: return launch_batched_l<T, 4>(descs, items, nitems, k, rpi, E, blocks, threads, s);
    case 8: return launch_batched_l<T, 8>(descs, items, nitems, k, rpi, E, blocks, threads, s);
    case 16: return launch_batched_l<T, 16>(descs, items, nitems, k, rpi, E, blocks, threads, s);
    default: return launch_batched_l<T, 32>(descs, items, nitems, k, rpi, E, blocks, threads, s);
  }
}

template <typename T, int L, int E>
int launch_streamed_le(const DevDesc *descs, const int2 *items, int nitems, int k, int rpi,
                       int blocks, int threads, cudaStream_t s) {
  if ((k + L - 1) / L <= 1)
    k_spmm_streamed<T, L, 1, E><<<blocks, threads, 0, s>>>(descs, items, nitems, k, rpi);
  else
    k_spmm_streamed<T, L, 2, E><<<blocks, threads, 0, s>>>(descs, items, nitems, k, rpi);
  DAMN_CHECK_LAUNCH("k_spmm_streamed");
  return DAMN_OK;
}

template <typename T, int L>
int launch_streamed_l(const DevDesc *descs, const int2 *items, int nitems, int k, int rpi, int E,
                      int blocks, int threads, cudaStream_t s) {
  if constexpr (L <= 16)
    if (E >= 2) {
      if constexpr (L <= 4)
        if (E >= 8) return launch_streamed_le<T, L, 8>(descs, items, nitems, k, rpi, blocks, threads, s);
      if constexpr (L <= 8)
        if (E >= 4) return launch_streamed_le<T, L, 4>(descs, items, nitems, k, rpi, blocks, threads, s);
      return launch_streamed_le<T, L, 2>(descs, items, nitems, k, rpi, blocks, threads, s);
    }
  return launch_streamed_le<T, L, 1>(descs, items, nitems, k, rpi, blocks, threads, s);
}

template <typename T>
int launch_streamed(const DevDesc *descs, const int2 *items, int nitems, int k, int rpi, int E,
                    int blocks, int threads, cudaStream_t s) {
  switch (lanes_for(k)) {
    case 1: return launch_streamed_l<T, 1>(descs, items, nitems, k, rpi, E, blocks, threads, s);
    case 2: return launch_streamed_l<T, 2>(descs, items, nitems, k, rpi, E, blocks, threads, s);
    case 4: return launch_streamed_l<T, 4>(descs, items, nitems, k, rpi, E, blocks, threads, s);
    case 8: return launch_streamed_l<T, 8>(descs, items, nitems, k, rpi, E, blocks, threads, s);
    case 16: return launch_streamed_l<T, 16>(descs, items, nitems, k, rpi, E, blocks, threads, s);
    default: return launch_streamed_l<T, 32>(descs, items, nitems, k, rpi, E, blocks, threads, s);
  }
}

// Entry positions are int and step past a row's end by up to 32 (U entries
// for each of the E entry lanes): nnz keeps that headroom below INT_MAX.
constexpr long long kMaxSpmmNnz = (long long)INT_MAX - 64;

bool desc_ok(const damn_mat_desc &m) {
  if (m.nrows < 0 || m.ncols < 0 || m.nnz < 0 || m.nnz > kMaxSpmmNnz) return false;
  if (m.nrows > 0 && (!m.rowptr || !m.Y)) return false;
  if (m.nnz > 0 && (!m.off || !m.val || !m.X || m.ncols == 0)) return false;
  return true;
}

}  // namespace
}  // namespace damn

using namespace damn;

constexpr int kMaxRowsPerItem = 1024;

struct damn_batch_plan {
  int count, k, dtype;
  DevDesc *d_descs;
  int2 *d_items;
  int nitems;
  int rows_per_item;
  int streamed;            // 1: row groups take the next row as they finish
  int entry_lanes;         // E: lanes splitting each row's entries
  int threads, blocks;
  std::vector<int> nrows;  // per matrix, to rebuild items
  cudaGraphExec_t graph;
  double tune_ms;
};

static int batch_build_items(damn_batch_plan *pl, int rpi) {
  std::vector<int2> items;
  for (int m = 0; m < pl->count; ++m)
    for (int r = 0; r < pl->nrows[m]; r += rpi) items.push_back(make_int2(m, r));
  if (pl->d_items) cudaFree(pl->d_items);
  pl->d_items = nullptr;
  pl->nitems = (int)items.size();
  pl->rows_per_item = rpi;
  if (items.empty()) return DAMN_OK;
  DAMN_CUDA(cudaMalloc(&pl->d_items, sizeof(int2) * items.size()));
  DAMN_CUDA(cudaMemcpy(pl->d_items, items.data(), sizeof(int2) * items.size(),
                       cudaMemcpyHostToDevice));
  return DAMN_OK;
}

// Persistent grid: one warp per item, at most 16 blocks per SM.
static void batch_set_grid(damn_batch_plan *pl) {
  const int wpb = pl->threads / 32;
  pl->blocks = std::max(1, std::min(16 * sm_count(), (pl->nitems + wpb - 1) / wpb));
}

static int batch_launch(const damn_batch_plan *pl, cudaStream_t s);

// Captures the persistent launch of the plan's current shape in a CUDA graph
// (replacing an earlier one).
static int batch_capture(damn_batch_plan *pl) {
  if (pl->graph) cudaGraphExecDestroy(pl->graph);
  pl->graph = nullptr;
  if (pl->nitems == 0) return DAMN_OK;
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamCreate");
  cudaGraph_t g = nullptr;
  int rc = DAMN_OK;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = batch_launch(pl, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess && rc == DAMN_OK) e = cudaGraphInstantiate(&pl->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_error(e, "batch plan graph capture");
  return DAMN_OK;
}

static int batch_launch(const damn_batch_plan *pl, cudaStream_t s) {
  if (pl->nitems == 0) return DAMN_OK;
  if (pl->streamed)
    return pl->dtype == DAMN_F64
               ? launch_streamed<double>(pl->d_descs, pl->d_items, pl->nitems, pl->k,
                                         pl->rows_per_item, pl->entry_lanes, pl->blocks,
                                         pl->threads, s)
               : launch_streamed<float>(pl->d_descs, pl->d_items, pl->nitems, pl->k,
                                        pl->rows_per_item, pl->entry_lanes, pl->blocks,
                                        pl->threads, s);
  if (pl->dtype == DAMN_F64)
    return launch_batched<double>(pl->d_descs, pl->d_items, pl->nitems, pl->k, pl->rows_per_item,
                                  pl->entry_lanes, pl->blocks, pl->threads, s);
  return launch_batched<float>(pl->d_descs, pl->d_items, pl->nitems, pl->k, pl->rows_per_item,
                               pl->entry_lanes, pl->blocks, pl->threads, s);
}

static void batch_free(damn_batch_plan *pl) {
  if (pl->graph) cudaGraphExecDestroy(pl->graph);
  if (pl->d_items) cudaFree(pl->d_items);
  if (pl->d_descs) cudaFree(pl->d_descs);
  pl->graph = nullptr;
  pl->d_items = nullptr;
  pl->d_descs = nullptr;
}

extern "C" int damn_spmm_dacsr16(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                                 const int16_t *off, const void *val, int dtype, int32_t k,
                                 const void *X, void *Y, void *stream) {
  damn_mat_desc m{nrows, ncols, nnz, rowptr, off, val, X, Y};
  if (!desc_ok(m)) return set_error(DAMN_ERR_INVALID_ARG, "damn_spmm_dacsr16: bad arguments");
  if (dtype != DAMN_F64 && dtype != DAMN_F32)
    return set_error(DAMN_ERR_UNSUPPORTED, "damn_spmm_dacsr16: dtype must be DAMN_F64 or DAMN_F32");
  if (k < 1 || k > 64) return set_error(DAMN_ERR_INVALID_ARG, "damn_spmm_dacsr16: k must be 1..64");
  if (nrows == 0) return DAMN_OK;
  DevDesc d{nrows, ncols, nnz, rowptr, off, val, X, Y};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int E = entry_lanes_for(d, lanes_for(k));
  return dtype == DAMN_F64 ? launch_single<double>(d, k, E, s) : launch_single<float>(d, k, E, s);
}

extern "C" int damn_batch_plan_create(int32_t count, const damn_mat_desc *h_descs, int32_t k,
                                      int dtype, int autotune, void *stream,
                                      damn_batch_plan **out) {
  if (!out) return set_error(DAMN_ERR_INVALID_ARG, "damn_batch_plan_create: out is NULL");
  *out = nullptr;
  if (count < 0 || (count > 0 && !h_descs))
    return set_error(DAMN_ERR_INVALID_ARG, "damn_batch_plan_create: bad count / descriptors");
  if (dtype != DAMN_F64 && dtype != DAMN_F32)
    return set_error(DAMN_ERR_UNSUPPORTED, "damn_batch_plan_create: dtype must be F64 or F32");
  if (k < 1 || k > 64) return set_error(DAMN_ERR_INVALID_ARG, "damn_batch_plan_create: k must be 1..64");
  for (int m = 0; m < count; ++m)
    if (!desc_ok(h_descs[m]))
      return set_error(DAMN_ERR_INVALID_ARG, "damn_batch_plan_create: bad descriptor %d", m);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  damn_batch_plan *pl = new damn_batch_plan();
  pl->count = count; pl->k = k; pl->dtype = dtype;
  pl->d_descs = nullptr; pl->d_items = nullptr; pl->graph = nullptr; pl->tune_ms = 0.0;
  pl->nrows.resize(count);
  std::vector<DevDesc> dd(count);
  for (int m = 0; m < count; ++m) {
    const damn_mat_desc &h = h_descs[m];
    dd[m] = DevDesc{h.nrows, h.ncols, h.nnz, h.rowptr, h.off, h.val, h.X, h.Y};
    pl->nrows[m] = h.nrows;
  }
  auto fail = [&](int rc) { batch_free(pl); delete pl; return rc; };
  if (count > 0) {
    cudaError_t e = cudaMalloc(&pl->d_descs, sizeof(DevDesc) * count);
    if (e != cudaSuccess) return fail(cuda_error(e, "damn_batch_plan_create: cudaMalloc"));
    e = cudaMemcpy(pl->d_descs, dd.data(), sizeof(DevDesc) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_error(e, "damn_batch_plan_create: cudaMemcpy"));
  }
  // default shape: about four entries per lane and pass, items of 256 rows
  long long tot_rows = 0, tot_nnz = 0;
  for (int m = 0; m < count; ++m) { tot_rows += h_descs[m].nrows; tot_nnz += h_descs[m].nnz; }
  const int L = lanes_for(k);
  {
    DevDesc avg{(int)std::min<long long>(tot_rows, INT_MAX), 0, tot_nnz, nullptr, nullptr, nullptr,
                nullptr, nullptr};
    pl->entry_lanes = entry_lanes_for(avg, L);
  }
  pl->streamed = 0;
  int rc = batch_build_items(pl, 256);
  if (rc) return fail(rc);
  pl->threads = 256;
  batch_set_grid(pl);
  if (autotune && pl->nitems > 0) {
    // candidates: every E, row groups in fixed passes over items of 64 or
    // 256 rows and streamed rows over items of 256 or 1024 rows, 128 or 256
    // threads per block
    struct Shape { int streamed, rpi, E, threads; };
    std::vector<Shape> cand;
    for (int streamed : {0, 1})
      for (int rpi : {64, 256})
        for (int tp : {128, 256})
          for (int E = 1; E * L <= 32 && E <= 8; E *= 2)
            cand.push_back({streamed, streamed ? 4 * rpi : rpi, E, tp});
    float best = 1e30f;
    Shape bs = {pl->streamed, pl->rows_per_item, pl->entry_lanes, pl->threads};
    cudaEvent_t e0, e1;
    DAMN_CUDA(cudaEventCreate(&e0));
    DAMN_CUDA(cudaEventCreate(&e1));
    for (size_t c = 0; c < cand.size() && rc == DAMN_OK; ++c) {
      if (cand[c].rpi != pl->rows_per_item) rc = batch_build_items(pl, cand[c].rpi);
      if (rc) break;
      pl->streamed = cand[c].streamed;
      pl->entry_lanes = cand[c].E;
      pl->threads = cand[c].threads;
      batch_set_grid(pl);
      rc = batch_launch(pl, s);  // warm
      float tmin = 1e30f;
      for (int r = 0; r < 3 && rc == DAMN_OK; ++r) {
        cudaEventRecord(e0, s);
        rc = batch_launch(pl, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        tmin = std::min(tmin, ms);
      }
      if (tmin < best) { best = tmin; bs = cand[c]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return fail(rc);
    if (bs.rpi != pl->rows_per_item) rc = batch_build_items(pl, bs.rpi);
    if (rc) return fail(rc);
    pl->streamed = bs.streamed;
    pl->entry_lanes = bs.E;
    pl->threads = bs.threads;
    batch_set_grid(pl);
    pl->tune_ms = best;
  }
  rc = batch_capture(pl);
  if (rc) return fail(rc);
  DAMN_CUDA(cudaStreamSynchronize(s));
  *out = pl;
  return DAMN_OK;
}

extern "C" int damn_batch_plan_set_shape(damn_batch_plan *plan, int32_t streamed,
                                         int32_t rows_per_item, int32_t entry_lanes,
                                         int32_t threads, void *stream) {
  if (!plan) return set_error(DAMN_ERR_INVALID_ARG, "damn_batch_plan_set_shape: plan is NULL");
  if (rows_per_item < 1 || rows_per_item > kMaxRowsPerItem)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_batch_plan_set_shape: rows_per_item must be 1..%d",
                     kMaxRowsPerItem);
  if (threads != 32 && threads != 64 && threads != 128 && threads != 256)
    return set_error(DAMN_ERR_INVALID_ARG,
                     "damn_batch_plan_set_shape: threads must be 32, 64, 128 or 256");
  const int L = lanes_for(plan->k);
  if (entry_lanes < 1 || entry_lanes > 8 || (entry_lanes & (entry_lanes - 1)) ||
      L * entry_lanes > 32)
    return set_error(DAMN_ERR_INVALID_ARG,
                     "damn_batch_plan_set_shape: entry_lanes must be a power of two <= 8 with "
                     "%d * entry_lanes <= 32", L);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DAMN_CUDA(cudaStreamSynchronize(s));  // no launch of the old shape in flight
  int rc = batch_build_items(plan, rows_per_item);
  if (rc) return rc;
  plan->streamed = streamed ? 1 : 0;
  plan->entry_lanes = entry_lanes;
  plan->threads = threads;
  batch_set_grid(plan);
  plan->tune_ms = 0.0;
  return batch_capture(plan);
}

extern "C" int damn_batch_plan_describe(const damn_batch_plan *plan, damn_batch_desc *h) {
  if (!plan || !h) return set_error(DAMN_ERR_INVALID_ARG, "damn_batch_plan_describe: NULL");
  h->count = plan->count;
  h->k = plan->k;
  h->dtype = plan->dtype;
  h->ntiles = plan->nitems;
  h->grid = plan->blocks;
  h->threads = plan->threads;
  h->tile_items = plan->rows_per_item;
  h->graph_ready = plan->graph ? 1 : 0;
  h->entry_lanes = plan->entry_lanes;
  h->streamed = plan->streamed;
  h->tune_ms = plan->tune_ms;
  return DAMN_OK;
}

extern "C" int damn_batch_plan_destroy(damn_batch_plan *plan) {
  if (!plan) return DAMN_OK;
  batch_free(plan);
  delete plan;
  return DAMN_OK;
}

extern "C" int damn_spmm_dacsr16_batched(const damn_batch_plan *plan, void *stream) {
  if (!plan) return set_error(DAMN_ERR_INVALID_ARG, "damn_spmm_dacsr16_batched: plan is NULL");
  return batch_launch(plan, static_cast<cudaStream_t>(stream));
}

extern "C" int damn_batch_graph_launch(damn_batch_plan *plan, void *stream) {
  if (!plan) return set_error(DAMN_ERR_INVALID_ARG, "damn_batch_graph_launch: plan is NULL");
  if (!plan->graph) return DAMN_OK;  // empty batch
  DAMN_CUDA(cudaGraphLaunch(plan->graph, static_cast<cudaStream_t>(stream)));
  return DAMN_OK;
}
