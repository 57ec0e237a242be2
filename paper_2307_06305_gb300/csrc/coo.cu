// COO SpMV with absolute columns (COO-32) or columns addressed from the
// diagonal (DA-COO-16: the column vector of COO storage stored as c - r in
// int16; the paper notes the technique applies to one of COO's vectors,
// Section 1).  Entries are sorted by row; the row vector stays int32.
//
// Deterministic two-pass scheme, no atomics:
//  1. one CTA per tile of kTile consecutive entries, kChunk of them per
//     thread, read with 16-byte loads.  A thread sums each run of equal rows
//     of its chunk in stored order.  Tile T owns the rows
//     (row[first entry of T] - 1 ... row[last entry of T]], empty rows
//     included (the last tile also owns every row after the last entry), so
//     the tiles' row ranges partition [0, nrows).  A row crossing threads is
//     finished by the thread holding its first entry, which adds the
//     following threads' first-run sums left to right from shared memory.
//     The CTA then writes y for all its rows in one coalesced pass:
//     y[r] = alpha * sum + beta * y[r] (y[r] not read when beta = 0).  Two
//     partial sums leave the tile: the sum of its leading run when that run
//     continues a row owned by an earlier tile (carry_first), and the sum of
//     its own last row when that row goes on into the next tile
//     (carry_last);
//  2. a row crossing tiles is finished by its owner tile: carry_last plus
//     the carry_first of the following tiles the row continues into, added
//     left to right.
// Every y[r] has exactly one writer in pass 1 or 2.
#include <algorithm>
#include <climits>

#include "damn_common.cuh"

namespace damn {
namespace {

constexpr int kChunk = 8;                  // entries per thread
constexpr int kThreads = 256;
constexpr int kTile = kChunk * kThreads;   // entries per CTA
constexpr int kRowCap = 2048;              // owned rows summed in shared memory per pass

template <typename A>
__global__ void k_coo_scale(long long n, A *y, double beta) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = beta == 0.0 ? A(0) : static_cast<A>(beta) * y[i];
}

template <typename T> __device__ __forceinline__ T from_bits(unsigned long long b);
template <> __device__ __forceinline__ int from_bits<int>(unsigned long long b) { return (int)(unsigned)b; }
template <> __device__ __forceinline__ int16_t from_bits<int16_t>(unsigned long long b) {
  return (int16_t)(unsigned short)b;
}
template <> __device__ __forceinline__ float from_bits<float>(unsigned long long b) {
  return __uint_as_float((unsigned)b);
}
template <> __device__ __forceinline__ double from_bits<double>(unsigned long long b) {
  return __longlong_as_double((long long)b);
}
template <> __device__ __forceinline__ __nv_bfloat16 from_bits<__nv_bfloat16>(unsigned long long b) {
  return __ushort_as_bfloat16((unsigned short)b);
}

// kChunk elements starting at p (16-byte aligned) with 16-byte streaming loads
template <typename T>
__device__ __forceinline__ void load_chunk(const T *p, T (&out)[kChunk]) {
  constexpr int S = (int)sizeof(T);
  constexpr int NV = kChunk * S / 16;
  static_assert(NV * 16 == kChunk * S, "chunk is whole 16-byte words");
  unsigned w[4 * NV];
  const int4 *q = reinterpret_cast<const int4 *>(p);
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const int4 v = __ldcs(q + i);
    w[4 * i] = (unsigned)v.x;
    w[4 * i + 1] = (unsigned)v.y;
    w[4 * i + 2] = (unsigned)v.z;
    w[4 * i + 3] = (unsigned)v.w;
  }
#pragma unroll
  for (int i = 0; i < kChunk; ++i) {
    if (S == 8)
      out[i] = from_bits<T>((unsigned long long)w[2 * i] | ((unsigned long long)w[2 * i + 1] << 32));
    else if (S == 4)
      out[i] = from_bits<T>(w[i]);
    else
      out[i] = from_bits<T>(w[i / 2] >> (16 * (i % 2)));
  }
}

template <typename A>
__device__ __forceinline__ void coo_store(A *y, int r, A sum, double alpha, double beta) {
  const A yb = beta == 0.0 ? A(0) : static_cast<A>(beta) * y[r];
  y[r] = fma_acc(static_cast<A>(alpha), sum, yb);
}

template <typename V, typename I, bool VEC>
__global__ void __launch_bounds__(kThreads) k_coo_tiles(
    int nrows, long long nnz, const int *__restrict__ row, const I *__restrict__ idx,
    const V *__restrict__ val, const typename AccOf<V>::type *__restrict__ x,
    typename AccOf<V>::type *__restrict__ y, double alpha, double beta,
    typename AccOf<V>::type *carry_first, typename AccOf<V>::type *carry_last) {
  using A = typename AccOf<V>::type;
  constexpr bool DA = sizeof(I) < 4;
  __shared__ int s_fr[kThreads], s_lr[kThreads], s_n[kThreads];
  __shared__ A s_fs[kThreads];
  __shared__ A s_acc[kRowCap];
  const int tid = threadIdx.x;
  const long long T = blockIdx.x;
  const long long ntiles = gridDim.x;
  const long long t0 = T * kTile;
  const long long t1 = min(t0 + kTile, nnz);
  const long long e0 = t0 + (long long)tid * kChunk;
  const int n = (int)max(0LL, min((long long)kChunk, t1 - e0));

  // the chunk: rows, products of value and x in registers
  int r[kChunk];
  A pr[kChunk];
  int j1 = n, rlast = INT_MAX;
  A fs = 0, ls = 0;
  {
    I ix[kChunk];
    V vv[kChunk];
    if (VEC && n == kChunk) {
      load_chunk(row + e0, r);
      load_chunk(idx + e0, ix);
      load_chunk(val + e0, vv);
    } else {
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        r[u] = u < n ? __ldcs(row + e0 + u) : INT_MAX;
        ix[u] = u < n ? idx[e0 + u] : I(0);
        vv[u] = u < n ? val[e0 + u] : V(0);
      }
    }
    A xv[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u)
      if (u < n) xv[u] = __ldg(x + (DA ? r[u] + static_cast<int>(ix[u]) : static_cast<int>(ix[u])));
#pragma unroll
    for (int u = 0; u < kChunk; ++u) pr[u] = u < n ? to_acc(vv[u]) : A(0);
    // run sums in stored order; pr[u] becomes the run's sum up to entry u.
    // The first run is entries [0, j1) with sum fs; ls is the last run's sum.
    A acc = 0;
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      if (u < n) {
        if (u > 0 && r[u] != r[u - 1]) {
          if (j1 == n) { j1 = u; fs = acc; }
          acc = 0;
        }
        acc = fma_acc(pr[u], xv[u], acc);
        pr[u] = acc;
        rlast = r[u];
      }
    }
    ls = acc;
    if (j1 == n) fs = acc;
  }
  const int rfirst = n > 0 ? r[0] : INT_MAX;
  s_fr[tid] = rfirst;
  s_lr[tid] = rlast;
  s_n[tid] = n;
  s_fs[tid] = fs;

  // the tile's rows: (prev, rb]
  const int prev = t0 > 0 ? __ldg(row + t0 - 1) : -1;
  const int last_entry_row = __ldg(row + t1 - 1);
  const bool cont_out = t1 < nnz && __ldg(row + t1) == last_entry_row;
  const int ra = max(prev + 1, 0);  // rows outside [0, nrows) are never written
  const int rb = T == ntiles - 1 ? nrows - 1 : min(last_entry_row, nrows - 1);
  __syncthreads();

  // owned, complete runs: bit u = the run ending at entry u, value pr[u];
  // the last run's row, when owned and complete here: last_sum
  unsigned own = 0;
  bool out_last = false;
  A last_sum = 0;
  if (n > 0) {
#pragma unroll
    for (int u = 0; u < kChunk; ++u)  // interior runs
      if (u < n - 1 && u >= j1 && r[u] != r[u + 1]) own |= 1u << u;
    const bool single = j1 == n;
    const bool starts_here = tid == 0 ? rfirst >= ra : s_lr[tid - 1] != rfirst;
    if (!single && starts_here && rfirst >= ra) own |= 1u << (j1 - 1);
    if (!single || (starts_here && rfirst >= ra)) {
      // the last run's row starts in this thread: add the following threads'
      // first runs while the row goes on
      A tot = ls;
      int k = tid + 1;
      bool ended = false;
      for (; k < kThreads && s_n[k] > 0; ++k) {
        if (s_fr[k] != rlast) { ended = true; break; }
        tot += s_fs[k];
        if (s_lr[k] != rlast) { ended = true; break; }
      }
      if (!ended) ended = !(cont_out && rlast == last_entry_row);
      if (ended) {
        out_last = true;
        last_sum = tot;
      } else {
        carry_last[T] = tot;
      }
    }
    if (tid == 0 && T > 0) {
      // the leading run continues a row of an earlier tile
      A tot = 0;
      if (rfirst < ra) {
        tot = fs;
        if (single)
          for (int k = 1; k < kThreads && s_n[k] > 0 && s_fr[k] == rfirst; ++k) {
            tot += s_fs[k];
            if (s_lr[k] != rfirst) break;
          }
      }
      carry_first[T] = tot;
    }
  }

  // y for the owned rows, kRowCap at a time (one pass unless the tile owns
  // a long range of empty rows)
  const int nown = rb - ra + 1;
  for (int w0 = 0; w0 < nown; w0 += kRowCap) {
    const int wn = min(kRowCap, nown - w0);
    for (int i = tid; i < wn; i += kThreads) s_acc[i] = A(0);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      if (own & (1u << u)) {
        const int lr = r[u] - ra - w0;
        if (lr >= 0 && lr < wn) s_acc[lr] = pr[u];
      }
    }
    if (out_last) {
      const int lr = rlast - ra - w0;
      if (lr >= 0 && lr < wn) s_acc[lr] = last_sum;
    }
    __syncthreads();
    for (int i = tid; i < wn; i += kThreads) {
      const int rr = ra + w0 + i;
      if (cont_out && rr == last_entry_row) continue;  // finished by pass 2
      coo_store(y, rr, s_acc[i], alpha, beta);
    }
    __syncthreads();
  }
}

// Pass 2.  A row crossing a tile boundary belongs to the tile holding its
// first entry: tile T owns the row of its last entry when that row goes on
// into tile T + 1 and starts inside tile T.
template <typename A>
__global__ void k_coo_cross(int nrows, long long nnz, const int *__restrict__ row, A *y,
                            double alpha, double beta, const A *carry_first, const A *carry_last,
                            long long ntiles) {
  for (long long T = blockIdx.x * (long long)blockDim.x + threadIdx.x; T + 1 < ntiles;
       T += (long long)gridDim.x * blockDim.x) {
    const long long t0 = T * kTile, t1 = t0 + kTile;  // t1 < nnz since T + 1 < ntiles
    const int r = __ldg(row + t1 - 1);
    if (__ldg(row + t1) != r) continue;               // the row ends in tile T
    if (t0 > 0 && __ldg(row + t0 - 1) == r) continue;  // an earlier tile owns it
    A tot = carry_last[T];
    for (long long U = T + 1; U < ntiles; ++U) {
      const long long u1 = min((U + 1) * kTile, nnz);
      tot += carry_first[U];
      if (__ldg(row + u1 - 1) != r || u1 >= nnz || __ldg(row + u1) != r) break;
    }
    if (r >= 0 && r < nrows) coo_store(y, r, tot, alpha, beta);
  }
}

template <typename V, typename I>
int coo_launch(int32_t nrows, int64_t nnz, const int *row, const void *idx, const void *val,
               const void *x, void *y, double alpha, double beta, void *ws, cudaStream_t s) {
  using A = typename AccOf<V>::type;
  A *yy = static_cast<A *>(y);
  if (nnz == 0) {
    const int g0 = (int)std::max<long long>(1, std::min<long long>(8LL * sm_count(), (nrows + 255) / 256));
    k_coo_scale<A><<<g0, 256, 0, s>>>(nrows, yy, beta);
    DAMN_CHECK_LAUNCH("k_coo_scale");
    return DAMN_OK;
  }
  const long long ntiles = (nnz + kTile - 1) / kTile;
  A *cf = static_cast<A *>(ws);
  A *cl = cf + ntiles;
  const bool vec = aligned16(row) && aligned16(idx) && aligned16(val);
  if (vec)
    k_coo_tiles<V, I, true><<<(unsigned)ntiles, kThreads, 0, s>>>(
        nrows, nnz, row, static_cast<const I *>(idx), static_cast<const V *>(val),
        static_cast<const A *>(x), yy, alpha, beta, cf, cl);
  else
    k_coo_tiles<V, I, false><<<(unsigned)ntiles, kThreads, 0, s>>>(
        nrows, nnz, row, static_cast<const I *>(idx), static_cast<const V *>(val),
        static_cast<const A *>(x), yy, alpha, beta, cf, cl);
  DAMN_CHECK_LAUNCH("k_coo_tiles");
  if (ntiles > 1) {
    const int g1 = (int)std::min<long long>(4LL * sm_count(), (ntiles + 255) / 256);
    k_coo_cross<A><<<g1, 256, 0, s>>>(nrows, nnz, row, yy, alpha, beta, cf, cl, ntiles);
    DAMN_CHECK_LAUNCH("k_coo_cross");
  }
  return DAMN_OK;
}

template <typename I>
int coo_entry(const char *fn, int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *row,
              const I *idx, const void *val, int dtype, const void *x, void *y, double alpha,
              double beta, void *ws, size_t ws_bytes, void *stream) {
  if (nrows < 0 || ncols < 0 || nnz < 0 || nnz > INT_MAX)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: bad sizes", fn);
  if (dtype != DAMN_F64 && dtype != DAMN_F32 && dtype != DAMN_BF16)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: bad dtype %d", fn, dtype);
  if (nrows > 0 && !y) return set_error(DAMN_ERR_INVALID_ARG, "%s: NULL y", fn);
  if (nnz > 0 && (!row || !idx || !val || !x)) return set_error(DAMN_ERR_INVALID_ARG, "%s: NULL pointer", fn);
  const size_t need = damn_coo_workspace_size(nnz, dtype);
  if (nnz > 0 && (!ws || ws_bytes < need || !aligned16(ws)))
    return set_error(DAMN_ERR_INVALID_ARG, "%s: workspace too small or misaligned", fn);
  if (nrows == 0) return DAMN_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == DAMN_F64) return coo_launch<double, I>(nrows, nnz, row, idx, val, x, y, alpha, beta, ws, s);
  if (dtype == DAMN_F32) return coo_launch<float, I>(nrows, nnz, row, idx, val, x, y, alpha, beta, ws, s);
  return coo_launch<__nv_bfloat16, I>(nrows, nnz, row, idx, val, x, y, alpha, beta, ws, s);
}

}  // namespace
}  // namespace damn

using namespace damn;

extern "C" size_t damn_coo_workspace_size(int64_t nnz, int dtype) {
  if (nnz <= 0) return 16;
  const size_t a = dtype == DAMN_F64 ? 8 : 4;
  const size_t ntiles = (size_t)((nnz + kTile - 1) / kTile);
  return 2 * ntiles * a + 16;
}

extern "C" int damn_spmv_coo32(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *row,
                               const int32_t *col, const void *val, int dtype, const void *x,
                               void *y, double alpha, double beta, void *workspace,
                               size_t ws_bytes, void *stream) {
  return coo_entry("damn_spmv_coo32", nrows, ncols, nnz, row, col, val, dtype, x, y, alpha, beta,
                   workspace, ws_bytes, stream);
}

extern "C" int damn_spmv_dacoo16(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *row,
                                 const int16_t *off, const void *val, int dtype, const void *x,
                                 void *y, double alpha, double beta, void *workspace,
                                 size_t ws_bytes, void *stream) {
  return coo_entry("damn_spmv_dacoo16", nrows, ncols, nnz, row, off, val, dtype, x, y, alpha,
                   beta, workspace, ws_bytes, stream);
}
