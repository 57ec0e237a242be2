// COO SpMV with absolute columns (COO-32) or columns addressed from the
// diagonal (DA-COO-16: the column vector of COO storage stored as c - r in
// int16; the paper notes the technique applies to one of COO's vectors,
// Section 1).  Entries are sorted by row; the row vector stays int32.
//
// Deterministic three-pass scheme, no atomics:
//  1. y <- beta y (or 0);
//  2. entries are cut into chunks of kChunk consecutive entries, one per
//     thread.  A thread sums each run of equal rows of its chunk in stored
//     order; a run that is a whole row (it neither starts before the chunk
//     nor ends after it) is added to y at once (y[r] += alpha * sum); the
//     first and last runs' sums go to carry_first / carry_last;
//  3. a row that crosses chunks is finished by the chunk it starts in: its
//     last-run sum plus the first-run sums of the following chunks the row
//     continues into, added left to right, then y[r] += alpha * total.
// Every y[r] has exactly one writer in pass 2 or 3.
#include <algorithm>
#include <climits>

#include "damn_common.cuh"

namespace damn {
namespace {

constexpr int kChunk = 8;

template <typename A>
__global__ void k_coo_scale(long long n, A *y, double beta) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = beta == 0.0 ? A(0) : static_cast<A>(beta) * y[i];
}

template <typename V, typename I>
__global__ void k_coo_chunks(long long nnz, const int *__restrict__ row, const I *__restrict__ idx,
                             const V *__restrict__ val, const typename AccOf<V>::type *__restrict__ x,
                             typename AccOf<V>::type *__restrict__ y, double alpha,
                             typename AccOf<V>::type *carry_first,
                             typename AccOf<V>::type *carry_last, long long nchunks) {
  using A = typename AccOf<V>::type;
  constexpr bool DA = sizeof(I) < 4;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nchunks;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e0 = t * kChunk, e1 = min(e0 + kChunk, nnz);
    const int r_before = e0 > 0 ? __ldg(row + e0 - 1) : -1;
    const int r_after = e1 < nnz ? __ldg(row + e1) : -1;
    int r = __ldg(row + e0);
    A acc = 0;
    bool first_run = true;
    for (long long e = e0; e < e1; ++e) {
      const int re = __ldg(row + e);
      if (re != r) {  // run of row r ends inside the chunk
        if (first_run && r == r_before) carry_first[t] = acc;
        else y[r] = fma_acc(static_cast<A>(alpha), acc, y[r]);
        first_run = false;
        r = re;
        acc = 0;
      }
      const int c = DA ? re + static_cast<int>(__ldg(idx + e)) : static_cast<int>(__ldg(idx + e));
      acc = fma_acc(to_acc(__ldg(val + e)), __ldg(x + c), acc);
    }
    // the last run of the chunk
    if (first_run && r == r_before) {
      carry_first[t] = acc;       // the whole chunk continues an earlier row
      carry_last[t] = acc;
    } else if (r == r_after) {
      carry_last[t] = acc;        // the row goes on into the next chunk
    } else {
      y[r] = fma_acc(static_cast<A>(alpha), acc, y[r]);
    }
  }
}

// Pass 3.  A row that crosses a chunk boundary belongs to the chunk holding
// its first entry: chunk t owns the row of its last run when that row goes
// on into chunk t + 1 and its first entry lies in chunk t.
template <typename A>
__global__ void k_coo_finish(long long nnz, const int *__restrict__ row, A *y, double alpha,
                             const A *carry_first, const A *carry_last, long long nchunks) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t + 1 < nchunks;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e0 = t * kChunk, e1 = e0 + kChunk;  // e1 < nnz since t + 1 < nchunks
    const int r = __ldg(row + e1 - 1);
    if (__ldg(row + e1) != r) continue;                 // the row ends in chunk t
    // does the row start inside chunk t?  (else an earlier chunk owns it)
    const bool starts_here = (__ldg(row + e0) != r) || e0 == 0 || __ldg(row + e0 - 1) != r;
    if (!starts_here) continue;
    A tot = carry_last[t];
    long long u = t + 1;
    while (u < nchunks) {
      const long long f0 = u * kChunk, f1 = min(f0 + kChunk, nnz);
      tot += carry_first[u];
      if (__ldg(row + f1 - 1) != r || f1 >= nnz || __ldg(row + f1) != r) break;
      ++u;
    }
    y[r] = fma_acc(static_cast<A>(alpha), tot, y[r]);
  }
}

template <typename V, typename I>
int coo_launch(int32_t nrows, int64_t nnz, const int *row, const void *idx, const void *val,
               const void *x, void *y, double alpha, double beta, void *ws, cudaStream_t s) {
  using A = typename AccOf<V>::type;
  A *yy = static_cast<A *>(y);
  const int bs = 256;
  const int g0 = (int)std::max<long long>(1, std::min<long long>(8LL * sm_count(), (nrows + bs - 1) / bs));
  k_coo_scale<A><<<g0, bs, 0, s>>>(nrows, yy, beta);
  DAMN_CHECK_LAUNCH("k_coo_scale");
  if (nnz == 0) return DAMN_OK;
  const long long nchunks = (nnz + kChunk - 1) / kChunk;
  A *cf = static_cast<A *>(ws);
  A *cl = cf + nchunks;
  const int g1 = (int)std::max<long long>(1, std::min<long long>(16LL * sm_count(), (nchunks + bs - 1) / bs));
  k_coo_chunks<V, I><<<g1, bs, 0, s>>>(nnz, row, static_cast<const I *>(idx),
                                       static_cast<const V *>(val), static_cast<const A *>(x), yy,
                                       alpha, cf, cl, nchunks);
  DAMN_CHECK_LAUNCH("k_coo_chunks");
  k_coo_finish<A><<<g1, bs, 0, s>>>(nnz, row, yy, alpha, cf, cl, nchunks);
  DAMN_CHECK_LAUNCH("k_coo_finish");
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
  const size_t nchunks = (size_t)((nnz + kChunk - 1) / kChunk);
  return 2 * nchunks * a + 16;
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
