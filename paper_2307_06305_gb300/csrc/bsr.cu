// Block CSR SpMV, with absolute block columns (BSR-32) or block offsets
// relative to the block diagonal (DA-BSR-16 / DA-BSR-8): Section 2's
// translation applied to the block pattern, so one index serves b * b values
// (the paper notes the technique applies to BSR, Section 1).
//
// Each thread computes one scalar row r = R * b + i: for every block k of
// block row R (stored order) and j = 0..b-1 it accumulates
// val[k][i][j] * x[C_k * b + j] with FMA.  The b threads of a block row read
// the block's b * b values as one contiguous run and the same b values of x;
// two blocks are loaded ahead so several loads are in flight.
#include <algorithm>
#include <climits>

#include "damn_common.cuh"

namespace damn {
namespace {

template <typename V, typename I, int B>
__global__ void __launch_bounds__(256)
k_bsr_spmv(int nbr, const int *__restrict__ browptr, const I *__restrict__ bidx,
           const V *__restrict__ val, const typename AccOf<V>::type *__restrict__ x,
           typename AccOf<V>::type *__restrict__ y, double alpha, double beta, int ab_mode) {
  using A = typename AccOf<V>::type;
  constexpr bool DA = sizeof(I) < 4;
  const long long nrows = (long long)nbr * B;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrows;
       r += (long long)gridDim.x * blockDim.x) {
    const int R = static_cast<int>(r / B), i = static_cast<int>(r - (long long)R * B);
    const int k0 = __ldg(browptr + R), k1 = __ldg(browptr + R + 1);
    A acc = 0;
    int k = k0;
    for (; k + 1 < k1; k += 2) {
      const int c0 = (DA ? R : 0) + static_cast<int>(__ldg(bidx + k));
      const int c1 = (DA ? R : 0) + static_cast<int>(__ldg(bidx + k + 1));
      const V *v0 = val + ((size_t)k * B + i) * B;
      const V *v1 = v0 + (size_t)B * B;
      A a0[B], a1[B], x0[B], x1[B];
#pragma unroll
      for (int j = 0; j < B; ++j) {
        a0[j] = to_acc(__ldg(v0 + j));
        a1[j] = to_acc(__ldg(v1 + j));
        x0[j] = __ldg(x + (size_t)c0 * B + j);
        x1[j] = __ldg(x + (size_t)c1 * B + j);
      }
#pragma unroll
      for (int j = 0; j < B; ++j) acc = fma_acc(a0[j], x0[j], acc);
#pragma unroll
      for (int j = 0; j < B; ++j) acc = fma_acc(a1[j], x1[j], acc);
    }
    if (k < k1) {
      const int c0 = (DA ? R : 0) + static_cast<int>(__ldg(bidx + k));
      const V *v0 = val + ((size_t)k * B + i) * B;
#pragma unroll
      for (int j = 0; j < B; ++j)
        acc = fma_acc(to_acc(__ldg(v0 + j)), __ldg(x + (size_t)c0 * B + j), acc);
    }
    A out = acc;
    if (ab_mode == 1) out = static_cast<A>(alpha) * acc;
    if (ab_mode == 2) out = fma_acc(static_cast<A>(beta), y[r], static_cast<A>(alpha) * acc);
    y[r] = out;
  }
}

template <typename V, typename I, int B>
int launch_b(int nbr, const int *browptr, const void *bidx, const void *val, const void *x,
             void *y, double alpha, double beta, cudaStream_t s) {
  using A = typename AccOf<V>::type;
  const int ab_mode = beta != 0.0 ? 2 : (alpha == 1.0 ? 0 : 1);
  const long long nrows = (long long)nbr * B;
  const int blocks = (int)std::max<long long>(
      1, std::min<long long>(16LL * sm_count(), (nrows + 255) / 256));
  k_bsr_spmv<V, I, B><<<blocks, 256, 0, s>>>(nbr, browptr, static_cast<const I *>(bidx),
                                             static_cast<const V *>(val),
                                             static_cast<const A *>(x), static_cast<A *>(y),
                                             alpha, beta, ab_mode);
  DAMN_CHECK_LAUNCH("k_bsr_spmv");
  return DAMN_OK;
}

template <typename V, typename I>
int launch_v(int b, int nbr, const int *browptr, const void *bidx, const void *val, const void *x,
             void *y, double alpha, double beta, cudaStream_t s) {
  switch (b) {
    case 1: return launch_b<V, I, 1>(nbr, browptr, bidx, val, x, y, alpha, beta, s);
    case 2: return launch_b<V, I, 2>(nbr, browptr, bidx, val, x, y, alpha, beta, s);
    case 3: return launch_b<V, I, 3>(nbr, browptr, bidx, val, x, y, alpha, beta, s);
    case 4: return launch_b<V, I, 4>(nbr, browptr, bidx, val, x, y, alpha, beta, s);
    case 6: return launch_b<V, I, 6>(nbr, browptr, bidx, val, x, y, alpha, beta, s);
    case 8: return launch_b<V, I, 8>(nbr, browptr, bidx, val, x, y, alpha, beta, s);
    default: return set_error(DAMN_ERR_UNSUPPORTED, "BSR SpMV: block size %d (use 1, 2, 3, 4, 6, 8)", b);
  }
}

template <typename I>
int bsr_entry(const char *fn, int32_t nbr, int32_t nbc, int64_t nblk, int32_t b,
              const int32_t *browptr, const I *bidx, const void *val, int dtype, const void *x,
              void *y, double alpha, double beta, void *stream) {
  if (nbr < 0 || nbc < 0 || nblk < 0 || nblk > INT_MAX || b < 1 ||
      (long long)nbr * b > INT_MAX || (long long)nbc * b > INT_MAX)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: bad sizes", fn);
  if (dtype != DAMN_F64 && dtype != DAMN_F32 && dtype != DAMN_BF16)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: bad dtype %d", fn, dtype);
  if (nbr > 0 && (!browptr || !y)) return set_error(DAMN_ERR_INVALID_ARG, "%s: NULL pointer", fn);
  if (nblk > 0 && (!bidx || !val || !x)) return set_error(DAMN_ERR_INVALID_ARG, "%s: NULL pointer", fn);
  if (nbr == 0) return DAMN_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == DAMN_F64) return launch_v<double, I>(b, nbr, browptr, bidx, val, x, y, alpha, beta, s);
  if (dtype == DAMN_F32) return launch_v<float, I>(b, nbr, browptr, bidx, val, x, y, alpha, beta, s);
  return launch_v<__nv_bfloat16, I>(b, nbr, browptr, bidx, val, x, y, alpha, beta, s);
}

}  // namespace
}  // namespace damn

using namespace damn;

extern "C" int damn_spmv_bsr32(int32_t nbr, int32_t nbc, int64_t nblk, int32_t b,
                               const int32_t *browptr, const int32_t *bcol, const void *val,
                               int dtype, const void *x, void *y, double alpha, double beta,
                               void *stream) {
  return bsr_entry("damn_spmv_bsr32", nbr, nbc, nblk, b, browptr, bcol, val, dtype, x, y, alpha,
                   beta, stream);
}

extern "C" int damn_spmv_dabsr16(int32_t nbr, int32_t nbc, int64_t nblk, int32_t b,
                                 const int32_t *browptr, const int16_t *boff, const void *val,
                                 int dtype, const void *x, void *y, double alpha, double beta,
                                 void *stream) {
  return bsr_entry("damn_spmv_dabsr16", nbr, nbc, nblk, b, browptr, boff, val, dtype, x, y, alpha,
                   beta, stream);
}

extern "C" int damn_spmv_dabsr8(int32_t nbr, int32_t nbc, int64_t nblk, int32_t b,
                                const int32_t *browptr, const int8_t *boff, const void *val,
                                int dtype, const void *x, void *y, double alpha, double beta,
                                void *stream) {
  return bsr_entry("damn_spmv_dabsr8", nbr, nbc, nblk, b, browptr, boff, val, dtype, x, y, alpha,
                   beta, stream);
}
