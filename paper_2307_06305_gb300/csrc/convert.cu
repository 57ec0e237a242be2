// CSR -> DA-CSR translation with the 16-bit (or 8-bit) fit check (Section 2,
// Example 1, Eq. (2)), CSR validation, and round-to-nearest value casts.
//
// Each CTA owns a block of kRowsPerBlock rows: it stages their row pointers
// in shared memory and walks the block's entries with coalesced loads of col
// and coalesced stores of off, finding each entry's row by binary search in
// shared memory.  Per-entry work is an int32 subtraction, a narrowing store
// and min/max/count reductions; the kernel is bound by HBM traffic (4 bytes
// read + 2 (or 1) bytes written per entry, plus 4 bytes per row).
#include <algorithm>
#include <climits>
#include <mutex>

#include "damn_common.cuh"

namespace damn {
namespace {

constexpr int kConvThreads = 256;
constexpr int kRowsPerBlock = 512;

struct FitAccum {
  int min_off;
  int max_off;
  unsigned long long n_fit;
  unsigned long long n_bad;
};

__global__ void k_fit_init(FitAccum *acc) {
  acc->min_off = INT_MAX;
  acc->max_off = INT_MIN;
  acc->n_fit = 0;
  acc->n_bad = 0;
}

// Largest local row lr in [0, nr) with rp[lr] <= k (rows are non-empty at k).
__device__ __forceinline__ int row_of(const int *rp, int nr, int k) {
  int lo = 0, hi = nr - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (rp[mid] <= k) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// c - r saturated to the int32 range of the reported min / max offsets
// (reached only by columns outside [0, ncols)).
__device__ __forceinline__ int sat_int(long long d) {
  return static_cast<int>(d < INT_MIN ? (long long)INT_MIN : d > INT_MAX ? (long long)INT_MAX : d);
}

template <int NT>
__device__ __forceinline__ void block_reduce_fit(int mn, int mx, unsigned long long nf,
                                                 unsigned long long nb, FitAccum *acc) {
  __shared__ int s_mn[NT / 32], s_mx[NT / 32];
  __shared__ unsigned long long s_nf[NT / 32], s_nb[NT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nf += __shfl_xor_sync(0xffffffffu, nf, o);
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { s_mn[w] = mn; s_mx[w] = mx; s_nf[w] = nf; s_nb[w] = nb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < NT / 32; ++i) {
      mn = min(mn, s_mn[i]); mx = max(mx, s_mx[i]); nf += s_nf[i]; nb += s_nb[i];
    }
    if (mn != INT_MAX) {
      atomicMin(&acc->min_off, mn);
      atomicMax(&acc->max_off, mx);
    }
    if (nf) atomicAdd(&acc->n_fit, nf);
    if (nb) atomicAdd(&acc->n_bad, nb);
  }
}

// OffT = int16_t (DA-CSR-16) or int8_t (DA-CSR-8): an entry fits when its
// offset lies in OffT's range.
template <typename OffT>
__global__ void __launch_bounds__(kConvThreads)
k_csr_to_dacsr(int nrows, int ncols, const int *__restrict__ rowptr, const int *__restrict__ col,
               OffT *__restrict__ off, FitAccum *acc) {
  constexpr int kLo = -(1 << (8 * sizeof(OffT) - 1)), kHi = (1 << (8 * sizeof(OffT) - 1)) - 1;
  __shared__ int rp[kRowsPerBlock + 1];
  const int r0 = blockIdx.x * kRowsPerBlock;
  const int nr = min(kRowsPerBlock, nrows - r0);
  for (int i = threadIdx.x; i <= nr; i += kConvThreads) rp[i] = rowptr[r0 + i];
  __syncthreads();
  const int k0 = rp[0], k1 = rp[nr];
  int mn = INT_MAX, mx = INT_MIN;
  unsigned long long nf = 0, nb = 0;
  for (int k = k0 + threadIdx.x; k < k1; k += kConvThreads) {
    const int lr = row_of(rp, nr, k);
    const int c = __ldcs(col + k);
    // in 64 bits: a bad column near INT_MIN would overflow c - r in int32
    const long long d = (long long)c - (r0 + lr);
    off[k] = static_cast<OffT>(d);
    mn = min(mn, sat_int(d));
    mx = max(mx, sat_int(d));
    nf += (d >= kLo && d <= kHi) ? 1ull : 0ull;
    nb += (c < 0 || c >= ncols) ? 1ull : 0ull;
  }
  block_reduce_fit<kConvThreads>(mn, mx, nf, nb, acc);
}

struct ValidateAccum {
  unsigned long long bad_rows;
  unsigned long long bad_cols;
};

__global__ void k_validate(int nrows, int ncols, long long nnz, const int *__restrict__ rowptr,
                           const int *__restrict__ col, ValidateAccum *acc) {
  unsigned long long br = 0, bc = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long r = tid; r < nrows; r += stride) br += rowptr[r] > rowptr[r + 1] ? 1 : 0;
  if (tid == 0) br += (rowptr[0] != 0 ? 1 : 0) + ((long long)rowptr[nrows] != nnz ? 1 : 0);
  for (long long k = tid; k < nnz; k += stride) {
    const int c = col[k];
    bc += (c < 0 || c >= ncols) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    br += __shfl_xor_sync(0xffffffffu, br, o);
    bc += __shfl_xor_sync(0xffffffffu, bc, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (br) atomicAdd(&acc->bad_rows, br);
    if (bc) atomicAdd(&acc->bad_cols, bc);
  }
}

// Round-to-nearest-even narrowing written from the IEEE 754 encodings:
// the significand is cut to 8 bits (bfloat16) with the discarded bits
// compared against one half ulp; values below 2^-126 become bfloat16
// subnormals (spacing 2^-133); overflow becomes infinity.
__device__ __forceinline__ uint16_t bf16_bits_from_double(double v) {
  const unsigned long long b = __double_as_longlong(v);
  const uint16_t sign = static_cast<uint16_t>((b >> 48) & 0x8000u);
  const int ef = static_cast<int>((b >> 52) & 0x7ff);
  const unsigned long long frac = b & ((1ull << 52) - 1);
  if (ef == 0x7ff) return frac ? static_cast<uint16_t>(sign | 0x7fc0u) : static_cast<uint16_t>(sign | 0x7f80u);
  if (ef == 0) return sign;  // FP64 zero or subnormal (< 2^-1022): rounds to zero
  const int e = ef - 1023;
  const unsigned long long m = (1ull << 52) | frac;  // 53-bit significand
  int shift = 45;                                    // keep 8 bits for normals
  if (e < -126) shift += (-126 - e);                 // fewer bits for subnormals
  if (shift > 60) return sign;                       // far below half the smallest subnormal
  unsigned long long q = m >> shift;
  const unsigned long long rem = m & ((1ull << shift) - 1);
  const unsigned long long half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (q & 1ull))) ++q;
  if (e < -126) return static_cast<uint16_t>(sign | q);  // q <= 128: 128 is the smallest normal
  int eb = e + 127;
  if (q == 256) { q = 128; ++eb; }
  if (eb >= 255) return static_cast<uint16_t>(sign | 0x7f80u);
  return static_cast<uint16_t>(sign | (eb << 7) | (q & 127u));
}

// Round-to-nearest-even narrowing to FP8 E4M3, written from the encodings:
// |v| = m 2^e with m in [1, 2) (e read from the FP64 exponent field, clamped
// at -6, the subnormal range of E4M3); q = |v| 2^(3-e), rounded to an
// integer with ties to even, is |v| in units of the spacing 2^(e-3), and
// q = 16 carries into the next binade.  |v| > 464 (rounding past the largest
// finite 448), an infinity or a NaN give NaN: the format has no infinity.
__device__ __forceinline__ uint8_t e4m3_bits_from_double(double v) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const uint8_t sign = static_cast<uint8_t>((bits >> 56) & 0x80u);
  const double a = fabs(v);
  if (!(a <= 464.0)) return sign | 0x7Fu;
  if (a == 0.0) return sign;
  int e = static_cast<int>((bits >> 52) & 0x7FFu) - 1023;  // FP64 subnormals: e = -1023
  if (e < -6) e = -6;
  const double scale = __longlong_as_double(static_cast<long long>(1023 + 3 - e) << 52);
  int q = static_cast<int>(__double2ll_rn(a * scale));  // exact product, RNE
  if (e == -6 && q < 8) return sign | static_cast<uint8_t>(q);  // subnormal or zero
  if (q == 16) { q = 8; ++e; }
  return sign | static_cast<uint8_t>(((e + 7) << 3) | (q - 8));
}

__global__ void k_cast(long long n, const void *src, int st, void *dst, int dt) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double v = (st == DAMN_F64) ? static_cast<const double *>(src)[i]
                                      : static_cast<double>(static_cast<const float *>(src)[i]);
    if (dt == DAMN_F32)
      static_cast<float *>(dst)[i] = __double2float_rn(v);
    else if (dt == DAMN_F8E4M3)
      static_cast<uint8_t *>(dst)[i] = e4m3_bits_from_double(v);
    else
      static_cast<uint16_t *>(dst)[i] = bf16_bits_from_double(v);
  }
}

}  // namespace
}  // namespace damn

using namespace damn;

extern "C" size_t damn_csr_to_dacsr_workspace_size(void) { return 256; }

template <typename OffT>
static int csr_to_dacsr(const char *fn, int32_t nrows, int32_t ncols, int64_t nnz,
                        const int32_t *rowptr, const int32_t *col, OffT *off_out,
                        damn_fit_info *h_info, void *workspace, size_t ws_bytes, void *stream) {
  if (nrows < 0 || ncols < 0 || nnz < 0 || nnz > INT_MAX)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: bad sizes", fn);
  if (!h_info || !rowptr || (nnz > 0 && (!col || !off_out)))
    return set_error(DAMN_ERR_INVALID_ARG, "%s: NULL pointer", fn);
  if (!workspace || ws_bytes < damn_csr_to_dacsr_workspace_size() || !aligned16(workspace))
    return set_error(DAMN_ERR_INVALID_ARG, "%s: workspace too small or misaligned", fn);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FitAccum *acc = static_cast<FitAccum *>(workspace);
  k_fit_init<<<1, 1, 0, s>>>(acc);
  DAMN_CHECK_LAUNCH("k_fit_init");
  if (nrows > 0) {
    const int blocks = (nrows + kRowsPerBlock - 1) / kRowsPerBlock;
    k_csr_to_dacsr<OffT><<<blocks, kConvThreads, 0, s>>>(nrows, ncols, rowptr, col, off_out, acc);
    DAMN_CHECK_LAUNCH("k_csr_to_dacsr");
  }
  FitAccum h{};
  DAMN_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  if (nnz == 0) { h.min_off = 0; h.max_off = 0; }
  h_info->min_off = h.min_off;
  h_info->max_off = h.max_off;
  h_info->w = std::max<int64_t>(-(int64_t)h.min_off, (int64_t)h.max_off);
  h_info->n_fit = static_cast<int64_t>(h.n_fit);
  h_info->n_bad = static_cast<int64_t>(h.n_bad);
  h_info->fits = (static_cast<int64_t>(h.n_fit) == nnz && h.n_bad == 0) ? 1 : 0;
  h_info->reserved = 0;
  if (!h_info->fits)
    return set_error(DAMN_ERR_NOFIT,
                     "%s: %lld of %lld entries do not fit int%d (min %d, max %d), %lld bad columns",
                     fn, (long long)(nnz - h_info->n_fit), (long long)nnz, (int)(8 * sizeof(OffT)),
                     h.min_off, h.max_off, (long long)h.n_bad);
  return DAMN_OK;
}

extern "C" int damn_csr_to_dacsr(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                                 const int32_t *col, int16_t *off_out, damn_fit_info *h_info,
                                 void *workspace, size_t ws_bytes, void *stream) {
  return csr_to_dacsr<int16_t>("damn_csr_to_dacsr", nrows, ncols, nnz, rowptr, col, off_out,
                               h_info, workspace, ws_bytes, stream);
}

extern "C" int damn_csr_to_dacsr8(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                                  const int32_t *col, int8_t *off_out, damn_fit_info *h_info,
                                  void *workspace, size_t ws_bytes, void *stream) {
  return csr_to_dacsr<int8_t>("damn_csr_to_dacsr8", nrows, ncols, nnz, rowptr, col, off_out,
                              h_info, workspace, ws_bytes, stream);
}

extern "C" size_t damn_validate_csr_workspace_size(void) { return 256; }

extern "C" int damn_validate_csr(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                                 const int32_t *col, int64_t *h_bad_rows, int64_t *h_bad_cols,
                                 void *workspace, size_t ws_bytes, void *stream) {
  if (nrows < 0 || ncols < 0 || nnz < 0 || nnz > INT_MAX)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_validate_csr: bad sizes");
  if (!rowptr || (nnz > 0 && !col) || !h_bad_rows || !h_bad_cols)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_validate_csr: NULL pointer");
  if (!workspace || ws_bytes < damn_validate_csr_workspace_size() || !aligned16(workspace))
    return set_error(DAMN_ERR_INVALID_ARG, "damn_validate_csr: workspace too small or misaligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ValidateAccum *acc = static_cast<ValidateAccum *>(workspace);
  DAMN_CUDA(cudaMemsetAsync(acc, 0, sizeof(ValidateAccum), s));
  const int blocks = std::max(1, std::min(4 * sm_count(), (int)((std::max<int64_t>(nnz, nrows) + 255) / 256)));
  k_validate<<<blocks, 256, 0, s>>>(nrows, ncols, nnz, rowptr, col, acc);
  DAMN_CHECK_LAUNCH("k_validate");
  ValidateAccum h{};
  DAMN_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  *h_bad_rows = static_cast<int64_t>(h.bad_rows);
  *h_bad_cols = static_cast<int64_t>(h.bad_cols);
  if (h.bad_rows || h.bad_cols)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_validate_csr: %llu bad row pointers, %llu bad columns",
                     h.bad_rows, h.bad_cols);
  return DAMN_OK;
}

// DA-CSR validation: a block of kRowsPerBlock rows stages its row pointers,
// counts decreasing row pointers, and checks r + off in [0, ncols) for its
// entries (the entry range clamped to [0, nnz), so a broken rowptr cannot
// make it read outside off).
template <typename OffT>
__global__ void __launch_bounds__(kConvThreads)
k_validate_dacsr(int nrows, int ncols, long long nnz, const int *__restrict__ rowptr,
                 const OffT *__restrict__ off, ValidateAccum *acc) {
  __shared__ int rp[kRowsPerBlock + 1];
  const int r0 = blockIdx.x * kRowsPerBlock;
  const int nr = min(kRowsPerBlock, nrows - r0);
  for (int i = threadIdx.x; i <= nr; i += kConvThreads) rp[i] = rowptr[r0 + i];
  __syncthreads();
  unsigned long long br = 0, bc = 0;
  for (int i = threadIdx.x; i < nr; i += kConvThreads) br += rp[i] > rp[i + 1] ? 1 : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0)
    br += (rowptr[0] != 0 ? 1 : 0) + ((long long)rowptr[nrows] != nnz ? 1 : 0);
  const long long k0 = max(0LL, min((long long)rp[0], nnz));
  const long long k1 = max(k0, min((long long)rp[nr], nnz));
  for (long long k = k0 + threadIdx.x; k < k1; k += kConvThreads) {
    const int lr = row_of(rp, nr, static_cast<int>(k));
    const long long c = (long long)r0 + lr + static_cast<long long>(off[k]);
    bc += (c < 0 || c >= ncols) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    br += __shfl_xor_sync(0xffffffffu, br, o);
    bc += __shfl_xor_sync(0xffffffffu, bc, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (br) atomicAdd(&acc->bad_rows, br);
    if (bc) atomicAdd(&acc->bad_cols, bc);
  }
}

extern "C" int damn_validate_dacsr(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t *rowptr,
                                   const void *off, int32_t off_bits, int64_t *h_bad_rows,
                                   int64_t *h_bad_cols, void *workspace, size_t ws_bytes,
                                   void *stream) {
  if (nrows < 0 || ncols < 0 || nnz < 0 || nnz > INT_MAX)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_validate_dacsr: bad sizes");
  if (off_bits != 16 && off_bits != 8)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_validate_dacsr: off_bits must be 16 or 8");
  if (!rowptr || (nnz > 0 && !off) || !h_bad_rows || !h_bad_cols)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_validate_dacsr: NULL pointer");
  if (!workspace || ws_bytes < damn_validate_csr_workspace_size() || !aligned16(workspace))
    return set_error(DAMN_ERR_INVALID_ARG, "damn_validate_dacsr: workspace too small or misaligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ValidateAccum *acc = static_cast<ValidateAccum *>(workspace);
  DAMN_CUDA(cudaMemsetAsync(acc, 0, sizeof(ValidateAccum), s));
  const int blocks = (nrows + kRowsPerBlock - 1) / kRowsPerBlock;
  if (blocks > 0) {
    if (off_bits == 16)
      k_validate_dacsr<int16_t><<<blocks, kConvThreads, 0, s>>>(
          nrows, ncols, nnz, rowptr, static_cast<const int16_t *>(off), acc);
    else
      k_validate_dacsr<int8_t><<<blocks, kConvThreads, 0, s>>>(
          nrows, ncols, nnz, rowptr, static_cast<const int8_t *>(off), acc);
    DAMN_CHECK_LAUNCH("k_validate_dacsr");
  }
  ValidateAccum h{};
  DAMN_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  if (nrows == 0) h.bad_rows = nnz != 0 ? 1 : 0;  // no block ran: rowptr[0] == nnz must be 0
  *h_bad_rows = static_cast<int64_t>(h.bad_rows);
  *h_bad_cols = static_cast<int64_t>(h.bad_cols);
  if (h.bad_rows || h.bad_cols)
    return set_error(DAMN_ERR_INVALID_ARG,
                     "damn_validate_dacsr: %llu bad row pointers, %llu entries with r + off outside [0, %d)",
                     h.bad_rows, h.bad_cols, ncols);
  return DAMN_OK;
}

extern "C" int damn_cast_values(int64_t n, const void *src, int src_dtype, void *dst, int dst_dtype,
                                void *stream) {
  if (n < 0) return set_error(DAMN_ERR_INVALID_ARG, "damn_cast_values: n < 0");
  if (n == 0) return DAMN_OK;
  if (!src || !dst) return set_error(DAMN_ERR_INVALID_ARG, "damn_cast_values: NULL pointer");
  const bool ok =
      (src_dtype == DAMN_F64 &&
       (dst_dtype == DAMN_F32 || dst_dtype == DAMN_BF16 || dst_dtype == DAMN_F8E4M3)) ||
      (src_dtype == DAMN_F32 && (dst_dtype == DAMN_BF16 || dst_dtype == DAMN_F8E4M3));
  if (!ok) return set_error(DAMN_ERR_UNSUPPORTED, "damn_cast_values: unsupported dtype pair");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = (int)std::min<int64_t>(8LL * sm_count(), (n + 255) / 256);
  k_cast<<<blocks, 256, 0, s>>>(n, src, src_dtype, dst, dst_dtype);
  DAMN_CHECK_LAUNCH("k_cast");
  return DAMN_OK;
}

// ----------------------------------------------------------------------------
// Allocation-free conversion (no counterpart in the paper)
// ----------------------------------------------------------------------------
// Some callers cannot allocate device memory: a host application or framework
// that owns every device allocation through its own pool and forbids others,
// or a latency-critical loop where cudaMalloc (which can synchronise the whole
// device) is not acceptable.  damn_csr_to_dacsr_noalloc gives them the
// conversion without a workspace: its scratch -- one fit record per block of
// kRowsPerBlock rows plus one for the reduced result -- is a file-scope
// device array that every GPU loading the library holds until the process
// exits (kNoAllocMaxBlocks + 1 records of 32 bytes, about 64 KiB per device).
namespace damn {
namespace {

constexpr int kNoAllocMaxBlocks = 2048;  // at most 2048 * 512 = 1,048,576 rows

struct __align__(32) FitPartial {
  int min_off;
  int max_off;
  unsigned long long n_fit;
  unsigned long long n_bad;
  int pad[2];
};

static __device__ __align__(256) FitPartial g_noalloc_fit[kNoAllocMaxBlocks + 1];

// Same per-entry work as k_csr_to_dacsr<int16_t>; the block's result is written to
// its own record instead of being combined with atomics.
__global__ void __launch_bounds__(kConvThreads)
k_csr_to_dacsr16_part(int nrows, int ncols, const int *__restrict__ rowptr,
                      const int *__restrict__ col, int16_t *__restrict__ off, FitPartial *part) {
  __shared__ int rp[kRowsPerBlock + 1];
  __shared__ int s_mn[kConvThreads / 32], s_mx[kConvThreads / 32];
  __shared__ unsigned long long s_nf[kConvThreads / 32], s_nb[kConvThreads / 32];
  const int r0 = blockIdx.x * kRowsPerBlock;
  const int nr = min(kRowsPerBlock, nrows - r0);
  for (int i = threadIdx.x; i <= nr; i += kConvThreads) rp[i] = rowptr[r0 + i];
  __syncthreads();
  const int k0 = rp[0], k1 = rp[nr];
  int mn = INT_MAX, mx = INT_MIN;
  unsigned long long nf = 0, nb = 0;
  for (int k = k0 + threadIdx.x; k < k1; k += kConvThreads) {
    const int lr = row_of(rp, nr, k);
    const int c = __ldcs(col + k);
    const long long d = (long long)c - (r0 + lr);  // 64 bits, as above
    __stcs(off + k, static_cast<int16_t>(d));
    mn = min(mn, sat_int(d));
    mx = max(mx, sat_int(d));
    nf += (d >= -32768 && d <= 32767) ? 1ull : 0ull;
    nb += (c < 0 || c >= ncols) ? 1ull : 0ull;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nf += __shfl_xor_sync(0xffffffffu, nf, o);
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { s_mn[w] = mn; s_mx[w] = mx; s_nf[w] = nf; s_nb[w] = nb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kConvThreads / 32; ++i) {
      mn = min(mn, s_mn[i]); mx = max(mx, s_mx[i]); nf += s_nf[i]; nb += s_nb[i];
    }
    FitPartial r;
    r.min_off = mn; r.max_off = mx; r.n_fit = nf; r.n_bad = nb; r.pad[0] = r.pad[1] = 0;
    part[blockIdx.x] = r;
  }
}

// Combines the nblocks records into *out (written, not accumulated, so
// nothing from an earlier call survives into this one).
__global__ void k_fit_reduce_part(const FitPartial *part, int nblocks, FitPartial *out) {
  __shared__ int s_mn[32], s_mx[32];
  __shared__ unsigned long long s_nf[32], s_nb[32];
  int mn = INT_MAX, mx = INT_MIN;
  unsigned long long nf = 0, nb = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    mn = min(mn, part[b].min_off);
    mx = max(mx, part[b].max_off);
    nf += part[b].n_fit;
    nb += part[b].n_bad;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nf += __shfl_xor_sync(0xffffffffu, nf, o);
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { s_mn[w] = mn; s_mx[w] = mx; s_nf[w] = nf; s_nb[w] = nb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x / 32); ++i) {
      mn = min(mn, s_mn[i]); mx = max(mx, s_mx[i]); nf += s_nf[i]; nb += s_nb[i];
    }
    FitPartial r;
    r.min_off = mn; r.max_off = mx; r.n_fit = nf; r.n_bad = nb; r.pad[0] = r.pad[1] = 0;
    *out = r;
  }
}

// Device address of g_noalloc_fit on the current device, looked up with
// cudaGetSymbolAddress once per device (again after a device reset, which
// gives the device a new context).  In host code the array's name is only a
// stand-in for the symbol, so kernels get this address, never the name.
SymbolCache g_noalloc_cache;

FitPartial *noalloc_fit_scratch(int *rc) {
  return static_cast<FitPartial *>(symbol_address(g_noalloc_cache, &g_noalloc_fit,
                                                  "damn_csr_to_dacsr_noalloc: scratch address", rc));
}

}  // namespace
}  // namespace damn

extern "C" int damn_csr_to_dacsr_noalloc(int32_t nrows, int32_t ncols, int64_t nnz,
                                         const int32_t *rowptr, const int32_t *col,
                                         int16_t *off_out, damn_fit_info *h_info, void *stream) {
  if (nrows < 0 || ncols < 0 || nnz < 0 || nnz > INT_MAX)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_csr_to_dacsr_noalloc: bad sizes");
  const long long max_rows = (long long)kNoAllocMaxBlocks * kRowsPerBlock;
  if (nrows > max_rows)
    return set_error(DAMN_ERR_INVALID_ARG,
                     "damn_csr_to_dacsr_noalloc: %d rows exceed the %lld rows its static scratch "
                     "covers; use damn_csr_to_dacsr with a workspace",
                     nrows, max_rows);
  if (!h_info || !rowptr || (nnz > 0 && (!col || !off_out)))
    return set_error(DAMN_ERR_INVALID_ARG, "damn_csr_to_dacsr_noalloc: NULL pointer");
  int rc = DAMN_OK;
  FitPartial *part = noalloc_fit_scratch(&rc);
  if (!part) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = (nrows + kRowsPerBlock - 1) / kRowsPerBlock;
  if (blocks > 0) {
    k_csr_to_dacsr16_part<<<blocks, kConvThreads, 0, s>>>(nrows, ncols, rowptr, col, off_out, part);
    DAMN_CHECK_LAUNCH("k_csr_to_dacsr16_part");
  }
  k_fit_reduce_part<<<1, 256, 0, s>>>(part, blocks, part + kNoAllocMaxBlocks);
  DAMN_CHECK_LAUNCH("k_fit_reduce_part");
  FitPartial h{};
  DAMN_CUDA(cudaMemcpyAsync(&h, part + kNoAllocMaxBlocks, sizeof(h), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  if (nnz == 0) { h.min_off = 0; h.max_off = 0; }
  h_info->min_off = h.min_off;
  h_info->max_off = h.max_off;
  h_info->w = std::max<int64_t>(-(int64_t)h.min_off, (int64_t)h.max_off);
  h_info->n_fit = static_cast<int64_t>(h.n_fit);
  h_info->n_bad = static_cast<int64_t>(h.n_bad);
  h_info->fits = (static_cast<int64_t>(h.n_fit) == nnz && h.n_bad == 0) ? 1 : 0;
  h_info->reserved = 0;
  if (!h_info->fits)
    return set_error(DAMN_ERR_NOFIT,
                     "damn_csr_to_dacsr_noalloc: %lld of %lld entries do not fit int16 (min %d, max %d), %lld bad columns",
                     (long long)(nnz - h_info->n_fit), (long long)nnz, h.min_off, h.max_off,
                     (long long)h.n_bad);
  return DAMN_OK;
}
