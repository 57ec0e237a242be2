// Shared device and host helpers of the DA-CSR library (sm_103a).
//
// Device side: inline-PTX wrappers for mbarriers and the bulk asynchronous
// copy engine (cp.async.bulk, the non-tensor TMA path), named barriers, the
// global timer used to bound every wait, and value-type conversions.
// Host side: status codes, the per-thread error message and CUDA call checks.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <mutex>
#include <string>

#include "../../include/damn.h"

namespace damn {

// ----------------------------------------------------------------------------
// Host: errors
// ----------------------------------------------------------------------------
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
int *device_status_ptr();          // library status word on the current device
int sm_count();                    // SMs of the current device

// Identifier of the calling thread's current CUDA context, 0 when there is
// none yet.  A device reset destroys the context and its successor gets a new
// identifier.
unsigned long long context_id();

// Device addresses of one __device__ variable, one per device, each valid for
// the context it was looked up in.
struct SymbolCache {
  static constexpr int kDevices = 64;
  unsigned long long ctx[kDevices] = {};
  void *addr[kDevices] = {};
  std::mutex mu;
};

// Device address of `symbol` (the host-side stand-in of a __device__
// variable) on the current device: cudaGetSymbolAddress once per device
// context, cached in `cache`.  A kernel must be given this address, never
// the stand-in.  NULL on failure (*rc set).
void *symbol_address(SymbolCache &cache, const void *symbol, const char *what, int *rc);

// Reads the device status word (synchronises s): DAMN_OK, or the recorded
// error code (with a message) when a bounded wait gave up or a device-side
// check failed.  The word is not cleared.
int check_device_status(cudaStream_t s, const char *what);

#define DAMN_CUDA(call)                                                  \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return ::damn::cuda_error(e_, #call);         \
  } while (0)

#define DAMN_CHECK_LAUNCH(what)                                          \
  do {                                                                   \
    cudaError_t e_ = cudaGetLastError();                                 \
    if (e_ != cudaSuccess) return ::damn::cuda_error(e_, what);          \
  } while (0)

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Default limit of every device-side wait: a kernel that would otherwise hang
// records DAMN_ERR_TIMEOUT in the status word and returns.
constexpr uint64_t kWaitTimeoutNs = 2000000000ull;  // 2 s

// ----------------------------------------------------------------------------
// Device: PTX wrappers
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Same, but the thread may be suspended for up to hint_ns nanoseconds
// waiting for the phase to complete instead of returning at once, so a
// waiting warp takes no issue slots from the working ones.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint32_t addr, uint32_t parity,
                                                      uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity to complete, for at most
// timeout_ns.  On timeout records DAMN_ERR_TIMEOUT in *status and returns
// false.
// The clock is read once per 16 tries (each try may suspend the thread up to
// the hint), so that a waiting warp spends few issue slots.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *status,
                                                  uint64_t timeout_ns) {
  const uint32_t a = smem_addr(bar);
  if (mbar_try_wait(a, parity)) return true;
  const uint64_t t0 = global_timer_ns();
#pragma unroll 1
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 16; ++i)
      if (mbar_try_wait_suspend(a, parity, 100000u)) return true;
    if (global_timer_ns() - t0 > timeout_ns) {
      if (status) atomicExch(status, DAMN_ERR_TIMEOUT);
      return false;
    }
  }
}

// Programmatic dependent launch.  wait: blocks until the grids this one
// depends on in its stream have completed and their writes are visible (a
// no-op when the launch did not ask for programmatic serialisation); no
// global memory may be touched before it.  launch_dependents: lets the next
// kernel of the stream start launching its CTAs (they run their prologue,
// then wait in turn), hiding the launch gap between back-to-back kernels.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// L2 policy for data that is streamed once (matrix arrays).
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Bulk asynchronous copy global -> shared (this CTA), completing on `bar`
// with `bytes` transaction bytes.  dst, src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// Same without a cache hint (data that should stay in L2, e.g. x).
__device__ __forceinline__ void bulk_copy_g2s_nohint(void *dst, const void *src, uint32_t bytes,
                                                     uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also ORs a predicate over the participating threads.
__device__ __forceinline__ bool named_bar_or(int id, int nthreads, bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
      : "memory");
  return out != 0;
}

// ----------------------------------------------------------------------------
// Value types
// ----------------------------------------------------------------------------
// FP8 E4M3 value (the 'fn' variant: sign, 4 exponent bits with bias 7, 3
// significand bits, no infinity, NaN = S.1111.111), stored as its byte.
struct f8e4m3 {
  uint8_t b;
};

template <typename T> struct AccOf;
template <> struct AccOf<double> { using type = double; };
template <> struct AccOf<float> { using type = float; };
template <> struct AccOf<__nv_bfloat16> { using type = float; };
template <> struct AccOf<f8e4m3> { using type = float; };

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
// E4M3 -> FP32, exact, through the hardware E4M3 -> FP16 conversion: every
// E4M3 value (magnitudes 2^-9 .. 448) is an FP16 normal or zero, and NaN
// stays NaN.
__device__ __forceinline__ float to_acc(f8e4m3 v) {
  return __half2float(__half(__nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(v.b), __NV_E4M3)));
}

// Running dot product of a thread.  FP64 operands: FP64 FMA.  FP32 operands
// (the inner CG of the refinement): every product a b is split exactly into
// FP32 p + e (e = fma(a, b, -p)), p is added to a compensated FP32 pair with
// the error-free TwoSum, e and the TwoSum error go to the low part; the pair
// is combined in FP64 once at the end.  The relative error of a thread's
// sum of k products is below about (k + 2) 2^-47 (FP64 accumulation of the
// same k products: k 2^-53), far below the FP32 rounding of the vectors,
// and no FP64 instruction is spent per element (the FP64 unit of this part
// does 2 lane operations per SM-cycle, the FP32 units 128).  Products below
// FP32's normal range (|a b| < 2^-126) lose relative accuracy; the inner
// vectors are normalised, far from that range.
template <typename A> struct DotAcc;
template <> struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = __fma_rn(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);          // a b = p + pe exactly
    const float s = __fadd_rn(hi, p);               // TwoSum(hi, p) = s + t exactly
    const float bv = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(t, pe));
  }
  __device__ __forceinline__ double value() const {
    return static_cast<double>(hi) + static_cast<double>(lo);
  }
};

__device__ __forceinline__ double fma_acc(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_acc(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename T> __device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }
template <> __device__ __forceinline__ __nv_bfloat16 ldg(const __nv_bfloat16 *p) {
  unsigned short u = __ldg(reinterpret_cast<const unsigned short *>(p));
  return __ushort_as_bfloat16(u);
}
template <> __device__ __forceinline__ f8e4m3 ldg(const f8e4m3 *p) {
  return f8e4m3{__ldg(reinterpret_cast<const unsigned char *>(p))};
}

}  // namespace damn
