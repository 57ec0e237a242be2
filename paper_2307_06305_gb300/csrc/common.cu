// Library-wide host state: error messages, the device status word, the
// failure-detection self test, version.
#include <cuda.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "damn_common.cuh"

namespace damn {

namespace {
thread_local std::string g_last_error;

// One status word per device context (a kernel whose bounded wait gives up
// records DAMN_ERR_TIMEOUT here instead of hanging).
__device__ int g_status_word;

constexpr int kMaxDevices = 64;
SymbolCache g_status_cache;
int g_sm_count[kMaxDevices];
std::mutex g_mu;

using PfnCtxGetCurrent = CUresult (*)(CUcontext *);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long *);
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;
std::once_flag g_ctx_fn_once;
}  // namespace

unsigned long long context_id() {
  std::call_once(g_ctx_fn_once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(f);
  });
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  unsigned long long id = 0;
  if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

void *symbol_address(SymbolCache &cache, const void *symbol, const char *what, int *rc) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { *rc = cuda_error(e, what); return nullptr; }
  if (dev < 0 || dev >= SymbolCache::kDevices) {
    *rc = set_error(DAMN_ERR_UNSUPPORTED, "%s: device index %d", what, dev);
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(cache.mu);
  const unsigned long long ctx = context_id();
  if (!cache.addr[dev] || ctx == 0 || cache.ctx[dev] != ctx) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, symbol);
    if (e != cudaSuccess) { *rc = cuda_error(e, what); return nullptr; }
    cache.addr[dev] = p;
    cache.ctx[dev] = context_id();  // the lookup above created the context if needed
  }
  return cache.addr[dev];
}

int check_device_status(cudaStream_t s, const char *what) {
  int *p = device_status_ptr();
  if (!p) return set_error(DAMN_ERR_CUDA, "%s: no device status word", what);
  int v = 0;
  DAMN_CUDA(cudaMemcpyAsync(&v, p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  if (v != DAMN_OK)
    return set_error(v, "%s: the device status word reports %d (a bounded device-side wait gave "
                        "up, or a device-side check failed); results are incomplete",
                     what, v);
  return DAMN_OK;
}

int set_error(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_error(cudaError_t e, const char *what) {
  return set_error(DAMN_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int *device_status_ptr() {
  int rc = DAMN_OK;
  return static_cast<int *>(symbol_address(g_status_cache, &g_status_word, "device status word", &rc));
}

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_sm_count[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_sm_count[dev] = n > 0 ? n : 1;
  }
  return g_sm_count[dev];
}

// A barrier that nothing ever completes: the bounded wait must give up.
__global__ void k_selftest_wait(int *status, uint64_t timeout_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, status, timeout_ns);
}

}  // namespace damn

using namespace damn;

extern "C" const char *damn_last_error(void) { return g_last_error.c_str(); }

extern "C" int damn_version(void) { return 100; }

extern "C" int damn_device_status(int32_t *h_status, int reset, void *stream) {
  if (!h_status) return set_error(DAMN_ERR_INVALID_ARG, "damn_device_status: h_status is NULL");
  int *p = device_status_ptr();
  if (!p) return set_error(DAMN_ERR_CUDA, "damn_device_status: no device status word");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  DAMN_CUDA(cudaMemcpyAsync(&v, p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  if (reset) {
    DAMN_CUDA(cudaMemsetAsync(p, 0, sizeof(int), s));
    DAMN_CUDA(cudaStreamSynchronize(s));
  }
  *h_status = v;
  return DAMN_OK;
}

extern "C" int damn_selftest_wait_timeout(int64_t timeout_ns, void *stream) {
  if (timeout_ns < 1000 || timeout_ns > 10000000000ll)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_selftest_wait_timeout: timeout_ns out of range");
  int *p = device_status_ptr();
  if (!p) return set_error(DAMN_ERR_CUDA, "damn_selftest_wait_timeout: no device status word");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DAMN_CUDA(cudaMemsetAsync(p, 0, sizeof(int), s));
  k_selftest_wait<<<1, 32, 0, s>>>(p, static_cast<uint64_t>(timeout_ns));
  DAMN_CHECK_LAUNCH("k_selftest_wait");
  int v = 0;
  DAMN_CUDA(cudaMemcpyAsync(&v, p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  DAMN_CUDA(cudaMemsetAsync(p, 0, sizeof(int), s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  if (v == DAMN_ERR_TIMEOUT)
    return set_error(DAMN_ERR_TIMEOUT, "bounded device wait gave up after %lld ns (expected)",
                     static_cast<long long>(timeout_ns));
  return set_error(DAMN_ERR_CUDA, "self test: the wait did not report a timeout (status %d)", v);
}
