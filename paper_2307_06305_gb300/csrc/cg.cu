// Conjugate gradients in FP64 and mixed-precision iterative refinement
// (CG-IR) around a reduced-precision CG, on DA-CSR-16 matrices.
//
// The paper motivates DA storage for iterative solvers and multi-precision
// algorithms (Section 2, multi-precision remark; Section 3); the solver is
// textbook Hestenes-Stiefel CG:
//
//   q = A p;  a = rr / (p.q);  x += a p;  r -= a q;  rr' = r.r;
//   p = r + (rr'/rr) p;  rr = rr'
//
// One iteration is three launches: the SpMV (whose epilogue also forms the
// per-CTA partial sums of p.q in FP64), k_cg_update (a, x, r and partial
// r.r) and k_cg_direction (rr', beta, p, convergence flag).  Dot products are
// reduced deterministically: every CTA sums the same partials in the same
// order.  A device "done" flag turns the kernels of later iterations into
// no-ops, so chunks of iterations run as one CUDA graph and the host reads the
// flag once per chunk.
//
// CG-IR: the outer loop computes r = b - A x with the FP64 values and FP64
// accumulation (the SpMV with alpha = -1, beta = 1 and a fused ||r||^2),
// stops at ||r|| <= rtol ||b||, solves A_low d = r / ||r|| with the CG above
// in FP32 vectors (FP32 or BF16 values, FP32 accumulation, FP64 dot
// products) to inner_rtol, and updates x += ||r|| d in FP64.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "damn_common.cuh"
#include "spmv_internal.h"

namespace damn {
namespace {

constexpr int kVecThreads = 256;

// Scalars of a CG run (device).
struct CgScalars {
  double rr[2];      // r.r of the previous iteration, double-buffered by parity
  double tol2;       // stop when r.r <= tol2
  int done;          // 1: converged, 2: breakdown (p.q <= 0 or not finite), 3: cap reached
  int iters;         // iterations performed
  int max_iter;      // iteration cap
  int pad;
};

// Deterministic sum of n partials by one CTA: thread t adds partials
// t, t + blockDim, ... in order, then a fixed-shape tree.
__device__ double block_sum(const double *part, int n, double *red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = s;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

template <typename T>
__device__ __forceinline__ double to_d(T v) { return static_cast<double>(v); }

// 16 bytes of a vector: 4 floats or 2 doubles per load.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using type = float4;
  static constexpr int N = 4;
  __device__ static float get(const float4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
  __device__ static void set(float4 &v, int i, float f) {
    if (i == 0) v.x = f; else if (i == 1) v.y = f; else if (i == 2) v.z = f; else v.w = f;
  }
};
template <> struct Vec16<double> {
  using type = double2;
  static constexpr int N = 2;
  __device__ static double get(const double2 &v, int i) { return i == 0 ? v.x : v.y; }
  __device__ static void set(double2 &v, int i, double f) { if (i == 0) v.x = f; else v.y = f; }
};

__device__ __forceinline__ bool all_aligned16(const void *a, const void *b, const void *c,
                                              const void *d) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
           reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(d)) & 15u) == 0;
}

// Per-CTA sum of the threads' dot accumulators into part[blockIdx.x].
template <typename T>
__device__ __forceinline__ void block_partial(const DotAcc<T> &acc, double *red, double *part) {
  double s = acc.value();
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    part[blockIdx.x] = t;
  }
}

// a = rr / (p.q); x += a p; r -= a q; partial r.r -> part_rr[blockIdx].
// 16-byte loads when every vector is 16-byte aligned (the tail and
// misaligned vectors element by element).
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_cg_update(int n, const double *part_pq, int npq, CgScalars *sc, int parity, T *x, T *r,
            const T *p, const T *q, double *part_rr) {
  using VT = Vec16<T>;
  using V = typename VT::type;
  __shared__ double red[kVecThreads / 32];
  if (sc->done) return;
  const double pq = block_sum(part_pq, npq, red);
  const double rr = sc->rr[parity];
  const double a = rr / pq;
  if (!(pq > 0.0) || !isfinite(a)) {  // breakdown: stop without touching x
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->done = 2;
    if (threadIdx.x == 0) part_rr[blockIdx.x] = 0.0;
    return;
  }
  const T at = static_cast<T>(a);
  DotAcc<T> acc;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long head = 0;
  if (all_aligned16(x, r, p, q)) {
    const long long nv = n / VT::N;
    head = nv * VT::N;
    for (long long v = tid; v < nv; v += stride) {
      V xv = reinterpret_cast<const V *>(x)[v], rv = reinterpret_cast<const V *>(r)[v];
      const V pv = reinterpret_cast<const V *>(p)[v], qv = reinterpret_cast<const V *>(q)[v];
#pragma unroll
      for (int k = 0; k < VT::N; ++k) {
        VT::set(xv, k, VT::get(xv, k) + at * VT::get(pv, k));
        const T ri = VT::get(rv, k) - at * VT::get(qv, k);
        VT::set(rv, k, ri);
        acc.add(ri, ri);
      }
      reinterpret_cast<V *>(x)[v] = xv;
      reinterpret_cast<V *>(r)[v] = rv;
    }
  }
  for (long long i = head + tid; i < n; i += stride) {
    x[i] = x[i] + at * p[i];
    const T ri = r[i] - at * q[i];
    r[i] = ri;
    acc.add(ri, ri);
  }
  block_partial<T>(acc, red, part_rr);
}

// rr' = sum part_rr; b = rr'/rr; p = r + b p; flags convergence
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_cg_direction(int n, const double *part_rr, int nrr, CgScalars *sc, int parity, const T *r,
               T *p) {
  using VT = Vec16<T>;
  using V = typename VT::type;
  __shared__ double red[kVecThreads / 32];
  if (sc->done) return;
  const double rr_new = block_sum(part_rr, nrr, red);
  const double beta = rr_new / sc->rr[parity];
  const T bt = static_cast<T>(beta);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long head = 0;
  if (all_aligned16(r, p, r, p)) {
    const long long nv = n / VT::N;
    head = nv * VT::N;
    for (long long v = tid; v < nv; v += stride) {
      const V rv = reinterpret_cast<const V *>(r)[v];
      V pv = reinterpret_cast<const V *>(p)[v];
#pragma unroll
      for (int k = 0; k < VT::N; ++k) VT::set(pv, k, VT::get(rv, k) + bt * VT::get(pv, k));
      reinterpret_cast<V *>(p)[v] = pv;
    }
  }
  for (long long i = head + tid; i < n; i += stride) p[i] = r[i] + bt * p[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rr[parity ^ 1] = rr_new;
    sc->iters += 1;
    if (rr_new <= sc->tol2) sc->done = 1;
    else if (sc->iters >= sc->max_iter) sc->done = 3;
  }
}

// Starts a CG run: p = r, rr = sum part (r.r), done = (rr <= tol2); a
// negative tol2_rel asks for tol2 = -tol2_rel * rr (relative to the start)
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_cg_start(int n, const double *part, int npart, CgScalars *sc, double tol2_rel, int max_iter,
           const T *r, T *p) {
  __shared__ double red[kVecThreads / 32];
  const double rr = block_sum(part, npart, red);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = r[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // tol2_rel < 0: the tolerance is relative to the start, -tol2_rel * rr
    if (tol2_rel < 0.0) tol2_rel = -tol2_rel * rr;
    sc->rr[0] = rr;
    sc->rr[1] = rr;
    sc->tol2 = tol2_rel;
    sc->iters = 0;
    sc->max_iter = max_iter;
    sc->done = (rr <= tol2_rel) ? 1 : (max_iter <= 0 ? 3 : 0);
  }
}

// Partial sums of v.v (DotAcc: FP64 for FP64 vectors, compensated FP32 of
// exact products for FP32 vectors).
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_dot_self(int n, const T *v, double *part) {
  __shared__ double red[kVecThreads / 32];
  DotAcc<T> acc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc.add(v[i], v[i]);
  block_partial<T>(acc, red, part);
}

// out = sum of partials (one CTA)
__global__ void __launch_bounds__(kVecThreads) k_sum(const double *part, int n, double *out) {
  __shared__ double red[kVecThreads / 32];
  const double s = block_sum(part, n, red);
  if (threadIdx.x == 0) *out = s;
}

// s32 = fl32(r / nr), d = 0   (inner right-hand side of the refinement)
__global__ void k_scale_to_f32(int n, const double *r, const double *nr2, float *s32, float *d) {
  const double inv = 1.0 / sqrt(*nr2);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    s32[i] = __double2float_rn(r[i] * inv);
    d[i] = 0.0f;
  }
}

// x += ||r|| d  (FP64)
__global__ void k_ir_update(int n, const double *nr2, const float *d, double *x) {
  const double nr = sqrt(*nr2);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = __fma_rn(nr, static_cast<double>(d[i]), x[i]);
}

// x = 0
template <typename T>
__global__ void k_zero(int n, T *x) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = T(0);
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int vec_grid() { return 4 * sm_count(); }

// Workspace carving helper
struct Carve {
  char *base;
  size_t off = 0;
  template <typename T> T *take(size_t count) {
    T *p = reinterpret_cast<T *>(base + off);
    off += align256(count * sizeof(T));
    return p;
  }
};

size_t partials_count() { return (size_t)spmv_max_grid() + (size_t)vec_grid() + 8; }

// One matrix for the CG loop.
struct CgMatrix {
  int n;
  long long nnz;
  const int32_t *rowptr;
  const int16_t *off;
  const void *val;
  int dtype;  // DAMN_F64 (vectors double) or DAMN_F32 / DAMN_BF16 (vectors float)
  const damn_plan *plan;
};

// Runs CG iterations on A p = ... with vectors of type T, starting from the
// current x, r (p and rr set by k_cg_start).  Returns DAMN_OK or an error.
// `chunk` iterations run per graph launch (even, so that parities line up);
// the graph is captured on the first call and kept in *exec_cache (the
// caller destroys it) for later calls with the same vectors, as the inner
// solves of CG-IR are.
template <typename T>
int cg_loop(const CgMatrix &A, T *x, T *r, T *p, T *q, double *part_pq, double *part_rr,
            CgScalars *sc, int max_iter, cudaStream_t s, int *iters_out, int *done_out,
            int chunk, cudaGraphExec_t *exec_cache) {
  const int n = A.n;
  const int gv = vec_grid();
  // the SpMV q = A p with the fused p.q partials
  SpmvCall c;
  c.nrows = n; c.ncols = n; c.nnz = A.nnz; c.rowptr = A.rowptr; c.idx = A.off;
  c.fmt = DAMN_FMT_DACSR16; c.val = A.val; c.dtype = A.dtype; c.x = p; c.y0 = q; c.y = q;
  c.alpha = 1.0; c.beta = 0.0; c.dot_w = p; c.dot_partials = part_pq;
  int gs = 0;
  // one eager iteration pair: sets launch attributes and tells the SpMV grid
  auto iteration = [&](int parity) -> int {
    int rc = spmv_launch(c, A.plan, s, &gs);
    if (rc) return rc;
    k_cg_update<T><<<gv, kVecThreads, 0, s>>>(n, part_pq, gs, sc, parity, x, r, p, q, part_rr);
    k_cg_direction<T><<<gv, kVecThreads, 0, s>>>(n, part_rr, gv, sc, parity, r, p);
    DAMN_CHECK_LAUNCH("cg iteration");
    return DAMN_OK;
  };
  CgScalars h{};
  int done_iters = 0;
  // first two iterations eagerly (launch attributes, SpMV grid size), then
  // graphs of `chunk` iterations; the device flag stops at convergence, at a
  // breakdown or at max_iter, after which launched iterations do nothing
  for (int k = 0; k < 2 && done_iters < max_iter; ++k, ++done_iters) {
    int rc = iteration(k & 1);
    if (rc) return rc;
  }
  cudaGraphExec_t exec = *exec_cache;
  if (!exec && done_iters < max_iter) {
    cudaStream_t cs;
    DAMN_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    int rc = DAMN_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int k = 0; k < chunk && rc == DAMN_OK; ++k) {
        rc = spmv_launch(c, A.plan, cs, nullptr);
        if (rc) break;
        k_cg_update<T><<<gv, kVecThreads, 0, cs>>>(n, part_pq, gs, sc, k & 1, x, r, p, q, part_rr);
        k_cg_direction<T><<<gv, kVecThreads, 0, cs>>>(n, part_rr, gv, sc, k & 1, r, p);
      }
      e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess && rc == DAMN_OK) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_error(e, "cg graph capture");
    *exec_cache = exec;
  }
  // chunks: launch, then read the flag (one small copy per chunk)
  int rc = DAMN_OK;
  while (true) {
    cudaError_t e = cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { rc = cuda_error(e, "cg loop"); break; }
    if (h.done || done_iters >= max_iter || !exec) break;
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) { rc = cuda_error(e, "cudaGraphLaunch"); break; }
    done_iters += chunk;
  }
  *iters_out = h.iters;
  *done_out = h.done;
  return rc;
}

}  // namespace
}  // namespace damn

using namespace damn;

static int check_cg_args(const char *fn, int32_t n, int64_t nnz, const int32_t *rowptr,
                         const int16_t *off, const void *val, const void *b, const void *x,
                         damn_cg_result *h_res, void *ws, size_t ws_bytes, size_t need) {
  if (n < 0 || nnz < 0 || nnz > INT_MAX) return set_error(DAMN_ERR_INVALID_ARG, "%s: bad sizes", fn);
  if (!h_res) return set_error(DAMN_ERR_INVALID_ARG, "%s: h_res is NULL", fn);
  if (n > 0 && (!rowptr || !b || !x || (nnz > 0 && (!off || !val))))
    return set_error(DAMN_ERR_INVALID_ARG, "%s: NULL pointer", fn);
  if (!ws || ws_bytes < need || !aligned16(ws))
    return set_error(DAMN_ERR_INVALID_ARG, "%s: workspace too small (%zu < %zu) or misaligned", fn,
                     ws_bytes, need);
  return DAMN_OK;
}

extern "C" size_t damn_cg_workspace_size(int32_t n) {
  const size_t nn = n > 0 ? (size_t)n : 0;
  return 3 * align256(nn * sizeof(double)) + 2 * align256(partials_count() * sizeof(double)) +
         align256(sizeof(CgScalars)) + align256(16 * sizeof(double)) + 4096;
}

// ||b - A x||^2 / ||b||^2 in FP64 into h (uses r and partials as scratch)
static int true_relres(const CgMatrix &A64, const double *b, const double *x, double *r,
                       double *part, double *tmp, cudaStream_t s, double *out) {
  SpmvCall c;
  c.nrows = A64.n; c.ncols = A64.n; c.nnz = A64.nnz; c.rowptr = A64.rowptr; c.idx = A64.off;
  c.fmt = DAMN_FMT_DACSR16; c.val = A64.val; c.dtype = DAMN_F64; c.x = x; c.y0 = b; c.y = r;
  c.alpha = -1.0; c.beta = 1.0; c.dot_self = 1; c.dot_partials = part;
  int gs = 0;
  int rc = spmv_launch(c, A64.plan, s, &gs);
  if (rc) return rc;
  k_sum<<<1, kVecThreads, 0, s>>>(part, gs, tmp);
  k_dot_self<double><<<vec_grid(), kVecThreads, 0, s>>>(A64.n, b, part + spmv_max_grid());
  k_sum<<<1, kVecThreads, 0, s>>>(part + spmv_max_grid(), vec_grid(), tmp + 1);
  DAMN_CHECK_LAUNCH("true_relres");
  double h[2] = {0, 0};
  DAMN_CUDA(cudaMemcpyAsync(h, tmp, sizeof(h), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  *out = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
  return DAMN_OK;
}

extern "C" int damn_cg(int32_t n, int64_t nnz, const int32_t *rowptr, const int16_t *off,
                       const double *val, const double *b, double *x, double rtol,
                       int32_t max_iter, const damn_plan *plan, damn_cg_result *h_res,
                       void *workspace, size_t ws_bytes, void *stream) {
  int rc = check_cg_args("damn_cg", n, nnz, rowptr, off, val, b, x, h_res, workspace, ws_bytes,
                         damn_cg_workspace_size(n));
  if (rc) return rc;
  rc = plan_check("damn_cg", plan, DAMN_FMT_DACSR16, n, n, nnz, rowptr, off, DAMN_F64);
  if (rc) return rc;
  std::memset(h_res, 0, sizeof(*h_res));
  if (n == 0) { h_res->converged = 1; return DAMN_OK; }
  if (!(rtol > 0) || max_iter < 0) return set_error(DAMN_ERR_INVALID_ARG, "damn_cg: bad rtol / max_iter");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carve cv{static_cast<char *>(workspace)};
  double *r = cv.take<double>(n), *p = cv.take<double>(n), *q = cv.take<double>(n);
  double *part_a = cv.take<double>(partials_count()), *part_b = cv.take<double>(partials_count());
  CgScalars *sc = cv.take<CgScalars>(1);
  double *tmp = cv.take<double>(16);
  CgMatrix A{n, nnz, rowptr, off, val, DAMN_F64, plan};
  // r = b - A x with ||r||^2 partials; ||b||^2
  SpmvCall c;
  c.nrows = n; c.ncols = n; c.nnz = nnz; c.rowptr = rowptr; c.idx = off; c.fmt = DAMN_FMT_DACSR16;
  c.val = val; c.dtype = DAMN_F64; c.x = x; c.y0 = b; c.y = r; c.alpha = -1.0; c.beta = 1.0;
  c.dot_self = 1; c.dot_partials = part_a;
  int gs = 0;
  rc = spmv_launch(c, plan, s, &gs);
  if (rc) return rc;
  k_dot_self<double><<<vec_grid(), kVecThreads, 0, s>>>(n, b, part_b);
  k_sum<<<1, kVecThreads, 0, s>>>(part_b, vec_grid(), tmp);
  DAMN_CHECK_LAUNCH("damn_cg start");
  double bb = 0;
  DAMN_CUDA(cudaMemcpyAsync(&bb, tmp, sizeof(double), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  const double tol2 = rtol * rtol * (bb > 0 ? bb : 1.0);
  k_cg_start<double><<<vec_grid(), kVecThreads, 0, s>>>(n, part_a, gs, sc, tol2, max_iter, r, p);
  DAMN_CHECK_LAUNCH("k_cg_start");
  int iters = 0, done = 0;
  cudaGraphExec_t exec = nullptr;
  rc = cg_loop<double>(A, x, r, p, q, part_a, part_b, sc, max_iter, s, &iters, &done, 16, &exec);
  if (exec) cudaGraphExecDestroy(exec);
  if (rc) return rc;
  CgScalars h{};
  DAMN_CUDA(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  h_res->iterations = iters;
  h_res->outer = 0;
  h_res->converged = done == 1 ? 1 : 0;
  h_res->relres = std::sqrt(h.rr[iters & 1] / (bb > 0 ? bb : 1.0));
  rc = true_relres(A, b, x, r, part_a, tmp, s, &h_res->true_relres);
  if (rc) return rc;
  // a bounded wait that gave up inside an SpMV left vectors partly computed
  rc = check_device_status(s, "damn_cg");
  if (rc) return rc;
  if (done == 2) return set_error(DAMN_ERR_NOT_CONVERGED, "damn_cg: breakdown (p.q <= 0)");
  if (!h_res->converged)
    return set_error(DAMN_ERR_NOT_CONVERGED, "damn_cg: not converged after %d iterations", iters);
  return DAMN_OK;
}

extern "C" size_t damn_cg_ir_workspace_size(int32_t n) {
  const size_t nn = n > 0 ? (size_t)n : 0;
  return align256(nn * sizeof(double)) + 4 * align256(nn * sizeof(float)) +
         2 * align256(partials_count() * sizeof(double)) + 2 * align256(sizeof(CgScalars)) +
         align256(16 * sizeof(double)) + 4096;
}

extern "C" int damn_cg_ir(int32_t n, int64_t nnz, const int32_t *rowptr, const int16_t *off,
                          const double *val, const void *val_low, int low_dtype, const double *b,
                          double *x, double rtol, double inner_rtol, int32_t max_inner,
                          int32_t max_outer, const damn_plan *plan64, const damn_plan *plan_low,
                          damn_cg_result *h_res, void *workspace, size_t ws_bytes, void *stream) {
  int rc = check_cg_args("damn_cg_ir", n, nnz, rowptr, off, val, b, x, h_res, workspace, ws_bytes,
                         damn_cg_ir_workspace_size(n));
  if (rc) return rc;
  if (low_dtype != DAMN_F32 && low_dtype != DAMN_BF16)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_cg_ir: low_dtype must be DAMN_F32 or DAMN_BF16");
  if (nnz > 0 && !val_low) return set_error(DAMN_ERR_INVALID_ARG, "damn_cg_ir: val_low is NULL");
  if (!(rtol > 0) || !(inner_rtol > 0) || max_inner < 1 || max_outer < 0)
    return set_error(DAMN_ERR_INVALID_ARG, "damn_cg_ir: bad tolerances or iteration caps");
  rc = plan_check("damn_cg_ir", plan64, DAMN_FMT_DACSR16, n, n, nnz, rowptr, off, DAMN_F64);
  if (rc) return rc;
  rc = plan_check("damn_cg_ir", plan_low, DAMN_FMT_DACSR16, n, n, nnz, rowptr, off, low_dtype);
  if (rc) return rc;
  std::memset(h_res, 0, sizeof(*h_res));
  if (n == 0) { h_res->converged = 1; return DAMN_OK; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carve cv{static_cast<char *>(workspace)};
  double *r = cv.take<double>(n);
  float *d = cv.take<float>(n), *r32 = cv.take<float>(n), *p32 = cv.take<float>(n),
        *q32 = cv.take<float>(n);
  double *part_a = cv.take<double>(partials_count()), *part_b = cv.take<double>(partials_count());
  CgScalars *sc = cv.take<CgScalars>(1);
  cv.take<CgScalars>(1);
  double *tmp = cv.take<double>(16);
  CgMatrix A64{n, nnz, rowptr, off, val, DAMN_F64, plan64};
  CgMatrix Alow{n, nnz, rowptr, off, val_low, low_dtype, plan_low};
  // ||b||^2
  k_dot_self<double><<<vec_grid(), kVecThreads, 0, s>>>(n, b, part_b);
  k_sum<<<1, kVecThreads, 0, s>>>(part_b, vec_grid(), tmp + 1);
  DAMN_CHECK_LAUNCH("damn_cg_ir start");
  double bb = 0;
  DAMN_CUDA(cudaMemcpyAsync(&bb, tmp + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  const double nb = std::sqrt(bb > 0 ? bb : 1.0);
  int total_inner = 0, outer = 0;
  double relres = 0.0;
  bool converged = false;
  cudaGraphExec_t inner_exec = nullptr;  // the inner loop's graph, captured once
  while (true) {
    // r = b - A x (FP64) and ||r||^2
    SpmvCall c;
    c.nrows = n; c.ncols = n; c.nnz = nnz; c.rowptr = rowptr; c.idx = off;
    c.fmt = DAMN_FMT_DACSR16; c.val = val; c.dtype = DAMN_F64; c.x = x; c.y0 = b; c.y = r;
    c.alpha = -1.0; c.beta = 1.0; c.dot_self = 1; c.dot_partials = part_a;
    int gs = 0;
    rc = spmv_launch(c, plan64, s, &gs);
    if (rc) break;
    k_sum<<<1, kVecThreads, 0, s>>>(part_a, gs, tmp);
    double rr = 0;
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&rr, tmp, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (ce != cudaSuccess) { rc = cuda_error(ce, "cg_ir residual"); break; }
    // also synchronises: a bounded wait that gave up inside an SpMV (this
    // residual or the previous inner solve) left vectors partly computed
    rc = check_device_status(s, "damn_cg_ir");
    if (rc) break;
    relres = std::sqrt(rr) / nb;
    if (relres <= rtol) { converged = true; break; }
    if (outer >= max_outer || !std::isfinite(relres)) break;
    // inner: A_low d = fl32(r / ||r||), d0 = 0, FP32 vectors, FP64 dots;
    // tolerance relative to ||fl32(r / ||r||)||: k_cg_start forms
    // tol2 = inner_rtol^2 * r32.r32 on the device from the same partials
    k_scale_to_f32<<<vec_grid(), kVecThreads, 0, s>>>(n, r, tmp, r32, d);
    k_dot_self<float><<<vec_grid(), kVecThreads, 0, s>>>(n, r32, part_a);
    k_cg_start<float><<<vec_grid(), kVecThreads, 0, s>>>(n, part_a, vec_grid(), sc,
                                                         -inner_rtol * inner_rtol, max_inner,
                                                         r32, p32);
    DAMN_CHECK_LAUNCH("cg_ir inner start");
    int it = 0, done = 0;
    rc = cg_loop<float>(Alow, d, r32, p32, q32, part_a, part_b, sc, max_inner, s, &it, &done, 8,
                        &inner_exec);
    if (rc) break;
    total_inner += it;
    // x += ||r|| d
    k_ir_update<<<vec_grid(), kVecThreads, 0, s>>>(n, tmp, d, x);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { rc = cuda_error(ce, "k_ir_update"); break; }
    ++outer;
  }
  if (inner_exec) cudaGraphExecDestroy(inner_exec);
  if (rc) return rc;
  h_res->iterations = total_inner;
  h_res->outer = outer;
  h_res->converged = converged ? 1 : 0;
  h_res->relres = relres;
  h_res->true_relres = relres;  // the outer residual is the true FP64 residual
  if (!converged)
    return set_error(DAMN_ERR_NOT_CONVERGED, "damn_cg_ir: relative residual %.3e after %d outer steps",
                     relres, outer);
  return DAMN_OK;
}
