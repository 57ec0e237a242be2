// Host-side launch of the SpMV kernels for one (value type, index type):
// kernel configuration per plan shape, ring depth and grid size.  Included
// by the instantiation units spmv_inst_*.cu, one per (index format, value
// type), so that the many kernel variants compile in parallel.
#pragma once

#include <algorithm>
#include <mutex>

#include "damn_common.cuh"
#include "spmv_band.cuh"
#include "spmv_kernel.cuh"

namespace damn {
namespace spmvk {

constexpr int kMaxDev = 64;

// Occupancy of one kernel for every ring depth on one device, found once.
struct Occ {
  int known = 0;
  int max_optin = 0;
  int occ[kMaxStages + 1] = {};  // CTAs per SM at that depth (0: does not fit)
};

// Ring depth and CTAs per SM: the requested depth when it fits, else the
// deepest ring that keeps `minb` CTAs per SM (at least two stages).  Kernels
// whose consumer groups take turns on the tiles (band, sorted rows) need a
// depth that is a multiple of the number of groups `mult`: then stage s is
// only ever reused by the group that consumed it last, so a group waiting
// for a stage's next phase is never two phases behind it (a parity wait
// would otherwise take an older completed phase of the same parity for the
// one it wants).  A requested depth is rounded down to such a multiple.
template <class KFn, class TotalFn>
int pick_geometry(KFn kernel, int threads, TotalFn total, int minb, int req, Occ (&cache)[kMaxDev],
                  std::mutex &mu, int *stages, int *occ, int mult = 1) {
  int dev = 0;
  DAMN_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return set_error(DAMN_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lock(mu);
  Occ &c = cache[dev];
  if (!c.known) {
    DAMN_CUDA(cudaDeviceGetAttribute(&c.max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    DAMN_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c.max_optin));
    for (int st = 2; st <= kMaxStages; ++st) {
      c.occ[st] = 0;
      if (total(st) > (size_t)c.max_optin) continue;
      int o = 0;
      DAMN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, threads, total(st)));
      c.occ[st] = o;
    }
    c.known = 1;
  }
  const int lo = mult > 2 ? mult : 2;
  if (req > 0) req = req / mult * mult;
  if (req >= lo && req <= kMaxStages && c.occ[req] > 0) {
    *stages = req;
    *occ = c.occ[req];
    return DAMN_OK;
  }
  int best_s = lo, best_o = 0;
  for (int st = kMaxStages; st >= lo; --st) {
    if (st % mult) continue;
    if (c.occ[st] >= minb) { best_s = st; best_o = c.occ[st]; break; }
    if (c.occ[st] > best_o) { best_s = st; best_o = c.occ[st]; }
  }
  if (best_o == 0) return set_error(DAMN_ERR_UNSUPPORTED, "SpMV kernel does not fit this device");
  *stages = best_s;
  *occ = best_o;
  return DAMN_OK;
}

// Launches kernel<<<grid, threads, smem, s>>>(p) with programmatic stream
// serialisation: the kernel may begin launching while the previous kernel
// of the stream finishes; it waits for it (griddepcontrol.wait) before
// touching global memory.
template <class KFn>
int launch_pdl(KFn kernel, int grid, int threads, size_t smem, cudaStream_t s,
               const SpmvParams &p, const char *what) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, p);
  if (e != cudaSuccess) return cuda_error(e, what);
  return DAMN_OK;
}

template <bool PLAIN, typename V, typename I, class C, int NS>
int launch_kernel(SpmvParams p, cudaStream_t s, int *gs_out) {
  using L = Layout<V, I, C>;
  static Occ cache[2][kMaxDev];
  static std::mutex mu;
  const int mode = p.mode == 1 ? 1 : 0;
  int st = 2, occ = 1;
  int rc = pick_geometry(k_spmv<PLAIN, V, I, C, NS>, C::NT + 32,
                         [mode](int k) { return L::total(k, mode); }, C::MINB, p.stages_req,
                         cache[mode], mu, &st, &occ);
  if (rc) return rc;
  p.stages = st;
  const int grid = std::max(1, std::min(p.ntiles, occ * sm_count()));
  if (gs_out) { gs_out[0] = grid; gs_out[1] = p.stages; }
  if (p.ntiles == 0) return DAMN_OK;
  return launch_pdl(k_spmv<PLAIN, V, I, C, NS>, grid, C::NT + 32, L::total(p.stages, mode), s, p,
                    "k_spmv");
}

template <bool PLAIN, typename V, typename I, class C>
int launch_band(SpmvParams p, cudaStream_t s, int *gs_out) {
  using L = BandLayout<V, I, C>;
  static Occ cache[2][kMaxDev];
  static std::mutex mu;
  // no column ranges: no tile reads x through the ring, whose shared memory
  // is then left to the L1 cache
  const int ring = p.colrange ? 1 : 0;
  auto total = [ring](int k) { return L::total(k) - (ring ? size_t(0) : L::RING_BYTES); };
  // without the ring every x value is gathered through L1: unless a depth is
  // requested, one stage per consumer group, so that the shared memory saved
  // goes to the L1 cache rather than to a deeper ring of stages
  const int req = p.stages_req > 0 ? p.stages_req : (ring ? 0 : C::G);
  int st = 2, occ = 1;
  int rc = pick_geometry(k_spmv_band<PLAIN, V, I, C>, C::G * C::NT + 32, total, 1, req,
                         cache[ring], mu, &st, &occ, C::G);
  if (rc) return rc;
  p.stages = st;
  // one chunk of consecutive tiles per CTA; at least a few tiles per chunk
  const int grid = std::max(1, std::min(occ * sm_count(), (p.ntiles + 3) / 4));
  if (gs_out) { gs_out[0] = grid; gs_out[1] = p.stages; }
  if (p.ntiles == 0) return DAMN_OK;
  return launch_pdl(k_spmv_band<PLAIN, V, I, C>, grid, C::G * C::NT + 32, total(p.stages), s, p,
                    "k_spmv_band");
}

template <bool PLAIN, typename V, typename I, class C>
int launch_sorted(SpmvParams p, cudaStream_t s, int *gs_out) {
  using L = BandLayout<V, I, C>;
  static Occ cache[kMaxDev];
  static std::mutex mu;
  int st = 2, occ = 1;
  int rc = pick_geometry(k_spmv_sorted<PLAIN, V, I, C>, C::G * C::NT + 32,
                         [](int k) { return L::total(k); }, 1, p.stages_req, cache, mu, &st, &occ,
                         C::G);
  if (rc) return rc;
  p.stages = st;
  const int grid = std::max(1, std::min(occ * sm_count(), (p.ntiles + 3) / 4));
  if (gs_out) { gs_out[0] = grid; gs_out[1] = p.stages; }
  if (p.ntiles == 0) return DAMN_OK;
  return launch_pdl(k_spmv_sorted<PLAIN, V, I, C>, grid, C::G * C::NT + 32, L::total(p.stages),
                    s, p, "k_spmv_sorted");
}

inline bool is_plain(const SpmvParams &p) {
  return p.ab_mode == 0 && !p.dot_w && !p.dot_self && !p.dot_partials;
}

template <typename V, typename I, class C>
int launch_cfg(const SpmvParams &p, cudaStream_t s, int *gs) {
  const bool plain = is_plain(p);
  // rows without x windows: x read from global memory in the batched path
  if constexpr (C::E <= 2) {
    if (p.mode == 0 && !p.xseg) {
      if (plain) return launch_kernel<true, V, I, C, 0>(p, s, gs);
      return launch_kernel<false, V, I, C, 0>(p, s, gs);
    }
  }
  // one row per lane (or two lanes per row with narrow values) with every x
  // window of at most 3 segments: one compare fewer per entry in the column
  // -> slot map
  if constexpr (C::E == 1 || (C::E == 2 && sizeof(V) < 8)) {
    if (p.mode == 0 && p.max_nseg <= 3) {
      if (plain) return launch_kernel<true, V, I, C, 3>(p, s, gs);
      return launch_kernel<false, V, I, C, 3>(p, s, gs);
    }
  }
  if (plain) return launch_kernel<true, V, I, C, kXSegMax>(p, s, gs);
  return launch_kernel<false, V, I, C, kXSegMax>(p, s, gs);
}

template <typename V, typename I>
int launch_types(const SpmvParams &p, int shape, cudaStream_t s, int *gs) {
  using CB = std::conditional_t<sizeof(V) == 8, CfgBand64, CfgBand32>;
  using CS = std::conditional_t<sizeof(V) == 8, CfgSorted64, CfgSorted32>;
  switch (shape) {
    case kShapeSorted:
      return is_plain(p) ? launch_sorted<true, V, I, CS>(p, s, gs)
                         : launch_sorted<false, V, I, CS>(p, s, gs);
    case kShapeLong:
      if constexpr (sizeof(V) < 8)
        return launch_cfg<V, I, CfgLongNarrow>(p, s, gs);
      else
        return launch_cfg<V, I, CfgLong>(p, s, gs);
    case kShapeSlices: return launch_cfg<V, I, CfgSlices>(p, s, gs);
    case kShapeBand:
      return is_plain(p) ? launch_band<true, V, I, CB>(p, s, gs)
                         : launch_band<false, V, I, CB>(p, s, gs);
    case kShapeShortX2:
      if constexpr (sizeof(V) < 8)
        return launch_cfg<V, I, CfgShortNarrowX2>(p, s, gs);
      else
        return launch_cfg<V, I, CfgShortX2>(p, s, gs);
    case kShapeLanes4: return launch_cfg<V, I, CfgLanes4>(p, s, gs);
    case kShapeLanes8: return launch_cfg<V, I, CfgLanes8>(p, s, gs);
    case kShapeLanes16: return launch_cfg<V, I, CfgLanes16>(p, s, gs);
    case kShapeLanes32: return launch_cfg<V, I, CfgLanes32>(p, s, gs);
    default: break;
  }
  if constexpr (sizeof(V) < 8)
    return launch_cfg<V, I, CfgShortNarrow>(p, s, gs);
  else
    return launch_cfg<V, I, CfgShort>(p, s, gs);
}

}  // namespace spmvk
}  // namespace damn

// Defines the launcher of one (value type, index type) pair.
#define DAMN_SPMV_INSTANCE(NAME, V, I)                                                   \
  namespace damn {                                                                      \
  int NAME(const spmvk::SpmvParams &p, int shape, cudaStream_t s, int *gs) {            \
    return spmvk::launch_types<V, I>(p, shape, s, gs);                                  \
  }                                                                                     \
  }
