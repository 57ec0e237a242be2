// Bandwidth reduction before the DA-CSR translation: reverse Cuthill-McKee
// ordering (host) and the symmetric permutation B = P A P^T (device).
//
// The paper reorders matrices that are not already bandwidth-reduced with RCM
// before translating them (Section 2, Example 2; Section 3), without fixing a
// start vertex, tie-break or treatment of disconnected graphs.  This library
// fixes one reading and documents it in include/damn.h:
//   * graph: pattern of A + A^T, self loops dropped, neighbours deduplicated;
//   * components in the order of their smallest vertex;
//   * start: George-Liu pseudo-peripheral search from the component's vertex
//     of minimum (degree, index), moving to the last BFS level's vertex of
//     minimum (degree, index) while the eccentricity strictly grows;
//   * Cuthill-McKee: a dequeued vertex appends its unvisited neighbours by
//     increasing (degree, index); the concatenated order is reversed.
//
// The ordering is a sequential breadth-first search (its result depends on
// the visit order at every step), so it runs on the host in O(nnz) per BFS.
// The permutation itself is data-parallel and runs on the device: inverse
// permutation with validation, new row lengths, a three-pass scan without
// inter-block waits, and one warp per new row that maps the columns and
// places every entry at its rank under (new column, stored position).
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "damn_common.cuh"

namespace damn {
namespace {

// ---------------------------------------------------------------------------
// host: symmetric graph and RCM
// ---------------------------------------------------------------------------

struct Graph {
  std::vector<int64_t> ptr;   // n + 1
  std::vector<int32_t> adj;   // neighbours, ascending, no duplicates, no self loops
  std::vector<int32_t> deg;   // distinct neighbours
};

void build_graph(int32_t n, const int32_t *rowptr, const int32_t *col, Graph &g) {
  std::vector<int64_t> cnt(static_cast<size_t>(n) + 1, 0);
  for (int32_t r = 0; r < n; ++r)
    for (int32_t i = rowptr[r]; i < rowptr[r + 1]; ++i) {
      const int32_t c = col[i];
      if (c == r) continue;
      ++cnt[r + 1];
      ++cnt[c + 1];
    }
  for (int32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
  std::vector<int32_t> raw(static_cast<size_t>(cnt[n]));
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int32_t r = 0; r < n; ++r)
    for (int32_t i = rowptr[r]; i < rowptr[r + 1]; ++i) {
      const int32_t c = col[i];
      if (c == r) continue;
      raw[fill[r]++] = c;
      raw[fill[c]++] = r;
    }
  g.ptr.assign(static_cast<size_t>(n) + 1, 0);
  g.deg.assign(n, 0);
  g.adj.clear();
  g.adj.reserve(raw.size());
  for (int32_t v = 0; v < n; ++v) {
    auto b = raw.begin() + cnt[v], e = raw.begin() + cnt[v + 1];
    std::sort(b, e);
    e = std::unique(b, e);
    g.adj.insert(g.adj.end(), b, e);
    g.ptr[v + 1] = static_cast<int64_t>(g.adj.size());
    g.deg[v] = static_cast<int32_t>(g.ptr[v + 1] - g.ptr[v]);
  }
}

// Breadth-first search with a visit stamp (no clearing between searches).
struct Bfs {
  const Graph &g;
  std::vector<int32_t> stamp, queue;
  int32_t cur = 0;
  explicit Bfs(const Graph &gr, int32_t n) : g(gr), stamp(n, 0) { queue.reserve(n); }

  // Level structure rooted at s: returns the number of levels; the vertices
  // of the last level are queue[last_begin, queue.size()).
  int32_t levels(int32_t s, size_t &last_begin) {
    ++cur;
    queue.clear();
    queue.push_back(s);
    stamp[s] = cur;
    size_t lb = 0, le = 1;
    int32_t nlev = 1;
    while (true) {
      for (size_t q = lb; q < le; ++q) {
        const int32_t v = queue[q];
        for (int64_t a = g.ptr[v]; a < g.ptr[v + 1]; ++a) {
          const int32_t u = g.adj[a];
          if (stamp[u] != cur) {
            stamp[u] = cur;
            queue.push_back(u);
          }
        }
      }
      if (queue.size() == le) break;
      lb = le;
      le = queue.size();
      ++nlev;
    }
    last_begin = lb;
    return nlev;
  }
};

inline bool deg_less(const Graph &g, int32_t a, int32_t b) {
  return g.deg[a] != g.deg[b] ? g.deg[a] < g.deg[b] : a < b;
}

int32_t min_deg_of(const Graph &g, const int32_t *v, size_t cnt) {
  int32_t best = v[0];
  for (size_t i = 1; i < cnt; ++i)
    if (deg_less(g, v[i], best)) best = v[i];
  return best;
}

int32_t pseudo_peripheral(const Graph &g, Bfs &bfs, int32_t start) {
  int32_t v = start;
  size_t lb = 0;
  int32_t nlev = bfs.levels(v, lb);
  while (true) {
    const int32_t u = min_deg_of(g, bfs.queue.data() + lb, bfs.queue.size() - lb);
    size_t lbu = 0;
    const int32_t nlu = bfs.levels(u, lbu);
    if (nlu > nlev) {
      v = u;
      nlev = nlu;
      lb = lbu;
    } else {
      return v;
    }
  }
}

void rcm(int32_t n, const Graph &g, int32_t *perm) {
  Bfs bfs(g, n);
  std::vector<char> visited(n, 0);
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<int32_t> nb;
  for (int32_t v0 = 0; v0 < n; ++v0) {
    if (visited[v0]) continue;
    size_t lb = 0;
    bfs.levels(v0, lb);  // the whole component of v0
    const int32_t s = min_deg_of(g, bfs.queue.data(), bfs.queue.size());
    const int32_t p = pseudo_peripheral(g, bfs, s);
    size_t head = order.size();
    order.push_back(p);
    visited[p] = 1;
    while (head < order.size()) {
      const int32_t v = order[head++];
      nb.clear();
      for (int64_t a = g.ptr[v]; a < g.ptr[v + 1]; ++a)
        if (!visited[g.adj[a]]) nb.push_back(g.adj[a]);
      std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) { return deg_less(g, a, b); });
      for (int32_t u : nb) {
        visited[u] = 1;
        order.push_back(u);
      }
    }
  }
  for (int32_t i = 0; i < n; ++i) perm[i] = order[n - 1 - i];
}

bool host_csr_ok(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col) {
  if (rowptr[0] != 0 || rowptr[n] != nnz) return false;
  for (int32_t r = 0; r < n; ++r)
    if (rowptr[r + 1] < rowptr[r]) return false;
  for (int64_t i = 0; i < nnz; ++i)
    if (col[i] < 0 || col[i] >= n) return false;
  return true;
}

int64_t host_bandwidth(int32_t n, const int32_t *rowptr, const int32_t *col, const int32_t *iperm) {
  int64_t w = 0;
  for (int32_t r = 0; r < n; ++r) {
    const int64_t rr = iperm ? iperm[r] : r;
    for (int32_t i = rowptr[r]; i < rowptr[r + 1]; ++i) {
      const int64_t c = iperm ? iperm[col[i]] : col[i];
      w = std::max(w, c > rr ? c - rr : rr - c);
    }
  }
  return w;
}

// ---------------------------------------------------------------------------
// device: B = P A P^T
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanBlock = kScanThreads * kScanPer;  // elements per scan block

// flag bits: 1 = perm not a permutation, 2 = bad column / row range in A
__global__ void k_iperm(int32_t n, const int32_t *__restrict__ perm, int32_t *__restrict__ iperm,
                        int *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = perm[i];
    if (p < 0 || p >= n)
      atomicOr(flag, 1);
    else
      iperm[p] = static_cast<int32_t>(i);
  }
}

// Checks iperm[perm[i]] == i (a repeated value of perm fails it for all but
// one of its positions) and writes the new row lengths to lens[i].
__global__ void k_lengths(int32_t n, const int32_t *__restrict__ rowptr,
                          const int32_t *__restrict__ perm, const int32_t *__restrict__ iperm,
                          int32_t *__restrict__ lens, int *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = perm[i];
    int32_t len = 0;
    if (p >= 0 && p < n) {
      if (iperm[p] != i) atomicOr(flag, 1);
      len = rowptr[p + 1] - rowptr[p];
      if (len < 0) {
        atomicOr(flag, 2);
        len = 0;
      }
    }
    lens[i] = len;
  }
}

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *total) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += t;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    int32_t s = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const int32_t before = (w > 0 ? warp_tot[w - 1] : 0) + inc - v;
  *total = warp_tot[kScanThreads / 32 - 1];
  __syncthreads();
  return before;
}

// Pass 1: inclusive scan of a[0..m) inside each block of kScanBlock
// elements; block totals to bsum.
__global__ void __launch_bounds__(kScanThreads) k_scan_local(int32_t m, int32_t *a, int32_t *bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanPer;
  int32_t v[kScanPer];
  int32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    v[j] = base + j < m ? a[base + j] : 0;
    s += v[j];
    v[j] = s;
  }
  int32_t total;
  const int32_t before = block_exclusive_scan(s, &total);
#pragma unroll
  for (int j = 0; j < kScanPer; ++j)
    if (base + j < m) a[base + j] = v[j] + before;
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Pass 2: exclusive scan of the block totals, one block walking chunks.
__global__ void __launch_bounds__(kScanThreads) k_scan_totals(int32_t nb, int32_t *bsum) {
  int32_t carry = 0;
  for (int32_t c0 = 0; c0 < nb; c0 += kScanThreads) {
    const int32_t i = c0 + threadIdx.x;
    const int32_t v = i < nb ? bsum[i] : 0;
    int32_t total;
    const int32_t before = block_exclusive_scan(v, &total);
    if (i < nb) bsum[i] = carry + before;
    carry += total;
  }
}

// Pass 3: add each block's offset; rowptr_out = [0, a...].
__global__ void k_scan_add(int32_t m, int32_t *a, const int32_t *bsum, int32_t *rowptr0) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) *rowptr0 = 0;
  if (i < m) a[i] += bsum[i / kScanBlock];
}

// One warp per new row i: entries of old row perm[i], column c -> iperm[c],
// each placed at its rank under (new column, stored position), computed by
// comparing against the row's keys 32 at a time through shuffles.
template <typename VT>
__global__ void k_fill(int32_t n, int64_t nnz, const int32_t *__restrict__ rowptr,
                       const int32_t *__restrict__ col, const VT *__restrict__ val,
                       const int32_t *__restrict__ perm, const int32_t *__restrict__ iperm,
                       const int32_t *__restrict__ rowptr_out, int32_t *__restrict__ col_out,
                       VT *__restrict__ val_out, int *flag, int *status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (*flag != 0 || rowptr_out[n] != nnz) {
    if (warp == 0 && lane == 0) {
      atomicOr(flag, 1);
      atomicCAS(status, DAMN_OK, DAMN_ERR_INVALID_ARG);
    }
    return;
  }
  for (int64_t i = warp; i < n; i += nwarps) {
    const int32_t p = perm[i];
    const int32_t b = rowptr[p];
    const int32_t len = rowptr[p + 1] - b;
    const int32_t ob = rowptr_out[i];
    for (int32_t jc = 0; jc < len; jc += 32) {
      const int32_t j = jc + lane;
      const bool has = j < len;
      int32_t key = INT_MAX;
      if (has) {
        const int32_t c = col[b + j];
        if (c >= 0 && c < n) {
          key = iperm[c];
        } else {
          atomicOr(flag, 2);
          atomicCAS(status, DAMN_OK, DAMN_ERR_INVALID_ARG);
        }
      }
      int32_t rank = 0;
      for (int32_t tc = 0; tc < len; tc += 32) {
        const int32_t t = tc + lane;
        int32_t kt = INT_MAX;
        if (tc == jc) {
          kt = key;
        } else if (t < len) {
          const int32_t c = col[b + t];
          kt = (c >= 0 && c < n) ? iperm[c] : INT_MAX;
        }
        const int lim = min(32, len - tc);
        for (int s = 0; s < lim; ++s) {
          const int32_t ks = __shfl_sync(0xffffffffu, kt, s);
          rank += (ks < key) | ((ks == key) & (tc + s < j));
        }
      }
      if (has) {
        col_out[ob + rank] = key;
        if (val) val_out[ob + rank] = val[b + j];
      }
    }
  }
}

inline size_t round_up256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

struct PermWs {
  int32_t *iperm, *bsum;
  int *flag;
};

size_t permute_ws_size(int32_t n) {
  const size_t nb = (static_cast<size_t>(n) + kScanBlock - 1) / kScanBlock + 1;
  return round_up256(sizeof(int32_t) * static_cast<size_t>(n)) + round_up256(sizeof(int32_t) * nb) +
         256;
}

PermWs carve_permute_ws(void *ws, int32_t n) {
  char *p = static_cast<char *>(ws);
  PermWs w;
  w.iperm = reinterpret_cast<int32_t *>(p);
  p += round_up256(sizeof(int32_t) * static_cast<size_t>(n));
  w.bsum = reinterpret_cast<int32_t *>(p);
  const size_t nb = (static_cast<size_t>(n) + kScanBlock - 1) / kScanBlock + 1;
  p += round_up256(sizeof(int32_t) * nb);
  w.flag = reinterpret_cast<int *>(p);
  return w;
}

template <typename VT>
int launch_fill(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col, const void *val,
                const int32_t *perm, const PermWs &w, const int32_t *rowptr_out, int32_t *col_out,
                void *val_out, int *status, cudaStream_t s) {
  const int threads = 256;
  const int64_t warps = std::max<int64_t>(1, n);
  const int blocks = static_cast<int>(
      std::min<int64_t>(32LL * sm_count(), (warps * 32 + threads - 1) / threads));
  k_fill<VT><<<blocks, threads, 0, s>>>(n, nnz, rowptr, col, static_cast<const VT *>(val), perm,
                                        w.iperm, rowptr_out, col_out, static_cast<VT *>(val_out),
                                        w.flag, status);
  DAMN_CHECK_LAUNCH("k_fill");
  return DAMN_OK;
}

int permute_sym(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col, const void *val,
                int dtype, const int32_t *perm, int32_t *rowptr_out, int32_t *col_out,
                void *val_out, void *workspace, cudaStream_t s) {
  const PermWs w = carve_permute_ws(workspace, n);
  int *status = device_status_ptr();
  if (!status) return set_error(DAMN_ERR_CUDA, "damn_permute_sym: no device status word");
  DAMN_CUDA(cudaMemsetAsync(w.flag, 0, sizeof(int), s));
  if (n == 0) {
    DAMN_CUDA(cudaMemsetAsync(rowptr_out, 0, sizeof(int32_t), s));
    return DAMN_OK;
  }
  const int threads = 256;
  const int blocks = static_cast<int>(
      std::min<int64_t>(8LL * sm_count(), ((int64_t)n + threads - 1) / threads));
  k_iperm<<<blocks, threads, 0, s>>>(n, perm, w.iperm, w.flag);
  DAMN_CHECK_LAUNCH("k_iperm");
  k_lengths<<<blocks, threads, 0, s>>>(n, rowptr, perm, w.iperm, rowptr_out + 1, w.flag);
  DAMN_CHECK_LAUNCH("k_lengths");
  const int32_t nb = static_cast<int32_t>(((int64_t)n + kScanBlock - 1) / kScanBlock);
  k_scan_local<<<nb, kScanThreads, 0, s>>>(n, rowptr_out + 1, w.bsum);
  DAMN_CHECK_LAUNCH("k_scan_local");
  k_scan_totals<<<1, kScanThreads, 0, s>>>(nb, w.bsum);
  DAMN_CHECK_LAUNCH("k_scan_totals");
  k_scan_add<<<static_cast<int>(((int64_t)n + 255) / 256), 256, 0, s>>>(n, rowptr_out + 1, w.bsum,
                                                                        rowptr_out);
  DAMN_CHECK_LAUNCH("k_scan_add");
  if (!val) dtype = DAMN_F32;  // pattern only: the value type is irrelevant
  switch (dtype) {
    case DAMN_F64:
      return launch_fill<unsigned long long>(n, nnz, rowptr, col, val, perm, w, rowptr_out,
                                             col_out, val_out, status, s);
    case DAMN_F32:
      return launch_fill<unsigned int>(n, nnz, rowptr, col, val, perm, w, rowptr_out, col_out,
                                       val_out, status, s);
    default:
      return launch_fill<unsigned short>(n, nnz, rowptr, col, val, perm, w, rowptr_out, col_out,
                                         val_out, status, s);
  }
}

}  // namespace
}  // namespace damn

using namespace damn;

extern "C" int damn_rcm_order(int32_t n, int64_t nnz, const int32_t *h_rowptr,
                              const int32_t *h_col, int32_t *h_perm, int64_t *h_w_before,
                              int64_t *h_w_after) {
  if (n < 0 || nnz < 0 || nnz > INT_MAX || !h_rowptr || !h_perm || (nnz > 0 && !h_col))
    return set_error(DAMN_ERR_INVALID_ARG, "damn_rcm_order: bad arguments");
  if (!host_csr_ok(n, nnz, h_rowptr, h_col))
    return set_error(DAMN_ERR_INVALID_ARG,
                     "damn_rcm_order: rowptr/col do not describe a square n x n CSR pattern");
  if (n == 0) {
    if (h_w_before) *h_w_before = 0;
    if (h_w_after) *h_w_after = 0;
    return DAMN_OK;
  }
  Graph g;
  build_graph(n, h_rowptr, h_col, g);
  rcm(n, g, h_perm);
  if (h_w_before) *h_w_before = host_bandwidth(n, h_rowptr, h_col, nullptr);
  if (h_w_after) {
    std::vector<int32_t> iperm(n);
    for (int32_t i = 0; i < n; ++i) iperm[h_perm[i]] = i;
    *h_w_after = host_bandwidth(n, h_rowptr, h_col, iperm.data());
  }
  return DAMN_OK;
}

extern "C" size_t damn_permute_sym_workspace_size(int32_t n) {
  return n < 0 ? 0 : permute_ws_size(n);
}

static int check_permute_args(const char *who, int32_t n, int64_t nnz, const int32_t *rowptr,
                              const int32_t *col, const void *val, int dtype,
                              const int32_t *rowptr_out, const int32_t *col_out,
                              const void *val_out, const void *workspace, size_t ws_bytes) {
  if (n < 0 || nnz < 0 || nnz > INT_MAX)
    return set_error(DAMN_ERR_INVALID_ARG, "%s: bad sizes n=%d nnz=%lld", who, n, (long long)nnz);
  if (!rowptr || !rowptr_out || !workspace || (nnz > 0 && (!col || !col_out)))
    return set_error(DAMN_ERR_INVALID_ARG, "%s: NULL pointer", who);
  if (val && (dtype < DAMN_F64 || dtype > DAMN_BF16 || (nnz > 0 && !val_out)))
    return set_error(DAMN_ERR_INVALID_ARG, "%s: bad value dtype / NULL val_out", who);
  if (ws_bytes < permute_ws_size(n))
    return set_error(DAMN_ERR_INVALID_ARG, "%s: workspace too small (%zu < %zu)", who, ws_bytes,
                     permute_ws_size(n));
  if (!aligned16(workspace)) return set_error(DAMN_ERR_INVALID_ARG, "%s: workspace not 16-byte aligned", who);
  return DAMN_OK;
}

extern "C" int damn_permute_sym(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                                const void *val, int dtype, const int32_t *perm,
                                int32_t *rowptr_out, int32_t *col_out, void *val_out,
                                void *workspace, size_t ws_bytes, void *stream) {
  int rc = check_permute_args("damn_permute_sym", n, nnz, rowptr, col, val, dtype, rowptr_out,
                              col_out, val_out, workspace, ws_bytes);
  if (rc) return rc;
  if (n > 0 && !perm) return set_error(DAMN_ERR_INVALID_ARG, "damn_permute_sym: perm is NULL");
  return permute_sym(n, nnz, rowptr, col, val, dtype, perm, rowptr_out, col_out, val_out,
                     workspace, static_cast<cudaStream_t>(stream));
}

extern "C" int damn_rcm_permute(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                                const void *val, int dtype, int32_t *perm_out,
                                int32_t *rowptr_out, int32_t *col_out, void *val_out,
                                damn_bw_info *h_info, void *workspace, size_t ws_bytes,
                                void *stream) {
  int rc = check_permute_args("damn_rcm_permute", n, nnz, rowptr, col, val, dtype, rowptr_out,
                              col_out, val_out, workspace, ws_bytes);
  if (rc) return rc;
  if (n > 0 && !perm_out) return set_error(DAMN_ERR_INVALID_ARG, "damn_rcm_permute: perm_out is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<int32_t> h_rowptr(static_cast<size_t>(n) + 1), h_col(static_cast<size_t>(nnz));
  std::vector<int32_t> h_perm(n);
  DAMN_CUDA(cudaMemcpyAsync(h_rowptr.data(), rowptr, sizeof(int32_t) * (n + 1),
                            cudaMemcpyDeviceToHost, s));
  if (nnz > 0)
    DAMN_CUDA(cudaMemcpyAsync(h_col.data(), col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  damn_bw_info info{0, 0};
  rc = damn_rcm_order(n, nnz, h_rowptr.data(), h_col.data(), h_perm.data(), &info.w_before,
                      &info.w_after);
  if (rc) return rc;
  if (n > 0)
    DAMN_CUDA(cudaMemcpyAsync(perm_out, h_perm.data(), sizeof(int32_t) * n,
                              cudaMemcpyHostToDevice, s));
  rc = permute_sym(n, nnz, rowptr, col, val, dtype, perm_out, rowptr_out, col_out, val_out,
                   workspace, s);
  if (rc) return rc;
  int flag = 0;
  const PermWs w = carve_permute_ws(workspace, n);
  DAMN_CUDA(cudaMemcpyAsync(&flag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DAMN_CUDA(cudaStreamSynchronize(s));
  if (flag) return set_error(DAMN_ERR_INVALID_ARG, "damn_rcm_permute: permutation check failed (%d)", flag);
  if (h_info) *h_info = info;
  return DAMN_OK;
}
