// C ABI of libprdf: graph handle, batch updates, partitions, frontier, and
// the Static / DF / DF-P drivers (Alg. static, Alg. frontier of
// arXiv 2404.08299). See include/prdf.h for the contract of each call.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"

namespace prdf {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int Workspace::init() {
  if (host_i64) return PRDF_OK;
  PRDF_CUDA(cudaMallocHost((void**)&host_i64, kHostSlots * sizeof(int64_t)));
  return PRDF_OK;
}

Workspace::~Workspace() {
  if (host_i64) cudaFreeHost(host_i64);
}

namespace {

constexpr int kThreads = 256;

// x[i] = R0[perm[i]] / |out(perm[i])| in the sweep numbering (R0 = NULL: 1/n)
__global__ void k_init_x(const double* __restrict__ R0, const int32_t* __restrict__ perm, int32_t n,
                         const double* __restrict__ inv, double* __restrict__ xa, double* __restrict__ xb) {
  const double r = 1.0 / (double)n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = (R0 ? R0[perm[i]] : r) * inv[i];
    xa[i] = x;
    if (xb) xb[i] = x;
  }
}

// Eq. 2 factor per vertex, 1 / (1 - alpha / |out(i)|)
__global__ void k_eq2_factor(const double* __restrict__ deg, int32_t n, double alpha, double* __restrict__ kf) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    kf[i] = 1.0 / (1.0 - alpha / deg[i]);
}

// FP32 stage set-up: y[i] = R0[perm[i]] / |out| (R0 = NULL: 1/n), rounded
// once from the FP64 quotient, into ya (and yb), FP32 degrees, and for DF-P
// the Eq. 2 factor (kf32 = NULL: not needed)
__global__ void k_init_y(const double* __restrict__ R0, const int32_t* __restrict__ perm, int32_t n,
                         const double* __restrict__ deg, const double* __restrict__ inv,
                         const double* __restrict__ kf, float* __restrict__ ya, float* __restrict__ yb,
                         float* __restrict__ degf, float* __restrict__ invf, float* __restrict__ kf32) {
  const double r = 1.0 / (double)n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float y = (float)((R0 ? R0[perm[i]] : r) * inv[i]);
    ya[i] = y;
    if (yb) yb[i] = y;
    degf[i] = (float)deg[i];
    invf[i] = (float)inv[i];
    if (kf32) kf32[i] = (float)kf[i];
  }
}

// FP64 stage start of Static: x = y (exact widening)
__global__ void k_widen(const float* __restrict__ y, int32_t n, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (double)y[i];
}

// FP64 stage start of DF / DF-P / DT: xa holds R^{t-1} / |out| in FP64. A
// vertex whose FP32 value still equals that start rounded to FP32 was not
// changed by the FP32 stage (never affected, or changed below FP32
// resolution) and keeps its FP64 value; the others take the widened FP32
// value and are affected again, so that the FP64 sweeps decide their
// prune test in FP64. Both buffers get the result (the copy-through of
// unaffected vertices relies on them being equal at the start of a loop).
__global__ void k_widen_keep(const float* __restrict__ y, int32_t n, double* __restrict__ xa, double* __restrict__ xb,
                             uint8_t* __restrict__ dV) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x0 = xa[i];
    const float yi = y[i];
    const bool same = (float)x0 == yi;
    const double x = same ? x0 : (double)yi;
    xa[i] = x;
    xb[i] = x;
    if (!same && !dV[i]) dV[i] = 1;
  }
}

// dst[i, :] = src[perm[i], :] for [n, K] row-major matrices
__global__ void k_rows_gather(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t n, int K,
                              double* __restrict__ dst) {
  const int64_t cnt = n * K;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / K, c = t - i * K;
    dst[t] = src[(int64_t)perm[i] * K + c];
  }
}

// dst[perm[i], :] = scale * src[i, :]
__global__ void k_rows_scatter(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t n, int K,
                               double* __restrict__ dst, double scale = 1.0) {
  const int64_t cnt = n * K;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / K, c = t - i * K;
    dst[(int64_t)perm[i] * K + c] = scale * src[t];
  }
}

// dst[i, :] = scale * src[perm[i], :]
__global__ void k_rows_gather_scaled(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t n,
                                     int K, double scale, double* __restrict__ dst) {
  const int64_t cnt = n * K;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / K, c = t - i * K;
    dst[t] = scale * src[(int64_t)perm[i] * K + c];
  }
}

// in-CSR weights from out-CSR weights: slot (u -> v) of row u holds w; find u in in-row v
__global__ void k_weights_to_in(const int64_t* __restrict__ ooff, const int32_t* __restrict__ oadj,
                                const float* __restrict__ w, int32_t n, const int64_t* __restrict__ ioff,
                                const int32_t* __restrict__ iadj, float* __restrict__ win, int* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int flag = 0;
  for (int64_t u = warp; u < n; u += nwarps) {
    for (int64_t j = ooff[u] + lane; j < ooff[u + 1]; j += 32) {
      const float x = w[j];
      if (!(x > 0.f) || !isfinite(x)) flag = 1;
      const int32_t v = oadj[j];
      int64_t lo = ioff[v], hi = ioff[v + 1];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (iadj[mid] < (int32_t)u) lo = mid + 1; else hi = mid;
      }
      win[lo] = x;  // (v, u) is in G' because (u, v) is in G
    }
  }
  flag = __reduce_or_sync(0xffffffffu, flag);
  if (lane == 0 && flag) atomicOr(bad, 1);
}

// R[perm[i]] = x[i] * |out(perm[i])|; dV_out[perm[i]] = dV[i]
__global__ void k_finalize(const double* __restrict__ x, const double* __restrict__ deg,
                           const int32_t* __restrict__ perm, int32_t n, double* __restrict__ R,
                           const uint8_t* __restrict__ dV, uint8_t* __restrict__ dV_out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = perm[i];
    R[v] = x[i] * deg[i];
    if (dV_out) dV_out[v] = dV[i];
  }
}

__global__ void k_check_ids(const int32_t* a, const int32_t* b, int64_t cnt, int32_t n, unsigned long long* bad) {
  int f = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    if (a && (a[i] < 0 || a[i] >= n)) f = 1;
    if (b && (b[i] < 0 || b[i] >= n)) f = 1;
  }
  f = __reduce_or_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0 && f) atomicOr(bad, 1ull);
}

// Start-vector check: bad[1] |= 1 for an entry that is negative, NaN or infinite;
// *sum accumulates the entries (one FP64 atomic per block).
__global__ void k_check_ranks(const double* __restrict__ R, int64_t n, unsigned long long* bad, double* sum) {
  __shared__ double sh[32];
  double acc = 0;
  int f = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = R[i];
    if (!(x >= 0.0) || !isfinite(x)) f = 1;
    else acc += x;
  }
  f = __reduce_or_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0 && f) atomicOr(bad + 1, 1ull);
  acc = warp_sum_f64(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum_f64(t);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(sum, t);
  }
}

// position of (u, v) in a sorted CSR row, or -1
__device__ __forceinline__ int64_t find_edge(const int64_t* off, const int32_t* adj, int32_t u, int32_t v) {
  int64_t lo = off[u], hi = off[u + 1];
  const int64_t e = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (adj[mid] < v) lo = mid + 1; else hi = mid;
  }
  return (lo < e && adj[lo] == v) ? lo : -1;
}

__global__ void k_mark_deleted(const int32_t* __restrict__ ds, const int32_t* __restrict__ dd, int64_t n_del,
                               const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                               uint8_t* __restrict__ deleted) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_del; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = ds[i], v = dd[i];
    if (u == v) continue;  // self-loops are never deleted
    const int64_t p = find_edge(off, adj, u, v);
    if (p >= 0) deleted[p] = 1;
  }
}

// edge list of the surviving old edges (deleted slots get row -1) followed by the insertions
__global__ void k_old_edges(int32_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            const float* __restrict__ w, const uint8_t* __restrict__ deleted,
                            int32_t* __restrict__ rows, int32_t* __restrict__ cols, float* __restrict__ wo) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nw) {
    for (int64_t j = off[u] + lane; j < off[u + 1]; j += 32) {
      rows[j] = deleted[j] ? -1 : (int32_t)u;
      cols[j] = adj[j];
      if (wo) wo[j] = w[j];
    }
  }
}

__global__ void k_append(const int32_t* __restrict__ is, const int32_t* __restrict__ id, const float* __restrict__ iw,
                         int64_t n_ins, int64_t at, int32_t* __restrict__ rows, int32_t* __restrict__ cols,
                         float* __restrict__ wo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_ins; i += (int64_t)gridDim.x * blockDim.x) {
    rows[at + i] = is[i];
    cols[at + i] = id[i];
    if (wo) wo[at + i] = iw[i];
  }
}

__global__ void k_effective(const int32_t* __restrict__ s, const int32_t* __restrict__ d, int64_t cnt, int deletion,
                            const int64_t* __restrict__ o_off, const int32_t* __restrict__ o_adj,
                            const int64_t* __restrict__ n_off, const int32_t* __restrict__ n_adj,
                            uint8_t* __restrict__ eff) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const bool in_old = find_edge(o_off, o_adj, s[i], d[i]) >= 0;
    const bool in_new = find_edge(n_off, n_adj, s[i], d[i]) >= 0;
    eff[i] = deletion ? (in_old && !in_new) : (!in_old && in_new);
  }
}

// ids of a batch list in the sweep numbering: out[i] = inv[a[i]]
__global__ void k_map_ids(const int32_t* __restrict__ a, int64_t cnt, const int32_t* __restrict__ inv,
                          int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = inv[a[i]];
}

// position of (u, v) (original ids) in a CSR of the sweep numbering, whose row inv[u] lists renumbered ids in
// original-id order, or -1
__device__ __forceinline__ int64_t find_edge_keyed(const int64_t* off, const int32_t* adj, const int32_t* perm,
                                                   const int32_t* inv, int32_t u, int32_t v) {
  const int32_t r = inv[u];
  int64_t lo = off[r], hi = off[r + 1];
  const int64_t e = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (perm[adj[mid]] < v) lo = mid + 1; else hi = mid;
  }
  return (lo < e && perm[adj[lo]] == v) ? lo : -1;
}

__global__ void k_effective_keyed(const int32_t* __restrict__ s, const int32_t* __restrict__ d, int64_t cnt,
                                  int deletion, const int32_t* __restrict__ perm, const int32_t* __restrict__ inv,
                                  const int64_t* __restrict__ o_off, const int32_t* __restrict__ o_adj,
                                  const int64_t* __restrict__ n_off, const int32_t* __restrict__ n_adj,
                                  uint8_t* __restrict__ eff) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const bool in_old = find_edge_keyed(o_off, o_adj, perm, inv, s[i], d[i]) >= 0;
    const bool in_new = find_edge_keyed(n_off, n_adj, perm, inv, s[i], d[i]) >= 0;
    eff[i] = deletion ? (in_old && !in_new) : (!in_old && in_new);
  }
}

// Vertices of the in-degree <= 1 classes (the sweep numbering's ids [0, end1))
// that receive an in-edge: their bit of multi is set, and the number of bits
// newly set is added to *count.
__global__ void k_mark_multi(const int32_t* __restrict__ ins_dst, int64_t cnt, const int32_t* __restrict__ inv,
                             int64_t end1, uint32_t* __restrict__ multi, unsigned long long* __restrict__ count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = inv[ins_dst[i]];
    if (r >= end1) continue;
    const uint32_t bit = 1u << (r & 31);
    if (!(atomicOr(multi + (r >> 5), bit) & bit)) atomicAdd(count, 1ull);
  }
}

int check_params(const prdf_params* p) {
  if (!p) {
    set_error("params is NULL");
    return PRDF_EINVAL;
  }
  if (!(p->alpha > 0.0 && p->alpha < 1.0)) {
    set_error("alpha must be in (0, 1)");
    return PRDF_EINVAL;
  }
  if (!(p->tol > 0.0) || std::isnan(p->tol)) {
    set_error("tol must be > 0");
    return PRDF_EINVAL;
  }
  if (p->max_iter < 1) {
    set_error("max_iter must be >= 1");
    return PRDF_EINVAL;
  }
  if (std::isnan(p->tau_f) || std::isnan(p->tau_p)) {
    set_error("tau_f / tau_p must not be NaN");
    return PRDF_EINVAL;
  }
  if (!(p->expand_pull >= 0.0)) {
    set_error("expand_pull must be >= 0");
    return PRDF_EINVAL;
  }
  if (p->expand_list < -1) {
    set_error("expand_list must be >= -1");
    return PRDF_EINVAL;
  }
  if (p->precision != PRDF_FP64 && p->precision != PRDF_FP32_REFINE) {
    set_error("unknown precision %d", p->precision);
    return PRDF_EINVAL;
  }
  if (p->accumulate != PRDF_ACC_EXACT && p->accumulate != PRDF_ACC_FP64) {
    set_error("unknown accumulate mode %d", p->accumulate);
    return PRDF_EINVAL;
  }
  return PRDF_OK;
}

int ensure_partition(prdf_graph* g, int which, cudaStream_t s) {
  PRDF_TRY(ensure_orig(g, s));
  if (g->pvalid[which]) return PRDF_OK;
  PRDF_TRY(g->P[which].reserve(g->n, s));
  PRDF_TRY(partition_by_degree(g->csr[which].off.p, g->n, g->thr[which], g->P[which].p, g->pcount[which], g->ws, s));
  g->pvalid[which] = true;
  return PRDF_OK;
}

int ensure_relabelled(prdf_graph* g, bool need_pout, cudaStream_t s) {
  Relabel& r = g->rl;
  bool same = r.valid && r.thr.n == g->thr[PRDF_IN].n;
  for (int i = 0; same && i < r.thr.n; ++i) same = r.thr.thr[i] == g->thr[PRDF_IN].thr[i];
  if (!same) PRDF_TRY(build_relabelled(g, s));
  if (need_pout && !r.pout_valid) {
    PRDF_TRY(r.pout.reserve(g->n, s));
    PRDF_TRY(partition_by_degree(r.out.off.p, g->n, g->thr[PRDF_OUT], r.pout.p, r.pout_count, g->ws, s));
    r.pout_valid = true;
  }
  return PRDF_OK;
}

void begins_from_counts(const int64_t* count, int C, int64_t* cb) {
  cb[0] = 0;
  for (int c = 0; c < C; ++c) cb[c + 1] = cb[c] + count[c];
}

void class_begins(const prdf_graph* g, int which, int64_t* cb) {
  const int C = g->thr[which].n + 1;
  cb[0] = 0;
  for (int c = 0; c < C; ++c) cb[c + 1] = cb[c] + g->pcount[which][c];
}

// Largest sum of a start vector the sweeps accept. The exact accumulator
// holds in-neighbour sums below 16, and an in-neighbour sum never exceeds the
// sum of all ranks (Eq. 1 keeps that sum near 1); a PageRank vector sums to 1.
constexpr double kMaxRankSum = 4.0;

// Check caller inputs with one device pass and one host synchronisation:
// the ids of (a, b)[0, na) and (c, d)[0, nc) in [0, n) (NULL arrays skipped),
// and a start vector R (NULL: none) with finite, non-negative entries that
// sum to at most kMaxRankSum. what names the vector in the message.
int check_inputs(prdf_graph* g, const int32_t* a, const int32_t* b, int64_t na, const int32_t* c, const int32_t* d,
                 int64_t nc, const double* R, const char* what, cudaStream_t s) {
  const bool ids1 = na > 0 && (a || b), ids2 = nc > 0 && (c || d);
  if (!ids1 && !ids2 && !R) return PRDF_OK;
  PRDF_TRY(g->chk.reserve(4, s));
  PRDF_CUDA(cudaMemsetAsync(g->chk.p, 0, 4 * sizeof(unsigned long long), s));
  if (ids1) k_check_ids<<<grid_for(na, kThreads), kThreads, 0, s>>>(a, b, na, g->n, g->chk.p);
  if (ids2) k_check_ids<<<grid_for(nc, kThreads), kThreads, 0, s>>>(c, d, nc, g->n, g->chk.p);
  if (R)
    k_check_ranks<<<grid_for(g->n, kThreads, kSMs * 4), kThreads, 0, s>>>(R, g->n, g->chk.p,
                                                                          reinterpret_cast<double*>(g->chk.p + 2));
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64, g->chk.p, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  const int64_t* h = g->ws.host_i64;
  if (h[0]) {
    set_error("vertex id outside [0, %d)", g->n);
    return PRDF_EINVAL;
  }
  if (R) {
    double sum;
    memcpy(&sum, &h[2], sizeof(double));
    if (h[1]) {
      set_error("%s: entries must be finite and >= 0", what);
      return PRDF_EINVAL;
    }
    if (!(sum <= kMaxRankSum)) {
      set_error("%s: entries sum to %g, above %g", what, sum, kMaxRankSum);
      return PRDF_EINVAL;
    }
  }
  return PRDF_OK;
}


struct Timer {
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  ~Timer() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
  int init() {
    for (auto& x : e) PRDF_CUDA(cudaEventCreate(&x));
    return PRDF_OK;
  }
};

struct IterResult {
  int iters = 0;          // sweeps up to and including the first converged one (or max_iter)
  int converged = 0;
  double final_delta = 0; // FP64 loop: L-inf change of the last sweep; FP32 stage: max |dR| of it
  int final_buf = 0;      // 0: xa (ya) holds the result, 1: xb (yb)
  int launched = 0;       // sweeps issued
  float ms_sweep = 0;     // device time of the first `iters` sweeps (time_sweeps)
  long long kernels = 0;  // kernels launched
};

int nonempty_classes(const int64_t* cb, int nclass) {
  int k = 0;
  for (int c = 0; c < nclass; ++c) k += cb[c + 1] > cb[c] ? 1 : 0;
  return k;
}

int ensure_hub(prdf_graph* g, const Csr& c, PprHubTable& t, cudaStream_t s);
int64_t hub_begin(const Relabel& rl);

// ----------------------------------------------------------- the loop ----
// One loop of synchronous sweeps, Alg. static (every vertex, Eq. 1) or
// Alg. frontier / Alg. traversal (affected vertices, Eq. 1 or Eq. 2, with an
// expansion round of Alg. affected after each sweep when `expand`), in FP64
// or as the FP32 stage of the mixed-precision solve. It runs until the stop
// rule holds for a sweep or max_iter sweeps ran: FP64, L-inf change <= tol;
// FP32, max|dR| <= tol_rel * max R.
//
// Two drivers run the same kernels:
//   - host loop: check_every sweeps are launched ahead and one residual is
//     read; sweeps launched past convergence exit at once on the device.
//     With time_sweeps each sweep is bracketed by CUDA events.
//   - CUDA graph: a while node whose body is one iteration (sweep, expansion)
//     and a one-thread check that advances the device iteration counter; the
//     kernels find their buffers from that counter. One launch per loop, no
//     host round trips. The instantiated graph is cached on the graph handle
//     and rebuilt when any buffer, numbering or parameter it holds changes.
struct Loop {
  bool fp32 = false, dynamic = false, expand = false, exact = true;
  int max_iter = 0;
  double tol = 0;
  float tol_rel = 0;
  SweepArgs a;      // FP64 sweep arguments (per-iteration buffers filled per launch)
  Sweep32Args a32;  // FP32 sweep arguments
  int64_t cb[kMaxThr + 2] = {}, cbo[kMaxThr + 2] = {};
  int nci = 0, nco = 0;
  int64_t pull_warp_b = 0;
  unsigned long long fthr = ~0ull;
  FrontList fl;              // listed small frontiers
  int kernels_per_iter = 0;  // kernels of one iteration (without the graph's check)
};

// An expansion round lists a frontier of at most cap vertices and expands it
// from the list (frontier.cu); larger ones take the partition kernels. The
// automatic cap is min(32768, n / 8) on graphs of at least 2^22 vertices; on
// smaller ones the partition kernels' scan costs less than the list's extra
// launches, so the list is off (cap 0: fl left empty).
int front_list(prdf_graph* g, const prdf_params* p, cudaStream_t s, FrontList* fl) {
  int64_t cap = p->expand_list;
  if (cap < 0) cap = g->n >= (1 << 22) ? (g->n / 8 < 32768 ? g->n / 8 : 32768) : 0;
  if (cap > g->n) cap = g->n;
  *fl = FrontList();
  if (cap == 0) return PRDF_OK;
  PRDF_TRY(g->flist.reserve((size_t)cap, s));
  PRDF_TRY(g->fcnt.reserve(1, s));
  fl->list = g->flist.p;
  fl->cnt = g->fcnt.p;
  fl->cap = (unsigned int)cap;
  return PRDF_OK;
}

int loop_setup(prdf_graph* g, const prdf_params* p, bool fp32, bool dynamic, bool expand, int max_iter, Loop* L,
               cudaStream_t s) {
  const int n = g->n;
  const Relabel& rl = g->rl;
  L->fp32 = fp32;
  L->dynamic = dynamic;
  L->expand = dynamic && expand;
  L->exact = p->accumulate == PRDF_ACC_EXACT;
  L->max_iter = max_iter;
  L->tol = p->tol;
  L->tol_rel = (float)p->tol_fp32_rel;
  L->nci = rl.thr.n + 1;
  begins_from_counts(rl.count, L->nci, L->cb);
  L->kernels_per_iter = nonempty_classes(L->cb, L->nci);
  // the highest in-degree class's rows are cut into the hub chunks of G' (a
  // partial sum per chunk); the table and the partial buffer are made here,
  // outside any stream capture
  PRDF_TRY(ensure_hub(g, rl.in, g->hub_in, s));
  const size_t nchunk = (size_t)(g->hub_in.nchunk > 0 ? g->hub_in.nchunk : 1);
  if (g->hub_in.nchunk > 0) L->kernels_per_iter += 1;  // the highest class takes two kernels
  if (fp32) {
    PRDF_TRY(g->sweep_hub_part32.reserve(nchunk, s));
    PRDF_TRY(g->resid32.reserve(2 * ((size_t)max_iter + 1), s));
    PRDF_CUDA(cudaMemsetAsync(g->resid32.p, 0, sizeof(uint32_t) * 2 * ((size_t)max_iter + 1), s));
    Sweep32Args& a = L->a32;
    memset(&a, 0, sizeof(a));
    a.off = rl.in.off.p;
    a.adj = rl.in.adj.p;
    a.degf = g->degf.p;
    a.invf = g->invf.p;
    a.alpha = (float)p->alpha;
    a.c0 = (float)((1.0 - p->alpha) / (double)n);
    a.self_loops = g->self_loops ? 1 : 0;
    a.tol_rel = L->tol_rel;
    a.multi = rl.multi_count > 0 ? rl.multi.p : nullptr;
    a.hub = g->hub_in.view();
    a.hub_part = g->sweep_hub_part32.p;
    if (dynamic) {
      a.kf = g->kf32.p;
      a.dV = g->dV.p;
      a.dN = g->dN.p;
      a.wrote = g->wrote.p;
      a.tau_f = (float)p->tau_f;
      a.tau_p = (float)p->tau_p;
      a.prune = p->prune;
    }
  } else {
    PRDF_TRY(g->sweep_hub_part.reserve(nchunk, s));
    PRDF_TRY(g->resid.reserve((size_t)max_iter + 1, s));
    PRDF_CUDA(cudaMemsetAsync(g->resid.p, 0, sizeof(uint64_t) * ((size_t)max_iter + 1), s));
    SweepArgs& a = L->a;
    memset(&a, 0, sizeof(a));
    a.off = rl.in.off.p;
    a.adj = rl.in.adj.p;
    a.degd = rl.degd.p;
    a.inv_deg = rl.inv_deg.p;
    a.kf = rl.kf.p;
    a.alpha = p->alpha;
    a.c0 = (1.0 - p->alpha) / (double)n;
    a.self_loops = g->self_loops ? 1 : 0;
    a.tol = p->tol;
    a.multi = rl.multi_count > 0 ? rl.multi.p : nullptr;
    a.hub = g->hub_in.view();
    a.hub_part = g->sweep_hub_part.p;
    if (dynamic) {
      a.dV = g->dV.p;
      a.dN = g->dN.p;
      a.wrote = g->wrote.p;
      // + 0.0 turns a tolerance of -0 into +0: the sweep compares products with
      // the tolerance by their bit patterns, which order -0 below +0
      a.tau_f = p->tau_f + 0.0;
      a.tau_p = p->tau_p + 0.0;
      a.prune = p->prune;
    }
  }
  if (L->expand) {
    // pull-form expansion: frontier count, thread rows below the two highest in-degree classes, warp rows above
    L->nco = g->thr[PRDF_OUT].n + 1;
    begins_from_counts(rl.pout_count, L->nco, L->cbo);
    L->pull_warp_b = hub_begin(rl);
    PRDF_TRY(g->fwork.reserve((size_t)max_iter + 1, s));
    PRDF_CUDA(cudaMemsetAsync(g->fwork.p, 0, sizeof(unsigned long long) * ((size_t)max_iter + 1), s));
    const double lim = p->expand_pull * (double)rl.in.m;
    L->fthr = lim >= 1.8e19 ? ~0ull : (unsigned long long)lim;
    PRDF_TRY(front_list(g, p, s, &L->fl));  // allocated here, outside any stream capture
    L->kernels_per_iter += nonempty_classes(L->cbo, L->nco) + (L->pull_warp_b > 0 ? 1 : 0) +
                           (n > L->pull_warp_b ? 1 : 0) + (L->fl.list ? 2 : 0);
  }
  return PRDF_OK;
}

// The sweep of iteration i (i >= 0: host loop, explicit buffers; i < 0:
// graph-driven, buffers from the device counter).
int launch_loop_sweep(prdf_graph* g, const Loop& L, int i, cudaStream_t s) {
  const Relabel& rl = g->rl;
  if (L.fp32) {
    Sweep32Args a = L.a32;
    // the sweep counts the out-edges of its deltaN for the expansion round after it
    if (i >= 0) {
      a.y = (i & 1) ? g->yb.p : g->ya.p;
      a.yn = (i & 1) ? g->ya.p : g->yb.p;
      a.resid = g->resid32.p + 2 * i;
      a.prev = i > 0 ? g->resid32.p + 2 * (i - 1) : nullptr;
      a.fw = L.expand ? g->fwork.p + i : nullptr;
    } else {
      a.ctl = g->ctl.p;
      a.ya = g->ya.p;
      a.yb = g->yb.p;
      a.resid_base = g->resid32.p;
      a.fw_base = L.expand ? g->fwork.p : nullptr;
    }
    return launch_sweep32(a, rl.thr, L.cb, L.dynamic, s);
  }
  SweepArgs a = L.a;
  if (i >= 0) {
    a.x = (i & 1) ? g->xb.p : g->xa.p;
    a.xn = (i & 1) ? g->xa.p : g->xb.p;
    a.resid = g->resid.p + i;
    a.prev = i > 0 ? g->resid.p + i - 1 : nullptr;
    a.fw = L.expand ? g->fwork.p + i : nullptr;
  } else {
    a.ctl = g->ctl.p;
    a.xa = g->xa.p;
    a.xb = g->xb.p;
    a.resid_base = g->resid.p;
    a.fw_base = L.expand ? g->fwork.p : nullptr;
  }
  return launch_sweep(a, rl.thr, L.cb, L.exact, L.dynamic, s);
}

// The expansion round after sweep i (Alg. affected over the frontier deltaN
// the sweep left), skipped on the device once the loop has converged.
int launch_loop_expansion(prdf_graph* g, const Loop& L, int i, cudaStream_t s) {
  if (!L.expand) return PRDF_OK;
  const Relabel& rl = g->rl;
  Stop st;
  if (L.fp32) {
    st.r32 = g->resid32.p + 2 * (i >= 0 ? i : 0);
    st.tol_rel = L.tol_rel;
  } else {
    st.r64 = g->resid.p + (i >= 0 ? i : 0);
    st.tol = L.tol;
  }
  st.ctl = i >= 0 ? nullptr : g->ctl.p;
  unsigned long long* fw = g->fwork.p + (i >= 0 ? i : 0);
  PRDF_TRY(launch_expand_pull(rl.in.off.p, rl.in.adj.p, g->n, L.pull_warp_b, g->dN.p, g->dV.p, fw, L.fthr, st, s));
  return launch_expand(rl.out.off.p, rl.out.adj.p, rl.pout.p, L.cbo, L.nco, g->dN.p, g->dV.p, nullptr, st, s, fw,
                       L.fthr, L.fl);
}

// stop rule of sweep i from the residual words read back
bool loop_stopped(const Loop& L, const void* words, int i, double* delta) {
  if (L.fp32) {
    const uint32_t* r = static_cast<const uint32_t*>(words) + 2 * i;
    float d, m;
    memcpy(&d, &r[0], 4);
    memcpy(&m, &r[1], 4);
    *delta = d;
    return d <= L.tol_rel * m;
  }
  double d;
  memcpy(&d, static_cast<const uint64_t*>(words) + i, sizeof(double));
  *delta = d;
  return d <= L.tol;
}

int run_host_loop(prdf_graph* g, const Loop& L, const prdf_params* p, IterResult* res, cudaStream_t s) {
  const int max_iter = L.max_iter;
  const int check = p->check_every > 0 ? p->check_every : 8;
  const bool timed = p->time_sweeps != 0;
  const size_t wsz = L.fp32 ? 2 * sizeof(uint32_t) : sizeof(uint64_t);
  const void* resid_dev = L.fp32 ? (const void*)g->resid32.p : (const void*)g->resid.p;
  std::vector<cudaEvent_t> ev;
  struct EvGuard {
    std::vector<cudaEvent_t>& v;
    ~EvGuard() {
      for (auto e : v) cudaEventDestroy(e);
    }
  } guard{ev};
  int launched = 0;
  bool done = false;
  while (launched < max_iter && !done) {
    const int upto = (launched + check < max_iter) ? launched + check : max_iter;
    for (int i = launched; i < upto; ++i) {
      if (timed) {
        cudaEvent_t e0, e1;
        PRDF_CUDA(cudaEventCreate(&e0));
        ev.push_back(e0);
        PRDF_CUDA(cudaEventCreate(&e1));
        ev.push_back(e1);
        PRDF_CUDA(cudaEventRecord(e0, s));
      }
      PRDF_TRY(launch_loop_sweep(g, L, i, s));
      if (timed) PRDF_CUDA(cudaEventRecord(ev.back(), s));  // the sweep alone, not its expansion
      PRDF_TRY(launch_loop_expansion(g, L, i, s));
    }
    launched = upto;
    PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64, (const char*)resid_dev + wsz * (launched - 1), wsz,
                              cudaMemcpyDeviceToHost, s));
    PRDF_CUDA(cudaStreamSynchronize(s));
    double d;
    done = loop_stopped(L, g->ws.host_i64, 0, &d);
  }
  std::vector<uint64_t> hr((size_t)launched);
  PRDF_CUDA(cudaMemcpyAsync(hr.data(), resid_dev, wsz * launched, cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  int k = launched - 1;
  res->converged = 0;
  for (int i = 0; i < launched; ++i) {
    double d;
    if (loop_stopped(L, hr.data(), i, &d)) {
      k = i;
      res->converged = 1;
      break;
    }
  }
  loop_stopped(L, hr.data(), k, &res->final_delta);
  res->iters = k + 1;
  res->final_buf = (k & 1) ? 0 : 1;  // sweep k wrote the second buffer if k is even
  res->launched = launched;
  res->kernels = (long long)launched * L.kernels_per_iter;
  res->ms_sweep = 0;
  if (timed)
    for (int i = 0; i < res->iters; ++i) {
      float ms = 0;
      PRDF_CUDA(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
      res->ms_sweep += ms;
    }
  return PRDF_OK;
}

// Launch on s the cached while-loop graph of `slot`, first building it when
// it was made for another key: a conditional while node whose body is
// recorded by body(capture stream, conditional handle) (the body ends with a
// one-thread check that sets the condition).
template <class Body>
int launch_while_graph(prdf_graph* g, int slot, const std::vector<uint64_t>& key, Body body, cudaStream_t s) {
  if (!g->loop_exec[slot] || g->loop_key[slot] != key) {
    if (g->loop_exec[slot]) {
      cudaGraphExecDestroy(g->loop_exec[slot]);
      g->loop_exec[slot] = nullptr;
    }
    if (!g->cap_stream) PRDF_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    PRDF_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    alignas(cudaGraphNodeParams) unsigned char np_storage[sizeof(cudaGraphNodeParams)];
    memset(np_storage, 0, sizeof(np_storage));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_storage);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    cudaGraph_t bodyg = e == cudaSuccess ? np.conditional.phGraph_out[0] : nullptr;
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(g->cap_stream, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    int rc = PRDF_OK;
    if (e == cudaSuccess) {
      rc = body(g->cap_stream, h);
      cudaGraph_t captured = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &captured);
      if (e == cudaSuccess) e = e2;
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && rc == PRDF_OK) e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (rc != PRDF_OK) return rc;
    if (e != cudaSuccess) {
      set_error("building the iteration graph: %s", cudaGetErrorString(e));
      return PRDF_ECUDA;
    }
    g->loop_exec[slot] = exec;
    g->loop_key[slot] = key;
  }
  PRDF_CUDA(cudaGraphLaunch(g->loop_exec[slot], s));
  return PRDF_OK;
}

// key words of a graph: the raw bytes of the values it was captured with
struct KeyWriter {
  std::vector<uint64_t> key;
  void put(const void* p, size_t nb) {
    const size_t at = key.size();
    key.resize(at + (nb + 7) / 8, 0);
    memcpy(key.data() + at, p, nb);
  }
  void putv(uint64_t v) { put(&v, sizeof(v)); }
};

// The same loop as one CUDA graph (see above).
int run_graph_loop(prdf_graph* g, const Loop& L, IterResult* res, cudaStream_t s) {
  PRDF_TRY(g->ctl.reserve(2, s));
  PRDF_CUDA(cudaMemsetAsync(g->ctl.p, 0, 2 * sizeof(int), s));
  // what the captured kernels hold: their arguments and the buffers of the graph-driven iteration
  KeyWriter kw;
  kw.putv(((uint64_t)L.fp32 << 3) | ((uint64_t)L.dynamic << 2) | ((uint64_t)L.expand << 1) | (uint64_t)L.exact);
  kw.putv((uint64_t)L.max_iter);
  kw.put(&L.tol, sizeof(L.tol));
  kw.put(&L.tol_rel, sizeof(L.tol_rel));
  if (L.fp32) kw.put(&L.a32, sizeof(L.a32));
  else kw.put(&L.a, sizeof(L.a));
  kw.put(L.cb, sizeof(L.cb));
  kw.put(L.cbo, sizeof(L.cbo));
  kw.putv((uint64_t)L.nci | ((uint64_t)L.nco << 32));
  kw.putv((uint64_t)L.pull_warp_b);
  kw.putv(L.fthr);
  kw.putv((uint64_t)L.fl.cap);
  const Relabel& rl = g->rl;
  const void* ptrs[] = {g->ctl.p,     g->xa.p,       g->xb.p,        g->ya.p,       g->yb.p,      g->resid.p,
                        g->resid32.p, g->fwork.p,    g->dN.p,        g->dV.p,       rl.in.off.p,  rl.in.adj.p,
                        rl.out.off.p, rl.out.adj.p,  rl.pout.p,     g->flist.p,    g->fcnt.p};
  kw.put(ptrs, sizeof(ptrs));
  kw.putv(rl.version);
  kw.putv((uint64_t)g->n);
  const int slot = (L.fp32 ? 4 : 0) + (L.dynamic ? 2 : 0) + (L.expand ? 1 : 0);
  PRDF_TRY(launch_while_graph(g, slot, kw.key, [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
    int rc = launch_loop_sweep(g, L, -1, cs);
    if (rc == PRDF_OK) rc = launch_loop_expansion(g, L, -1, cs);
    if (rc == PRDF_OK)
      rc = L.fp32 ? launch_iter_check32(g->ctl.p, g->resid32.p, L.tol_rel, L.max_iter, h, cs)
                  : launch_iter_check(g->ctl.p, g->resid.p, L.tol, L.max_iter, h, cs);
    return rc;
  }, s));
  PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64, g->ctl.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  int hit = 0;
  memcpy(&hit, g->ws.host_i64, sizeof(int));
  if (hit < 1 || hit > L.max_iter) {
    set_error("iteration graph ran %d sweeps", hit);
    return PRDF_ECUDA;
  }
  const size_t wsz = L.fp32 ? 2 * sizeof(uint32_t) : sizeof(uint64_t);
  const char* resid_dev = L.fp32 ? (const char*)g->resid32.p : (const char*)g->resid.p;
  PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64, resid_dev + wsz * (hit - 1), wsz, cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  res->converged = loop_stopped(L, g->ws.host_i64, 0, &res->final_delta) ? 1 : 0;
  res->iters = hit;
  const int k = hit - 1;
  res->final_buf = (k & 1) ? 0 : 1;
  res->launched = hit;
  res->kernels = (long long)hit * (L.kernels_per_iter + 1);
  res->ms_sweep = 0;
  return PRDF_OK;
}

// One loop with the driver the parameters select: the host loop when every
// sweep is to be timed (time_sweeps), else the CUDA graph.
int run_loop(prdf_graph* g, const prdf_params* p, bool fp32, bool dynamic, bool expand, int max_iter, IterResult* res,
             cudaStream_t s) {
  Loop L;
  PRDF_TRY(loop_setup(g, p, fp32, dynamic, expand, max_iter, &L, s));
  if (p->time_sweeps) return run_host_loop(g, L, p, res, s);
  return run_graph_loop(g, L, res, s);
}

int auto_tile(int K) { return K >= 64 ? 64 : (K >= 32 ? 32 : (K > 8 ? 16 : 8)); }

// the K-column fixed-point operator: forward pull over G' (P on in-slots) or
// adjoint pull over G (P on out-slots)
struct KOp {
  const int64_t* off;
  const int32_t* adj;
  const float* p32;
  const double* p64;
  int64_t hub_begin;  // first vertex of the two highest in-degree classes
  const PprHubTable* hub;  // chunks of the highest class's rows of this CSR
  const double* S64;  // right-hand side (dense [n, K]), also the start of the iteration
  bool sparse_rhs;    // look for few non-zero rows in S64 (a teleport on a few seed vertices)
  int slot;           // first of the four graph-cache slots of this operator's loops
};

int64_t hub_begin(const Relabel& rl) {
  const int C = rl.thr.n + 1;
  int64_t cb[kMaxThr + 2];
  begins_from_counts(rl.count, C, cb);
  return C >= 3 ? cb[C - 2] : cb[C - 1];
}

int64_t blk_begin(const Relabel& rl) {
  const int C = rl.thr.n + 1;
  int64_t cb[kMaxThr + 2];
  begins_from_counts(rl.count, C, cb);
  return cb[C - 1];
}

// kernels of one K-column FP32 tile: groups, warps, hub partials and hub finish
int ppr32_kernels(int64_t hub_b, int64_t blk_b, int64_t n) {
  return (hub_b > 0 ? 1 : 0) + (blk_b > hub_b ? 1 : 0) + (n > blk_b ? 2 : 0);
}

// chunk table of the highest in-degree class's rows of one CSR, rebuilt when the numbering changes
int ensure_hub(prdf_graph* g, const Csr& c, PprHubTable& t, cudaStream_t s) {
  if (t.valid && t.version == g->rl.version) return PRDF_OK;
  PRDF_TRY(build_ppr_hub(c.off.p, blk_begin(g->rl), g->n, t, g->ws, s));
  t.version = g->rl.version;
  t.valid = true;
  return PRDF_OK;
}

// FP32 K-column solve of R = alpha P^T R + (1 - alpha) rhs from the start held
// in *cur; on return *cur holds the result (the other buffer is scratch).
int ppr32_solve(prdf_graph* g, const KOp& op, const prdf_params* p, int K, int tile, const float* rhs,
                const int32_t* srow, float** cur, float** other, int max_iter, int* iters, long long* kernels,
                cudaStream_t s) {
  PRDF_TRY(g->resid32.reserve(2 * ((size_t)max_iter + 1), s));
  PRDF_CUDA(cudaMemsetAsync(g->resid32.p, 0, sizeof(uint32_t) * 2 * ((size_t)max_iter + 1), s));
  PRDF_TRY(g->ppr_part.reserve((size_t)(op.hub->nchunk > 0 ? op.hub->nchunk : 1) * (size_t)tile, s));
  Ppr32Args a;
  memset(&a, 0, sizeof(a));
  a.off = op.off;
  a.adj = op.adj;
  a.P = op.p32;
  a.S = rhs;
  a.srow = srow;
  a.K = K;
  a.alpha = (float)p->alpha;
  a.beta = (float)(1.0 - p->alpha);
  a.tol_rel = (float)p->tol_fp32_rel;
  const int64_t hb = op.hub_begin;
  const int check = p->check_every > 0 ? p->check_every : 8;
  float* buf[2] = {*cur, *other};
  const int tiles = (K + tile - 1) / tile;
  if (!p->time_sweeps) {
    // one CUDA graph: a while node over one sweep (every column tile) and the stop check
    PRDF_TRY(g->ctl.reserve(2, s));
    PRDF_CUDA(cudaMemsetAsync(g->ctl.p, 0, 2 * sizeof(int), s));
    a.ctl = g->ctl.p;
    a.Ra = buf[0];
    a.Rb = buf[1];
    a.resid_base = g->resid32.p;
    const PprHub hv = op.hub->view();
    KeyWriter kw;
    kw.put(&a, sizeof(a));
    kw.put(&hv, sizeof(hv));
    kw.putv((uint64_t)tile | ((uint64_t)max_iter << 32));
    kw.putv((uint64_t)hb);
    kw.putv((uint64_t)(uintptr_t)g->ppr_part.p);
    kw.putv((uint64_t)g->n);
    PRDF_TRY(launch_while_graph(g, op.slot + (srow ? 1 : 0), kw.key, [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
      int rc = launch_ppr32_sweep(a, tile, g->n, hb, hv, g->ppr_part.p, cs);
      if (rc == PRDF_OK) rc = launch_iter_check32(g->ctl.p, g->resid32.p, a.tol_rel, max_iter, h, cs);
      return rc;
    }, s));
    int hit = 0;
    PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64, g->ctl.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PRDF_CUDA(cudaStreamSynchronize(s));
    memcpy(&hit, g->ws.host_i64, sizeof(int));
    if (hit < 1 || hit > max_iter) {
      set_error("K-column graph ran %d sweeps", hit);
      return PRDF_ECUDA;
    }
    const int k = hit - 1;
    *iters = hit;
    *cur = buf[(k + 1) & 1];
    *other = buf[k & 1];
    *kernels += (long long)hit * (tiles * ppr32_kernels(hb, op.hub->begin, g->n) + 1);
    return PRDF_OK;
  }
  int launched = 0;
  bool done = false;
  while (launched < max_iter && !done) {
    const int upto = (launched + check < max_iter) ? launched + check : max_iter;
    for (int i = launched; i < upto; ++i) {
      a.R = buf[i & 1];
      a.Rn = buf[(i + 1) & 1];
      a.resid = g->resid32.p + 2 * i;
      a.prev = i > 0 ? g->resid32.p + 2 * (i - 1) : nullptr;
      PRDF_TRY(launch_ppr32_sweep(a, tile, g->n, hb, op.hub->view(), g->ppr_part.p, s));
    }
    launched = upto;
    PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64, g->resid32.p + 2 * (launched - 1), 2 * sizeof(uint32_t),
                              cudaMemcpyDeviceToHost, s));
    PRDF_CUDA(cudaStreamSynchronize(s));
    uint32_t h[2];
    memcpy(h, g->ws.host_i64, sizeof(h));
    float d, r;
    memcpy(&d, &h[0], 4);
    memcpy(&r, &h[1], 4);
    done = d <= (float)p->tol_fp32_rel * r;
  }
  std::vector<uint32_t> hr(2 * (size_t)launched);
  PRDF_CUDA(cudaMemcpyAsync(hr.data(), g->resid32.p, sizeof(uint32_t) * 2 * launched, cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  int k = launched - 1;
  for (int i = 0; i < launched; ++i) {
    float d, r;
    memcpy(&d, &hr[2 * i], 4);
    memcpy(&r, &hr[2 * i + 1], 4);
    if (d <= (float)p->tol_fp32_rel * r) {
      k = i;
      break;
    }
  }
  *iters = k + 1;
  *cur = buf[(k + 1) & 1];
  *other = buf[k & 1];
  *kernels += (long long)launched * tiles * ppr32_kernels(hb, op.hub->begin, g->n);
  return PRDF_OK;
}

// one FP64 Jacobi step Rn = T(R); returns max |T(R) - R|
int ppr64_step(prdf_graph* g, const KOp& op, const prdf_params* p, int K, int tile, const double* rhs,
               const int32_t* srow, const double* R, double* Rn, float* res32, double* dmax, long long* kernels,
               cudaStream_t s) {
  PRDF_TRY(g->resid.reserve(2, s));
  PRDF_CUDA(cudaMemsetAsync(g->resid.p, 0, sizeof(uint64_t), s));
  Ppr64Args a;
  memset(&a, 0, sizeof(a));
  a.off = op.off;
  a.adj = op.adj;
  a.P = op.p64;
  a.R = R;
  a.Rn = Rn;
  a.S = rhs;
  a.srow = srow;
  a.res32 = res32;
  a.K = K;
  a.alpha = p->alpha;
  a.beta = 1.0 - p->alpha;
  a.inv_beta = 1.0 / (1.0 - p->alpha);
  a.dmax = g->resid.p;
  PRDF_TRY(g->ppr_part64.reserve((size_t)(op.hub->nchunk > 0 ? op.hub->nchunk : 1) * (size_t)tile, s));
  PRDF_TRY(launch_ppr64_step(a, tile, g->n, op.hub_begin, op.hub->view(), g->ppr_part64.p, s));
  PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64, g->resid.p, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  memcpy(dmax, g->ws.host_i64, sizeof(double));
  *kernels += (long long)((K + tile - 1) / tile) * ppr32_kernels(op.hub_begin, op.hub->begin, g->n);
  return PRDF_OK;
}

// Solve X = alpha * A X + (1 - alpha) * op.S64 (A = P^T on G' or P on G) from
// X = S64, K columns in the class-contiguous numbering; result in *out
// (one of R64a / R64b). Mixed: FP32 solve, then iterative refinement with an
// FP64 step for the residual and an FP32 solve for the correction.
struct KSolve {
  int iters32 = 0, steps64 = 0, converged = 0;
  double dmax = 0;
  long long kernels = 0;
};

int ksolve(prdf_graph* g, const KOp& op, const prdf_params* p, int K, int tile, double** out, KSolve* r,
           cudaStream_t s) {
  const int64_t cnt = (int64_t)g->n * K;
  PprSparseRhs& sp = g->ppr_rhs;
  sp.rows = 0;
  if (p->precision == PRDF_FP64) {
    PRDF_CUDA(cudaMemcpyAsync(g->R64a.p, op.S64, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s));
    if (op.sparse_rhs) {
      PRDF_TRY(ppr_sparse_rhs(op.S64, g->n, K, g->ws, &sp, nullptr, s));
      r->kernels += 2 + (sp.rows ? 1 : 0);
    }
    const double* rhs = sp.rows ? sp.Sc64.p : op.S64;
    const int32_t* srow = sp.rows ? sp.srow.p : nullptr;
    if (!p->time_sweeps) {
      // one CUDA graph: a while node over one FP64 Jacobi step (every column tile) and the stop check
      const int max_iter = p->max_iter;
      PRDF_TRY(g->resid.reserve((size_t)max_iter + 1, s));
      PRDF_CUDA(cudaMemsetAsync(g->resid.p, 0, sizeof(uint64_t) * ((size_t)max_iter + 1), s));
      PRDF_TRY(g->ctl.reserve(2, s));
      PRDF_CUDA(cudaMemsetAsync(g->ctl.p, 0, 2 * sizeof(int), s));
      PRDF_TRY(g->ppr_part64.reserve((size_t)(op.hub->nchunk > 0 ? op.hub->nchunk : 1) * (size_t)tile, s));
      Ppr64Args pa;
      memset(&pa, 0, sizeof(pa));
      pa.off = op.off;
      pa.adj = op.adj;
      pa.P = op.p64;
      pa.S = rhs;
      pa.srow = srow;
      pa.K = K;
      pa.alpha = p->alpha;
      pa.beta = 1.0 - p->alpha;
      pa.inv_beta = 1.0 / (1.0 - p->alpha);
      pa.ctl = g->ctl.p;
      pa.Ra = g->R64a.p;
      pa.Rb = g->R64b.p;
      pa.dmax_base = g->resid.p;
      const PprHub hv = op.hub->view();
      KeyWriter kw;
      kw.put(&pa, sizeof(pa));
      kw.put(&hv, sizeof(hv));
      kw.putv((uint64_t)tile | ((uint64_t)max_iter << 32));
      kw.put(&p->tol, sizeof(p->tol));
      kw.putv((uint64_t)op.hub_begin);
      kw.putv((uint64_t)(uintptr_t)g->ppr_part64.p);
      kw.putv((uint64_t)g->n);
      PRDF_TRY(launch_while_graph(g, op.slot + 2, kw.key, [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
        int rc = launch_ppr64_step(pa, tile, g->n, op.hub_begin, hv, g->ppr_part64.p, cs);
        if (rc == PRDF_OK) rc = launch_iter_check(g->ctl.p, g->resid.p, p->tol, max_iter, h, cs);
        return rc;
      }, s));
      int hit = 0;
      PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64, g->ctl.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      PRDF_CUDA(cudaStreamSynchronize(s));
      memcpy(&hit, g->ws.host_i64, sizeof(int));
      if (hit < 1 || hit > max_iter) {
        set_error("K-column graph ran %d steps", hit);
        return PRDF_ECUDA;
      }
      PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64, g->resid.p + hit - 1, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
      PRDF_CUDA(cudaStreamSynchronize(s));
      memcpy(&r->dmax, g->ws.host_i64, sizeof(double));
      r->steps64 += hit;
      r->converged = r->dmax <= p->tol ? 1 : 0;
      r->kernels += (long long)hit * (((K + tile - 1) / tile) * ppr32_kernels(op.hub_begin, op.hub->begin, g->n) + 1);
      *out = ((hit - 1) & 1) ? g->R64a.p : g->R64b.p;  // step k writes R64b when k is even
      return PRDF_OK;
    }
    double* a = g->R64a.p;
    double* b = g->R64b.p;
    for (int it = 0; it < p->max_iter; ++it) {
      PRDF_TRY(ppr64_step(g, op, p, K, tile, rhs, srow, a, b, nullptr, &r->dmax, &r->kernels, s));
      ++r->steps64;
      double* tmp = a;
      a = b;
      b = tmp;
      if (r->dmax <= p->tol) {
        r->converged = 1;
        break;
      }
    }
    *out = a;
    return PRDF_OK;
  }
  PRDF_TRY(g->S32.reserve(cnt, s));
  PRDF_TRY(g->R32a.reserve(cnt, s));
  PRDF_TRY(g->R32b.reserve(cnt, s));
  if (op.sparse_rhs) {
    // a teleport on few vertices: the first solve reads a 4-byte row index per vertex instead of its row
    PRDF_TRY(ppr_sparse_rhs(op.S64, g->n, K, g->ws, &sp, g->R32a.p, s));
    r->kernels += 2 + (sp.rows ? 1 : 0);
  }
  const double* rhs64 = sp.rows ? sp.Sc64.p : op.S64;
  const int32_t* srow = sp.rows ? sp.srow.p : nullptr;
  if (!sp.rows) {
    PRDF_TRY(ppr_narrow(op.S64, cnt, g->S32.p, s));
    PRDF_CUDA(cudaMemcpyAsync(g->R32a.p, g->S32.p, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, s));
  }
  float* cur = g->R32a.p;
  float* oth = g->R32b.p;
  int it32 = 0;
  PRDF_TRY(ppr32_solve(g, op, p, K, tile, sp.rows ? sp.Sc32.p : g->S32.p, srow, &cur, &oth, p->max_iter, &it32,
                       &r->kernels, s));
  r->iters32 += it32;
  PRDF_TRY(ppr_widen(cur, cnt, g->R64a.p, s));
  r->kernels += 2;
  const int kRounds = 8;
  for (int round = 0; round < kRounds; ++round) {
    // FP64 Jacobi step: T(R) and the residual (T(R) - R) / (1 - alpha), dense, in S32
    PRDF_TRY(ppr64_step(g, op, p, K, tile, rhs64, srow, g->R64a.p, g->R64b.p, g->S32.p, &r->dmax, &r->kernels, s));
    ++r->steps64;
    if (r->dmax <= p->tol) {
      r->converged = 1;
      break;
    }
    PRDF_CUDA(cudaMemcpyAsync(g->R32a.p, g->S32.p, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, s));
    cur = g->R32a.p;
    oth = g->R32b.p;
    PRDF_TRY(ppr32_solve(g, op, p, K, tile, g->S32.p, nullptr, &cur, &oth, p->max_iter, &it32, &r->kernels, s));
    r->iters32 += it32;
    PRDF_TRY(ppr_add_correction(g->R64a.p, cur, cnt, s));
    r->kernels += 1;
  }
  *out = g->R64b.p;  // T(X) of the last step
  return PRDF_OK;
}

// FP32 stage buffers (state, degrees, and for DF-P the Eq. 2 factor)
int alloc_fp32(prdf_graph* g, bool eq2, cudaStream_t s) {
  PRDF_TRY(g->ya.reserve(g->n, s));
  PRDF_TRY(g->yb.reserve(g->n, s));
  PRDF_TRY(g->degf.reserve(g->n, s));
  PRDF_TRY(g->invf.reserve(g->n, s));
  if (eq2) PRDF_TRY(g->kf32.reserve(g->n, s));
  return PRDF_OK;
}

// FP32 stage of a dynamic solve (DF / DF-P with expansion, DT without): the
// affected set and flags are already marked and xa = xb = R^{t-1} / |out|.
// Runs FP32 sweeps from R^{t-1} to the relative stop, then sets xa = xb to
// their result (FP64 values kept where the FP32 stage changed nothing),
// affects every vertex it changed, and clears the copy-through marks, so the
// FP64 loop continues from there: the affected set the FP32 stage left plus
// the vertices it moved, whose prune tests the FP64 sweeps then decide.
int dynamic_fp32_stage(prdf_graph* g, const prdf_params* p, const double* prev_ranks, bool expand, IterResult* it32,
                       cudaStream_t s) {
  const int n = g->n;
  const Relabel& rl = g->rl;
  const bool eq2 = p->prune != 0;
  PRDF_TRY(alloc_fp32(g, eq2, s));
  k_init_y<<<grid_for(n, kThreads), kThreads, 0, s>>>(prev_ranks, rl.perm.p, n, rl.degd.p, rl.inv_deg.p,
                                                     eq2 ? rl.kf.p : nullptr, g->ya.p, g->yb.p, g->degf.p, g->invf.p,
                                                     eq2 ? g->kf32.p : nullptr);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(run_loop(g, p, true, true, expand, p->max_iter, it32, s));
  k_widen_keep<<<grid_for(n, kThreads), kThreads, 0, s>>>(it32->final_buf ? g->yb.p : g->ya.p, n, g->xa.p, g->xb.p,
                                                         g->dV.p);
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaMemsetAsync(g->wrote.p, 0, (size_t)n, s));
  return PRDF_OK;
}

int alloc_solver(prdf_graph* g, bool dynamic, cudaStream_t s) {
  PRDF_TRY(g->xa.reserve(g->n, s));
  PRDF_TRY(g->xb.reserve(g->n, s));
  if (dynamic) {
    PRDF_TRY(g->dV.reserve(g->n, s));
    PRDF_TRY(g->dN.reserve(g->n, s));
    PRDF_TRY(g->wrote.reserve(g->n, s));
  }
  PRDF_TRY(g->counter.reserve(1, s));
  return PRDF_OK;
}

}  // namespace
}  // namespace prdf

namespace prdf {
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};
}  // namespace

cudaMemPool_t device_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}
}  // namespace prdf

using namespace prdf;

extern "C" {

void prdf_params_default(prdf_params* p) {
  if (!p) return;
  p->alpha = 0.85;
  p->tol = 1e-10;
  p->tau_f = 1e-6;
  p->tau_p = 1e-6;
  p->max_iter = 500;
  p->precision = PRDF_FP64;
  p->tol_fp32_rel = 1e-6;
  p->accumulate = PRDF_ACC_EXACT;
  p->prune = 1;
  p->check_every = 8;
  p->time_sweeps = 0;
  p->tile = 0;
  p->expand_pull = 1.0 / 16.0;
  p->expand_list = -1;
  p->stream = nullptr;
}

const char* prdf_last_error(void) { return g_err; }

int prdf_release_cached_memory(void) {
  std::lock_guard<std::mutex> lock(prdf::g_pool_mu);
  for (int d = 0; d < prdf::kMaxDevices; ++d)
    if (prdf::g_pool[d]) PRDF_CUDA(cudaMemPoolTrimTo(prdf::g_pool[d], 0));
  return PRDF_OK;
}

const char* prdf_strerror(int code) {
  switch (code) {
    case PRDF_OK: return "ok";
    case PRDF_EINVAL: return "invalid argument";
    case PRDF_ENOMEM: return "out of device memory";
    case PRDF_ECUDA: return "CUDA error";
    case PRDF_ETIMEOUT: return "bounded device wait expired";
    case PRDF_ESTATE: return "call out of order";
    default: return "unknown error";
  }
}

int prdf_graph_create(int32_t n, const int32_t* src, const int32_t* dst, const float* w, int64_t m0, unsigned flags,
                      void* stream, prdf_graph** out) {
  if (!out || n < 1 || m0 < 0 || (m0 > 0 && (!src || !dst))) {
    set_error("prdf_graph_create: bad arguments (n=%d, m0=%lld)", n, (long long)m0);
    return PRDF_EINVAL;
  }
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  prdf_graph* g = new (std::nothrow) prdf_graph();
  if (!g) {
    set_error("host allocation failed");
    return PRDF_ENOMEM;
  }
  g->n = n;
  g->weighted = w != nullptr;
  g->stream = s;
  // default class thresholds. In-degree (rank sweep): self-loop only, <= 4,
  // <= 16 (4 lanes), <= 32 (8 lanes), <= 128 (16 lanes), <= 4096 (warp),
  // block above. Out-degree (marking): thread <= 8, 8 lanes <= 64, warp <=
  // 2048, block above.
  {
    const int64_t tin[6] = {1, 4, 16, 32, 128, 4096};
    g->thr[PRDF_IN].n = 6;
    for (int i = 0; i < 6; ++i) g->thr[PRDF_IN].thr[i] = tin[i];
    const int64_t tout[3] = {8, 64, 2048};
    g->thr[PRDF_OUT].n = 3;
    for (int i = 0; i < 3; ++i) g->thr[PRDF_OUT].thr[i] = tout[i];
  }
  int r = g->ws.init();
  const bool loops = (flags & PRDF_ADD_SELF_LOOPS) != 0;
  g->self_loops = loops;
  if (r == PRDF_OK) r = build_csr(n, m0, src, dst, w, loops, false, g->csr[PRDF_OUT], g->ws, s);
  if (r == PRDF_OK) r = build_csr(n, m0, dst, src, w, loops, false, g->csr[PRDF_IN], g->ws, s);
  g->m = g->csr[PRDF_OUT].m;
  if (r == PRDF_OK) r = build_relabelled(g, s);
  if (r == PRDF_OK && cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("graph build: %s", cudaGetErrorString(cudaGetLastError()));
    r = PRDF_ECUDA;
  }
  if (r != PRDF_OK) {
    delete g;
    return r;
  }
  *out = g;
  return PRDF_OK;
}

void prdf_graph_destroy(prdf_graph* g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  cudaDeviceSynchronize();
  for (auto& e : g->loop_exec)
    if (e) cudaGraphExecDestroy(e);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  delete g;
}

int prdf_graph_size(const prdf_graph* g, int32_t* n_host, int64_t* m_host) {
  if (!g) {
    set_error("graph is NULL");
    return PRDF_EINVAL;
  }
  if (n_host) *n_host = g->n;
  if (m_host) *m_host = g->m;
  return PRDF_OK;
}

int prdf_graph_export_csr(const prdf_graph* g, int which, int64_t* off, int32_t* adj, float* w, void* stream) {
  if (!g || (which != PRDF_OUT && which != PRDF_IN)) {
    set_error("bad graph or CSR selector");
    return PRDF_EINVAL;
  }
  if (w && !g->weighted) {
    set_error("graph has no weights");
    return PRDF_ESTATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  PRDF_TRY(ensure_orig(const_cast<prdf_graph*>(g), s));
  const Csr& c = g->csr[which];
  if (off) PRDF_CUDA(cudaMemcpyAsync(off, c.off.p, sizeof(int64_t) * ((size_t)g->n + 1), cudaMemcpyDeviceToDevice, s));
  if (adj && c.m) PRDF_CUDA(cudaMemcpyAsync(adj, c.adj.p, sizeof(int32_t) * (size_t)c.m, cudaMemcpyDeviceToDevice, s));
  if (w && c.m) PRDF_CUDA(cudaMemcpyAsync(w, c.w.p, sizeof(float) * (size_t)c.m, cudaMemcpyDeviceToDevice, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  return PRDF_OK;
}

int prdf_graph_apply_batch(prdf_graph* g, const int32_t* del_src, const int32_t* del_dst, int64_t n_del,
                           const int32_t* ins_src, const int32_t* ins_dst, const float* ins_w, int64_t n_ins,
                           uint8_t* del_eff, uint8_t* ins_eff, void* stream) {
  if (!g || n_del < 0 || n_ins < 0 || (n_del > 0 && (!del_src || !del_dst)) || (n_ins > 0 && (!ins_src || !ins_dst))) {
    set_error("prdf_graph_apply_batch: bad arguments");
    return PRDF_EINVAL;
  }
  if (g->weighted && n_ins > 0 && !ins_w) {
    set_error("weighted graph: insertions need weights");
    return PRDF_ESTATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  PRDF_TRY(check_inputs(g, del_src, del_dst, n_del, ins_src, ins_dst, n_ins, nullptr, nullptr, s));
  const int32_t n = g->n;
  Relabel& rl = g->rl;
  const int64_t nb = n_del + n_ins;
  if (g->self_loops && rl.valid && (rl.drift + nb) * 64 <= g->m) {
    // Every vertex already has its self-loop: each row of G and of G' becomes
    // (old \ D) u I, merged in order (batch_update.cu), directly on the copies
    // in the sweep numbering (rows ordered by original id, columns compared
    // through perm). The numbering, its partitions and the chunk tables are
    // kept; the original-id CSRs are derived again when asked for.
    DBuf<int32_t> rows;
    PRDF_TRY(rows.alloc((size_t)(2 * nb > 0 ? 2 * nb : 1), s));
    int32_t* del_r_out = rows.p;           // inv[del_src]
    int32_t* del_r_in = rows.p + n_del;    // inv[del_dst]
    int32_t* ins_r_out = rows.p + 2 * n_del;
    int32_t* ins_r_in = rows.p + 2 * n_del + n_ins;
    if (n_del) {
      k_map_ids<<<grid_for(n_del, kThreads), kThreads, 0, s>>>(del_src, n_del, rl.inv.p, del_r_out);
      k_map_ids<<<grid_for(n_del, kThreads), kThreads, 0, s>>>(del_dst, n_del, rl.inv.p, del_r_in);
    }
    if (n_ins) {
      k_map_ids<<<grid_for(n_ins, kThreads), kThreads, 0, s>>>(ins_src, n_ins, rl.inv.p, ins_r_out);
      k_map_ids<<<grid_for(n_ins, kThreads), kThreads, 0, s>>>(ins_dst, n_ins, rl.inv.p, ins_r_in);
    }
    PRDF_LAUNCH_CHECK();
    Csr nout, nin;
    PRDF_TRY(update_csr(n, rl.out, del_r_out, del_dst, n_del, ins_r_out, ins_dst, ins_w, n_ins, nout, g->ws, s,
                        rl.perm.p, rl.inv.p));
    PRDF_TRY(update_csr(n, rl.in, del_r_in, del_src, n_del, ins_r_in, ins_src, ins_w, n_ins, nin, g->ws, s,
                        rl.perm.p, rl.inv.p));
    if (del_eff && n_del)
      k_effective_keyed<<<grid_for(n_del, kThreads), kThreads, 0, s>>>(del_src, del_dst, n_del, 1, rl.perm.p,
                                                                       rl.inv.p, rl.out.off.p, rl.out.adj.p,
                                                                       nout.off.p, nout.adj.p, del_eff);
    if (ins_eff && n_ins)
      k_effective_keyed<<<grid_for(n_ins, kThreads), kThreads, 0, s>>>(ins_src, ins_dst, n_ins, 0, rl.perm.p,
                                                                       rl.inv.p, rl.out.off.p, rl.out.adj.p,
                                                                       nout.off.p, nout.adj.p, ins_eff);
    PRDF_LAUNCH_CHECK();
    rl.out = static_cast<Csr&&>(nout);
    rl.in = static_cast<Csr&&>(nin);
    g->m = rl.out.m;
    // vertices of the classes of in-degree <= 1 (ids [0, end1)) that gain an in-edge take the general path
    // of their kernel
    int64_t end1 = 0;
    for (int c = 0; c < rl.thr.n && rl.thr.thr[c] <= 1; ++c) end1 += rl.count[c];
    const bool self1 = end1 > 0;
    if (self1 && n_ins) {
      PRDF_TRY(g->counter.reserve(1, s));
      PRDF_CUDA(cudaMemsetAsync(g->counter.p, 0, sizeof(unsigned long long), s));
      k_mark_multi<<<grid_for(n_ins, kThreads), kThreads, 0, s>>>(ins_dst, n_ins, rl.inv.p, end1, rl.multi.p,
                                                                  g->counter.p);
      PRDF_LAUNCH_CHECK();
      PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64 + 1, g->counter.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                s));
    }
    // out-degrees change only for the batch's sources: their degrees and Eq. 2 factors are refreshed
    PRDF_TRY(update_degrees_of(g, del_src, n_del, s));
    PRDF_TRY(update_degrees_of(g, ins_src, n_ins, s));
    rl.drift += nb;
    ++rl.version;
    g->orig_valid = false;
    g->pvalid[0] = g->pvalid[1] = false;
    g->ppr_valid = false;
    PRDF_CUDA(cudaStreamSynchronize(s));
    if (self1 && n_ins) rl.multi_count += g->ws.host_i64[1];
    return PRDF_OK;
  }
  // A fresh numbering is due: the batches applied since the last one, this
  // one included, add up to more than 1/64 of the edges (degree classes and
  // out-degree tiers drift), or the graph was made without self-loops. The
  // rows are merged on the original-id CSRs (or rebuilt from the edge list,
  // which also gives every vertex its self-loop) and then renumbered.
  PRDF_TRY(ensure_orig(g, s));
  Csr& old = g->csr[PRDF_OUT];
  const int64_t m = old.m;
  Csr nout, nin;
  if (g->self_loops) {
    PRDF_TRY(update_csr(n, g->csr[PRDF_OUT], del_src, del_dst, n_del, ins_src, ins_dst, ins_w, n_ins, nout, g->ws, s));
    PRDF_TRY(update_csr(n, g->csr[PRDF_IN], del_dst, del_src, n_del, ins_dst, ins_src, ins_w, n_ins, nin, g->ws, s));
  } else {
    DBuf<uint8_t> deleted;
    PRDF_TRY(deleted.alloc((size_t)m, s));
    PRDF_CUDA(cudaMemsetAsync(deleted.p, 0, (size_t)m, s));
    if (n_del)
      k_mark_deleted<<<grid_for(n_del, kThreads), kThreads, 0, s>>>(del_src, del_dst, n_del, old.off.p, old.adj.p,
                                                                     deleted.p);
    const int64_t tot = m + n_ins;
    DBuf<int32_t> rows, cols;
    DBuf<float> ww;
    PRDF_TRY(rows.alloc(tot, s));
    PRDF_TRY(cols.alloc(tot, s));
    if (g->weighted) PRDF_TRY(ww.alloc(tot, s));
    k_old_edges<<<grid_for((int64_t)n * 32, kThreads), kThreads, 0, s>>>(n, old.off.p, old.adj.p,
                                                                          g->weighted ? old.w.p : nullptr, deleted.p,
                                                                          rows.p, cols.p, ww.p);
    if (n_ins)
      k_append<<<grid_for(n_ins, kThreads), kThreads, 0, s>>>(ins_src, ins_dst, ins_w, n_ins, m, rows.p, cols.p, ww.p);
    PRDF_LAUNCH_CHECK();
    PRDF_TRY(build_csr(n, tot, rows.p, cols.p, ww.p, true, true, nout, g->ws, s));
    PRDF_TRY(build_csr(n, tot, cols.p, rows.p, ww.p, true, true, nin, g->ws, s));
  }
  if (del_eff && n_del)
    k_effective<<<grid_for(n_del, kThreads), kThreads, 0, s>>>(del_src, del_dst, n_del, 1, old.off.p, old.adj.p,
                                                               nout.off.p, nout.adj.p, del_eff);
  if (ins_eff && n_ins)
    k_effective<<<grid_for(n_ins, kThreads), kThreads, 0, s>>>(ins_src, ins_dst, n_ins, 0, old.off.p, old.adj.p,
                                                               nout.off.p, nout.adj.p, ins_eff);
  PRDF_LAUNCH_CHECK();
  g->self_loops = true;  // the rebuild gives every vertex its self-loop
  g->csr[PRDF_OUT] = static_cast<Csr&&>(nout);
  g->csr[PRDF_IN] = static_cast<Csr&&>(nin);
  g->m = g->csr[PRDF_OUT].m;
  g->orig_valid = true;
  g->pvalid[0] = g->pvalid[1] = false;
  PRDF_TRY(build_relabelled(g, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  return PRDF_OK;
}

int prdf_graph_set_thresholds(prdf_graph* g, int which, int n_thr, const int64_t* thr_host) {
  if (!g || (which != PRDF_OUT && which != PRDF_IN) || n_thr < 1 || n_thr > kMaxThr || !thr_host) {
    set_error("prdf_graph_set_thresholds: bad arguments");
    return PRDF_EINVAL;
  }
  if (thr_host[0] < 0) {
    set_error("thresholds must be >= 0");
    return PRDF_EINVAL;
  }
  for (int i = 1; i < n_thr; ++i)
    if (thr_host[i] <= thr_host[i - 1]) {
      set_error("thresholds must be strictly increasing");
      return PRDF_EINVAL;
    }
  g->thr[which].n = n_thr;
  for (int i = 0; i < kMaxThr; ++i) g->thr[which].thr[i] = i < n_thr ? thr_host[i] : 0;
  g->pvalid[which] = false;
  if (which == PRDF_OUT) g->rl.pout_valid = false;  // the marking partition follows the out-degree classes
  return PRDF_OK;
}

int prdf_partition(prdf_graph* g, int which, int32_t* P, int64_t* counts_host, void* stream) {
  if (!g || (which != PRDF_OUT && which != PRDF_IN) || !P || !counts_host) {
    set_error("prdf_partition: bad arguments");
    return PRDF_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  g->pvalid[which] = false;
  PRDF_TRY(ensure_partition(g, which, s));
  PRDF_CUDA(cudaMemcpyAsync(P, g->P[which].p, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToDevice, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; c <= g->thr[which].n; ++c) counts_host[c] = g->pcount[which][c];
  return PRDF_OK;
}

int prdf_initial_affected(prdf_graph* g, const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask,
                          int64_t n_del, const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins, uint8_t* dV,
                          uint8_t* dN, void* stream) {
  if (!g || !dV || !dN || n_del < 0 || n_ins < 0 || (n_del && (!del_src || !del_dst)) || (n_ins && !ins_src)) {
    set_error("prdf_initial_affected: bad arguments");
    return PRDF_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  PRDF_TRY(check_inputs(g, del_src, del_dst, n_del, ins_src, nullptr, n_ins, nullptr, nullptr, s));
  PRDF_TRY(launch_initial_affected(del_src, del_dst, del_mask, n_del, ins_src, ins_mask, n_ins, nullptr, dV, dN, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  return PRDF_OK;
}

int prdf_expand_affected(prdf_graph* g, const uint8_t* dN, uint8_t* dV, void* stream) {
  if (!g || !dN || !dV) {
    set_error("prdf_expand_affected: bad arguments");
    return PRDF_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  PRDF_TRY(ensure_partition(g, PRDF_OUT, s));
  int64_t cb[kMaxThr + 2];
  class_begins(g, PRDF_OUT, cb);
  PRDF_TRY(launch_expand(g->csr[PRDF_OUT].off.p, g->csr[PRDF_OUT].adj.p, g->P[PRDF_OUT].p, cb, g->thr[PRDF_OUT].n + 1,
                         dN, dV, nullptr, Stop(), s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  return PRDF_OK;
}

int prdf_pagerank_static(prdf_graph* g, const prdf_params* p, const double* R0, double* ranks, prdf_stats* stats) {
  if (!g || !ranks) {
    set_error("prdf_pagerank_static: bad arguments");
    return PRDF_EINVAL;
  }
  PRDF_TRY(check_params(p));
  cudaStream_t s = (cudaStream_t)p->stream;
  if (R0) PRDF_TRY(check_inputs(g, nullptr, nullptr, 0, nullptr, nullptr, 0, R0, "R0", s));
  Timer t;
  PRDF_TRY(t.init());
  PRDF_TRY(alloc_solver(g, false, s));
  PRDF_CUDA(cudaEventRecord(t.e[0], s));
  // Alg. static: initialise ranks, partition G' by in-degree, iterate
  // the in-degree partition is the class-contiguous numbering, built with the
  // graph and rebuilt here only if the thresholds changed
  PRDF_TRY(ensure_relabelled(g, false, s));
  int iters32 = 0;
  long long kernels32 = 0;
  prdf_params p64 = *p;
  if (p->precision == PRDF_FP32_REFINE) {
    // FP32 stage, then FP64 sweeps from its result
    PRDF_TRY(alloc_fp32(g, false, s));
    k_init_y<<<grid_for(g->n, kThreads), kThreads, 0, s>>>(R0, g->rl.perm.p, g->n, g->rl.degd.p, g->rl.inv_deg.p,
                                                           nullptr, g->ya.p, nullptr, g->degf.p, g->invf.p, nullptr);
    PRDF_LAUNCH_CHECK();
    PRDF_CUDA(cudaEventRecord(t.e[1], s));
    IterResult it32;
    PRDF_TRY(run_loop(g, p, true, false, false, p->max_iter, &it32, s));
    iters32 = it32.iters;
    k_widen<<<grid_for(g->n, kThreads), kThreads, 0, s>>>(it32.final_buf ? g->yb.p : g->ya.p, g->n, g->xa.p);
    PRDF_LAUNCH_CHECK();
    p64.max_iter = p->max_iter - iters32 > 0 ? p->max_iter - iters32 : 1;
    kernels32 = it32.kernels + 2;
  } else {
    k_init_x<<<grid_for(g->n, kThreads), kThreads, 0, s>>>(R0, g->rl.perm.p, g->n, g->rl.inv_deg.p, g->xa.p, nullptr);
    PRDF_LAUNCH_CHECK();
    PRDF_CUDA(cudaEventRecord(t.e[1], s));
  }
  IterResult it;
  PRDF_TRY(run_loop(g, &p64, false, false, false, p64.max_iter, &it, s));
  k_finalize<<<grid_for(g->n, kThreads), kThreads, 0, s>>>(it.final_buf ? g->xb.p : g->xa.p, g->rl.degd.p,
                                                           g->rl.perm.p, g->n, ranks, nullptr, nullptr);
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaEventRecord(t.e[2], s));
  PRDF_CUDA(cudaEventSynchronize(t.e[2]));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iterations = it.iters + iters32;
    stats->iterations_fp32 = iters32;
    stats->converged = it.converged;
    stats->final_delta = it.final_delta;
    stats->sweeps_launched = it.launched;
    cudaEventElapsedTime(&stats->ms_total, t.e[0], t.e[2]);
    cudaEventElapsedTime(&stats->ms_partition, t.e[0], t.e[1]);
    cudaEventElapsedTime(&stats->ms_iterate, t.e[1], t.e[2]);
    stats->ms_sweep = it.ms_sweep > 0 ? it.ms_sweep : 0.f;
    stats->edges_processed = (long long)(it.iters + iters32) * g->m;
    // init + sweeps + finalize
    stats->kernel_launches = 1 + kernels32 + it.kernels + 1;
  }
  return PRDF_OK;
}

int prdf_pagerank_dfp(prdf_graph* g, const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask,
                      int64_t n_del, const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins,
                      const double* prev_ranks, double* ranks, const prdf_params* p, uint8_t* dV_out,
                      prdf_stats* stats) {
  if (!g || !prev_ranks || !ranks || n_del < 0 || n_ins < 0 || (n_del && (!del_src || !del_dst)) ||
      (n_ins && !ins_src)) {
    set_error("prdf_pagerank_dfp: bad arguments");
    return PRDF_EINVAL;
  }
  PRDF_TRY(check_params(p));
  cudaStream_t s = (cudaStream_t)p->stream;
  PRDF_TRY(check_inputs(g, del_src, del_dst, n_del, ins_src, nullptr, n_ins, prev_ranks, "prev_ranks", s));
  Timer t;
  PRDF_TRY(t.init());
  PRDF_TRY(alloc_solver(g, true, s));
  const int n = g->n;
  PRDF_CUDA(cudaEventRecord(t.e[0], s));
  // Alg. frontier: R = Rnew = R^{t-1}; partition G and G'; mark; iterate.
  // The partitions are kept with the graph: G' by in-degree is the sweep
  // numbering, G by out-degree (for marking) is made with it and stays valid
  // until the graph or the thresholds change.
  const bool pout_made = !g->rl.pout_valid;
  PRDF_TRY(ensure_relabelled(g, true, s));
  Relabel& rl = g->rl;
  bool kf_made = false;
  if (p->prune && rl.kf_alpha != p->alpha) {
    // Eq. 2's per-vertex factor, kept until the numbering or alpha changes
    PRDF_TRY(rl.kf.reserve((size_t)n, s));
    k_eq2_factor<<<grid_for(n, kThreads), kThreads, 0, s>>>(rl.degd.p, n, p->alpha, rl.kf.p);
    PRDF_LAUNCH_CHECK();
    rl.kf_alpha = p->alpha;
    kf_made = true;
  }
  k_init_x<<<grid_for(n, kThreads), kThreads, 0, s>>>(prev_ranks, rl.perm.p, n, rl.inv_deg.p, g->xa.p, g->xb.p);
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaEventRecord(t.e[1], s));
  PRDF_CUDA(cudaMemsetAsync(g->dV.p, 0, (size_t)n, s));
  PRDF_CUDA(cudaMemsetAsync(g->dN.p, 0, (size_t)n, s));
  PRDF_CUDA(cudaMemsetAsync(g->wrote.p, 0, (size_t)n, s));
  PRDF_TRY(launch_initial_affected(del_src, del_dst, del_mask, n_del, ins_src, ins_mask, n_ins, rl.inv.p, g->dV.p,
                                   g->dN.p, s));
  int64_t cbo[kMaxThr + 2];
  begins_from_counts(rl.pout_count, g->thr[PRDF_OUT].n + 1, cbo);
  FrontList fl;
  PRDF_TRY(front_list(g, p, s, &fl));
  PRDF_TRY(launch_expand(rl.out.off.p, rl.out.adj.p, rl.pout.p, cbo, g->thr[PRDF_OUT].n + 1, g->dN.p, g->dV.p,
                         nullptr, Stop(), s, nullptr, 0, fl));
  PRDF_TRY(count_flags(g->dV.p, n, g->counter.p, s));
  PRDF_CUDA(cudaEventRecord(t.e[2], s));
  PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64 + 8, g->counter.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  IterResult it, it32;
  prdf_params p64 = *p;
  long long kernels32 = 0;
  if (p->precision == PRDF_FP32_REFINE) {
    // FP32 DF-P sweeps to the relative stop, then FP64 DF-P sweeps from their
    // result with the affected set they leave
    PRDF_TRY(dynamic_fp32_stage(g, p, prev_ranks, true, &it32, s));
    p64.max_iter = p->max_iter - it32.iters > 0 ? p->max_iter - it32.iters : 1;
    kernels32 = it32.kernels + 3;
  }
  PRDF_TRY(run_loop(g, &p64, false, true, true, p64.max_iter, &it, s));  // synchronises the stream
  const long long aff0 = (long long)g->ws.host_i64[8];
  k_finalize<<<grid_for(n, kThreads), kThreads, 0, s>>>(it.final_buf ? g->xb.p : g->xa.p, rl.degd.p, rl.perm.p, n,
                                                       ranks, g->dV.p, dV_out);
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaEventRecord(t.e[3], s));
  PRDF_CUDA(cudaEventSynchronize(t.e[3]));
  PRDF_CUDA(cudaStreamSynchronize(s));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iterations = it.iters + it32.iters;
    stats->iterations_fp32 = it32.iters;
    stats->converged = it.converged;
    stats->final_delta = it.final_delta;
    stats->sweeps_launched = it.launched + it32.launched;
    cudaEventElapsedTime(&stats->ms_total, t.e[0], t.e[3]);
    cudaEventElapsedTime(&stats->ms_partition, t.e[0], t.e[1]);
    cudaEventElapsedTime(&stats->ms_mark, t.e[1], t.e[2]);
    cudaEventElapsedTime(&stats->ms_iterate, t.e[2], t.e[3]);
    stats->ms_sweep = it.ms_sweep + it32.ms_sweep;
    stats->edges_processed = -1;
    stats->affected_initial = aff0;
    // (out-degree partition) + init (+ Eq. 2 factor) + initial marking + expand + count + sweeps/expands + finalize
    stats->kernel_launches = (pout_made ? 5 : 0) + 1 + (kf_made ? 1 : 0) + (n_del + n_ins > 0 ? 1 : 0) +
                             nonempty_classes(cbo, g->thr[PRDF_OUT].n + 1) + (fl.list ? 2 : 0) + 1 + kernels32 + it.kernels + 1;
  }
  return PRDF_OK;
}

int prdf_pagerank_dt(prdf_graph* g, const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask,
                     int64_t n_del, const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins,
                     const double* prev_ranks, double* ranks, const prdf_params* p, uint8_t* dV_out,
                     prdf_stats* stats) {
  if (!g || !prev_ranks || !ranks || n_del < 0 || n_ins < 0 || (n_del && (!del_src || !del_dst)) ||
      (n_ins && !ins_src)) {
    set_error("prdf_pagerank_dt: bad arguments");
    return PRDF_EINVAL;
  }
  PRDF_TRY(check_params(p));
  cudaStream_t s = (cudaStream_t)p->stream;
  PRDF_TRY(check_inputs(g, del_src, del_dst, n_del, ins_src, nullptr, n_ins, prev_ranks, "prev_ranks", s));
  Timer t;
  PRDF_TRY(t.init());
  PRDF_TRY(alloc_solver(g, true, s));
  const int n = g->n;
  PRDF_TRY(g->dF.reserve(n, s));
  PRDF_CUDA(cudaEventRecord(t.e[0], s));
  // Alg. traversal: R = Rnew = R^{t-1}; partitions (kept with the graph); mark; close; iterate
  const bool pout_made = !g->rl.pout_valid;
  PRDF_TRY(ensure_relabelled(g, true, s));
  const Relabel& rl = g->rl;
  k_init_x<<<grid_for(n, kThreads), kThreads, 0, s>>>(prev_ranks, rl.perm.p, n, rl.inv_deg.p, g->xa.p, g->xb.p);
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaEventRecord(t.e[1], s));
  PRDF_CUDA(cudaMemsetAsync(g->dV.p, 0, (size_t)n, s));
  PRDF_CUDA(cudaMemsetAsync(g->dN.p, 0, (size_t)n, s));
  PRDF_CUDA(cudaMemsetAsync(g->wrote.p, 0, (size_t)n, s));
  PRDF_TRY(launch_initial_affected(del_src, del_dst, del_mask, n_del, ins_src, ins_mask, n_ins, rl.inv.p, g->dV.p,
                                   g->dN.p, s));
  const int nco = g->thr[PRDF_OUT].n + 1;
  int64_t cbo[kMaxThr + 2];
  begins_from_counts(rl.pout_count, nco, cbo);
  FrontList fl;
  PRDF_TRY(front_list(g, p, s, &fl));
  PRDF_TRY(launch_expand(rl.out.off.p, rl.out.adj.p, rl.pout.p, cbo, nco, g->dN.p, g->dV.p, nullptr, Stop(), s,
                         nullptr, 0, fl));
  // reachability closure over G^t: the frontier starts as every affected vertex; each
  // round marks the vertices it reaches that were not yet affected, which form the
  // next frontier, until a round adds none (the affected count stops changing)
  long long kernels = (pout_made ? 5 : 0) + 1 + (n_del + n_ins > 0 ? 1 : 0) + nonempty_classes(cbo, nco) + (fl.list ? 2 : 0);
  PRDF_CUDA(cudaMemcpyAsync(g->dN.p, g->dV.p, (size_t)n, cudaMemcpyDeviceToDevice, s));
  uint8_t* front = g->dN.p;
  uint8_t* next = g->dF.p;
  for (int round = 0; round < n; ++round) {
    PRDF_CUDA(cudaMemsetAsync(next, 0, (size_t)n, s));
    PRDF_TRY(launch_expand(rl.out.off.p, rl.out.adj.p, rl.pout.p, cbo, nco, front, g->dV.p, next, Stop(), s, nullptr,
                           0, fl));
    PRDF_TRY(count_flags(next, n, g->counter.p, s));
    kernels += nonempty_classes(cbo, nco) + 1 + (fl.list ? 2 : 0);
    unsigned long long added = 0;
    PRDF_CUDA(cudaMemcpyAsync(&added, g->counter.p, sizeof(added), cudaMemcpyDeviceToHost, s));
    PRDF_CUDA(cudaStreamSynchronize(s));
    if (added == 0) break;
    uint8_t* tmp = front;
    front = next;
    next = tmp;
  }
  PRDF_TRY(count_flags(g->dV.p, n, g->counter.p, s));
  PRDF_CUDA(cudaEventRecord(t.e[2], s));
  PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64 + 8, g->counter.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  // Eq. 1 on the affected vertices, no prune and no expansion (FP32 stage first in mixed precision)
  prdf_params q = *p;
  q.prune = 0;
  q.tau_f = INFINITY;
  IterResult it, it32;
  if (p->precision == PRDF_FP32_REFINE) {
    PRDF_TRY(dynamic_fp32_stage(g, &q, prev_ranks, false, &it32, s));
    q.max_iter = p->max_iter - it32.iters > 0 ? p->max_iter - it32.iters : 1;
    kernels += it32.kernels + 3;
  }
  PRDF_TRY(run_loop(g, &q, false, true, false, q.max_iter, &it, s));  // synchronises the stream
  const long long aff = (long long)g->ws.host_i64[8];
  k_finalize<<<grid_for(n, kThreads), kThreads, 0, s>>>(it.final_buf ? g->xb.p : g->xa.p, rl.degd.p, rl.perm.p, n,
                                                       ranks, g->dV.p, dV_out);
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaEventRecord(t.e[3], s));
  PRDF_CUDA(cudaEventSynchronize(t.e[3]));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iterations = it.iters + it32.iters;
    stats->iterations_fp32 = it32.iters;
    stats->converged = it.converged;
    stats->final_delta = it.final_delta;
    stats->sweeps_launched = it.launched + it32.launched;
    cudaEventElapsedTime(&stats->ms_total, t.e[0], t.e[3]);
    cudaEventElapsedTime(&stats->ms_partition, t.e[0], t.e[1]);
    cudaEventElapsedTime(&stats->ms_mark, t.e[1], t.e[2]);
    cudaEventElapsedTime(&stats->ms_iterate, t.e[2], t.e[3]);
    stats->ms_sweep = it.ms_sweep + it32.ms_sweep;
    stats->edges_processed = -1;
    stats->affected_initial = aff;
    stats->kernel_launches = kernels + 1 + it.kernels + 1;
  }
  return PRDF_OK;
}

int prdf_pagerank_ppr(prdf_graph* g, const double* S, int K, double* R, const prdf_params* p, prdf_stats* stats) {
  if (!g || !S || !R) {
    set_error("prdf_pagerank_ppr: bad arguments");
    return PRDF_EINVAL;
  }
  if (K < 1) {
    set_error("prdf_pagerank_ppr: K must be >= 1");
    return PRDF_EINVAL;
  }
  if (!g->weighted) {
    set_error("prdf_pagerank_ppr: the graph has no edge weights");
    return PRDF_ESTATE;
  }
  PRDF_TRY(check_params(p));
  if (p->tile != 0 && p->tile != 8 && p->tile != 16 && p->tile != 32 && p->tile != 64) {
    set_error("prdf_pagerank_ppr: tile must be 0, 8, 16, 32 or 64");
    return PRDF_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)p->stream;
  Timer t;
  PRDF_TRY(t.init());
  PRDF_CUDA(cudaEventRecord(t.e[0], s));
  PRDF_TRY(ensure_relabelled(g, false, s));
  if (!g->ppr_valid) PRDF_TRY(build_ppr_weights(g, s));
  const int tile = p->tile ? p->tile : auto_tile(K);
  const int64_t cnt = (int64_t)g->n * K;
  PRDF_TRY(g->S64.reserve(cnt, s));
  PRDF_TRY(g->R64a.reserve(cnt, s));
  PRDF_TRY(g->R64b.reserve(cnt, s));
  k_rows_gather<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(S, g->rl.perm.p, g->n, K, g->S64.p);
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaEventRecord(t.e[1], s));
  PRDF_TRY(ensure_hub(g, g->rl.in, g->hub_in, s));
  const KOp op{g->rl.in.off.p, g->rl.in.adj.p, g->pin32.p, g->pin64.p, hub_begin(g->rl), &g->hub_in, g->S64.p, true,
               8};
  KSolve ks;
  ks.kernels = 1;
  double* Rfinal = nullptr;
  PRDF_TRY(ksolve(g, op, p, K, tile, &Rfinal, &ks, s));
  long long kernels = ks.kernels;
  const int iters32 = ks.iters32, steps64 = ks.steps64, conv = ks.converged;
  const double dmax = ks.dmax;
  k_rows_scatter<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(Rfinal, g->rl.perm.p, g->n, K, R);
  PRDF_LAUNCH_CHECK();
  kernels += 1;
  PRDF_CUDA(cudaEventRecord(t.e[2], s));
  PRDF_CUDA(cudaEventSynchronize(t.e[2]));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iterations = steps64 + iters32;
    stats->iterations_fp32 = iters32;
    stats->converged = conv;
    stats->final_delta = dmax;
    cudaEventElapsedTime(&stats->ms_total, t.e[0], t.e[2]);
    cudaEventElapsedTime(&stats->ms_partition, t.e[0], t.e[1]);
    cudaEventElapsedTime(&stats->ms_iterate, t.e[1], t.e[2]);
    stats->edges_processed = (long long)(steps64 + iters32) * g->rl.in.m * K;
    stats->kernel_launches = kernels;
  }
  return PRDF_OK;
}

int prdf_graph_set_weights(prdf_graph* g, const float* w, void* stream) {
  if (!g || !w) {
    set_error("prdf_graph_set_weights: bad arguments");
    return PRDF_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  PRDF_TRY(ensure_orig(g, s));  // w is given in the original out-CSR's slot order
  Csr& o = g->csr[PRDF_OUT];
  Csr& in = g->csr[PRDF_IN];
  DBuf<float> wo, wi;
  PRDF_TRY(wo.alloc(o.m > 0 ? (size_t)o.m : 1, s));
  PRDF_TRY(wi.alloc(in.m > 0 ? (size_t)in.m : 1, s));
  DBuf<int> bad;
  PRDF_TRY(bad.alloc(1, s));
  PRDF_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  PRDF_CUDA(cudaMemcpyAsync(wo.p, w, sizeof(float) * (size_t)o.m, cudaMemcpyDeviceToDevice, s));
  k_weights_to_in<<<grid_for((int64_t)g->n * 32, kThreads), kThreads, 0, s>>>(o.off.p, o.adj.p, w, g->n, in.off.p,
                                                                               in.adj.p, wi.p, bad.p);
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaMemcpyAsync(g->ws.host_i64, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  if (*(int*)g->ws.host_i64) {
    set_error("edge weights must be finite and > 0");
    return PRDF_EINVAL;
  }
  o.w = static_cast<DBuf<float>&&>(wo);
  in.w = static_cast<DBuf<float>&&>(wi);
  g->weighted = true;
  PRDF_TRY(build_relabelled(g, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  return PRDF_OK;
}

int prdf_pagerank_backward(prdf_graph* g, const double* R, const double* G, int K, double* grad_S, double* grad_w,
                           const prdf_params* p, prdf_stats* stats) {
  if (!g || !G || (grad_w && !R)) {
    set_error("prdf_pagerank_backward: bad arguments");
    return PRDF_EINVAL;
  }
  if (K < 1) {
    set_error("prdf_pagerank_backward: K must be >= 1");
    return PRDF_EINVAL;
  }
  if (!g->weighted) {
    set_error("prdf_pagerank_backward: the graph has no edge weights");
    return PRDF_ESTATE;
  }
  PRDF_TRY(check_params(p));
  if (p->tile != 0 && p->tile != 8 && p->tile != 16 && p->tile != 32 && p->tile != 64) {
    set_error("prdf_pagerank_backward: tile must be 0, 8, 16, 32 or 64");
    return PRDF_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)p->stream;
  Timer t;
  PRDF_TRY(t.init());
  PRDF_CUDA(cudaEventRecord(t.e[0], s));
  PRDF_TRY(ensure_relabelled(g, false, s));
  if (!g->ppr_valid) PRDF_TRY(build_ppr_weights(g, s));
  const int tile = p->tile ? p->tile : auto_tile(K);
  const int64_t cnt = (int64_t)g->n * K;
  const double beta = 1.0 - p->alpha;
  PRDF_TRY(g->S64.reserve(cnt, s));
  PRDF_TRY(g->R64a.reserve(cnt, s));
  PRDF_TRY(g->R64b.reserve(cnt, s));
  // lambda = alpha P lambda + G, i.e. X = alpha A X + (1 - alpha) * G / (1 - alpha) over the out-CSR
  k_rows_gather_scaled<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(G, g->rl.perm.p, g->n, K, 1.0 / beta, g->S64.p);
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaEventRecord(t.e[1], s));
  PRDF_TRY(ensure_hub(g, g->rl.out, g->hub_out, s));
  const KOp op{g->rl.out.off.p, g->rl.out.adj.p, g->pout32.p, g->pout64.p, hub_begin(g->rl), &g->hub_out, g->S64.p,
               false, 12};
  KSolve ks;
  ks.kernels = 1;
  double* lam = nullptr;
  PRDF_TRY(ksolve(g, op, p, K, tile, &lam, &ks, s));
  if (grad_S) {
    k_rows_scatter<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(lam, g->rl.perm.p, g->n, K, grad_S, beta);
    PRDF_LAUNCH_CHECK();
    ks.kernels += 1;
  }
  if (grad_w) {
    PRDF_TRY(ensure_orig(g, s));  // grad_w is written in the original out-CSR's slot order
    double* Rr = (lam == g->R64a.p) ? g->R64b.p : g->R64a.p;
    k_rows_gather_scaled<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(R, g->rl.perm.p, g->n, K, 1.0, Rr);
    PRDF_LAUNCH_CHECK();
    PRDF_TRY(launch_grad_w(g->rl.out.off.p, g->rl.out.adj.p, g->rl.perm.p, g->csr[PRDF_OUT].off.p, lam, g->S64.p, beta,
                           Rr, g->wsum.p, g->n, K, p->alpha, grad_w, s));
    ks.kernels += 2;
  }
  PRDF_CUDA(cudaEventRecord(t.e[2], s));
  PRDF_CUDA(cudaEventSynchronize(t.e[2]));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iterations = ks.steps64 + ks.iters32;
    stats->iterations_fp32 = ks.iters32;
    stats->converged = ks.converged;
    stats->final_delta = ks.dmax;
    cudaEventElapsedTime(&stats->ms_total, t.e[0], t.e[2]);
    cudaEventElapsedTime(&stats->ms_partition, t.e[0], t.e[1]);
    cudaEventElapsedTime(&stats->ms_iterate, t.e[1], t.e[2]);
    stats->kernel_launches = ks.kernels;
  }
  return PRDF_OK;
}

int prdf_autotune(prdf_graph* g, const prdf_params* p, int sweeps, int* best_index, float* best_ms_per_sweep) {
  if (!g || sweeps < 1) {
    set_error("prdf_autotune: bad arguments");
    return PRDF_EINVAL;
  }
  PRDF_TRY(check_params(p));
  // candidate in-degree class thresholds (the sweep numbering is rebuilt for each)
  static const int64_t cand[][8] = {
      {6, 1, 4, 16, 32, 128, 4096}, {5, 1, 4, 16, 128, 4096},   {6, 1, 4, 16, 64, 128, 4096},
      {6, 1, 4, 8, 32, 128, 2048},  {6, 1, 4, 16, 32, 256, 8192}, {4, 1, 4, 32, 1024},
      {3, 1, 16, 4096},             {2, 16, 2048}};
  const int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
  cudaStream_t s = (cudaStream_t)p->stream;
  DBuf<double> R;
  PRDF_TRY(R.alloc((size_t)g->n, s));
  prdf_params q = *p;
  q.max_iter = sweeps;
  q.tol = 1e-300;  // run exactly `sweeps` sweeps
  q.precision = PRDF_FP64;
  q.time_sweeps = 0;
  int best = 0;
  float best_ms = 0;
  for (int c = 0; c < ncand; ++c) {
    PRDF_TRY(prdf_graph_set_thresholds(g, PRDF_IN, (int)cand[c][0], &cand[c][1]));
    prdf_stats st;
    PRDF_TRY(prdf_pagerank_static(g, &q, nullptr, R.p, &st));  // builds numbering and graph
    PRDF_TRY(prdf_pagerank_static(g, &q, nullptr, R.p, &st));  // timed
    const float ms = st.ms_iterate / (float)st.iterations;
    if (c == 0 || ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  PRDF_TRY(prdf_graph_set_thresholds(g, PRDF_IN, (int)cand[best][0], &cand[best][1]));
  PRDF_TRY(ensure_relabelled(g, false, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  if (best_index) *best_index = best;
  if (best_ms_per_sweep) *best_ms_per_sweep = best_ms;
  return PRDF_OK;
}

int prdf_autotune_tile(prdf_graph* g, const double* S, int K, const prdf_params* p, int sweeps, int* best_tile) {
  if (!g || !S || K < 1 || sweeps < 1 || !best_tile) {
    set_error("prdf_autotune_tile: bad arguments");
    return PRDF_EINVAL;
  }
  if (!g->weighted) {
    set_error("prdf_autotune_tile: the graph has no edge weights");
    return PRDF_ESTATE;
  }
  PRDF_TRY(check_params(p));
  cudaStream_t s = (cudaStream_t)p->stream;
  DBuf<double> R;
  PRDF_TRY(R.alloc((size_t)g->n * K, s));
  prdf_params q = *p;
  q.precision = PRDF_FP64;
  q.max_iter = sweeps;
  q.tol = 1e-300;
  const int tiles[4] = {8, 16, 32, 64};
  float best_ms = 0;
  *best_tile = 32;
  for (int i = 0; i < 4; ++i) {
    if (tiles[i] > 2 * K && i > 0) break;
    q.tile = tiles[i];
    prdf_stats st;
    PRDF_TRY(prdf_pagerank_ppr(g, S, K, R.p, &q, &st));
    PRDF_TRY(prdf_pagerank_ppr(g, S, K, R.p, &q, &st));
    if (i == 0 || st.ms_iterate < best_ms) {
      best_ms = st.ms_iterate;
      *best_tile = tiles[i];
    }
  }
  return PRDF_OK;
}

}  // extern "C"
