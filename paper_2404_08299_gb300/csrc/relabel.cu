// Class-contiguous vertex numbering for the rank sweep.
//
// The in-degree partition P (Alg. partition) lists the vertices of each
// degree class together. The sweep runs on a copy of the graph renumbered by
// that list: new id i is vertex P[i]. Every class then occupies a contiguous
// id range, so the per-vertex arrays (offsets, degrees, ranks) stream
// sequentially within a class and the kernels need no list indirection.
// Within a class, vertices are ordered by out-degree tier, highest first:
// the sources gathered most often sit together, so their x values share
// cache lines and stay in L1 / L2 (the sweep is bound by the rate of L1
// misses of its random gathers, not by HBM bandwidth).
// Within a row the mapped neighbour ids keep the original row order; the
// exact accumulation makes the result independent of that order, so ranks
// are bit-identical to a sweep on the original numbering.
#include "internal.cuh"

namespace prdf {

namespace {

constexpr int kThreads = 256;
// out-degree tiers of the numbering inside each in-degree class
constexpr int kOutTiers = 7;
constexpr int64_t kOutTierThr[kOutTiers] = {8, 32, 128, 512, 2048, 8192, 32768};

__global__ void k_inverse_perm(const int32_t* __restrict__ perm, int32_t n, int32_t* __restrict__ inv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    inv[perm[i]] = (int32_t)i;
}

__global__ void k_perm_rowlen(const int64_t* __restrict__ off, const int32_t* __restrict__ perm, int32_t n,
                              int64_t* __restrict__ len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = perm[i];
    len[i] = off[v + 1] - off[v];
  }
}

// new row i = old row perm[i], neighbour ids mapped through inv (weights
// carried along when present). Balanced by entries, not rows: a warp takes
// kPermChunk consecutive entries of the new CSR (lane-strided, so stores stay
// coalesced), finds the row of the first one by binary search, and each lane
// walks rows forward for its own entries (a few steps, then a binary search
// past runs of empty rows). Long rows spread over many warps, short rows pack
// densely.
constexpr int64_t kPermChunk = 1024;

__global__ void k_perm_rows(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            const float* __restrict__ w, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ inv, int32_t n, int64_t m, const int64_t* __restrict__ noff,
                            int32_t* __restrict__ nadj, float* __restrict__ nw) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p0 = warp * kPermChunk; p0 < m; p0 += nwarps * kPermChunk) {
    // row of entry p0: the last r with noff[r] <= p0
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (noff[mid] <= p0) lo = mid; else hi = mid;
    }
    int64_t r = lo, re = noff[r + 1], rs = noff[r];
    int64_t src = off[perm[r]];
    for (int64_t p = p0 + lane; p < p0 + kPermChunk && p < m; p += 32) {
      if (p >= re) {
        // a few steps forward, then a binary search past runs of empty rows
        int steps = 0;
        do {
          ++r;
          re = noff[r + 1];
        } while (p >= re && ++steps < 8);
        if (p >= re) {
          int64_t a = r, z = n;  // the last row with noff[row] <= p
          while (z - a > 1) {
            const int64_t mid = (a + z) >> 1;
            if (noff[mid] <= p) a = mid; else z = mid;
          }
          r = a;
          re = noff[r + 1];
        }
        rs = noff[r];
        src = off[perm[r]];
      }
      nadj[p] = inv[adj[src + (p - rs)]];
      if (w) nw[p] = w[src + (p - rs)];
    }
  }
}

// sum of out-weights per row, one warp per row
__global__ void k_row_wsum(const int64_t* __restrict__ off, const float* __restrict__ w, int32_t n,
                           double* __restrict__ W) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    double s = 0;
    for (int64_t j = off[v] + lane; j < off[v + 1]; j += 32) s += (double)w[j];
    s = warp_sum_f64(s);
    if (lane == 0) W[v] = s;
  }
}

// P on the in-slots of the renumbered G': slot (u -> v) gets w_uv / W[u]
// (new_src and W in the sweep numbering)
__global__ void k_pin(const int32_t* __restrict__ new_src, const float* __restrict__ w, const double* __restrict__ W,
                      int64_t m, double* __restrict__ p64, float* __restrict__ p32) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const double p = (double)w[j] / W[new_src[j]];
    p64[j] = p;
    p32[j] = (float)p;
  }
}

// P on the out-slots of the renumbered G: row i divides by its own W
__global__ void k_pout(const int64_t* __restrict__ off, const float* __restrict__ w, const double* __restrict__ W,
                       int32_t n, double* __restrict__ p64, float* __restrict__ p32) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const double Wi = W[i];
    for (int64_t j = off[i] + lane; j < off[i + 1]; j += 32) {
      const double p = (double)w[j] / Wi;
      p64[j] = p;
      p32[j] = (float)p;
    }
  }
}

// |out(i)| and 1 / |out(i)| from the row lengths of a CSR
__global__ void k_row_degrees(const int64_t* __restrict__ off, int32_t n, double* __restrict__ deg,
                              double* __restrict__ inv) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = off[v + 1] - off[v];
    deg[v] = (double)d;
    inv[v] = d > 0 ? 1.0 / (double)d : 0.0;
  }
}

int permute_csr(const Csr& src, const int32_t* perm, const int32_t* inv, int32_t n, Csr& dst, Workspace& ws,
                cudaStream_t s) {
  DBuf<int64_t> len;
  PRDF_TRY(len.alloc((size_t)n, s));
  k_perm_rowlen<<<grid_for(n, kThreads), kThreads, 0, s>>>(src.off.p, perm, n, len.p);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(dst.off.alloc((size_t)n + 1, s));
  PRDF_TRY(exclusive_scan_i64(len.p, n, dst.off.p, ws, s));
  dst.m = src.m;
  PRDF_TRY(dst.adj.alloc(src.m > 0 ? (size_t)src.m : 1, s));
  if (src.w.p) PRDF_TRY(dst.w.alloc(src.m > 0 ? (size_t)src.m : 1, s));
  else dst.w.release();
  if (src.m > 0)
    k_perm_rows<<<grid_for((src.m + kPermChunk - 1) / kPermChunk * 32, kThreads), kThreads, 0, s>>>(
        src.off.p, src.adj.p, src.w.p, perm, inv, n, src.m, dst.off.p, dst.adj.p, dst.w.p);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

// degrees (and the Eq. 2 factor when kf is not null) of the rows of the listed
// vertices (original ids, mapped through inv); duplicates write equal values
__global__ void k_row_degrees_of(const int32_t* __restrict__ a, int64_t cnt, const int32_t* __restrict__ inv,
                                 const int64_t* __restrict__ off, double alpha, double* __restrict__ deg,
                                 double* __restrict__ inv_deg, double* __restrict__ kf) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < cnt; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = inv[a[k]];
    const int64_t d = off[i + 1] - off[i];
    deg[i] = (double)d;
    inv_deg[i] = d > 0 ? 1.0 / (double)d : 0.0;
    if (kf) kf[i] = 1.0 / (1.0 - alpha / (double)d);
  }
}


}  // namespace

int ensure_orig(prdf_graph* g, cudaStream_t s) {
  if (g->orig_valid) return PRDF_OK;
  Relabel& r = g->rl;
  // original row u is row inv[u] of the numbering, its entries mapped back through perm
  PRDF_TRY(permute_csr(r.out, r.inv.p, r.perm.p, g->n, g->csr[PRDF_OUT], g->ws, s));
  PRDF_TRY(permute_csr(r.in, r.inv.p, r.perm.p, g->n, g->csr[PRDF_IN], g->ws, s));
  g->orig_valid = true;
  g->pvalid[0] = g->pvalid[1] = false;
  return PRDF_OK;
}

int update_degrees_of(prdf_graph* g, const int32_t* a, int64_t cnt, cudaStream_t s) {
  if (cnt <= 0) return PRDF_OK;
  Relabel& r = g->rl;
  double* kf = r.kf_alpha >= 0 ? r.kf.p : nullptr;
  k_row_degrees_of<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(a, cnt, r.inv.p, r.out.off.p, r.kf_alpha, r.degd.p,
                                                                 r.inv_deg.p, kf);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int update_degrees(prdf_graph* g, cudaStream_t s) {
  Relabel& r = g->rl;
  PRDF_TRY(r.degd.reserve((size_t)g->n, s));
  PRDF_TRY(r.inv_deg.reserve((size_t)g->n, s));
  k_row_degrees<<<grid_for(g->n, kThreads), kThreads, 0, s>>>(r.out.off.p, g->n, r.degd.p, r.inv_deg.p);
  PRDF_LAUNCH_CHECK();
  r.kf_alpha = -1;
  return PRDF_OK;
}

int build_relabelled(prdf_graph* g, cudaStream_t s) {
  const int32_t n = g->n;
  Relabel& r = g->rl;
  PRDF_TRY(ensure_orig(g, s));  // the numbering is made from the original-id CSRs
  // out-degree tiers first (highest first), then a stable in-degree partition
  // of that list: classes by in-degree, tiers inside each class
  DBuf<int32_t> hot;
  PRDF_TRY(hot.alloc((size_t)n, s));
  PartThr tiers;
  tiers.n = kOutTiers;
  for (int i = 0; i < kOutTiers; ++i) tiers.thr[i] = kOutTierThr[i];
  int64_t tier_count[kMaxThr + 1];
  PRDF_TRY(partition_list(g->csr[PRDF_OUT].off.p, nullptr, n, tiers, true, hot.p, tier_count, g->ws, s));
  PRDF_TRY(r.perm.alloc((size_t)n, s));
  PRDF_TRY(partition_list(g->csr[PRDF_IN].off.p, hot.p, n, g->thr[PRDF_IN], false, r.perm.p, r.count, g->ws, s));
  r.thr = g->thr[PRDF_IN];
  PRDF_TRY(r.inv.alloc((size_t)n, s));
  k_inverse_perm<<<grid_for(n, kThreads), kThreads, 0, s>>>(r.perm.p, n, r.inv.p);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(permute_csr(g->csr[PRDF_IN], r.perm.p, r.inv.p, n, r.in, g->ws, s));
  PRDF_TRY(permute_csr(g->csr[PRDF_OUT], r.perm.p, r.inv.p, n, r.out, g->ws, s));
  PRDF_TRY(update_degrees(g, s));
  PRDF_TRY(r.multi.reserve((size_t)n / 32 + 1, s));
  PRDF_CUDA(cudaMemsetAsync(r.multi.p, 0, sizeof(uint32_t) * ((size_t)n / 32 + 1), s));
  r.multi_count = 0;
  r.drift = 0;
  r.valid = true;
  // the out-degree partition of the marking kernels (Alg. partition over G) is
  // made with the numbering, so that DF / DF-P / DT find it ready after a batch
  PRDF_TRY(r.pout.reserve((size_t)n, s));
  PRDF_TRY(partition_by_degree(r.out.off.p, n, g->thr[PRDF_OUT], r.pout.p, r.pout_count, g->ws, s));
  r.pout_valid = true;
  ++r.version;
  g->ppr_valid = false;
  return PRDF_OK;
}

int build_ppr_weights(prdf_graph* g, cudaStream_t s) {
  const int32_t n = g->n;
  const Relabel& r = g->rl;
  const int64_t m = r.in.m;
  PRDF_TRY(g->wsum.alloc((size_t)n, s));
  // each row holds its vertex's entries in original-id order: the same sum as over the original CSR
  k_row_wsum<<<grid_for((int64_t)n * 32, kThreads), kThreads, 0, s>>>(r.out.off.p, r.out.w.p, n, g->wsum.p);
  PRDF_TRY(g->pin64.alloc((size_t)m, s));
  PRDF_TRY(g->pin32.alloc((size_t)m, s));
  PRDF_TRY(g->pout64.alloc((size_t)m, s));
  PRDF_TRY(g->pout32.alloc((size_t)m, s));
  k_pin<<<grid_for(m, kThreads), kThreads, 0, s>>>(r.in.adj.p, r.in.w.p, g->wsum.p, m, g->pin64.p, g->pin32.p);
  k_pout<<<grid_for((int64_t)n * 32, kThreads), kThreads, 0, s>>>(r.out.off.p, r.out.w.p, g->wsum.p, n,
                                                                   g->pout64.p, g->pout32.p);
  PRDF_LAUNCH_CHECK();
  g->ppr_valid = true;
  return PRDF_OK;
}

}  // namespace prdf
