// Class-contiguous vertex numbering for the rank sweep.
//
// The in-degree partition P (Alg. partition) lists the vertices of each
// degree class together. The sweep runs on a copy of the graph renumbered by
// that list: new id i is vertex P[i]. Every class then occupies a contiguous
// id range, so the per-vertex arrays (offsets, degrees, ranks) stream
// sequentially within a class and the kernels need no list indirection.
// Within a row the mapped neighbour ids keep the original row order; the
// exact accumulation makes the result independent of that order, so ranks
// are bit-identical to a sweep on the original numbering.
#include "internal.cuh"

namespace prdf {

namespace {

constexpr int kThreads = 256;

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

// new row i = old row perm[i], neighbour ids mapped through inv; one warp per row
__global__ void k_perm_rows(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ inv, int32_t n,
                            const int64_t* __restrict__ noff, int32_t* __restrict__ nadj) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int32_t v = perm[i];
    const int64_t b = off[v], L = off[v + 1] - b, o = noff[i];
    for (int64_t j = lane; j < L; j += 32) nadj[o + j] = inv[adj[b + j]];
  }
}

__global__ void k_perm_degrees(const double* __restrict__ deg, const double* __restrict__ inv_deg,
                               const int32_t* __restrict__ perm, int32_t n, double* __restrict__ ndeg,
                               double* __restrict__ ninv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = perm[i];
    ndeg[i] = deg[v];
    ninv[i] = inv_deg[v];
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
  k_perm_rows<<<grid_for((int64_t)n * 32, kThreads), kThreads, 0, s>>>(src.off.p, src.adj.p, perm, inv, n, dst.off.p,
                                                                        dst.adj.p);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

}  // namespace

int build_relabelled(prdf_graph* g, cudaStream_t s) {
  const int32_t n = g->n;
  Relabel& r = g->rl;
  // the in-degree partition defines the numbering and the class ranges
  PRDF_TRY(r.perm.alloc((size_t)n, s));
  PRDF_TRY(partition_by_degree(g->csr[PRDF_IN].off.p, n, g->thr[PRDF_IN], r.perm.p, r.count, g->ws, s));
  r.thr = g->thr[PRDF_IN];
  PRDF_TRY(r.inv.alloc((size_t)n, s));
  k_inverse_perm<<<grid_for(n, kThreads), kThreads, 0, s>>>(r.perm.p, n, r.inv.p);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(permute_csr(g->csr[PRDF_IN], r.perm.p, r.inv.p, n, r.in, g->ws, s));
  PRDF_TRY(permute_csr(g->csr[PRDF_OUT], r.perm.p, r.inv.p, n, r.out, g->ws, s));
  PRDF_TRY(r.degd.alloc((size_t)n, s));
  PRDF_TRY(r.inv_deg.alloc((size_t)n, s));
  k_perm_degrees<<<grid_for(n, kThreads), kThreads, 0, s>>>(g->outdeg.p, g->inv_outdeg.p, r.perm.p, n, r.degd.p,
                                                            r.inv_deg.p);
  PRDF_LAUNCH_CHECK();
  r.valid = true;
  r.pout_valid = false;
  return PRDF_OK;
}

}  // namespace prdf
