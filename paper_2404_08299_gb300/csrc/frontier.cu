// Affected-vertex marking (Alg. affected, Appendix A.3 of arXiv 2404.08299):
// initialAffected over the batch, expandAffected over the out-degree
// partition of G with thread-, sub-warp- and warp-per-vertex kernels, and
// 16 blocks per row for the highest class. Flags are uint8; every store writes 1, so concurrent marks of the
// same vertex need no atomics, and a flag already set is not stored again.
// With a third flag array dF the same kernels are one round of the
// reachability closure of Dynamic Traversal (Alg. traversal): a vertex that
// was not yet affected is marked in dV and in dF (the next frontier).
#include "internal.cuh"

namespace prdf {

namespace {

constexpr int kThreads = 256;
constexpr int kExpandSlices = 16;  // blocks sharing one row of the highest out-degree class

__global__ void k_initial_affected(const int32_t* __restrict__ del_src, const int32_t* __restrict__ del_dst,
                                   const uint8_t* __restrict__ del_mask, int64_t n_del,
                                   const int32_t* __restrict__ ins_src, const uint8_t* __restrict__ ins_mask,
                                   int64_t n_ins, const int32_t* __restrict__ map, uint8_t* __restrict__ dV,
                                   uint8_t* __restrict__ dN) {
  const int64_t tot = n_del + n_ins;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n_del) {
      if (del_mask && !del_mask[i]) continue;
      const int32_t u = del_src[i], v = del_dst[i];
      dN[map ? map[u] : u] = 1;  // out-neighbours of the source are affected
      dV[map ? map[v] : v] = 1;  // the target is affected
    } else {
      const int64_t k = i - n_del;
      if (ins_mask && !ins_mask[k]) continue;
      const int32_t u = ins_src[k];
      dN[map ? map[u] : u] = 1;
    }
  }
}

// The sweep this round follows already met its loop's stop rule: the round does nothing.
__device__ __forceinline__ bool converged(const Stop& st) {
  const int it = st.ctl ? st.ctl[0] : 0;
  if (st.r64) return bitsd(st.r64[it]) <= st.tol;
  if (st.r32) {
    const uint32_t* r = st.r32 + 2 * it;
    return __uint_as_float(r[0]) <= st.tol_rel * __uint_as_float(r[1]);
  }
  return false;
}

// this round's frontier out-edge counter (one per sweep; the graph-driven loop indexes it by ctl[0])
__device__ __forceinline__ const unsigned long long* round_fw(const unsigned long long* fw, const Stop& st) {
  return fw ? fw + (st.ctl ? st.ctl[0] : 0) : nullptr;
}

// Direction of one expansion round, chosen on the device: the pull form when
// the frontier's out-edges (*fw) exceed fthr, else the push form.
__device__ __forceinline__ bool pull_chosen(const unsigned long long* fw, unsigned long long fthr) {
  return fw && *fw > fthr;
}

// Pull form of one expansion round over G' (the same marks as the push form,
// since w is an out-neighbour of u exactly when u is an in-neighbour of w): a
// vertex outside dV joins it when an in-neighbour is in the frontier. Only
// w's own thread (or warp) reads or writes dV[w]; the scan stops at the first
// frontier in-neighbour.
__global__ void __launch_bounds__(kThreads) k_pull_thread(const int64_t* __restrict__ off,
                                                          const int32_t* __restrict__ adj, int64_t begin, int64_t end,
                                                          const uint8_t* __restrict__ dN, uint8_t* __restrict__ dV,
                                                          const unsigned long long* fw, unsigned long long fthr,
                                                          const Stop st) {
  if (converged(st) || !pull_chosen(round_fw(fw, st), fthr)) return;
  for (int64_t w = begin + blockIdx.x * (int64_t)kThreads + threadIdx.x; w < end; w += (int64_t)gridDim.x * kThreads) {
    if (dV[w]) continue;
    const int64_t e = off[w + 1];
    for (int64_t j = off[w]; j < e; ++j)
      if (dN[adj[j]]) {
        dV[w] = 1;
        break;
      }
  }
}

__global__ void __launch_bounds__(kThreads) k_pull_warp(const int64_t* __restrict__ off,
                                                        const int32_t* __restrict__ adj, int64_t begin, int64_t end,
                                                        const uint8_t* __restrict__ dN, uint8_t* __restrict__ dV,
                                                        const unsigned long long* fw, unsigned long long fthr,
                                                        const Stop st) {
  if (converged(st) || !pull_chosen(round_fw(fw, st), fthr)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t w = begin + warp; w < end; w += nwarps) {
    if (dV[w]) continue;  // the same value on every lane
    const int64_t b = off[w], e = off[w + 1];
    for (int64_t j0 = b; j0 < e; j0 += 32) {
      const int64_t j = j0 + lane;
      const bool hit = j < e && dN[adj[j]];
      if (__any_sync(0xffffffffu, hit)) {
        if (lane == 0) dV[w] = 1;
        break;
      }
    }
  }
}

// Mark the targets of edges [j0, e) of one row, `step` apart, kU per lane in
// flight: the index loads of a round issue together, then their flag loads.
template <int kU>
__device__ __forceinline__ void mark_targets(const int32_t* __restrict__ adj, int64_t j0, int64_t e, int step,
                                             uint8_t* __restrict__ dV, uint8_t* __restrict__ dF) {
  for (; j0 < e; j0 += (int64_t)step * kU) {
    int32_t w[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      const int64_t j = j0 + (int64_t)k * step;
      w[k] = j < e ? adj[j] : -1;
    }
    uint8_t f[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) f[k] = w[k] >= 0 ? dV[w[k]] : (uint8_t)1;
#pragma unroll
    for (int k = 0; k < kU; ++k)
      if (!f[k]) {  // most targets are already marked when the frontier is large
        dV[w[k]] = 1;
        if (dF) dF[w[k]] = 1;
      }
  }
}

constexpr int kExpandU = 4;

// the frontier was listed (at most cap vertices) and expanded from the list
__device__ __forceinline__ bool listed(const unsigned int* cnt, unsigned int cap) { return cnt && *cnt <= cap; }

template <int G>
__global__ void __launch_bounds__(kThreads) k_expand_group(const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ adj,
                                                           const int32_t* __restrict__ P, int64_t begin, int64_t end,
                                                           const uint8_t* __restrict__ dN, uint8_t* __restrict__ dV,
                                                           uint8_t* __restrict__ dF, const Stop st,
                                                           const unsigned long long* fw, unsigned long long fthr,
                                                           const unsigned int* lcnt, unsigned int cap) {
  if (converged(st) || pull_chosen(round_fw(fw, st), fthr) || listed(lcnt, cap)) return;
  const int lane = (G == 1) ? 0 : (threadIdx.x & (G - 1));
  const int64_t gid = (blockIdx.x * (int64_t)kThreads + threadIdx.x) / G;
  const int64_t ng = ((int64_t)gridDim.x * kThreads) / G;
  for (int64_t i = begin + gid; i < end; i += ng) {
    const int32_t u = P[i];
    if (!dN[u]) continue;
    mark_targets<kExpandU>(adj, off[u] + lane, off[u + 1], G, dV, dF);
  }
}

// highest out-degree class: blockIdx.y picks one of gridDim.y equal slices of
// each row, so the longest rows are spread over that many blocks
__global__ void __launch_bounds__(kThreads) k_expand_block(const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ adj,
                                                           const int32_t* __restrict__ P, int64_t begin, int64_t end,
                                                           const uint8_t* __restrict__ dN, uint8_t* __restrict__ dV,
                                                           uint8_t* __restrict__ dF, const Stop st,
                                                           const unsigned long long* fw, unsigned long long fthr,
                                                           const unsigned int* lcnt, unsigned int cap) {
  if (converged(st) || pull_chosen(round_fw(fw, st), fthr) || listed(lcnt, cap)) return;
  const int64_t S = gridDim.y, y = blockIdx.y;
  for (int64_t i = begin + blockIdx.x; i < end; i += gridDim.x) {
    const int32_t u = P[i];
    if (!dN[u]) continue;
    const int64_t b = off[u], len = off[u + 1] - b;
    const int64_t span = (len + S - 1) / S;
    const int64_t sb = b + y * span;
    const int64_t se = sb + span < b + len ? sb + span : b + len;
    mark_targets<kExpandU>(adj, sb + threadIdx.x, se, kThreads, dV, dF);
  }
}

// Small frontiers. The class kernels above find the frontier by reading dN
// through the out-degree partition: n scattered byte loads per round however
// few vertices are in it. k_frontier_list lists the frontier instead (a
// coalesced read of dN, warp-aggregated appends) while it holds at most cap
// vertices, and k_expand_list gives each listed vertex a block; the class
// kernels then return at once. Past cap the list is abandoned (only counted)
// and the class kernels run as before. The marks are the same either way.
__global__ void __launch_bounds__(kThreads) k_frontier_list(const uint8_t* __restrict__ dN, int64_t n,
                                                            int32_t* __restrict__ list, unsigned int* __restrict__ cnt,
                                                            unsigned int cap, const Stop st,
                                                            const unsigned long long* fw, unsigned long long fthr) {
  if (converged(st) || pull_chosen(round_fw(fw, st), fthr)) return;
  const int lane = threadIdx.x & 31;
  const int64_t nw = n >> 2;  // whole 4-flag words; the tail is read by thread 0
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t base = i0 - lane; base < nw; base += stride) {  // warp-uniform trip count
    const int64_t i = base + lane;
    uint32_t word = 0;
    if (i < nw) word = reinterpret_cast<const uint32_t*>(dN)[i];
    int c = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) c += ((word >> (8 * q)) & 0xFFu) ? 1 : 0;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) continue;
    unsigned int wbase = 0;
    if (lane == 31) wbase = atomicAdd(cnt, (unsigned int)total);
    wbase = __shfl_sync(0xffffffffu, wbase, 31);
    unsigned int pos = wbase + (unsigned int)(incl - c);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if ((word >> (8 * q)) & 0xFFu) {
        if (pos < cap) list[pos] = (int32_t)(4 * i + q);
        ++pos;
      }
  }
  if (i0 == 0)
    for (int64_t v = nw << 2; v < n; ++v)
      if (dN[v]) {
        const unsigned int pos = atomicAdd(cnt, 1u);
        if (pos < cap) list[pos] = (int32_t)v;
      }
}

__global__ void __launch_bounds__(kThreads) k_expand_list(const int64_t* __restrict__ off,
                                                          const int32_t* __restrict__ adj,
                                                          const int32_t* __restrict__ list,
                                                          const unsigned int* __restrict__ cnt, unsigned int cap,
                                                          uint8_t* __restrict__ dV, uint8_t* __restrict__ dF,
                                                          const Stop st, const unsigned long long* fw,
                                                          unsigned long long fthr) {
  if (converged(st) || pull_chosen(round_fw(fw, st), fthr)) return;
  const unsigned int c = *cnt;
  if (c > cap) return;
  for (unsigned int k = blockIdx.x; k < c; k += gridDim.x) {
    const int32_t u = list[k];
    mark_targets<kExpandU>(adj, off[u] + threadIdx.x, off[u + 1], kThreads, dV, dF);
  }
}

__global__ void k_count_flags(const uint8_t* __restrict__ f, int64_t n, unsigned long long* __restrict__ out) {
  int64_t c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += f[i] ? 1 : 0;
  c = warp_sum_i64(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, (unsigned long long)c);
}

}  // namespace

int launch_initial_affected(const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask, int64_t n_del,
                            const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins, const int32_t* map,
                            uint8_t* dV, uint8_t* dN, cudaStream_t s) {
  if (n_del + n_ins == 0) return PRDF_OK;
  k_initial_affected<<<grid_for(n_del + n_ins, kThreads), kThreads, 0, s>>>(del_src, del_dst, del_mask, n_del, ins_src,
                                                                             ins_mask, n_ins, map, dV, dN);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int launch_expand(const int64_t* off, const int32_t* adj, const int32_t* P, const int64_t* cb, int nclass,
                  const uint8_t* dN, uint8_t* dV, uint8_t* dF, const Stop& st, cudaStream_t s,
                  const unsigned long long* fw, unsigned long long fthr, const FrontList& fl) {
  const int maxg = kSMs * 8;
  const unsigned int* lcnt = fl.list ? fl.cnt : nullptr;
  if (fl.list) {
    const int64_t n = cb[nclass];
    PRDF_CUDA(cudaMemsetAsync(fl.cnt, 0, sizeof(unsigned int), s));
    k_frontier_list<<<grid_for(n / 4 + 1, kThreads, kSMs * 4), kThreads, 0, s>>>(dN, n, fl.list, fl.cnt, fl.cap, st,
                                                                                fw, fthr);
    k_expand_list<<<kSMs * 8, kThreads, 0, s>>>(off, adj, fl.list, fl.cnt, fl.cap, dV, dF, st, fw, fthr);
  }
  for (int c = 0; c < nclass; ++c) {
    const int64_t b = cb[c], e = cb[c + 1];
    if (e <= b) continue;
    const int64_t cnt = e - b;
    const int kind = (nclass == 4) ? c : (c == nclass - 1 ? 3 : c);
    switch (kind) {
      case 0: k_expand_group<1><<<grid_for(cnt, kThreads, maxg), kThreads, 0, s>>>(off, adj, P, b, e, dN, dV, dF, st, fw, fthr, lcnt, fl.cap); break;
      case 1: k_expand_group<8><<<grid_for(cnt * 8, kThreads, maxg), kThreads, 0, s>>>(off, adj, P, b, e, dN, dV, dF, st, fw, fthr, lcnt, fl.cap); break;
      case 2: k_expand_group<32><<<grid_for(cnt * 32, kThreads, maxg), kThreads, 0, s>>>(off, adj, P, b, e, dN, dV, dF, st, fw, fthr, lcnt, fl.cap); break;
      default: {
        const dim3 grid(grid_for(cnt, 1, maxg / kExpandSlices), kExpandSlices);
        k_expand_block<<<grid, kThreads, 0, s>>>(off, adj, P, b, e, dN, dV, dF, st, fw, fthr, lcnt, fl.cap);
        break;
      }
    }
  }
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int launch_expand_pull(const int64_t* in_off, const int32_t* in_adj, int64_t n, int64_t warp_begin,
                       const uint8_t* dN, uint8_t* dV, const unsigned long long* fw, unsigned long long fthr,
                       const Stop& st, cudaStream_t s) {
  const int maxg = kSMs * 8;
  if (warp_begin > 0)
    k_pull_thread<<<grid_for(warp_begin, kThreads, maxg), kThreads, 0, s>>>(in_off, in_adj, 0, warp_begin, dN, dV, fw,
                                                                            fthr, st);
  if (n > warp_begin)
    k_pull_warp<<<grid_for((n - warp_begin) * 32, kThreads, maxg), kThreads, 0, s>>>(in_off, in_adj, warp_begin, n,
                                                                                      dN, dV, fw, fthr, st);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int count_flags(const uint8_t* f, int64_t n, unsigned long long* dev_out, cudaStream_t s) {
  PRDF_CUDA(cudaMemsetAsync(dev_out, 0, sizeof(unsigned long long), s));
  k_count_flags<<<grid_for(n, kThreads, kSMs * 4), kThreads, 0, s>>>(f, n, dev_out);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

}  // namespace prdf
