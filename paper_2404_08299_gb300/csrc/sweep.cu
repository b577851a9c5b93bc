// Synchronous, pull-based, atomics-free rank sweeps (Alg. update of
// arXiv 2404.08299) for Static (Eq. 1, every vertex) and DF / DF-P
// (Eq. 1 / Eq. 2 on affected vertices, with prune and expand flags).
//
// State: x[u] = R[u] / |out(u)|, so a sweep gathers one FP64 value per
// in-edge. Each vertex v is processed by a group of G lanes (G = 1, 8, 32)
// or a whole block, chosen by in-degree class (the paper's thread-per-vertex
// and block-per-vertex kernels, with two middle classes added). The L-inf
// change of the sweep is reduced in the epilogue (warp max, block max, one
// 64-bit atomic max per block on the bit pattern of a non-negative double);
// rank writes stay one plain store per vertex.
//
// A sweep whose predecessor already met the tolerance exits at once, so the
// host can launch several sweeps ahead of its convergence check.
#include "internal.cuh"

namespace prdf {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 8;

template <bool EXACT>
struct Acc;

template <>
struct Acc<true> {
  fix128 v = 0;
  __device__ __forceinline__ void add(double x) { fix_add(v, x); }
  template <int G>
  __device__ __forceinline__ void group_reduce() {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)v, o);
      uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(v >> 64), o);
      v += ((fix128)hi << 64) | lo;
    }
  }
  __device__ __forceinline__ double value() const { return fix_to_double(v); }
  __device__ __forceinline__ void merge_raw(uint64_t lo, uint64_t hi) { v += ((fix128)hi << 64) | lo; }
  __device__ __forceinline__ uint64_t lo() const { return (uint64_t)v; }
  __device__ __forceinline__ uint64_t hi() const { return (uint64_t)(v >> 64); }
};

template <>
struct Acc<false> {
  double v = 0;
  __device__ __forceinline__ void add(double x) { v += x; }
  template <int G>
  __device__ __forceinline__ void group_reduce() {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __device__ __forceinline__ double value() const { return v; }
  __device__ __forceinline__ void merge_raw(uint64_t lo, uint64_t) { v += bitsd(lo); }
  __device__ __forceinline__ uint64_t lo() const { return dbits(v); }
  __device__ __forceinline__ uint64_t hi() const { return 0; }
};

// Per-lane gather over row [b, e) of G' with stride G and kUnroll loads in flight.
template <int G, bool EXACT>
__device__ __forceinline__ void gather_row(const SweepArgs& a, int64_t b, int64_t e, int lane, int32_t v,
                                           Acc<EXACT>& acc, double& xself, uint64_t pf, uint64_t pl) {
  for (int64_t j0 = b + lane; j0 < e; j0 += (int64_t)G * kUnroll) {
    int32_t u[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int64_t j = j0 + (int64_t)k * G;
      u[k] = j < e ? ld_stream_i32(a.adj + j, pf) : -1;
    }
    double xv[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) xv[k] = u[k] >= 0 ? ld_gather_f64(a.x + u[k], pl) : 0.0;
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      if (u[k] >= 0) acc.add(xv[k]);
      if (u[k] == v) xself = xv[k];
    }
  }
}

// Vectorised variant for a row handled by NT lanes: 16-byte index loads for
// the aligned body, scalar loads for the head and tail.
template <int NT, bool EXACT>
__device__ __forceinline__ void gather_row_vec(const SweepArgs& a, int64_t b, int64_t e, int lane, int32_t v,
                                               Acc<EXACT>& acc, double& xself, uint64_t pf, uint64_t pl) {
  int64_t ba = (b + 3) & ~(int64_t)3;
  if (ba > e) ba = e;
  const int64_t ea = ba + ((e - ba) & ~(int64_t)3);
  // head and tail: at most 3 + 3 scalar elements
  {
    const int64_t nh = ba - b, nt = e - ea;
    if (lane < nh) {
      const int32_t u = ld_stream_i32(a.adj + b + lane, pf);
      const double xv = ld_gather_f64(a.x + u, pl);
      acc.add(xv);
      if (u == v) xself = xv;
    } else if (lane >= 4 && lane < 4 + nt) {
      const int32_t u = ld_stream_i32(a.adj + ea + (lane - 4), pf);
      const double xv = ld_gather_f64(a.x + u, pl);
      acc.add(xv);
      if (u == v) xself = xv;
    }
  }
  constexpr int kV = 2;  // int4 loads in flight per lane
  for (int64_t q0 = ba + 4 * (int64_t)lane; q0 < ea; q0 += 4 * (int64_t)NT * kV) {
    int4 u4[kV];
#pragma unroll
    for (int k = 0; k < kV; ++k) {
      const int64_t q = q0 + 4 * (int64_t)NT * k;
      u4[k] = q < ea ? ld_stream_i32x4(a.adj + q, pf) : make_int4(-1, -1, -1, -1);
    }
    double xv[4 * kV];
#pragma unroll
    for (int k = 0; k < kV; ++k) {
      xv[4 * k + 0] = u4[k].x >= 0 ? ld_gather_f64(a.x + u4[k].x, pl) : 0.0;
      xv[4 * k + 1] = u4[k].y >= 0 ? ld_gather_f64(a.x + u4[k].y, pl) : 0.0;
      xv[4 * k + 2] = u4[k].z >= 0 ? ld_gather_f64(a.x + u4[k].z, pl) : 0.0;
      xv[4 * k + 3] = u4[k].w >= 0 ? ld_gather_f64(a.x + u4[k].w, pl) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < kV; ++k) {
      const int us[4] = {u4[k].x, u4[k].y, u4[k].z, u4[k].w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (us[t] >= 0) acc.add(xv[4 * k + t]);
        if (us[t] == v) xself = xv[4 * k + t];
      }
    }
  }
}

// Vertex epilogue: Eq. 1 (Static, DF) or Eq. 2 (DF-P), prune / expand flags,
// next x, and this vertex's |r - R[v]|.
template <bool DYN>
__device__ __forceinline__ uint64_t finish_vertex(const SweepArgs& a, int32_t v, double c, double xself) {
  const double d = (double)a.deg[v];
  const double rold = xself * d;  // R[v] of the previous iteration
  double r;
  if (DYN && a.prune) {
    // Eq. 2: the self-loop term is solved in closed form
    const double kf = 1.0 / (1.0 - a.alpha / d);
    r = kf * (a.c0 + a.alpha * (c - xself));
  } else {
    r = fma(a.alpha, c, a.c0);  // Eq. 1
  }
  const double dr = fabs(r - rold);
  if (DYN) {
    const double m = fmax(r, rold);
    if (a.prune && dr <= a.tau_p * m) a.dV[v] = 0;
    if (dr > a.tau_f * m) a.dN[v] = 1;
    a.wrote[v] = 1;
  }
  a.xn[v] = r * a.inv_deg[v];
  return dbits(dr);
}

// DF / DF-P: an unaffected vertex keeps its rank; its slot in xn is stale
// only if the previous sweep wrote it (then copy it through).
__device__ __forceinline__ bool skip_unaffected(const SweepArgs& a, int32_t v) {
  if (a.dV[v]) return false;
  if (a.wrote[v]) {
    a.xn[v] = a.x[v];
    a.wrote[v] = 0;
  }
  return true;
}

__device__ __forceinline__ void block_max_to(uint64_t dmax, uint64_t* out) {
  __shared__ uint64_t sh[32];
  dmax = warp_max_u64(dmax);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = dmax;
  __syncthreads();
  if (wid == 0) {
    uint64_t x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
    x = warp_max_u64(x);
    if (lane == 0 && x) atomicMax((unsigned long long*)out, (unsigned long long)x);
  }
}

// G lanes per vertex (G = 1, 8, 32). The loop is uniform across each warp
// (a warp owns 32/G consecutive list entries per step), so the group
// shuffles always see all 32 lanes.
template <int G, bool EXACT, bool DYN>
__global__ void __launch_bounds__(kThreads) k_sweep_group(const SweepArgs a, int64_t begin, int64_t end) {
  if (a.prev && bitsd(*a.prev) <= a.tol) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  constexpr int kGroupsPerWarp = 32 / G;
  const int lane = (G == 1) ? 0 : (threadIdx.x & (G - 1));
  const int gw = (threadIdx.x & 31) / G;  // group within warp
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  uint64_t dmax = 0;
  for (int64_t base = begin + warp * kGroupsPerWarp; base < end; base += nwarps * kGroupsPerWarp) {
    const int64_t i = base + gw;
    bool active = i < end;
    int32_t v = active ? a.P[i] : -1;
    if (DYN && active && skip_unaffected(a, v)) active = false;
    Acc<EXACT> acc;
    double xself = 0.0;
    if (active) {
      const int64_t b = a.off[v], e = a.off[v + 1];
      if (G == 32) gather_row_vec<32, EXACT>(a, b, e, lane, v, acc, xself, pf, pl);
      else gather_row<G, EXACT>(a, b, e, lane, v, acc, xself, pf, pl);
    }
    if (G > 1) {
      acc.template group_reduce<G>();
      uint64_t xb = dbits(xself);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        const uint64_t t = __shfl_xor_sync(0xffffffffu, xb, o);
        xb = t > xb ? t : xb;
      }
      xself = bitsd(xb);
    }
    if (active && lane == 0) {
      const uint64_t db = finish_vertex<DYN>(a, v, acc.value(), xself);
      dmax = db > dmax ? db : dmax;
    }
  }
  block_max_to(dmax, a.resid);
}

// one block per vertex (high in-degree)
template <bool EXACT, bool DYN>
__global__ void __launch_bounds__(kThreads) k_sweep_block(const SweepArgs a, int64_t begin, int64_t end) {
  if (a.prev && bitsd(*a.prev) <= a.tol) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  __shared__ uint64_t s_lo[kThreads / 32], s_hi[kThreads / 32], s_x[kThreads / 32];
  __shared__ int s_skip;
  uint64_t dmax = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t i = begin + blockIdx.x; i < end; i += gridDim.x) {
    const int32_t v = a.P[i];
    if (DYN) {
      if (threadIdx.x == 0) s_skip = skip_unaffected(a, v) ? 1 : 0;
      __syncthreads();
      const int sk = s_skip;
      __syncthreads();
      if (sk) continue;
    }
    const int64_t b = a.off[v], e = a.off[v + 1];
    Acc<EXACT> acc;
    double xself = 0.0;
    gather_row_vec<kThreads, EXACT>(a, b, e, threadIdx.x, v, acc, xself, pf, pl);
    acc.template group_reduce<32>();
    const uint64_t xb = warp_max_u64(dbits(xself));
    if (lane == 0) {
      s_lo[wid] = acc.lo();
      s_hi[wid] = acc.hi();
      s_x[wid] = xb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Acc<EXACT> tot;
      uint64_t xm = 0;
      for (int k = 0; k < kThreads / 32; ++k) {
        tot.merge_raw(s_lo[k], s_hi[k]);
        xm = s_x[k] > xm ? s_x[k] : xm;
      }
      const uint64_t db = finish_vertex<DYN>(a, v, tot.value(), bitsd(xm));
      dmax = db > dmax ? db : dmax;
    }
    __syncthreads();
  }
  block_max_to(dmax, a.resid);
}

template <bool EXACT, bool DYN>
int launch_all(const SweepArgs& a, const int64_t* cb, int nclass, cudaStream_t s) {
  // class c covers P[cb[c], cb[c+1]); the group size per class: 1, 8, 32, block
  const int maxg = kSMs * 8;
  for (int c = 0; c < nclass; ++c) {
    const int64_t b = cb[c], e = cb[c + 1];
    if (e <= b) continue;
    const int64_t cnt = e - b;
    const int kind = (nclass == 4) ? c : (c == nclass - 1 ? 3 : c);  // last class is always block-per-vertex
    switch (kind) {
      case 0: k_sweep_group<1, EXACT, DYN><<<grid_for(cnt, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      case 1: k_sweep_group<8, EXACT, DYN><<<grid_for(cnt * 8, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      case 2: k_sweep_group<32, EXACT, DYN><<<grid_for(cnt * 32, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      default: k_sweep_block<EXACT, DYN><<<grid_for(cnt, 1, maxg), kThreads, 0, s>>>(a, b, e); break;
    }
  }
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

}  // namespace

int launch_sweep(const SweepArgs& a, const int64_t* class_begin, int nclass, bool exact, bool dynamic,
                 cudaStream_t s) {
  if (exact) return dynamic ? launch_all<true, true>(a, class_begin, nclass, s) : launch_all<true, false>(a, class_begin, nclass, s);
  return dynamic ? launch_all<false, true>(a, class_begin, nclass, s) : launch_all<false, false>(a, class_begin, nclass, s);
}

}  // namespace prdf
