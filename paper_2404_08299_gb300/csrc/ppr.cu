// K-column weighted personalised PageRank (an extension of Eq. 1 and
// Alg. static): R[:, c] = alpha * P^T R[:, c] + (1 - alpha) * S[:, c] with the
// row-stochastic P_uv = w_uv / sum_k w_uk, for K personalisation columns at
// once. State is row-major [n, K] in the class-contiguous numbering, so one
// index and weight fetch serves a tile of T columns (T = 2 * lanes per
// vertex); rows above kHubDeg in-edges use a block per vertex.
//
// FP32 sweeps use a compensated dot product (each product's rounding error
// from an FMA, TwoSum for the additions). The FP64 stage is mixed-precision
// iterative refinement: an FP64 sweep computes the Jacobi step T(R) and the
// residual T(R) - R; an FP32 solve of E = alpha P^T E + residual gives the
// correction. The stop rule is the same as Static's: the L-inf change of an
// FP64 Jacobi step <= tol.
#include "internal.cuh"

namespace prdf {

namespace {

constexpr int kThreads = 256;

// compensated FP32 dot product accumulator
struct Dot2 {
  float s = 0.f, e = 0.f;
  __device__ __forceinline__ void add_prod(float p, float r) {
    const float h = p * r;
    const float eh = fmaf(p, r, -h);
    const float t = s + h;
    const float bp = t - s;
    e += ((s - (t - bp)) + (h - bp)) + eh;
    s = t;
  }
  __device__ __forceinline__ void add(float y) {
    const float t = s + y;
    const float bp = t - s;
    e += (s - (t - bp)) + (y - bp);
    s = t;
  }
  __device__ __forceinline__ float value() const { return s + e; }
};

__device__ __forceinline__ void block_max2_u32(uint32_t dmax, uint32_t rmax, uint32_t* out) {
  __shared__ uint32_t sd[32], sr[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sd[wid] = dmax;
    sr[wid] = rmax;
  }
  __syncthreads();
  if (wid == 0) {
    uint32_t x = lane < (int)(blockDim.x >> 5) ? sd[lane] : 0u;
    uint32_t y = lane < (int)(blockDim.x >> 5) ? sr[lane] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
      y = max(y, __shfl_xor_sync(0xffffffffu, y, o));
    }
    if (lane == 0) {
      if (x) atomicMax(out, x);
      if (y) atomicMax(out + 1, y);
    }
  }
}

__device__ __forceinline__ bool ppr32_converged(const Ppr32Args& a) {
  if (!a.prev) return false;
  return __uint_as_float(a.prev[0]) <= a.tol_rel * __uint_as_float(a.prev[1]);
}

// new values of 2 columns of vertex v from their accumulated sums
__device__ __forceinline__ void ppr32_finish(const Ppr32Args& a, int32_t v, int col, float acc0, float acc1,
                                             uint32_t& dmax, uint32_t& rmax) {
  const int64_t o = (int64_t)v * a.K + col;
  if (col >= a.K) return;
  const bool two = col + 1 < a.K;
  const float s0 = a.S[o], s1 = two ? a.S[o + 1] : 0.f;
  const float r0 = fmaf(a.alpha, acc0, a.beta * s0), r1 = fmaf(a.alpha, acc1, a.beta * s1);
  const float o0 = a.R[o], o1 = two ? a.R[o + 1] : 0.f;
  a.Rn[o] = r0;
  if (two) a.Rn[o + 1] = r1;
  dmax = max(dmax, __float_as_uint(fabsf(r0 - o0)));
  rmax = max(rmax, __float_as_uint(fabsf(r0)));
  if (two) {
    dmax = max(dmax, __float_as_uint(fabsf(r1 - o1)));
    rmax = max(rmax, __float_as_uint(fabsf(r1)));
  }
}

// G lanes per vertex, 2 columns per lane (tile of 2G columns starting at c0)
template <int G, int U>
__global__ void __launch_bounds__(kThreads) k_ppr32_group(const Ppr32Args a, int64_t begin, int64_t end, int c0) {
  if (ppr32_converged(a)) return;
  constexpr int kGroupsPerWarp = 32 / G;
  const int lane = threadIdx.x & (G - 1);
  const int gw = (threadIdx.x & 31) / G;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int col = c0 + 2 * lane;
  const bool colok = col < a.K, two = col + 1 < a.K;
  uint32_t dmax = 0, rmax = 0;
  for (int64_t base = begin + warp * kGroupsPerWarp; base < end; base += nwarps * kGroupsPerWarp) {
    const int64_t i = base + gw;
    if (i >= end) continue;
    const int32_t v = (int32_t)i;
    const int64_t b = a.off[v], e = a.off[v + 1];
    Dot2 s0, s1;
    for (int64_t j0 = b; j0 < e; j0 += U) {
      int32_t u[U];
      float p[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const bool ok = j0 + k < e;
        u[k] = ok ? __ldg(a.adj + j0 + k) : -1;
        p[k] = ok ? __ldg(a.P + j0 + k) : 0.f;
      }
      float r0[U], r1[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        r0[k] = 0.f;
        r1[k] = 0.f;
        if (u[k] >= 0 && colok) {
          const float* src = a.R + (int64_t)u[k] * a.K + col;
          if (two) {
            r0[k] = __ldg(src);
            r1[k] = __ldg(src + 1);
          } else {
            r0[k] = __ldg(src);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (u[k] < 0) continue;
        s0.add_prod(p[k], r0[k]);
        s1.add_prod(p[k], r1[k]);
      }
    }
    ppr32_finish(a, v, col, s0.value(), s1.value(), dmax, rmax);
  }
  block_max2_u32(dmax, rmax, a.resid);
}

// block per vertex for rows above kHubDeg edges: the block's edge slots
// (kThreads / G of them) stride over the row, partial sums meet in shared memory
template <int G>
__global__ void __launch_bounds__(kThreads) k_ppr32_block(const Ppr32Args a, int64_t begin, int64_t end, int c0) {
  if (ppr32_converged(a)) return;
  constexpr int kSlots = kThreads / G;
  __shared__ float ss[kSlots][2 * G];
  const int lane = threadIdx.x % G, slot = threadIdx.x / G;
  const int col = c0 + 2 * lane;
  const bool colok = col < a.K, two = col + 1 < a.K;
  uint32_t dmax = 0, rmax = 0;
  for (int64_t i = begin + blockIdx.x; i < end; i += gridDim.x) {
    const int32_t v = (int32_t)i;
    const int64_t b = a.off[v], e = a.off[v + 1];
    Dot2 s0, s1;
    constexpr int U = 4;  // edges in flight per slot
    for (int64_t j0 = b + slot; j0 < e; j0 += (int64_t)kSlots * U) {
      int32_t u[U];
      float p[U], r0[U], r1[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int64_t j = j0 + (int64_t)k * kSlots;
        u[k] = j < e ? __ldg(a.adj + j) : -1;
        p[k] = j < e ? __ldg(a.P + j) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        r0[k] = 0.f;
        r1[k] = 0.f;
        if (u[k] >= 0 && colok) {
          const float* src = a.R + (int64_t)u[k] * a.K + col;
          r0[k] = __ldg(src);
          if (two) r1[k] = __ldg(src + 1);
        }
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (u[k] < 0) continue;
        s0.add_prod(p[k], r0[k]);
        s1.add_prod(p[k], r1[k]);
      }
    }
    ss[slot][2 * lane] = s0.value();
    ss[slot][2 * lane + 1] = s1.value();
    __syncthreads();
    if (slot == 0) {
      Dot2 t0, t1;
      for (int k = 0; k < kSlots; ++k) {
        t0.add(ss[k][2 * lane]);
        t1.add(ss[k][2 * lane + 1]);
      }
      ppr32_finish(a, v, col, t0.value(), t1.value(), dmax, rmax);
    }
    __syncthreads();
  }
  block_max2_u32(dmax, rmax, a.resid);
}

// FP64 Jacobi step T(R) = alpha P^T R + (1 - alpha) S for a tile of 2G columns:
// writes T(R) to Rn, the residual (T(R) - R) / (1 - alpha) as FP32 to res32 (if
// not null) and max |T(R) - R| to *dmax (FP64 bits, atomic max).
template <int G, bool HUB>
__global__ void __launch_bounds__(kThreads) k_ppr64_step(const Ppr64Args a, int64_t begin, int64_t end, int c0) {
  constexpr int kSlots = kThreads / G;
  __shared__ double ss[HUB ? kSlots : 1][HUB ? 2 * G : 1];
  const int lane = threadIdx.x % G;
  const int col = c0 + 2 * lane;
  const bool colok = col < a.K, two = col + 1 < a.K;
  uint64_t dmax = 0;
  const int64_t gstride = HUB ? gridDim.x : ((int64_t)gridDim.x * kThreads) / G;
  const int64_t g0 = HUB ? blockIdx.x : (blockIdx.x * (int64_t)kThreads + threadIdx.x) / G;
  const int slot = HUB ? (int)(threadIdx.x / G) : 0;
  for (int64_t i = begin + g0; HUB ? (i < end) : true; i += gstride) {
    bool active = i < end;
    if (!HUB && !active) break;
    const int32_t v = (int32_t)i;
    const int64_t b = a.off[v], e = a.off[v + 1];
    double s0 = 0, s1 = 0;
    constexpr int U = 4;  // edges in flight per slot
    const int64_t stride = HUB ? kSlots : 1;
    for (int64_t j0 = b + slot; j0 < e; j0 += stride * U) {
      int32_t u[U];
      double p[U], r0[U], r1[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int64_t j = j0 + (int64_t)k * stride;
        u[k] = j < e ? __ldg(a.adj + j) : -1;
        p[k] = j < e ? __ldg(a.P + j) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        r0[k] = 0.0;
        r1[k] = 0.0;
        if (u[k] >= 0 && colok) {
          const double* src = a.R + (int64_t)u[k] * a.K + col;
          r0[k] = __ldg(src);
          if (two) r1[k] = __ldg(src + 1);
        }
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (u[k] < 0) continue;
        s0 = fma(p[k], r0[k], s0);
        s1 = fma(p[k], r1[k], s1);
      }
    }
    if (HUB) {
      ss[slot][2 * lane] = s0;
      ss[slot][2 * lane + 1] = s1;
      __syncthreads();
      if (slot == 0) {
        s0 = 0;
        s1 = 0;
        for (int k = 0; k < kSlots; ++k) {
          s0 += ss[k][2 * lane];
          s1 += ss[k][2 * lane + 1];
        }
      }
    }
    if ((!HUB || slot == 0) && colok) {
      const int64_t o = (int64_t)v * a.K + col;
      const double t0 = fma(a.alpha, s0, a.beta * a.S[o]);
      const double d0 = t0 - a.R[o];
      a.Rn[o] = t0;
      if (a.res32) a.res32[o] = (float)(d0 * a.inv_beta);
      dmax = max(dmax, dbits(fabs(d0)));
      if (two) {
        const double t1 = fma(a.alpha, s1, a.beta * a.S[o + 1]);
        const double d1 = t1 - a.R[o + 1];
        a.Rn[o + 1] = t1;
        if (a.res32) a.res32[o + 1] = (float)(d1 * a.inv_beta);
        dmax = max(dmax, dbits(fabs(d1)));
      }
    }
    if (HUB) __syncthreads();
  }
  // block max
  __shared__ uint64_t sm[32];
  dmax = warp_max_u64(dmax);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = dmax;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint64_t x = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0;
    x = warp_max_u64(x);
    if (threadIdx.x == 0 && x) atomicMax((unsigned long long*)a.dmax, (unsigned long long)x);
  }
}

// Edge gradient of L = sum_c G_c . R_c with respect to w_uv (out-slot j of
// renumbered row i, vertex u = perm[i], target v = adj[j]):
//   dL/dw_uv = (1 / W_u) * sum_c R[u, c] * (alpha * lambda[v, c] - (lambda[u, c] - G[u, c]))
// using sum_k P_uk lambda[k] = (lambda[u] - G[u]) / alpha. The per-row constant
// b_u = sum_c R[u, c] * (lambda[u, c] - G[u, c]) is formed once per row; one
// warp per row, lanes over edges; written to the original out-slot order.
__global__ void k_grad_w(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                         const int32_t* __restrict__ perm, const int64_t* __restrict__ orig_off,
                         const double* __restrict__ lam, const double* __restrict__ Gs, double g_scale,
                         const double* __restrict__ Rr, const double* __restrict__ W, int32_t n, int K, double alpha,
                         double* __restrict__ grad_w) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const double* Ri = Rr + i * K;
    // b = sum_c R[i, c] * (lambda[i, c] - G[i, c]), lanes over columns
    double b = 0;
    for (int c = lane; c < K; c += 32) b = fma(Ri[c], lam[i * K + c] - g_scale * Gs[i * K + c], b);
    b = warp_sum_f64(b);
    const int32_t u = perm[i];
    const double invW = 1.0 / W[u];
    const int64_t rb = off[i], re = off[i + 1], ob = orig_off[u];
    for (int64_t j = rb + lane; j < re; j += 32) {
      const double* Lv = lam + (int64_t)adj[j] * K;
      double d = 0;
      for (int c = 0; c < K; ++c) d = fma(Ri[c], __ldg(Lv + c), d);
      grad_w[ob + (j - rb)] = (alpha * d - b) * invW;
    }
  }
}

// R64 += (double) E32
__global__ void k_add_correction(double* __restrict__ R, const float* __restrict__ E, int64_t cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
    R[i] += (double)E[i];
}

__global__ void k_narrow(const double* __restrict__ x, int64_t cnt, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void k_widen_n(const float* __restrict__ y, int64_t cnt, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (double)y[i];
}

template <int G>
void launch32_tile(const Ppr32Args& a, int64_t lo_b, int64_t lo_e, int64_t hi_e, int c0, cudaStream_t s) {
  const int maxg = kSMs * 8;
  if (lo_e > lo_b) k_ppr32_group<G, 4><<<grid_for((lo_e - lo_b) * G, kThreads, maxg), kThreads, 0, s>>>(a, lo_b, lo_e, c0);
  if (hi_e > lo_e) k_ppr32_block<G><<<grid_for(hi_e - lo_e, 1, maxg), kThreads, 0, s>>>(a, lo_e, hi_e, c0);
}

template <int G>
void launch64_tile(const Ppr64Args& a, int64_t lo_b, int64_t lo_e, int64_t hi_e, int c0, cudaStream_t s) {
  const int maxg = kSMs * 8;
  if (lo_e > lo_b) k_ppr64_step<G, false><<<grid_for((lo_e - lo_b) * G, kThreads, maxg), kThreads, 0, s>>>(a, lo_b, lo_e, c0);
  if (hi_e > lo_e) k_ppr64_step<G, true><<<grid_for(hi_e - lo_e, 1, maxg), kThreads, 0, s>>>(a, lo_e, hi_e, c0);
}

}  // namespace

int launch_ppr32_sweep(const Ppr32Args& a, int tile, int64_t n, int64_t hub_begin, cudaStream_t s) {
  for (int c0 = 0; c0 < a.K; c0 += tile) {
    switch (tile) {
      case 8: launch32_tile<4>(a, 0, hub_begin, n, c0, s); break;
      case 16: launch32_tile<8>(a, 0, hub_begin, n, c0, s); break;
      case 32: launch32_tile<16>(a, 0, hub_begin, n, c0, s); break;
      default: launch32_tile<32>(a, 0, hub_begin, n, c0, s); break;
    }
  }
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int launch_ppr64_step(const Ppr64Args& a, int tile, int64_t n, int64_t hub_begin, cudaStream_t s) {
  for (int c0 = 0; c0 < a.K; c0 += tile) {
    switch (tile) {
      case 8: launch64_tile<4>(a, 0, hub_begin, n, c0, s); break;
      case 16: launch64_tile<8>(a, 0, hub_begin, n, c0, s); break;
      case 32: launch64_tile<16>(a, 0, hub_begin, n, c0, s); break;
      default: launch64_tile<32>(a, 0, hub_begin, n, c0, s); break;
    }
  }
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int launch_grad_w(const int64_t* off, const int32_t* adj, const int32_t* perm, const int64_t* orig_off,
                  const double* lam, const double* Gs, double g_scale, const double* Rr, const double* W, int32_t n,
                  int K, double alpha, double* grad_w, cudaStream_t s) {
  k_grad_w<<<grid_for((int64_t)n * 32, kThreads), kThreads, 0, s>>>(off, adj, perm, orig_off, lam, Gs, g_scale, Rr, W, n,
                                                                     K, alpha, grad_w);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int ppr_add_correction(double* R, const float* E, int64_t cnt, cudaStream_t s) {
  k_add_correction<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(R, E, cnt);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int ppr_narrow(const double* x, int64_t cnt, float* y, cudaStream_t s) {
  k_narrow<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(x, cnt, y);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int ppr_widen(const float* y, int64_t cnt, double* x, cudaStream_t s) {
  k_widen_n<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(y, cnt, x);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

}  // namespace prdf
