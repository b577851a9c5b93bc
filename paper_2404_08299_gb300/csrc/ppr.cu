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

// Compensated FP32 sum (s + e): TwoSum folds each term's rounding error into e.
struct Dot2 {
  float s = 0.f, e = 0.f;
  __device__ __forceinline__ void add(float y) {
    const float t = s + y;
    const float bp = t - s;
    e += (s - (t - bp)) + (y - bp);
    s = t;
  }
  __device__ __forceinline__ void merge(const Dot2& o) {
    add(o.s);
    e += o.e;
  }
  __device__ __forceinline__ float value() const { return s + e; }
};

// Column accumulator of the FP32 sweeps: the products of a block of up to U
// edges are summed with FMAs in b, and each block sum is folded into a
// compensated pair, so the rounding error does not grow with the row length
// (about two FP32 instructions per edge and column instead of ten for a
// compensated product per edge).
struct BlockSum {
  Dot2 d;
  float b = 0.f;
  __device__ __forceinline__ void prod(float p, float r) { b = fmaf(p, r, b); }
  __device__ __forceinline__ void fold() {
    d.add(b);
    b = 0.f;
  }
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

// per-iteration buffers of the graph-driven loops
__device__ __forceinline__ Ppr32Args resolve_ppr32(const Ppr32Args& in) {
  if (!in.ctl) return in;
  Ppr32Args a = in;
  const int it = in.ctl[0];
  a.R = (it & 1) ? in.Rb : in.Ra;
  a.Rn = (it & 1) ? const_cast<float*>(in.Ra) : in.Rb;
  a.resid = in.resid_base + 2 * it;
  a.prev = it > 0 ? in.resid_base + 2 * (it - 1) : nullptr;
  return a;
}
__device__ __forceinline__ Ppr64Args resolve_ppr64(const Ppr64Args& in) {
  if (!in.ctl) return in;
  Ppr64Args a = in;
  const int it = in.ctl[0];
  a.R = (it & 1) ? in.Rb : in.Ra;
  a.Rn = (it & 1) ? const_cast<double*>(in.Ra) : in.Rb;
  a.dmax = in.dmax_base + it;
  return a;
}

__device__ __forceinline__ bool ppr32_converged(const Ppr32Args& a) {
  if (!a.prev) return false;
  return __uint_as_float(a.prev[0]) <= a.tol_rel * __uint_as_float(a.prev[1]);
}

// ------------------------------------------------- FP32 K-column sweep ----
// A lane owns 4 consecutive columns of a tile (one 16-byte load per gathered
// row when K % 4 == 0), so LPE = tile / 4 lanes cover one edge and a warp
// load serves 32 / LPE edges ("slots").

struct Col4 {
  float v[4];
};

__device__ __forceinline__ Col4 zero4() {
  Col4 c;
#pragma unroll
  for (int q = 0; q < 4; ++q) c.v[q] = 0.f;
  return c;
}

// columns col .. col + 3 of row u (zero past K)
__device__ __forceinline__ Col4 ld_cols(const float* R, int64_t u, int K, int col) {
  Col4 c;
  const float* src = R + u * K + col;
  if ((K & 3) == 0) {  // col is a multiple of 4: 16-byte aligned
    const float4 f = __ldg(reinterpret_cast<const float4*>(src));
    c.v[0] = f.x;
    c.v[1] = f.y;
    c.v[2] = f.z;
    c.v[3] = f.w;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) c.v[q] = col + q < K ? __ldg(src + q) : 0.f;
  }
  return c;
}

// S and the previous R of the 4 columns of vertex v, loaded before the row's
// gathers so their latency overlaps
struct Own4 {
  float s[4], o[4];
};
__device__ __forceinline__ Own4 ppr32_own(const Ppr32Args& a, int32_t v, int col) {
  Own4 w;
#pragma unroll
  for (int q = 0; q < 4; ++q) w.s[q] = w.o[q] = 0.f;
  if (col >= a.K) return w;
  const int64_t o = (int64_t)v * a.K + col;
  // right-hand side row: dense, or (srow) the compact row of v, none when v has no teleport mass
  const int64_t sr = a.srow ? (int64_t)a.srow[v] : (int64_t)v;
  const float* S = sr >= 0 ? a.S + sr * a.K + col : nullptr;
  if ((a.K & 3) == 0) {
    const float4 o4 = *reinterpret_cast<const float4*>(a.R + o);
    w.o[0] = o4.x; w.o[1] = o4.y; w.o[2] = o4.z; w.o[3] = o4.w;
    if (S) {
      const float4 s4 = *reinterpret_cast<const float4*>(S);
      w.s[0] = s4.x; w.s[1] = s4.y; w.s[2] = s4.z; w.s[3] = s4.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      w.s[q] = (S && col + q < a.K) ? S[q] : 0.f;
      w.o[q] = col + q < a.K ? a.R[o + q] : 0.f;
    }
  }
  return w;
}

// new values of the 4 columns of vertex v from their accumulated sums
__device__ __forceinline__ void ppr32_finish4(const Ppr32Args& a, int32_t v, int col, const float* acc, const Own4& w,
                                              uint32_t& dmax, uint32_t& rmax) {
  if (col >= a.K) return;
  const int64_t o = (int64_t)v * a.K + col;
  float r[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    r[q] = fmaf(a.alpha, acc[q], a.beta * w.s[q]);
    if (col + q < a.K) {
      dmax = max(dmax, __float_as_uint(fabsf(r[q] - w.o[q])));
      rmax = max(rmax, __float_as_uint(fabsf(r[q])));
    }
  }
  if ((a.K & 3) == 0) {
    *reinterpret_cast<float4*>(a.Rn + o) = make_float4(r[0], r[1], r[2], r[3]);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (col + q < a.K) a.Rn[o + q] = r[q];
  }
}

// U edges of one slot in flight: edges j0 + k * stride (k < U) below e
template <int U>
__device__ __forceinline__ void ppr32_edges(const Ppr32Args& a, int64_t j0, int64_t stride, int64_t e, int col,
                                            bool colok, BlockSum* acc) {
  int32_t u[U];
  float p[U];
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const int64_t j = j0 + (int64_t)k * stride;
    u[k] = j < e ? __ldg(a.adj + j) : -1;
    p[k] = j < e ? __ldg(a.P + j) : 0.f;
  }
  Col4 r[U];
#pragma unroll
  for (int k = 0; k < U; ++k) r[k] = (u[k] >= 0 && colok) ? ld_cols(a.R, u[k], a.K, col) : zero4();
#pragma unroll
  for (int k = 0; k < U; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q].prod(p[k], r[k].v[q]);
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q].fold();
}

// merge the compensated sums of the slots of a warp (slot 0 ends with the total)
template <int LPE>
__device__ __forceinline__ void merge_slots(Dot2* t) {
#pragma unroll
  for (int o = LPE; o < 32; o <<= 1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Dot2 x;
      x.s = __shfl_xor_sync(0xffffffffu, t[q].s, o);
      x.e = __shfl_xor_sync(0xffffffffu, t[q].e, o);
      t[q].merge(x);
    }
  }
}

// One vertex per slot (rows of at most a few hundred edges), U edges in flight.
template <int LPE, int U>
__global__ void __launch_bounds__(kThreads) k_ppr32_group(const Ppr32Args a_in, int64_t begin, int64_t end, int c0) {
  const Ppr32Args a = resolve_ppr32(a_in);
  if (ppr32_converged(a)) return;
  constexpr int kSlots = 32 / LPE;
  const int sub = threadIdx.x & (LPE - 1);
  const int slot = (threadIdx.x & 31) / LPE;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int col = c0 + 4 * sub;
  const bool colok = col < a.K;
  uint32_t dmax = 0, rmax = 0;
  // The row offsets of the next vertex a slot takes load while the current
  // vertex's rows are gathered, so a vertex starts with its offsets known.
  const int64_t step = nwarps * kSlots;
  int64_t base = begin + warp * kSlots;
  int64_t i = base + slot;
  int64_t b = i < end ? a.off[i] : 0, e = i < end ? a.off[i + 1] : 0;
  for (; base < end; base += step, i += step) {
    const int64_t in = i + step;
    const int64_t bn = in < end ? a.off[in] : 0, en = in < end ? a.off[in + 1] : 0;
    if (i < end) {
      const int32_t v = (int32_t)i;
      const Own4 w = ppr32_own(a, v, col);
      BlockSum acc[4];
      for (int64_t j0 = b; j0 < e; j0 += U) ppr32_edges<U>(a, j0, 1, e, col, colok, acc);
      float c[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) c[q] = acc[q].d.value();
      ppr32_finish4(a, v, col, c, w, dmax, rmax);
    }
    b = bn;
    e = en;
  }
  block_max2_u32(dmax, rmax, a.resid);
}

// One warp per vertex (mid-degree rows): the slots stride over the row, U
// edges in flight each, and meet by shuffles.
template <int LPE, int U>
__global__ void __launch_bounds__(kThreads) k_ppr32_warp(const Ppr32Args a_in, int64_t begin, int64_t end, int c0) {
  const Ppr32Args a = resolve_ppr32(a_in);
  if (ppr32_converged(a)) return;
  constexpr int kSlots = 32 / LPE;
  const int sub = threadIdx.x & (LPE - 1);
  const int slot = (threadIdx.x & 31) / LPE;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int col = c0 + 4 * sub;
  const bool colok = col < a.K;
  uint32_t dmax = 0, rmax = 0;
  // the next row's offsets load while the current row is gathered
  int64_t i = begin + warp;
  int64_t b = i < end ? a.off[i] : 0, e = i < end ? a.off[i + 1] : 0;
  for (; i < end; i += nwarps) {
    const int32_t v = (int32_t)i;
    const int64_t in = i + nwarps;
    const int64_t bn = in < end ? a.off[in] : 0, en = in < end ? a.off[in + 1] : 0;
    Own4 w;
    if (slot == 0) w = ppr32_own(a, v, col);
    BlockSum acc[4];
    for (int64_t j0 = b + slot; j0 < e; j0 += (int64_t)kSlots * U) ppr32_edges<U>(a, j0, kSlots, e, col, colok, acc);
    b = bn;
    e = en;
    Dot2 t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = acc[q].d;
    merge_slots<LPE>(t);
    if (slot == 0) {
      float c[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) c[q] = t[q].value();
      ppr32_finish4(a, v, col, c, w, dmax, rmax);
    }
  }
  block_max2_u32(dmax, rmax, a.resid);
}

// Rows of the highest in-degree class are cut into chunks of kHubChunk edges
// handled by different warps; each chunk's compensated partial sums go to
// part[chunk][column] and a second kernel merges them in chunk order.
template <int LPE, int U>
__global__ void __launch_bounds__(kThreads) k_ppr32_hub_part(const Ppr32Args a_in, PprHub h, int c0, int tile,
                                                             float2* __restrict__ part) {
  const Ppr32Args a = resolve_ppr32(a_in);
  if (ppr32_converged(a)) return;
  constexpr int kSlots = 32 / LPE;
  const int sub = threadIdx.x & (LPE - 1);
  const int slot = (threadIdx.x & 31) / LPE;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int col = c0 + 4 * sub;
  const bool colok = col < a.K;
  for (int64_t c = warp; c < h.nchunk; c += nwarps) {
    const int32_t v = (int32_t)(h.begin + h.chunk_hub[c]);
    const int64_t j_begin = h.chunk_j0[c];
    const int64_t row_end = a.off[v + 1];
    const int64_t e = j_begin + kHubChunk < row_end ? j_begin + kHubChunk : row_end;
    BlockSum acc[4];
    for (int64_t j0 = j_begin + slot; j0 < e; j0 += (int64_t)kSlots * U) ppr32_edges<U>(a, j0, kSlots, e, col, colok, acc);
    Dot2 t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = acc[q].d;
    merge_slots<LPE>(t);
    if (slot == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) part[c * tile + 4 * sub + q] = make_float2(t[q].s, t[q].e);
    }
  }
}

template <int LPE>
__global__ void __launch_bounds__(kThreads) k_ppr32_hub_finish(const Ppr32Args a_in, PprHub h, int c0, int tile,
                                                               const float2* __restrict__ part) {
  const Ppr32Args a = resolve_ppr32(a_in);
  if (ppr32_converged(a)) return;
  constexpr int kSlots = 32 / LPE;
  const int sub = threadIdx.x & (LPE - 1);
  const int slot = (threadIdx.x & 31) / LPE;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int col = c0 + 4 * sub;
  uint32_t dmax = 0, rmax = 0;
  for (int64_t base = warp * kSlots; base < h.nhub; base += nwarps * kSlots) {
    const int64_t hi = base + slot;
    if (hi >= h.nhub) continue;
    Dot2 t[4];
    for (int64_t c = h.hub_first[hi]; c < h.hub_first[hi + 1]; ++c) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 x = part[c * tile + 4 * sub + q];
        Dot2 y;
        y.s = x.x;
        y.e = x.y;
        t[q].merge(y);
      }
    }
    float cv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) cv[q] = t[q].value();
    const int32_t v = (int32_t)(h.begin + hi);
    ppr32_finish4(a, v, col, cv, ppr32_own(a, v, col), dmax, rmax);
  }
  block_max2_u32(dmax, rmax, a.resid);
}

// hub chunk table: count, then fill (hub_first is the scan of the counts)
__global__ void k_hub_count(const int64_t* __restrict__ off, int64_t begin, int64_t nhub, int64_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nhub; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = off[begin + i + 1] - off[begin + i];
    cnt[i] = d > 0 ? (d + kHubChunk - 1) / kHubChunk : 0;
  }
}

__global__ void k_hub_fill(const int64_t* __restrict__ off, int64_t begin, int64_t nhub,
                           const int64_t* __restrict__ first, int32_t* __restrict__ chunk_hub,
                           int64_t* __restrict__ chunk_j0) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nhub; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = off[begin + i];
    for (int64_t c = first[i]; c < first[i + 1]; ++c) {
      chunk_hub[c] = (int32_t)i;
      chunk_j0[c] = b + (c - first[i]) * kHubChunk;
    }
  }
}

// ---------------------------------------------------- FP64 Jacobi step ----
// T(R) = alpha P^T R + (1 - alpha) S for a tile of columns, with the layout of
// the FP32 sweep (4 columns per lane, LPE = tile / 4 lanes per edge): writes
// T(R) to Rn, the residual (T(R) - R) / (1 - alpha) as FP32 to res32 (if not
// null) and max |T(R) - R| to *dmax (FP64 bits, atomic max). Sums are plain
// FP64 FMAs in a fixed order (edge order within a slot, then slots, then
// chunks), so every run gives the same bits.

struct Col4d {
  double v[4];
};

__device__ __forceinline__ Col4d zero4d() {
  Col4d c;
#pragma unroll
  for (int q = 0; q < 4; ++q) c.v[q] = 0.0;
  return c;
}

// columns col .. col + 3 of row u (zero past K); K even: two 16-byte loads
__device__ __forceinline__ Col4d ld_cols64(const double* R, int64_t u, int K, int col) {
  Col4d c;
  const double* src = R + u * K + col;
  if ((K & 1) == 0 && col + 4 <= K) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(src));
    const double2 b = __ldg(reinterpret_cast<const double2*>(src + 2));
    c.v[0] = a.x;
    c.v[1] = a.y;
    c.v[2] = b.x;
    c.v[3] = b.y;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) c.v[q] = col + q < K ? __ldg(src + q) : 0.0;
  }
  return c;
}

template <int U>
__device__ __forceinline__ void ppr64_edges(const Ppr64Args& a, int64_t j0, int64_t stride, int64_t e, int col,
                                            bool colok, double* acc) {
  int32_t u[U];
  double p[U];
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const int64_t j = j0 + (int64_t)k * stride;
    u[k] = j < e ? __ldg(a.adj + j) : -1;
    p[k] = j < e ? __ldg(a.P + j) : 0.0;
  }
  Col4d r[U];
#pragma unroll
  for (int k = 0; k < U; ++k) r[k] = (u[k] >= 0 && colok) ? ld_cols64(a.R, u[k], a.K, col) : zero4d();
#pragma unroll
  for (int k = 0; k < U; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(p[k], r[k].v[q], acc[q]);
}

// T(R), residual and |T(R) - R| for the 4 columns of vertex v
__device__ __forceinline__ void ppr64_finish4(const Ppr64Args& a, int32_t v, int col, const double* acc,
                                              uint64_t& dmax) {
  const int64_t sr = a.srow ? (int64_t)a.srow[v] : (int64_t)v;  // as in ppr32_own
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (col + q >= a.K) break;
    const int64_t o = (int64_t)v * a.K + col + q;
    const double sv = sr >= 0 ? a.S[sr * a.K + col + q] : 0.0;
    const double t = fma(a.alpha, acc[q], a.beta * sv);
    const double d = t - a.R[o];
    a.Rn[o] = t;
    if (a.res32) a.res32[o] = (float)(d * a.inv_beta);
    dmax = max(dmax, dbits(fabs(d)));
  }
}

__device__ __forceinline__ void block_max_u64(uint64_t dmax, uint64_t* out) {
  __shared__ uint64_t sm[32];
  dmax = warp_max_u64(dmax);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = dmax;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint64_t x = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0;
    x = warp_max_u64(x);
    if (threadIdx.x == 0 && x) atomicMax((unsigned long long*)out, (unsigned long long)x);
  }
}

template <int LPE>
__device__ __forceinline__ void merge_slots64(double* t) {
#pragma unroll
  for (int o = LPE; o < 32; o <<= 1)
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] += __shfl_xor_sync(0xffffffffu, t[q], o);
}

// one vertex per slot (in-degree up to the two highest classes)
template <int LPE, int U>
__global__ void __launch_bounds__(kThreads) k_ppr64_group(const Ppr64Args a_in, int64_t begin, int64_t end, int c0) {
  const Ppr64Args a = resolve_ppr64(a_in);
  constexpr int kSlots = 32 / LPE;
  const int sub = threadIdx.x & (LPE - 1);
  const int slot = (threadIdx.x & 31) / LPE;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int col = c0 + 4 * sub;
  const bool colok = col < a.K;
  uint64_t dmax = 0;
  for (int64_t base = begin + warp * kSlots; base < end; base += nwarps * kSlots) {
    const int64_t i = base + slot;
    if (i >= end) continue;
    const int32_t v = (int32_t)i;
    const int64_t b = a.off[v], e = a.off[v + 1];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t j0 = b; j0 < e; j0 += U) ppr64_edges<U>(a, j0, 1, e, col, colok, acc);
    if (colok) ppr64_finish4(a, v, col, acc, dmax);
  }
  block_max_u64(dmax, a.dmax);
}

// a warp per vertex (mid-degree rows), slots meet by shuffles
template <int LPE, int U>
__global__ void __launch_bounds__(kThreads) k_ppr64_warp(const Ppr64Args a_in, int64_t begin, int64_t end, int c0) {
  const Ppr64Args a = resolve_ppr64(a_in);
  constexpr int kSlots = 32 / LPE;
  const int sub = threadIdx.x & (LPE - 1);
  const int slot = (threadIdx.x & 31) / LPE;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int col = c0 + 4 * sub;
  const bool colok = col < a.K;
  uint64_t dmax = 0;
  for (int64_t i = begin + warp; i < end; i += nwarps) {
    const int32_t v = (int32_t)i;
    const int64_t b = a.off[v], e = a.off[v + 1];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t j0 = b + slot; j0 < e; j0 += (int64_t)kSlots * U) ppr64_edges<U>(a, j0, kSlots, e, col, colok, acc);
    merge_slots64<LPE>(acc);
    if (slot == 0 && colok) ppr64_finish4(a, v, col, acc, dmax);
  }
  block_max_u64(dmax, a.dmax);
}

// hub rows in 1024-edge chunks: partial sums per chunk, then merged in chunk order
template <int LPE, int U>
__global__ void __launch_bounds__(kThreads) k_ppr64_hub_part(const Ppr64Args a_in, PprHub h, int c0, int tile,
                                                             double* __restrict__ part) {
  const Ppr64Args a = resolve_ppr64(a_in);
  constexpr int kSlots = 32 / LPE;
  const int sub = threadIdx.x & (LPE - 1);
  const int slot = (threadIdx.x & 31) / LPE;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int col = c0 + 4 * sub;
  const bool colok = col < a.K;
  for (int64_t c = warp; c < h.nchunk; c += nwarps) {
    const int32_t v = (int32_t)(h.begin + h.chunk_hub[c]);
    const int64_t jb = h.chunk_j0[c];
    const int64_t re = a.off[v + 1];
    const int64_t e = jb + kHubChunk < re ? jb + kHubChunk : re;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t j0 = jb + slot; j0 < e; j0 += (int64_t)kSlots * U) ppr64_edges<U>(a, j0, kSlots, e, col, colok, acc);
    merge_slots64<LPE>(acc);
    if (slot == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) part[c * tile + 4 * sub + q] = acc[q];
    }
  }
}

template <int LPE>
__global__ void __launch_bounds__(kThreads) k_ppr64_hub_finish(const Ppr64Args a_in, PprHub h, int c0, int tile,
                                                               const double* __restrict__ part) {
  const Ppr64Args a = resolve_ppr64(a_in);
  constexpr int kSlots = 32 / LPE;
  const int sub = threadIdx.x & (LPE - 1);
  const int slot = (threadIdx.x & 31) / LPE;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int col = c0 + 4 * sub;
  uint64_t dmax = 0;
  for (int64_t base = warp * kSlots; base < h.nhub; base += nwarps * kSlots) {
    const int64_t hi = base + slot;
    if (hi >= h.nhub) continue;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t c = h.hub_first[hi]; c < h.hub_first[hi + 1]; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += part[c * tile + 4 * sub + q];
    if (col < a.K) ppr64_finish4(a, (int32_t)(h.begin + hi), col, acc, dmax);
  }
  block_max_u64(dmax, a.dmax);
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
    const double invW = 1.0 / W[i];
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
// rows of a [n, K] matrix with a non-zero entry (flag per row)
__global__ void k_row_nonzero(const double* __restrict__ S, int64_t n, int K, uint32_t* __restrict__ flag) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    bool nz = false;
    for (int c = lane; c < K; c += 32) nz = nz || S[v * K + c] != 0.0;
    nz = __any_sync(0xffffffffu, nz);
    if (lane == 0) flag[v] = nz ? 1u : 0u;
  }
}

// srow[v] = compact row of v or -1; Sc64 / Sc32 (FP64 / FP32) get the non-zero rows, and R32 (zero on
// entry) the FP32 rows at their place
__global__ void k_row_compact(const double* __restrict__ S, int64_t n, int K, const uint32_t* __restrict__ flag,
                              const int64_t* __restrict__ pos, int32_t* __restrict__ srow, double* __restrict__ Sc64,
                              float* __restrict__ Sc32, float* __restrict__ R32) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const bool nz = flag[v] != 0;
    const int64_t r = nz ? pos[v] : -1;
    if (lane == 0) srow[v] = (int32_t)r;
    if (!nz) continue;
    for (int c = lane; c < K; c += 32) {
      const double x = S[v * K + c];
      Sc64[r * K + c] = x;
      Sc32[r * K + c] = (float)x;
      if (R32) R32[v * K + c] = (float)x;
    }
  }
}

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

template <int LPE>
void launch32_tile(const Ppr32Args& a, const PprHub& h, float2* part, int64_t hub_b, int64_t n, int c0, int tile,
                   cudaStream_t s) {
  const int maxg = kSMs * 8;
  if (hub_b > 0) k_ppr32_group<LPE, 4><<<grid_for(hub_b * LPE, kThreads, maxg), kThreads, 0, s>>>(a, 0, hub_b, c0);
  if (h.begin > hub_b)
    k_ppr32_warp<LPE, 8><<<grid_for((h.begin - hub_b) * 32, kThreads, maxg), kThreads, 0, s>>>(a, hub_b, h.begin, c0);
  if (n > h.begin) {
    k_ppr32_hub_part<LPE, 8><<<grid_for(h.nchunk * 32, kThreads, maxg), kThreads, 0, s>>>(a, h, c0, tile, part);
    k_ppr32_hub_finish<LPE><<<grid_for(h.nhub * LPE, kThreads, maxg), kThreads, 0, s>>>(a, h, c0, tile, part);
  }
}

template <int LPE>
void launch64_tile(const Ppr64Args& a, const PprHub& h, double* part, int64_t hub_b, int64_t n, int c0, int tile,
                   cudaStream_t s) {
  const int maxg = kSMs * 8;
  if (hub_b > 0) k_ppr64_group<LPE, 4><<<grid_for(hub_b * LPE, kThreads, maxg), kThreads, 0, s>>>(a, 0, hub_b, c0);
  if (h.begin > hub_b)
    k_ppr64_warp<LPE, 4><<<grid_for((h.begin - hub_b) * 32, kThreads, maxg), kThreads, 0, s>>>(a, hub_b, h.begin, c0);
  if (n > h.begin) {
    k_ppr64_hub_part<LPE, 4><<<grid_for(h.nchunk * 32, kThreads, maxg), kThreads, 0, s>>>(a, h, c0, tile, part);
    k_ppr64_hub_finish<LPE><<<grid_for(h.nhub * LPE, kThreads, maxg), kThreads, 0, s>>>(a, h, c0, tile, part);
  }
}

}  // namespace

int launch_ppr32_sweep(const Ppr32Args& a, int tile, int64_t n, int64_t hub_begin, const PprHub& h, float2* part,
                       cudaStream_t s) {
  for (int c0 = 0; c0 < a.K; c0 += tile) {
    switch (tile) {
      case 8: launch32_tile<2>(a, h, part, hub_begin, n, c0, tile, s); break;
      case 16: launch32_tile<4>(a, h, part, hub_begin, n, c0, tile, s); break;
      case 32: launch32_tile<8>(a, h, part, hub_begin, n, c0, tile, s); break;
      default: launch32_tile<16>(a, h, part, hub_begin, n, c0, tile, s); break;
    }
  }
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int build_ppr_hub(const int64_t* off, int64_t begin, int64_t n, PprHubTable& t, Workspace& ws, cudaStream_t s) {
  const int64_t nhub = n - begin;
  t.begin = begin;
  t.nhub = nhub > 0 ? nhub : 0;
  t.nchunk = 0;
  if (t.nhub == 0) return PRDF_OK;
  DBuf<int64_t> cnt;
  PRDF_TRY(cnt.alloc((size_t)t.nhub, s));
  PRDF_TRY(t.hub_first.alloc((size_t)t.nhub + 1, s));
  k_hub_count<<<grid_for(t.nhub, kThreads), kThreads, 0, s>>>(off, begin, t.nhub, cnt.p);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(exclusive_scan_i64(cnt.p, t.nhub, t.hub_first.p, ws, s));
  PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, t.hub_first.p + t.nhub, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  t.nchunk = ws.host_i64[0];
  PRDF_TRY(t.chunk_hub.alloc((size_t)(t.nchunk > 0 ? t.nchunk : 1), s));
  PRDF_TRY(t.chunk_j0.alloc((size_t)(t.nchunk > 0 ? t.nchunk : 1), s));
  k_hub_fill<<<grid_for(t.nhub, kThreads), kThreads, 0, s>>>(off, begin, t.nhub, t.hub_first.p, t.chunk_hub.p,
                                                              t.chunk_j0.p);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int launch_ppr64_step(const Ppr64Args& a, int tile, int64_t n, int64_t hub_begin, const PprHub& h, double* part,
                      cudaStream_t s) {
  for (int c0 = 0; c0 < a.K; c0 += tile) {
    switch (tile) {
      case 8: launch64_tile<2>(a, h, part, hub_begin, n, c0, tile, s); break;
      case 16: launch64_tile<4>(a, h, part, hub_begin, n, c0, tile, s); break;
      case 32: launch64_tile<8>(a, h, part, hub_begin, n, c0, tile, s); break;
      default: launch64_tile<16>(a, h, part, hub_begin, n, c0, tile, s); break;
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

int ppr_sparse_rhs(const double* S, int64_t n, int K, Workspace& ws, PprSparseRhs* out, float* R32, cudaStream_t s) {
  out->rows = 0;
  DBuf<uint32_t> flag;
  DBuf<int64_t> pos;
  PRDF_TRY(flag.alloc((size_t)n, s));
  PRDF_TRY(pos.alloc((size_t)n + 1, s));
  k_row_nonzero<<<grid_for(n * 32, kThreads), kThreads, 0, s>>>(S, n, K, flag.p);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(exclusive_scan_u32(flag.p, n, pos.p, ws, s));
  PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, pos.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  const int64_t rows = ws.host_i64[0];
  if (rows * 4 > n) return PRDF_OK;  // dense enough: keep the dense form
  PRDF_TRY(out->srow.reserve((size_t)n, s));
  PRDF_TRY(out->Sc64.reserve((size_t)(rows > 0 ? rows : 1) * K, s));
  PRDF_TRY(out->Sc32.reserve((size_t)(rows > 0 ? rows : 1) * K, s));
  if (R32) PRDF_CUDA(cudaMemsetAsync(R32, 0, sizeof(float) * (size_t)n * K, s));
  k_row_compact<<<grid_for(n * 32, kThreads), kThreads, 0, s>>>(S, n, K, flag.p, pos.p, out->srow.p, out->Sc64.p,
                                                                out->Sc32.p, R32);
  PRDF_LAUNCH_CHECK();
  out->rows = rows;
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
