// FP32 stage of the mixed-precision PageRank (an extension of the paper's
// Alg. static / Alg. frontier with Eq. 1 and Eq. 2): rank state y = R / |out|
// stored in FP32, so a sweep gathers 4 bytes per in-edge, and in-neighbour
// sums accumulated with compensated summation (Kahan-Babuska: TwoSum of every
// term, errors summed separately) on the FP32 pipes. Each sweep reports
// max |r - R[v]| and max r over the vertices it updates as FP32 bit
// patterns; the stage stops when max|dR| <= tol_fp32_rel * max R and the
// solve continues in FP64 (api.cu). The DF / DF-P form updates only the
// affected vertices, with Alg. update's prune and expand tests evaluated in
// FP32, and copies the others through, as the FP64 sweep does.
// Same class-contiguous numbering and kernel shapes as the FP64 sweep.
#include "internal.cuh"

namespace prdf {

namespace {

constexpr int kThreads = 256;

// compensated FP32 sum: value = s + e
struct Kahan {
  float s = 0.f, e = 0.f;
  __device__ __forceinline__ void add(float y) {
    const float t = s + y;
    const float bp = t - s;
    e += (s - (t - bp)) + (y - bp);
    s = t;
  }
  __device__ __forceinline__ void merge(float s2, float e2) {
    add(s2);
    e += e2;
  }
  template <int G>
  __device__ __forceinline__ void group_reduce() {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
      const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
      merge(s2, e2);
    }
  }
  __device__ __forceinline__ float value() const { return s + e; }
};

__device__ __forceinline__ uint32_t ld_gather_b32(const float* p, uint64_t pol) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_stream_f32(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}

template <int G, int U>
__device__ __forceinline__ void gather32(const Sweep32Args& a, int64_t b, int64_t e, int lane, int32_t v, Kahan& acc,
                                         uint32_t& yself, uint64_t pf, uint64_t pl) {
  for (int64_t j0 = b + lane; j0 < e; j0 += (int64_t)G * U) {
    int32_t u[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t j = j0 + (int64_t)k * G;
      u[k] = j < e ? ld_stream_i32(a.adj + j, pf) : -1;
    }
    uint32_t yv[U];
#pragma unroll
    for (int k = 0; k < U; ++k) yv[k] = u[k] >= 0 ? ld_gather_b32(a.y + u[k], pl) : 0u;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (u[k] >= 0) acc.add(__uint_as_float(yv[k]));
      yself = (u[k] == v) ? yv[k] : yself;
    }
  }
}

// Row handled by NT lanes: 16-byte index loads for the aligned body (KV of
// them in flight per lane), scalar head and tail. The head / tail term's
// index is loaded with the body's first indices and its gather issued with
// the body's first gathers (added after them), and each chunk's gathers are
// in flight while the next chunk's indices load, so a row costs one index and
// one gather round trip before its first add, as in the FP64 sweep.
template <int NT, int KV>
__device__ __forceinline__ void gather32_vec(const Sweep32Args& a, int64_t b, int64_t e, int lane, int32_t v,
                                             Kahan& acc, uint32_t& yself, uint64_t pf, uint64_t pl) {
  int64_t ba = (b + 3) & ~(int64_t)3;
  if (ba > e) ba = e;
  const int64_t ea = ba + ((e - ba) & ~(int64_t)3);
  int32_t uh = -1;
  {
    const int64_t nh = ba - b, nt = e - ea;
    int64_t j = -1;
    if (lane < nh) j = b + lane;
    else if (lane >= 4 && lane < 4 + nt) j = ea + (lane - 4);
    if (j >= 0) uh = ld_stream_i32(a.adj + j, pf);
  }
  const int64_t step = 4 * (int64_t)NT * KV;
  int4 u4[KV];
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    const int64_t q = ba + 4 * (int64_t)lane + 4 * (int64_t)NT * k;
    u4[k] = q < ea ? ld_stream_i32x4(a.adj + q, pf) : make_int4(-1, -1, -1, -1);
  }
  const uint32_t yh = uh >= 0 ? ld_gather_b32(a.y + uh, pl) : 0u;
  bool head = uh >= 0;
  for (int64_t base = ba; base < ea; base += step) {
    const int64_t q0 = base + 4 * (int64_t)lane;
    uint32_t yv[4 * KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      yv[4 * k + 0] = u4[k].x >= 0 ? ld_gather_b32(a.y + u4[k].x, pl) : 0u;
      yv[4 * k + 1] = u4[k].y >= 0 ? ld_gather_b32(a.y + u4[k].y, pl) : 0u;
      yv[4 * k + 2] = u4[k].z >= 0 ? ld_gather_b32(a.y + u4[k].z, pl) : 0u;
      yv[4 * k + 3] = u4[k].w >= 0 ? ld_gather_b32(a.y + u4[k].w, pl) : 0u;
    }
    int4 nx[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int64_t q = q0 + step + 4 * (int64_t)NT * k;
      nx[k] = q < ea ? ld_stream_i32x4(a.adj + q, pf) : make_int4(-1, -1, -1, -1);
    }
    if (head) {
      acc.add(__uint_as_float(yh));
      yself = (uh == v) ? yh : yself;
      head = false;
    }
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      if (u4[k].x < 0) continue;  // a whole int4 is valid or not
      acc.add(__uint_as_float(yv[4 * k + 0]));
      acc.add(__uint_as_float(yv[4 * k + 1]));
      acc.add(__uint_as_float(yv[4 * k + 2]));
      acc.add(__uint_as_float(yv[4 * k + 3]));
      yself = (u4[k].x == v) ? yv[4 * k + 0] : yself;
      yself = (u4[k].y == v) ? yv[4 * k + 1] : yself;
      yself = (u4[k].z == v) ? yv[4 * k + 2] : yself;
      yself = (u4[k].w == v) ? yv[4 * k + 3] : yself;
    }
#pragma unroll
    for (int k = 0; k < KV; ++k) u4[k] = nx[k];
  }
  if (head) {  // rows without a body chunk
    acc.add(__uint_as_float(yh));
    yself = (uh == v) ? yh : yself;
  }
}

// Eq. 1 (Static, DF) or Eq. 2 (DF-P) in FP32, with Alg. update's prune and
// expand tests for DF / DF-P; returns |r - R[v]| and r (both non-negative) as
// bit patterns
template <bool DYN>
__device__ __forceinline__ void finish32(const Sweep32Args& a, int32_t v, float c, uint32_t yself_b, uint64_t pf,
                                        uint32_t& db, uint32_t& rb, uint64_t& fwsum) {
  const float d = ld_stream_f32(a.degf + v, pf);
  const float yself = __uint_as_float(yself_b);
  const float rold = yself * d;
  float r;
  if (DYN && a.prune) r = ld_stream_f32(a.kf + v, pf) * fmaf(a.alpha, c - yself, a.c0);  // Eq. 2
  else r = fmaf(a.alpha, c, a.c0);                                                        // Eq. 1
  const float dr = fabsf(r - rold);
  if (DYN) {
    const float m = fmaxf(r, rold);
    if (a.prune && dr <= a.tau_p * m) a.dV[v] = 0;
    if (dr > a.tau_f * m) {
      a.dN[v] = 1;
      fwsum += (uint64_t)d;
    } else if (a.dN[v]) {
      a.dN[v] = 0;
    }
    a.wrote[v] = 1;
  }
  a.yn[v] = r * ld_stream_f32(a.invf + v, pf);
  db = __float_as_uint(dr);
  rb = __float_as_uint(r);
}

// DF / DF-P: an unaffected vertex keeps its rank (copied through when the
// previous sweep wrote its slot of yn) and leaves this sweep's expand set
__device__ __forceinline__ bool skip_unaffected32(const Sweep32Args& a, int32_t v) {
  if (a.dV[v]) return false;
  if (a.wrote[v]) {
    a.yn[v] = a.y[v];
    a.wrote[v] = 0;
  }
  if (a.dN[v]) a.dN[v] = 0;
  return true;
}

// per-iteration pointers of the graph-driven loop
__device__ __forceinline__ Sweep32Args resolve32(const Sweep32Args& in) {
  if (!in.ctl) return in;
  Sweep32Args a = in;
  const int it = in.ctl[0];
  a.y = (it & 1) ? in.yb : in.ya;
  a.yn = (it & 1) ? const_cast<float*>(in.ya) : in.yb;
  a.resid = in.resid_base + 2 * it;
  a.prev = it > 0 ? in.resid_base + 2 * (it - 1) : nullptr;
  a.fw = in.fw_base ? in.fw_base + it : nullptr;
  return a;
}

__device__ __forceinline__ bool converged32(const Sweep32Args& a) {
  if (!a.prev) return false;
  const float d = __uint_as_float(a.prev[0]), rm = __uint_as_float(a.prev[1]);
  return d <= a.tol_rel * rm;
}

__global__ void k_iter_check32(int* ctl, const uint32_t* resid_base, float tol_rel, int max_iter,
                               cudaGraphConditionalHandle h) {
  const int it = ctl[0];
  const uint32_t* r = resid_base + 2 * it;
  const bool done = __uint_as_float(r[0]) <= tol_rel * __uint_as_float(r[1]) || it + 1 >= max_iter;
  ctl[0] = it + 1;
  cudaGraphSetConditional(h, done ? 0u : 1u);
}

__device__ __forceinline__ void block_max2_to(uint32_t dmax, uint32_t rmax, uint32_t* out) {
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

// block epilogue: the pair (max |dR|, max R) and, for DF / DF-P, the out-edges of the new deltaN
template <bool DYN>
__device__ __forceinline__ void block_epilogue32(const Sweep32Args& a, uint32_t dmax, uint32_t rmax, uint64_t fwsum) {
  block_max2_to(dmax, rmax, a.resid);
  if (DYN && a.fw) {
    __shared__ uint64_t shs[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    fwsum = (uint64_t)warp_sum_i64((int64_t)fwsum);
    if (lane == 0) shs[wid] = fwsum;
    __syncthreads();
    if (wid == 0) {
      uint64_t x = lane < (int)(blockDim.x >> 5) ? shs[lane] : 0;
      x = (uint64_t)warp_sum_i64((int64_t)x);
      if (lane == 0 && x) atomicAdd((unsigned long long*)a.fw, (unsigned long long)x);
    }
  }
}

template <int G, int U, bool SELF1, bool DYN>
__global__ void __launch_bounds__(kThreads) k_sweep32_group(const Sweep32Args a_in, int64_t begin, int64_t end) {
  const Sweep32Args a = resolve32(a_in);
  if (converged32(a)) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  constexpr int kGroupsPerWarp = 32 / G;
  const int lane = (G == 1) ? 0 : (threadIdx.x & (G - 1));
  const int gw = (threadIdx.x & 31) / G;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  uint32_t dmax = 0, rmax = 0;
  uint64_t fwsum = 0;
  if constexpr (!DYN && !SELF1) {
    // Static form, pipelined as the FP64 group kernel: while an item's first
    // G*U gathers are in flight, the next item's first indices and the row
    // offsets of the item after it load, so a step waits for one round trip.
    // Each lane adds its terms in the same order as gather32.
    const int64_t step = nwarps * kGroupsPerWarp;
    auto row_of = [&](int64_t i) -> int32_t { return i < end ? (int32_t)i : -1; };
    auto load_off = [&](int32_t v, int64_t& b, int64_t& e) {
      b = v >= 0 ? ld_stream_i64(a.off + v, pf) : 0;
      e = v >= 0 ? ld_stream_i64(a.off + v + 1, pf) : 0;
    };
    auto load_idx = [&](int32_t v, int64_t b, int64_t e, int32_t (&u)[U]) {
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int64_t j = b + lane + (int64_t)k * G;
        u[k] = (v >= 0 && j < e) ? ld_stream_i32(a.adj + j, pf) : -1;
      }
    };
    int64_t base = begin + warp * kGroupsPerWarp;
    int32_t v = row_of(base + gw);
    int64_t b, e;
    load_off(v, b, e);
    int32_t u[U];
    load_idx(v, b, e, u);
    int32_t vn = row_of(base + step + gw);
    int64_t bn, en;
    load_off(vn, bn, en);
    for (; base < end; base += step) {
      uint32_t yv[U];
#pragma unroll
      for (int k = 0; k < U; ++k) yv[k] = u[k] >= 0 ? ld_gather_b32(a.y + u[k], pl) : 0u;
      int32_t un[U];
      load_idx(vn, bn, en, un);
      const int32_t vnn = row_of(base + 2 * step + gw);
      int64_t bnn, enn;
      load_off(vnn, bnn, enn);
      Kahan acc;
      uint32_t yself = 0;
      if (v >= 0) {
#pragma unroll
        for (int k = 0; k < U; ++k) {
          if (u[k] >= 0) acc.add(__uint_as_float(yv[k]));
          yself = (u[k] == v) ? yv[k] : yself;
        }
        // rest of a row longer than G*U (rows that grew past their class's bound in a batch update)
        if (e - b > (int64_t)G * U) gather32<G, U>(a, b + (int64_t)G * U, e, lane, v, acc, yself, pf, pl);
      }
      if (G > 1) {
        acc.template group_reduce<G>();
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) yself = max(yself, __shfl_xor_sync(0xffffffffu, yself, o));
      }
      if (v >= 0 && lane == 0) {
        uint32_t db, rb;
        finish32<DYN>(a, v, acc.value(), yself, pf, db, rb, fwsum);
        dmax = max(dmax, db);
        rmax = max(rmax, rb);
      }
      v = vn;
      b = bn;
      e = en;
#pragma unroll
      for (int k = 0; k < U; ++k) u[k] = un[k];
      vn = vnn;
      bn = bnn;
      en = enn;
    }
    block_epilogue32<DYN>(a, dmax, rmax, fwsum);
  } else {
    for (int64_t base = begin + warp * kGroupsPerWarp; base < end; base += nwarps * kGroupsPerWarp) {
      const int64_t i = base + gw;
      bool active = i < end;
      const int32_t v = (int32_t)i;
      // every lane of the group reads the flag before the group's shuffles, and
      // only the group's lane 0 changes it (in finish32, after them)
      if (DYN && active && skip_unaffected32(a, v)) active = false;
      Kahan acc;
      uint32_t yself = 0;
      if (active) {
        // the row is [v] unless a batch gave the vertex in-edges (its bit in multi)
        if (SELF1 && !(a.multi && ((a.multi[v >> 5] >> (v & 31)) & 1u))) {
          yself = lane == 0 ? ld_gather_b32(a.y + v, pl) : 0u;
          if (lane == 0) acc.add(__uint_as_float(yself));
        } else {
          const int64_t b = ld_stream_i64(a.off + v, pf), e = ld_stream_i64(a.off + v + 1, pf);
          gather32<G, U>(a, b, e, lane, v, acc, yself, pf, pl);
        }
      }
      // DF / DF-P: nothing to reduce when no item of the warp's step is affected
      if (DYN && !__any_sync(0xffffffffu, active)) continue;
      if (G > 1) {
        acc.template group_reduce<G>();
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) yself = max(yself, __shfl_xor_sync(0xffffffffu, yself, o));
      }
      if (active && lane == 0) {
        uint32_t db, rb;
        finish32<DYN>(a, v, acc.value(), yself, pf, db, rb, fwsum);
        dmax = max(dmax, db);
        rmax = max(rmax, rb);
      }
    }
    block_epilogue32<DYN>(a, dmax, rmax, fwsum);
  }
}

template <int KV, bool DYN>
__global__ void __launch_bounds__(kThreads) k_sweep32_warp(const Sweep32Args a_in, int64_t begin, int64_t end) {
  const Sweep32Args a = resolve32(a_in);
  if (converged32(a)) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  uint32_t dmax = 0, rmax = 0;
  uint64_t fwsum = 0;
  // the next row's offsets load while the current row is gathered
  int64_t i = begin + warp;
  int64_t b = i < end ? ld_stream_i64(a.off + i, pf) : 0, e = i < end ? ld_stream_i64(a.off + i + 1, pf) : 0;
  for (; i < end; i += nwarps) {
    const int32_t v = (int32_t)i;
    const int64_t inx = i + nwarps;
    const int64_t bn = inx < end ? ld_stream_i64(a.off + inx, pf) : 0;
    const int64_t en = inx < end ? ld_stream_i64(a.off + inx + 1, pf) : 0;
    // the flag is the same for the whole warp; lane 0 alone changes it, after the shuffles below
    if (DYN && skip_unaffected32(a, v)) {
      __syncwarp();
      b = bn;
      e = en;
      continue;
    }
    Kahan acc;
    uint32_t yself = 0;
    gather32_vec<32, KV>(a, b, e, lane, v, acc, yself, pf, pl);
    acc.template group_reduce<32>();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) yself = max(yself, __shfl_xor_sync(0xffffffffu, yself, o));
    if (lane == 0) {
      uint32_t db, rb;
      finish32<DYN>(a, v, acc.value(), yself, pf, db, rb, fwsum);
      dmax = max(dmax, db);
      rmax = max(rmax, rb);
    }
    b = bn;
    e = en;
  }
  block_epilogue32<DYN>(a, dmax, rmax, fwsum);
}

template <int KV, bool DYN>
__global__ void __launch_bounds__(kThreads) k_sweep32_block(const Sweep32Args a_in, int64_t begin, int64_t end) {
  const Sweep32Args a = resolve32(a_in);
  if (converged32(a)) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  __shared__ float s_s[kThreads / 32], s_e[kThreads / 32];
  __shared__ uint32_t s_y[kThreads / 32];
  __shared__ int s_skip;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t dmax = 0, rmax = 0;
  uint64_t fwsum = 0;
  for (int64_t i = begin + blockIdx.x; i < end; i += gridDim.x) {
    const int32_t v = (int32_t)i;
    if (DYN) {
      if (threadIdx.x == 0) s_skip = skip_unaffected32(a, v) ? 1 : 0;
      __syncthreads();
      const int sk = s_skip;
      __syncthreads();
      if (sk) continue;
    }
    const int64_t b = a.off[v], e = a.off[v + 1];
    Kahan acc;
    uint32_t yself = 0;
    gather32_vec<kThreads, KV>(a, b, e, threadIdx.x, v, acc, yself, pf, pl);
    acc.template group_reduce<32>();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) yself = max(yself, __shfl_xor_sync(0xffffffffu, yself, o));
    if (lane == 0) {
      s_s[wid] = acc.s;
      s_e[wid] = acc.e;
      s_y[wid] = yself;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Kahan tot;
      uint32_t ym = 0;
      for (int k = 0; k < kThreads / 32; ++k) {
        tot.merge(s_s[k], s_e[k]);
        ym = max(ym, s_y[k]);
      }
      uint32_t db, rb;
      finish32<DYN>(a, v, tot.value(), ym, pf, db, rb, fwsum);
      dmax = max(dmax, db);
      rmax = max(rmax, rb);
    }
    __syncthreads();
  }
  block_epilogue32<DYN>(a, dmax, rmax, fwsum);
}

// Rows of the highest in-degree class in 1024-edge chunks (the hub chunk
// table): a warp per chunk stores the chunk's compensated sum (s, e); a warp
// per hub vertex merges its chunks' sums, lanes striding over the chunks and
// a fixed shuffle tree after them, so every run gives the same bits. Long
// rows no longer serialise on one block. DF / DF-P skip unaffected hubs as
// the FP64 hub kernels do.
template <bool DYN>
__global__ void __launch_bounds__(kThreads) k_sweep32_hub_part(const Sweep32Args a_in) {
  const Sweep32Args a = resolve32(a_in);
  if (converged32(a)) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t c = warp; c < a.hub.nchunk; c += nwarps) {
    const int32_t v = (int32_t)(a.hub.begin + a.hub.chunk_hub[c]);
    if (DYN && !a.dV[v]) continue;  // the same flag on every lane
    const int64_t jb = a.hub.chunk_j0[c];
    const int64_t re = a.off[v + 1];
    const int64_t je = jb + kHubChunk < re ? jb + kHubChunk : re;
    Kahan acc;
    uint32_t unused = 0;
    gather32_vec<32, 2>(a, jb, je, lane, v, acc, unused, pf, pl);
    acc.template group_reduce<32>();
    if (lane == 0) a.hub_part[c] = make_float2(acc.s, acc.e);
  }
}

template <bool DYN>
__global__ void __launch_bounds__(kThreads) k_sweep32_hub_finish(const Sweep32Args a_in) {
  const Sweep32Args a = resolve32(a_in);
  if (converged32(a)) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  uint32_t dmax = 0, rmax = 0;
  uint64_t fwsum = 0;
  for (int64_t h = warp; h < a.hub.nhub; h += nwarps) {
    const int32_t v = (int32_t)(a.hub.begin + h);
    if (DYN) {
      // every lane reads the flag before lane 0 may change it
      const bool skip = __shfl_sync(0xffffffffu, lane == 0 ? (int)(a.dV[v] == 0) : 0, 0) != 0;
      if (skip) {
        if (lane == 0) skip_unaffected32(a, v);
        continue;
      }
    }
    Kahan tot;
    for (int64_t c = a.hub.hub_first[h] + lane; c < a.hub.hub_first[h + 1]; c += 32) {
      const float2 x = a.hub_part[c];
      tot.merge(x.x, x.y);
    }
    tot.template group_reduce<32>();
    if (lane == 0) {
      uint32_t db, rb;
      finish32<DYN>(a, v, tot.value(), ld_gather_b32(a.y + v, pl), pf, db, rb, fwsum);
      dmax = max(dmax, db);
      rmax = max(rmax, rb);
    }
  }
  block_epilogue32<DYN>(a, dmax, rmax, fwsum);
}

enum Kind32 { kT1 = 0, kT4, kG4, kG8, kG16, kG16U8, kWarp, kBlock };

// the FP64 sweep's shapes: lanes x indices per lane sized to the class's rows
Kind32 class_kind32(const PartThr& t, int c) {
  const int C = t.n + 1;
  if (c == C - 1) return kBlock;
  if (c == C - 2 && C >= 3) return kWarp;
  const int64_t hi = t.thr[c];
  if (hi <= 1) return kT1;
  if (hi <= 4) return kT4;
  if (hi <= 16) return kG4;
  if (hi <= 32) return kG8;
  // 16 lanes; 8 indices per lane only when every row of the class is longer than 64
  if (hi <= 128) return (c > 0 && t.thr[c - 1] >= 64) ? kG16U8 : kG16;
  return kWarp;
}

// As in the FP64 sweep: almost no shared memory, so the unified L1 / shared
// storage goes to L1, which holds the gathered y of the hottest sources.
template <typename K>
void prefer_l1_32(K k) {
  // a preference the driver declines is not an error: clear what this call set
  if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 0) != cudaSuccess) cudaGetLastError();
}

template <bool DYN>
bool prefer_l1_all32() {
  prefer_l1_32(k_sweep32_group<1, 1, true, DYN>);
  prefer_l1_32(k_sweep32_group<1, 1, false, DYN>);
  prefer_l1_32(k_sweep32_group<1, 4, false, DYN>);
  prefer_l1_32(k_sweep32_group<4, 4, false, DYN>);
  prefer_l1_32(k_sweep32_group<8, 4, false, DYN>);
  prefer_l1_32(k_sweep32_group<16, 4, false, DYN>);
  prefer_l1_32(k_sweep32_group<16, 8, false, DYN>);
  prefer_l1_32(k_sweep32_warp<2, DYN>);
  prefer_l1_32(k_sweep32_block<4, DYN>);
  prefer_l1_32(k_sweep32_hub_part<DYN>);
  return true;
}

template <bool DYN>
int launch_all32(const Sweep32Args& a, const PartThr& t, const int64_t* cb, cudaStream_t s) {
  // Static form only: the DF / DF-P kernels run at 32-40 registers, eight
  // blocks per SM, and the smallest shared-memory carve-out leaves room for
  // fewer of them (measured: mixed DF-P 15 % slower with it)
  static const bool carveout_set = DYN ? false : prefer_l1_all32<DYN>();
  (void)carveout_set;
  const int maxg = kSMs * 8;
  const int C = t.n + 1;
  for (int c = 0; c < C; ++c) {
    const int64_t b = cb[c], e = cb[c + 1];
    if (e <= b) continue;
    const int64_t cnt = e - b;
    const Kind32 kind = class_kind32(t, c);
    const bool self1 = a.self_loops && kind == kT1 && t.thr[c] <= 1;
    switch (kind) {
      case kT1:
        if (self1) k_sweep32_group<1, 1, true, DYN><<<grid_for(cnt, kThreads, maxg), kThreads, 0, s>>>(a, b, e);
        else k_sweep32_group<1, 1, false, DYN><<<grid_for(cnt, kThreads, maxg), kThreads, 0, s>>>(a, b, e);
        break;
      case kT4: k_sweep32_group<1, 4, false, DYN><<<grid_for(cnt, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      case kG4: k_sweep32_group<4, 4, false, DYN><<<grid_for(cnt * 4, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      // The DF / DF-P form is not pipelined: a row longer than its item's G*U
      // slots costs extra round trips, so it keeps 16 lanes x 8 indices for
      // in-degree 17..128 (the Static form measured faster with 8 x 4 and 16 x 4)
      case kG8:
        if (DYN) k_sweep32_group<16, 8, false, DYN><<<grid_for(cnt * 16, kThreads, maxg), kThreads, 0, s>>>(a, b, e);
        else k_sweep32_group<8, 4, false, DYN><<<grid_for(cnt * 8, kThreads, maxg), kThreads, 0, s>>>(a, b, e);
        break;
      case kG16:
        if (DYN) k_sweep32_group<16, 8, false, DYN><<<grid_for(cnt * 16, kThreads, maxg), kThreads, 0, s>>>(a, b, e);
        else k_sweep32_group<16, 4, false, DYN><<<grid_for(cnt * 16, kThreads, maxg), kThreads, 0, s>>>(a, b, e);
        break;
      case kG16U8: k_sweep32_group<16, 8, false, DYN><<<grid_for(cnt * 16, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      case kWarp: k_sweep32_warp<2, DYN><<<grid_for(cnt * 32, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      default:
        if (a.hub.nchunk > 0 && a.hub.begin == b && a.hub.nhub == cnt && a.hub_part) {
          k_sweep32_hub_part<DYN><<<grid_for(a.hub.nchunk * 32, kThreads, maxg), kThreads, 0, s>>>(a);
          k_sweep32_hub_finish<DYN><<<grid_for(cnt * 32, kThreads, maxg), kThreads, 0, s>>>(a);
        } else {
          k_sweep32_block<4, DYN><<<grid_for(cnt, 1, maxg), kThreads, 0, s>>>(a, b, e);
        }
        break;
    }
  }
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

}  // namespace

int launch_sweep32(const Sweep32Args& a, const PartThr& t, const int64_t* cb, bool dynamic, cudaStream_t s) {
  return dynamic ? launch_all32<true>(a, t, cb, s) : launch_all32<false>(a, t, cb, s);
}

int launch_iter_check32(int* ctl, const uint32_t* resid_base, float tol_rel, int max_iter,
                        cudaGraphConditionalHandle h, cudaStream_t s) {
  k_iter_check32<<<1, 1, 0, s>>>(ctl, resid_base, tol_rel, max_iter, h);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

}  // namespace prdf
