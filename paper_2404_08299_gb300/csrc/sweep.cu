// Synchronous, pull-based, atomics-free rank sweeps (Alg. update of
// arXiv 2404.08299) for Static (Eq. 1, every vertex) and DF / DF-P
// (Eq. 1 / Eq. 2 on affected vertices, with prune and expand flags).
//
// State: x[u] = R[u] / |out(u)|, so a sweep gathers one FP64 value per
// in-edge. The sweeps run on the class-contiguous numbering (relabel.cu):
// class c is the id range [begin, end). Vertices are split by in-degree class (the paper's thread- and
// block-per-vertex kernels, refined into narrower classes so the lanes of a
// warp carry similar work): each vertex is processed by a group of G lanes
// (G = 1, 4, 16, 32) or by a whole block. The L-inf change of the sweep is
// reduced in the epilogue (warp max, block max, one 64-bit atomic max per
// block on the bit pattern of a non-negative double); rank writes stay one
// plain store per vertex.
//
// GB300 issues FP64 instructions at ~1.6 per clock per SM, so gathered
// values stay in 64-bit integer registers and are summed exactly on the
// integer pipes (common.cuh); FP64 arithmetic is limited to a few
// instructions per vertex.
//
// A sweep whose predecessor already met the tolerance exits at once, so the
// host can launch several sweeps ahead of its convergence check.
#include "internal.cuh"

namespace prdf {

namespace {

constexpr int kThreads = 256;
// four blocks of 256 threads per SM (64 registers a thread): the sweeps are
// bound by the latency of their gathers, so resident warps matter more than
// registers (at 70 registers a thread the DF-P warp kernel ran 3 blocks per SM
// and took 1.5x the time of the same work at 64). The block-per-vertex kernel
// and the 8-indices-per-lane group need more registers and keep three.
constexpr int kMinBlocks = 4;

// Exact accumulator (4 x 32-bit words, 2^-124 resolution) or plain FP64.
template <bool EXACT>
struct Acc;

template <>
struct Acc<true> {
  Fix4 v;
  __device__ __forceinline__ void add(uint64_t xb) { v.add(xb); }
  // add_w1: only for terms with in_w1 (the common window, three-word add)
  __device__ __forceinline__ static bool in_w1(uint64_t xb) { return Fix4::in_w1(xb); }
  __device__ __forceinline__ void add_w1(uint64_t xb) { v.add_w1(xb); }
  __device__ __forceinline__ void merge(const Acc& o) { v.add4(o.v.w0, o.v.w1, o.v.w2, o.v.w3); }
  __device__ __forceinline__ Acc shfl_up(int o) const {
    Acc r;
    r.v.w0 = __shfl_up_sync(0xffffffffu, v.w0, o);
    r.v.w1 = __shfl_up_sync(0xffffffffu, v.w1, o);
    r.v.w2 = __shfl_up_sync(0xffffffffu, v.w2, o);
    r.v.w3 = __shfl_up_sync(0xffffffffu, v.w3, o);
    return r;
  }
  __device__ __forceinline__ Acc shfl_idx(int l) const {
    Acc r;
    r.v.w0 = __shfl_sync(0xffffffffu, v.w0, l);
    r.v.w1 = __shfl_sync(0xffffffffu, v.w1, l);
    r.v.w2 = __shfl_sync(0xffffffffu, v.w2, l);
    r.v.w3 = __shfl_sync(0xffffffffu, v.w3, l);
    return r;
  }
  template <int G>
  __device__ __forceinline__ void group_reduce() { v.template group_reduce<G>(); }
  __device__ __forceinline__ double value() const { return v.to_double(); }
  __device__ __forceinline__ void to_shared(uint32_t* s) const { v.store(s); }
  __device__ __forceinline__ void from_shared(const uint32_t* s) { v.add_words(s); }
};

template <>
struct Acc<false> {
  double v = 0;
  __device__ __forceinline__ void add(uint64_t xb) { v += bitsd(xb); }
  __device__ __forceinline__ static bool in_w1(uint64_t) { return true; }
  __device__ __forceinline__ void add_w1(uint64_t xb) { v += bitsd(xb); }
  __device__ __forceinline__ void merge(const Acc& o) { v += o.v; }
  __device__ __forceinline__ Acc shfl_up(int o) const {
    Acc r;
    r.v = __shfl_up_sync(0xffffffffu, v, o);
    return r;
  }
  __device__ __forceinline__ Acc shfl_idx(int l) const {
    Acc r;
    r.v = __shfl_sync(0xffffffffu, v, l);
    return r;
  }
  template <int G>
  __device__ __forceinline__ void group_reduce() {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __device__ __forceinline__ double value() const { return v; }
  __device__ __forceinline__ void to_shared(uint32_t* s) const {
    const uint64_t b = dbits(v);
    s[0] = (uint32_t)b;
    s[1] = (uint32_t)(b >> 32);
  }
  __device__ __forceinline__ void from_shared(const uint32_t* s) {
    v += bitsd(((uint64_t)s[1] << 32) | s[0]);
  }
};

// Per-lane gather over row [b, e) of G' with stride G and U loads in flight.
template <int G, int U, bool EXACT>
__device__ __forceinline__ void gather_row(const SweepArgs& a, int64_t b, int64_t e, int lane, int32_t v,
                                           Acc<EXACT>& acc, uint64_t& xself, uint64_t pf, uint64_t pl) {
  for (int64_t j0 = b + lane; j0 < e; j0 += (int64_t)G * U) {
    int32_t u[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t j = j0 + (int64_t)k * G;
      u[k] = j < e ? ld_stream_i32(a.adj + j, pf) : -1;
    }
    uint64_t xv[U];
#pragma unroll
    for (int k = 0; k < U; ++k) xv[k] = u[k] >= 0 ? ld_gather_b64(a.x + u[k], pl) : 0ull;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (u[k] >= 0) acc.add(xv[k]);
      xself = (u[k] == v) ? xv[k] : xself;
    }
  }
}

// Vectorised variant for a row handled by NT lanes: 16-byte index loads for
// the aligned body (KV of them in flight per lane), scalar head and tail;
// row_indices issues a row's first indices, gather_row_from consumes them.
// (A warp kernel that loaded the next row's first indices a turn ahead needed
// 76 registers, ran three blocks per SM instead of four and was 4 % slower.)
template <int KV>
struct RowIdx {
  int64_t ba = 0, ea = 0;  // aligned body [ba, ea)
  int32_t uh = -1;         // this lane's head or tail entry (the unaligned ends), -1: none
  int4 u4[KV];             // this lane's first body indices
};

template <int NT, int KV>
__device__ __forceinline__ void row_indices(const SweepArgs& a, int64_t b, int64_t e, int lane, uint64_t pf,
                                            RowIdx<KV>& r) {
  int64_t ba = (b + 3) & ~(int64_t)3;
  if (ba > e) ba = e;
  const int64_t ea = ba + ((e - ba) & ~(int64_t)3);
  r.ba = ba;
  r.ea = ea;
  const int64_t nh = ba - b, nt = e - ea;
  int64_t j = -1;
  if (lane < nh) j = b + lane;
  else if (lane >= 4 && lane < 4 + nt) j = ea + (lane - 4);
  r.uh = j >= 0 ? ld_stream_i32(a.adj + j, pf) : -1;
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    const int64_t q = ba + 4 * (int64_t)lane + 4 * (int64_t)NT * k;
    r.u4[k] = q < ea ? ld_stream_i32x4(a.adj + q, pf) : make_int4(-1, -1, -1, -1);
  }
}

// The head / tail term's gather is issued with the body's first gathers and
// added after them, so the row costs one gather round trip before its first
// add. The body loads the next chunk's indices while this chunk's gathers are
// in flight; the loop runs the same trip count on all NT lanes, so each warp
// is converged at the vote below.
template <int NT, int KV, bool EXACT, bool SELF = true>
__device__ __forceinline__ void gather_row_from(const SweepArgs& a, const RowIdx<KV>& r, int lane, int32_t v,
                                                Acc<EXACT>& acc, uint64_t& xself, uint64_t pf, uint64_t pl) {
  const int64_t ba = r.ba, ea = r.ea;
  const int32_t uh = r.uh;
  const int64_t step = 4 * (int64_t)NT * KV;
  int4 u4[KV];
#pragma unroll
  for (int k = 0; k < KV; ++k) u4[k] = r.u4[k];
  uint64_t xh = uh >= 0 ? ld_gather_b64(a.x + uh, pl) : 0ull;
  bool head = uh >= 0;  // the head term is still to be added
  for (int64_t base = ba; base < ea; base += step) {
    const int64_t q0 = base + 4 * (int64_t)lane;
    uint64_t xv[4 * KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      xv[4 * k + 0] = u4[k].x >= 0 ? ld_gather_b64(a.x + u4[k].x, pl) : 0ull;
      xv[4 * k + 1] = u4[k].y >= 0 ? ld_gather_b64(a.x + u4[k].y, pl) : 0ull;
      xv[4 * k + 2] = u4[k].z >= 0 ? ld_gather_b64(a.x + u4[k].z, pl) : 0ull;
      xv[4 * k + 3] = u4[k].w >= 0 ? ld_gather_b64(a.x + u4[k].w, pl) : 0ull;
    }
    int4 nx[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int64_t q = q0 + step + 4 * (int64_t)NT * k;
      nx[k] = q < ea ? ld_stream_i32x4(a.adj + q, pf) : make_int4(-1, -1, -1, -1);
    }
    if (head) {
      acc.add(xh);
      if (SELF) xself = (uh == v) ? xh : xself;
      head = false;
    }
    bool w1 = true;
#pragma unroll
    for (int k = 0; k < KV; ++k)
#pragma unroll
      for (int q = 0; q < 4; ++q) w1 = w1 && (u4[k].x < 0 || Acc<EXACT>::in_w1(xv[4 * k + q]));
    if (__all_sync(0xffffffffu, w1)) {
#pragma unroll
      for (int k = 0; k < KV; ++k) {
        if (u4[k].x < 0) continue;  // a whole int4 is valid or not
#pragma unroll
        for (int q = 0; q < 4; ++q) acc.add_w1(xv[4 * k + q]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < KV; ++k) {
        if (u4[k].x < 0) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) acc.add(xv[4 * k + q]);
      }
    }
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      if (u4[k].x < 0) continue;
      if (SELF) {
        xself = (u4[k].x == v) ? xv[4 * k + 0] : xself;
        xself = (u4[k].y == v) ? xv[4 * k + 1] : xself;
        xself = (u4[k].z == v) ? xv[4 * k + 2] : xself;
        xself = (u4[k].w == v) ? xv[4 * k + 3] : xself;
      }
    }
#pragma unroll
    for (int k = 0; k < KV; ++k) u4[k] = nx[k];
  }
  if (head) {  // rows without a body chunk
    acc.add(xh);
    if (SELF) xself = (uh == v) ? xh : xself;
  }
}

template <int NT, int KV, bool EXACT, bool SELF = true>
__device__ __forceinline__ void gather_row_vec(const SweepArgs& a, int64_t b, int64_t e, int lane, int32_t v,
                                               Acc<EXACT>& acc, uint64_t& xself, uint64_t pf, uint64_t pl) {
  RowIdx<KV> r;
  row_indices<NT, KV>(a, b, e, lane, pf, r);
  gather_row_from<NT, KV, EXACT, SELF>(a, r, lane, v, acc, xself, pf, pl);
}

// Exact integer value of an out-degree held as a double (an integer below
// 2^53), decoded from its bit pattern on the integer pipes; 0 for 0.
__device__ __forceinline__ uint64_t degree_of(double d) {
  const uint64_t b = dbits(d);
  const int e = (int)(b >> 52) - 1023;
  const uint64_t mant = (b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
  return e >= 0 ? mant >> (52 - e) : 0ull;
}

// Vertex epilogue: Eq. 1 (Static, DF) or Eq. 2 (DF-P), prune / expand flags,
// next x, and this vertex's |r - R[v]| as bits. GB300's FP64 pipe is narrow,
// so FP64 instructions are kept to those that need FP64 rounding: three on the
// Static path (r, |r - R[v]| as one FMA, next x); on the DF-P path also
// Eq. 2's two extra steps, R[v] and the threshold tau * max(r, R[v]). The
// maximum and the comparisons run on the bit patterns of the non-negative
// doubles (integer instructions, the same order as the FP64 comparison; a
// negative threshold's pattern is negative as int64, so it orders below every
// non-negative value, as in FP64).
template <bool DYN>
__device__ __forceinline__ uint64_t finish_vertex(const SweepArgs& a, int32_t v, double c, uint64_t xself_b,
                                                  uint64_t pf, uint64_t& fwsum, uint8_t dn_old) {
  const double xself = bitsd(xself_b);
  const double d = ld_stream_f64(a.degd + v, pf);
  double r;
  if (DYN && a.prune) {
    // Eq. 2: the self-loop term is solved in closed form (factor precomputed per vertex)
    r = ld_stream_f64(a.kf + v, pf) * (a.c0 + a.alpha * (c - xself));
  } else {
    r = fma(a.alpha, c, a.c0);  // Eq. 1
  }
  // |r - R[v]| with R[v] = x[v] * |out(v)| of the previous iteration, one rounding
  const double dr = fabs(fma(xself, -d, r));
  if (DYN) {
    const uint64_t rb = dbits(r), ob = dbits(xself * d), drb = dbits(dr);
    const double m = bitsd(rb > ob ? rb : ob);  // max(r, R[v])
    const int64_t tp = (int64_t)dbits(a.tau_p * m);
    const int64_t tf = a.tau_f == a.tau_p ? tp : (int64_t)dbits(a.tau_f * m);
    if (a.prune && (int64_t)drb <= tp) a.dV[v] = 0;
    // deltaN holds exactly this sweep's expand set: set or cleared for every vertex; the out-edges of
    // the set are counted for the choice of the expansion round's direction
    // (dn_old: the vertex's deltaN flag before this sweep, read ahead; no load on this path)
    if ((int64_t)drb > tf) {
      if (!dn_old) a.dN[v] = 1;
      fwsum += degree_of(d);
    } else if (dn_old) {
      a.dN[v] = 0;
    }
    a.wrote[v] = 1;
  }
  a.xn[v] = r * ld_stream_f64(a.inv_deg + v, pf);
  return dbits(dr);
}

// per-iteration pointers of the graph-driven loop
__device__ __forceinline__ SweepArgs resolve(const SweepArgs& in) {
  if (!in.ctl) return in;
  SweepArgs a = in;
  const int it = in.ctl[0];
  a.x = (it & 1) ? in.xb : in.xa;
  a.xn = (it & 1) ? const_cast<double*>(in.xa) : in.xb;
  a.resid = in.resid_base + it;
  a.prev = it > 0 ? in.resid_base + it - 1 : nullptr;
  a.fw = in.fw_base ? in.fw_base + it : nullptr;
  return a;
}

__global__ void k_iter_check(int* ctl, const uint64_t* resid_base, double tol, int max_iter,
                             cudaGraphConditionalHandle h) {
  const int it = ctl[0];
  const bool done = bitsd(resid_base[it]) <= tol || it + 1 >= max_iter;
  ctl[0] = it + 1;
  cudaGraphSetConditional(h, done ? 0u : 1u);
}

// DF / DF-P: an unaffected vertex keeps its rank; its slot in xn is stale
// only if the previous sweep wrote it (then copy it through). It is not in
// this sweep's expand set, so its deltaN flag is cleared (the sweep keeps
// deltaN exact without a separate clearing pass).
__device__ __forceinline__ bool skip_unaffected(const SweepArgs& a, int32_t v) {
  if (a.dV[v]) return false;
  if (a.wrote[v]) {
    a.xn[v] = a.x[v];
    a.wrote[v] = 0;
  }
  if (a.dN[v]) a.dN[v] = 0;
  return true;
}

// The three flags of a vertex, read ahead of its turn: a vertex's flags change
// during a sweep only in its own epilogue or skip, so a read issued earlier in
// the sweep sees the values of the previous sweep, which is what the skip and
// the epilogue need, and the loads leave the critical path.
struct Flags {
  uint8_t dv = 1, wr = 0, dn = 0;
};
__device__ __forceinline__ Flags load_flags(const SweepArgs& a, int32_t v) {
  Flags f;
  f.dv = a.dV[v];
  f.wr = a.wrote[v];
  f.dn = a.dN[v];
  return f;
}
// skip_unaffected with the flags read ahead
__device__ __forceinline__ void skip_vertex(const SweepArgs& a, int32_t v, const Flags& f) {
  if (f.wr) {
    a.xn[v] = a.x[v];
    a.wrote[v] = 0;
  }
  if (f.dn) a.dN[v] = 0;
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

// Sweep epilogue of a block: the L-inf change (max) and, for DF / DF-P, the
// out-edges of the vertices put into deltaN (sum, when fw is given).
template <bool DYN>
__device__ __forceinline__ void block_epilogue(const SweepArgs& a, uint64_t dmax, uint64_t fwsum) {
  block_max_to(dmax, a.resid);
  if (DYN && a.fw) {
    __shared__ uint64_t shs[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    fwsum = (uint64_t)warp_sum_i64((int64_t)fwsum);
    __syncthreads();  // shs is written after every warp left block_max_to's shared reads
    if (lane == 0) shs[wid] = fwsum;
    __syncthreads();
    if (wid == 0) {
      uint64_t x = lane < (int)(blockDim.x >> 5) ? shs[lane] : 0;
      x = (uint64_t)warp_sum_i64((int64_t)x);
      if (lane == 0 && x) atomicAdd((unsigned long long*)a.fw, (unsigned long long)x);
    }
  }
}

// Work item of a group: list entry, vertex, its row of G' and the first
// G*U indices of the row (this lane's share), and (DF / DF-P) its flags.
template <int U>
struct Item {
  int32_t v;
  int64_t b, e;
  int32_t u[U];
  Flags f;
  bool self_only;  // the row is [v] (in-degree <= 1 class, no in-edges added since the numbering)
};

// G lanes per vertex (G = 1, 4, 16), U indices per lane per round. The loop is
// uniform across each warp (a warp owns 32/G consecutive list entries per
// step), so the group shuffles always see all 32 lanes. Software pipeline:
// the list entry of the item two steps ahead (and its affected flag) and the
// offsets, first indices and other flags of the next item are loaded while
// the current item's gathers are in flight, so a step costs about one memory
// round trip instead of four. With self-loops on every vertex, a row of length 1 is [v] itself and needs
// no offsets or indices.
template <int G, int U, bool EXACT, bool DYN, bool SELF1>
__global__ void __launch_bounds__(kThreads, U >= 8 ? 3 : kMinBlocks) k_sweep_group(const SweepArgs a_in, int64_t begin,
                                                                                  int64_t end) {
  const SweepArgs a = resolve(a_in);
  if (a.prev && bitsd(*a.prev) <= a.tol) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  constexpr int kGroupsPerWarp = 32 / G;
  const int lane = (G == 1) ? 0 : (threadIdx.x & (G - 1));
  const int gw = (threadIdx.x & 31) / G;  // group within warp
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int64_t step = nwarps * kGroupsPerWarp;
  uint64_t dmax = 0, fwsum = 0;

  auto load_v = [&](int64_t i) -> int32_t { return i < end ? (int32_t)i : -1; };
  auto load_dv = [&](int32_t v) -> uint8_t { return (DYN && v >= 0) ? a.dV[v] : (uint8_t)1; };
  // DF / DF-P: the row of an unaffected vertex is not read
  auto load_item = [&](int32_t v, uint8_t dv, Item<U>& it) {
    it.v = v;
    it.b = 0;
    it.e = 0;
    it.f = Flags();
    if (DYN && v >= 0) {
      it.f.dv = dv;
      it.f.wr = a.wrote[v];
      it.f.dn = a.dN[v];
    }
    const bool live = v >= 0 && dv;
    // the row is [v] unless a batch gave the vertex in-edges (its bit in multi)
    const bool self_only = SELF1 && !(live && a.multi && ((a.multi[v >> 5] >> (v & 31)) & 1u));
    it.self_only = self_only;
    if (live) {
      if (self_only) {
        it.b = 0;
        it.e = 1;
      } else {
        it.b = ld_stream_i64(a.off + v, pf);
        it.e = ld_stream_i64(a.off + v + 1, pf);
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t j = it.b + lane + (int64_t)k * G;
      if (self_only) it.u[k] = (live && k == 0 && lane == 0) ? v : -1;
      else it.u[k] = (live && j < it.e) ? ld_stream_i32(a.adj + j, pf) : -1;
    }
  };

  // The row offsets run one more step ahead (offsets of the item two steps
  // ahead, indices of the next), so a step waits for one round trip. In DF /
  // DF-P the affected flag runs three steps ahead, so that offsets and indices
  // are loaded only for affected vertices.
  constexpr bool kOffAhead = !DYN && !SELF1;
  constexpr bool kDynAhead = DYN && !SELF1;
  auto load_off = [&](int32_t v, int64_t& b, int64_t& e) {
    b = v >= 0 ? ld_stream_i64(a.off + v, pf) : 0;
    e = v >= 0 ? ld_stream_i64(a.off + v + 1, pf) : 0;
  };
  auto load_idx = [&](int32_t v, int64_t b, int64_t e, Item<U>& it) {
    it.v = v;
    it.b = b;
    it.e = e;
    it.f = Flags();
    it.self_only = false;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t j = b + lane + (int64_t)k * G;
      it.u[k] = (v >= 0 && j < e) ? ld_stream_i32(a.adj + j, pf) : -1;
    }
  };

  int64_t base = begin + warp * kGroupsPerWarp;
  Item<U> cur;
  {
    const int32_t v0 = load_v(base + gw);
    load_item(v0, load_dv(v0), cur);
  }
  int32_t v_next = load_v(base + step + gw);
  uint8_t dv_next = load_dv(v_next);
  int64_t nb = 0, ne = 0;  // kOffAhead, kDynAhead: row offsets of v_next (when affected)
  if (kOffAhead) load_off(v_next, nb, ne);
  int32_t v_n2 = -1;  // kDynAhead: the list entry two steps ahead and its affected flag
  uint8_t dv_n2 = 0;
  if (kDynAhead) {
    load_off((v_next >= 0 && dv_next) ? v_next : -1, nb, ne);
    v_n2 = load_v(base + 2 * step + gw);
    dv_n2 = load_dv(v_n2);
  }
  for (; base < end; base += step) {
    // gathers of the current item
    uint64_t xv[U];
#pragma unroll
    for (int k = 0; k < U; ++k) xv[k] = cur.u[k] >= 0 ? ld_gather_b64(a.x + cur.u[k], pl) : 0ull;
    // prefetch: next item's row, first indices and flags, and the list entry (and flag) after it
    Item<U> nxt;
    if (kOffAhead) {
      load_idx(v_next, nb, ne, nxt);
      v_next = load_v(base + 2 * step + gw);
      load_off(v_next, nb, ne);
    } else if (kDynAhead) {
      const bool live = v_next >= 0 && dv_next;
      load_idx(live ? v_next : -1, nb, ne, nxt);
      nxt.v = v_next;
      if (v_next >= 0) {
        nxt.f.dv = dv_next;
        nxt.f.wr = a.wrote[v_next];
        nxt.f.dn = a.dN[v_next];
      }
      v_next = v_n2;
      dv_next = dv_n2;
      load_off((v_next >= 0 && dv_next) ? v_next : -1, nb, ne);
      v_n2 = load_v(base + 3 * step + gw);
      dv_n2 = load_dv(v_n2);
    } else {
      load_item(v_next, dv_next, nxt);
      v_next = load_v(base + 2 * step + gw);
      dv_next = load_dv(v_next);
    }

    // the warp is converged here (uniform loop): one vote picks the
    // three-word add when every gathered term of the step is in the common window
    bool w1 = true;
#pragma unroll
    for (int k = 0; k < U; ++k) w1 = w1 && (cur.u[k] < 0 || Acc<EXACT>::in_w1(xv[k]));
    const bool all_w1 = __all_sync(0xffffffffu, w1);
    bool active = cur.v >= 0;
    if (DYN && active && !cur.f.dv) {
      if (lane == 0) skip_vertex(a, cur.v, cur.f);
      active = false;
    }
    if (SELF1 && cur.self_only) {
      // row [v] (one lane per item): the in-neighbour sum is the single term x[v], exactly
      if (active) {
        const uint64_t db = finish_vertex<DYN>(a, cur.v, bitsd(xv[0]), xv[0], pf, fwsum, cur.f.dn);
        dmax = db > dmax ? db : dmax;
      }
      cur = nxt;
      continue;
    }
    // DF / DF-P: a step in which no item of the warp is affected (most steps of
    // the first sweeps after a small batch) has nothing to reduce. (Every lane
    // reaches the vote: only the SELF1 form leaves the step early, per lane.)
    if (DYN && !SELF1 && !__any_sync(0xffffffffu, active)) {
      cur = nxt;
      continue;
    }
    Acc<EXACT> acc;
    uint64_t xself = 0;
    if (active) {
      if (all_w1) {
#pragma unroll
        for (int k = 0; k < U; ++k)
          if (cur.u[k] >= 0) acc.add_w1(xv[k]);
      } else {
#pragma unroll
        for (int k = 0; k < U; ++k)
          if (cur.u[k] >= 0) acc.add(xv[k]);
      }
#pragma unroll
      for (int k = 0; k < U; ++k) xself = (cur.u[k] == cur.v) ? xv[k] : xself;
      // rest of a row longer than G*U (rows that grew past their class's bound in a batch update)
      if (cur.e - cur.b > (int64_t)G * U)
        gather_row<G, U, EXACT>(a, cur.b + (int64_t)G * U, cur.e, lane, cur.v, acc, xself, pf, pl);
    }
    if (G > 1) {
      acc.template group_reduce<G>();
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        const uint64_t t = __shfl_xor_sync(0xffffffffu, xself, o);
        xself = t > xself ? t : xself;
      }
    }
    if (active && lane == 0) {
      const uint64_t db = finish_vertex<DYN>(a, cur.v, acc.value(), xself, pf, fwsum, cur.f.dn);
      dmax = db > dmax ? db : dmax;
    }
    cur = nxt;
  }
  block_epilogue<DYN>(a, dmax, fwsum);
}

// one warp per vertex, 16-byte index loads; the next vertex's list entry, row
// offsets and (DF / DF-P) flags are loaded while the current row is gathered
template <int KV, bool EXACT, bool DYN>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_sweep_warp(const SweepArgs a_in, int64_t begin, int64_t end) {
  const SweepArgs a = resolve(a_in);
  if (a.prev && bitsd(*a.prev) <= a.tol) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  uint64_t dmax = 0, fwsum = 0;
  int64_t i = begin + warp;
  int32_t v = i < end ? (int32_t)i : -1;
  int64_t b = v >= 0 ? ld_stream_i64(a.off + v, pf) : 0, e = v >= 0 ? ld_stream_i64(a.off + v + 1, pf) : 0;
  Flags f;
  if (DYN && v >= 0) f = load_flags(a, v);
  for (; i < end; i += nwarps) {
    const int64_t inx = i + nwarps;
    const int32_t vn = inx < end ? (int32_t)inx : -1;
    bool active = true;
    if (DYN && !f.dv) {
      if (lane == 0) skip_vertex(a, v, f);
      active = false;
    }
    Acc<EXACT> acc;
    // x[v], for R[v] of the previous iteration = x[v] * |out(v)|, issued ahead of the gathers
    uint64_t xself = (active && lane == 0) ? ld_gather_b64(a.x + v, pl) : 0ull;
    if (active) gather_row_vec<32, KV, EXACT, false>(a, b, e, lane, v, acc, xself, pf, pl);
    const int64_t bn = vn >= 0 ? ld_stream_i64(a.off + vn, pf) : 0, en = vn >= 0 ? ld_stream_i64(a.off + vn + 1, pf) : 0;
    Flags fn;
    if (DYN && vn >= 0) fn = load_flags(a, vn);
    if (active) acc.template group_reduce<32>();  // active is the same on every lane (one row per warp)
    if (active && lane == 0) {
      const uint64_t db = finish_vertex<DYN>(a, v, acc.value(), xself, pf, fwsum, f.dn);
      dmax = db > dmax ? db : dmax;
    }
    v = vn;
    b = bn;
    e = en;
    f = fn;
  }
  block_epilogue<DYN>(a, dmax, fwsum);
}

// one block per vertex (high in-degree)
template <int KV, bool EXACT, bool DYN>
__global__ void __launch_bounds__(kThreads, 3) k_sweep_block(const SweepArgs a_in, int64_t begin, int64_t end) {
  const SweepArgs a = resolve(a_in);
  if (a.prev && bitsd(*a.prev) <= a.tol) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  __shared__ uint32_t s_acc[kThreads / 32][4];
  __shared__ int s_skip;
  uint64_t dmax = 0, fwsum = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t i = begin + blockIdx.x; i < end; i += gridDim.x) {
    const int32_t v = (int32_t)i;
    if (DYN) {
      if (threadIdx.x == 0) s_skip = skip_unaffected(a, v) ? 1 : 0;
      __syncthreads();
      const int sk = s_skip;
      __syncthreads();
      if (sk) continue;
    }
    const int64_t b = a.off[v], e = a.off[v + 1];
    Acc<EXACT> acc;
    // x[v] for R[v] of the previous iteration, read by the thread that finishes the vertex
    uint64_t xb = (threadIdx.x == 0) ? ld_gather_b64(a.x + v, pl) : 0ull;
    gather_row_vec<kThreads, KV, EXACT, false>(a, b, e, threadIdx.x, v, acc, xb, pf, pl);
    acc.template group_reduce<32>();
    if (lane == 0) acc.to_shared(s_acc[wid]);
    __syncthreads();
    if (threadIdx.x == 0) {
      Acc<EXACT> tot;
      for (int k = 0; k < kThreads / 32; ++k) tot.from_shared(s_acc[k]);
      const uint64_t db = finish_vertex<DYN>(a, v, tot.value(), xb, pf, fwsum, DYN ? a.dN[v] : (uint8_t)0);
      dmax = db > dmax ? db : dmax;
    }
    __syncthreads();
  }
  block_epilogue<DYN>(a, dmax, fwsum);
}

// Rows of the highest in-degree class in 1024-edge chunks (the hub chunk
// table). A warp per chunk sums the chunk's terms and stores the partial sum;
// a warp per hub vertex adds its chunks' partials and finishes the vertex.
// With exact accumulation the partials are integers, so the result is the
// same bits as any other split; long rows no longer serialise on one block.
// DF / DF-P: chunks of unaffected hubs are skipped; the finishing warp copies
// an unaffected hub through. A hub's flag changes only in its finishing warp,
// which runs after every chunk of the sweep has read it.
template <bool EXACT, bool DYN>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_sweep_hub_part(const SweepArgs a_in) {
  const SweepArgs a = resolve(a_in);
  if (a.prev && bitsd(*a.prev) <= a.tol) return;
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
    Acc<EXACT> acc;
    uint64_t unused = 0;
    gather_row_vec<32, 2, EXACT, false>(a, jb, je, lane, v, acc, unused, pf, pl);
    acc.template group_reduce<32>();
    if (lane == 0) acc.to_shared(reinterpret_cast<uint32_t*>(a.hub_part + c));
  }
}

template <bool EXACT, bool DYN>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_sweep_hub_finish(const SweepArgs a_in) {
  const SweepArgs a = resolve(a_in);
  if (a.prev && bitsd(*a.prev) <= a.tol) return;
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  uint64_t dmax = 0, fwsum = 0;
  // a warp per hub vertex: lanes add strided chunk partials, then the warp reduces
  for (int64_t h = warp; h < a.hub.nhub; h += nwarps) {
    const int32_t v = (int32_t)(a.hub.begin + h);
    if (DYN) {
      // every lane reads the flag before lane 0 may change it
      const bool skip = __shfl_sync(0xffffffffu, lane == 0 ? (int)(a.dV[v] == 0) : 0, 0) != 0;
      if (skip) {
        if (lane == 0) skip_unaffected(a, v);
        continue;
      }
    }
    Acc<EXACT> tot;
    for (int64_t c = a.hub.hub_first[h] + lane; c < a.hub.hub_first[h + 1]; c += 32)
      tot.from_shared(reinterpret_cast<const uint32_t*>(a.hub_part + c));
    tot.template group_reduce<32>();
    if (lane == 0) {
      const uint64_t db =
          finish_vertex<DYN>(a, v, tot.value(), ld_gather_b64(a.x + v, pl), pf, fwsum, DYN ? a.dN[v] : (uint8_t)0);
      dmax = db > dmax ? db : dmax;
    }
  }
  block_epilogue<DYN>(a, dmax, fwsum);
}

// Kernel shape of class c: the last class is block-per-vertex, the one before
// it warp-per-vertex; lower classes by their upper degree bound.
enum Kind { kT1 = 0, kT4, kG4, kG8, kG16, kG16U8, kWarp, kBlock };

Kind class_kind(const PartThr& t, int c) {
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

// The sweep kernels use almost no shared memory: give the unified L1 /
// shared storage to L1, which holds the gathered x of the hottest sources.
template <typename K>
void prefer_l1(K k) {
  // a preference the driver declines is not an error: clear what this call set
  if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 0) != cudaSuccess) cudaGetLastError();
}

template <bool EXACT, bool DYN>
bool prefer_l1_all() {
  prefer_l1(k_sweep_group<1, 1, EXACT, DYN, true>);
  prefer_l1(k_sweep_group<1, 1, EXACT, DYN, false>);
  prefer_l1(k_sweep_group<1, 4, EXACT, DYN, false>);
  prefer_l1(k_sweep_group<4, 4, EXACT, DYN, false>);
  prefer_l1(k_sweep_group<8, 4, EXACT, DYN, false>);
  prefer_l1(k_sweep_group<16, 4, EXACT, DYN, false>);
  prefer_l1(k_sweep_group<16, 8, EXACT, DYN, false>);
  prefer_l1(k_sweep_warp<2, EXACT, DYN>);
  prefer_l1(k_sweep_block<4, EXACT, DYN>);
  prefer_l1(k_sweep_hub_part<EXACT, DYN>);
  return true;
}

template <bool EXACT, bool DYN>
int launch_all(const SweepArgs& a, const PartThr& t, const int64_t* cb, cudaStream_t s) {
  static const bool carveout_set = prefer_l1_all<EXACT, DYN>();
  (void)carveout_set;
  const int maxg = kSMs * 8;
  const int C = t.n + 1;
  for (int c = 0; c < C; ++c) {
    const int64_t b = cb[c], e = cb[c + 1];
    if (e <= b) continue;
    const int64_t cnt = e - b;
    const Kind kind = class_kind(t, c);
    // a class holding only rows of length <= 1 on a graph with all self-loops: the row is [v]
    const bool self1 = a.self_loops && kind == kT1 && t.thr[c] <= 1;
    switch (kind) {
      case kT1:
        if (self1) k_sweep_group<1, 1, EXACT, DYN, true><<<grid_for(cnt, kThreads, maxg), kThreads, 0, s>>>(a, b, e);
        else k_sweep_group<1, 1, EXACT, DYN, false><<<grid_for(cnt, kThreads, maxg), kThreads, 0, s>>>(a, b, e);
        break;
      case kT4: k_sweep_group<1, 4, EXACT, DYN, false><<<grid_for(cnt, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      case kG4: k_sweep_group<4, 4, EXACT, DYN, false><<<grid_for(cnt * 4, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      case kG8: k_sweep_group<8, 4, EXACT, DYN, false><<<grid_for(cnt * 8, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      case kG16: k_sweep_group<16, 4, EXACT, DYN, false><<<grid_for(cnt * 16, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      case kG16U8: k_sweep_group<16, 8, EXACT, DYN, false><<<grid_for(cnt * 16, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      case kWarp: k_sweep_warp<2, EXACT, DYN><<<grid_for(cnt * 32, kThreads, maxg), kThreads, 0, s>>>(a, b, e); break;
      default:
        if (a.hub.nchunk > 0 && a.hub.begin == b && a.hub.nhub == cnt && a.hub_part) {
          k_sweep_hub_part<EXACT, DYN><<<grid_for(a.hub.nchunk * 32, kThreads, maxg), kThreads, 0, s>>>(a);
          k_sweep_hub_finish<EXACT, DYN><<<grid_for(cnt * 32, kThreads, maxg), kThreads, 0, s>>>(a);
        } else {
          k_sweep_block<4, EXACT, DYN><<<grid_for(cnt, 1, maxg), kThreads, 0, s>>>(a, b, e);
        }
        break;
    }
  }
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

}  // namespace

int launch_iter_check(int* ctl, const uint64_t* resid_base, double tol, int max_iter,
                      cudaGraphConditionalHandle h, cudaStream_t s) {
  k_iter_check<<<1, 1, 0, s>>>(ctl, resid_base, tol, max_iter, h);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int launch_sweep(const SweepArgs& a, const PartThr& t, const int64_t* class_begin, bool exact, bool dynamic,
                 cudaStream_t s) {
  if (exact) return dynamic ? launch_all<true, true>(a, t, class_begin, s) : launch_all<true, false>(a, t, class_begin, s);
  return dynamic ? launch_all<false, true>(a, t, class_begin, s) : launch_all<false, false>(a, t, class_begin, s);
}

}  // namespace prdf
