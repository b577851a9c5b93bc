// Shared device/host helpers of libprdf (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>

#include "prdf.h"

namespace prdf {

// ------------------------------------------------------------ errors ----

void set_error(const char* fmt, ...);

struct Status {
  int code = PRDF_OK;
  bool ok() const { return code == PRDF_OK; }
};

#define PRDF_CUDA(call)                                                                             \
  do {                                                                                              \
    cudaError_t e__ = (call);                                                                       \
    if (e__ != cudaSuccess) {                                                                       \
      ::prdf::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e__));        \
      return e__ == cudaErrorMemoryAllocation ? PRDF_ENOMEM : PRDF_ECUDA;                           \
    }                                                                                               \
  } while (0)

#define PRDF_LAUNCH_CHECK() PRDF_CUDA(cudaGetLastError())

#define PRDF_TRY(expr)            \
  do {                            \
    int r__ = (expr);             \
    if (r__ != PRDF_OK) return r__; \
  } while (0)

// ------------------------------------------------------ device buffer ----
// The library's stream-ordered memory pool on the current device (created on
// first use, nullptr if that fails). Its release threshold is unbounded:
// blocks freed by one call stay mapped for the next, where the default pool
// hands them back to the driver at each synchronisation and large CSR and
// workspace buffers would be mapped again by every build and batch update.
// prdf_release_cached_memory() returns the unused reserve.
cudaMemPool_t device_pool();

// Stream-ordered device allocation (from device_pool()) owned by RAII.
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { *this = static_cast<DBuf&&>(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n; s = o.s;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  int alloc(size_t count, cudaStream_t stream) {
    release();
    s = stream;
    n = count;
    if (count == 0) return PRDF_OK;
    cudaMemPool_t pool = device_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync((void**)&p, count * sizeof(T), pool, stream)
                         : cudaMallocAsync((void**)&p, count * sizeof(T), stream);
    if (e != cudaSuccess) {
      p = nullptr;
      n = 0;
      set_error("device allocation of %zu bytes: %s", count * sizeof(T), cudaGetErrorString(e));
      return PRDF_ENOMEM;
    }
    return PRDF_OK;
  }
  // grow-only reuse
  int reserve(size_t count, cudaStream_t stream) {
    if (p && n >= count && s == stream) return PRDF_OK;
    return alloc(count, stream);
  }
};

// ------------------------------------------------------ launch shapes ----

constexpr int kSMs = 152;  // GB300: 2 dies x 76 SMs; grids are sized in multiples of this

inline int grid_for(int64_t work, int per_block, int cap_blocks = kSMs * 32) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap_blocks) b = cap_blocks;
  return (int)b;
}

// ----------------------------------------------------------- warp ops ----

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------- exact fixed-point summation ----
//
// GB300 issues FP64 additions at about 1.6 per clock per SM (measured), 70x
// below FP32, so an FP64 add per edge would bound the sweep by the FP64 pipe
// instead of HBM. In-neighbour sums of non-negative FP64 terms are therefore
// accumulated exactly in a 128-bit integer (four 32-bit words, resolution
// 2^-124) on the integer pipes, and the exact sum is rounded once to FP64
// (round to nearest, ties to even). The result is the correctly rounded sum,
// independent of summation order, so every kernel shape and thread count
// gives the same bits. Valid for terms in [0, 8) and sums below 16; a term
// below 2^-72 is dropped (absolute error < 2^-72 per term).

constexpr int kFixFrac = 124;

struct Fix4 {
  uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;  // value = (w3:w2:w1:w0) * 2^-124

  __device__ __forceinline__ void add4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3) {
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, %7;"
        : "+r"(w0), "+r"(w1), "+r"(w2), "+r"(w3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3));
  }

  // add the non-negative double whose bit pattern is xb
  __device__ __forceinline__ void add(uint64_t xb) {
    const uint32_t hi = (uint32_t)(xb >> 32), lo = (uint32_t)xb;
    const uint32_t e = (hi >> 20) & 0x7FFu;
    const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
    // the mantissa's least significant bit sits at 2^(e - 1075) = 2^-124 * 2^(e - 951)
    const int p = (int)e - (1075 - kFixFrac);
    const bool ok = p >= 0;
    const uint32_t pp = ok ? (uint32_t)p : 0u;
    const uint32_t b = pp & 31u, w = pp >> 5;
    const uint32_t t0 = lo << b;
    const uint32_t t1 = __funnelshift_l(lo, mh, b);
    const uint32_t t2 = __funnelshift_l(mh, 0u, b);
    const uint32_t ww = ok ? w : 3u;  // 3: a dropped term, every word zero
    const uint32_t a0 = ww == 0 ? t0 : 0u;
    const uint32_t a1 = ww == 0 ? t1 : (ww == 1 ? t0 : 0u);
    const uint32_t a2 = ww == 0 ? t2 : (ww == 1 ? t1 : (ww == 2 ? t0 : 0u));
    const uint32_t a3 = ww == 1 ? t2 : (ww == 2 ? t1 : 0u);
    add4(a0, a1, a2, a3);
  }

  // Terms in [2^-40, 2^-8) (biased exponent 983..1014) have their mantissa's
  // lowest bit in word 1 (w = 1 above): the image is (0, t0, t1, t2) with
  // b = e - 983, so the word selection and the dropped-term test fall away.
  // PageRank values of graphs with 2^8 .. 2^36 vertices divided by their
  // out-degree land in this window.
  __device__ __forceinline__ static bool in_w1(uint64_t xb) { return (uint32_t)(xb >> 52) - 983u < 32u; }
  __device__ __forceinline__ void add_w1(uint64_t xb) {
    const uint32_t hi = (uint32_t)(xb >> 32), lo = (uint32_t)xb;
    const uint32_t b = (hi >> 20) - 983u;
    const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
    const uint32_t t0 = lo << b;
    const uint32_t t1 = __funnelshift_l(lo, mh, b);
    const uint32_t t2 = __funnelshift_l(mh, 0u, b);
    asm("add.cc.u32 %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, %5;"
        : "+r"(w1), "+r"(w2), "+r"(w3)
        : "r"(t0), "r"(t1), "r"(t2));
  }

  __device__ __forceinline__ void add_words(const uint32_t* s) { add4(s[0], s[1], s[2], s[3]); }
  __device__ __forceinline__ void store(uint32_t* s) const {
    s[0] = w0;
    s[1] = w1;
    s[2] = w2;
    s[3] = w3;
  }

  template <int G>
  __device__ __forceinline__ void group_reduce() {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const uint32_t a0 = __shfl_xor_sync(0xffffffffu, w0, o);
      const uint32_t a1 = __shfl_xor_sync(0xffffffffu, w1, o);
      const uint32_t a2 = __shfl_xor_sync(0xffffffffu, w2, o);
      const uint32_t a3 = __shfl_xor_sync(0xffffffffu, w3, o);
      add4(a0, a1, a2, a3);
    }
  }

  // round to the nearest double, ties to even
  __device__ __forceinline__ double to_double() const {
    const uint64_t H = ((uint64_t)w3 << 32) | w2, L = ((uint64_t)w1 << 32) | w0;
    if ((H | L) == 0) return 0.0;
    const int lz = H ? __clzll((long long)H) : 64 + __clzll((long long)L);
    uint64_t nH, nL;
    if (lz == 0) {
      nH = H;
      nL = L;
    } else if (lz < 64) {
      nH = (H << lz) | (L >> (64 - lz));
      nL = L << lz;
    } else {
      nH = L << (lz - 64);
      nL = 0;
    }
    uint64_t mant = nH >> 11;  // 53 significant bits, leading one at bit 52
    const uint64_t rb = nH & 0x7FFull;
    const bool up = rb > 0x400ull || (rb == 0x400ull && (nL != 0 || (mant & 1ull)));
    mant += up ? 1ull : 0ull;
    int ex = (127 - lz) - kFixFrac;  // unbiased exponent of the leading one
    if (mant >> 53) {
      mant >>= 1;
      ++ex;
    }
    return __longlong_as_double((long long)(((uint64_t)(ex + 1023) << 52) | (mant & 0x000FFFFFFFFFFFFFull)));
  }
};

// non-negative doubles order like their bit patterns
__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(uint64_t b) { return __longlong_as_double((long long)b); }

// ----------------------------------------------------- cache hints ----
// The CSR index stream is read once per sweep: load it through an L2
// evict-first access policy so the gathered rank vector keeps the L2
// (evict-last policy on the gathers).
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int ld_stream_i32(const int32_t* p, uint64_t pol) {
  int v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int4 ld_stream_i32x4(const int32_t* p, uint64_t pol) {
  int4 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int64_t ld_stream_i64(const int64_t* p, uint64_t pol) {
  int64_t v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_stream_f64(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
// gathered FP64 value returned as its bit pattern (stays on the integer pipes)
__device__ __forceinline__ uint64_t ld_gather_b64(const double* p, uint64_t pol) {
  uint64_t v;
  asm("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_gather_f64(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_gather_f32(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}

}  // namespace prdf
