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
// Stream-ordered device allocation (cudaMallocAsync) owned by RAII.
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
    cudaError_t e = cudaMallocAsync((void**)&p, count * sizeof(T), stream);
    if (e != cudaSuccess) {
      p = nullptr;
      n = 0;
      set_error("cudaMallocAsync(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
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
// instead of HBM. In-neighbour sums of non-negative FP64 terms below 2^7 are
// therefore accumulated exactly in a 128-bit integer with 2^-120 resolution
// (integer pipes), and the exact sum is rounded once to FP64 (round to
// nearest even). The result is the correctly rounded sum, independent of
// summation order, so every kernel shape and thread count gives the same bits.
// Terms below 2^-120 are truncated (absolute error < 2^-120 per term).

constexpr int kFixFrac = 120;

typedef unsigned __int128 fix128;

__device__ __forceinline__ fix128 fix_from_double(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t e = (uint32_t)(b >> 52) & 0x7FFu;
  const uint64_t m = (b & 0x000FFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  // x = m * 2^(max(e,1) - 1075); in units of 2^-120 that is m << (max(e,1) - 955)
  const int s = (int)(e ? e : 1u) - (1075 - kFixFrac);
  fix128 t = (fix128)m;
  if (s >= 0) t <<= (unsigned)s;
  else t = (s > -64) ? (t >> (unsigned)(-s)) : (fix128)0;
  return t;
}

__device__ __forceinline__ void fix_add(fix128& acc, double x) { acc += fix_from_double(x); }

// Round a fixed-point value (units 2^-120) to the nearest double, ties to even.
__device__ __forceinline__ double fix_to_double(fix128 a) {
  if (a == 0) return 0.0;
  const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  const fix128 nrm = a << (unsigned)lz;  // leading one at bit 127
  const uint64_t top = (uint64_t)(nrm >> 64);
  const uint64_t rest = (uint64_t)nrm;
  uint64_t mant = top >> 11;  // 53 significant bits
  const uint64_t rb = top & 0x7FFull;
  const bool sticky = rest != 0;
  const bool up = rb > 0x400ull || (rb == 0x400ull && (sticky || (mant & 1ull)));
  mant += up ? 1ull : 0ull;
  int ex = (127 - lz) - kFixFrac;  // unbiased exponent of the leading one
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  const uint64_t bits = ((uint64_t)(ex + 1023) << 52) | (mant & 0x000FFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ fix128 warp_sum_fix(fix128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)v, o);
    uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(v >> 64), o);
    v += ((fix128)hi << 64) | lo;
  }
  return v;
}

// non-negative doubles order like their bit patterns
__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(uint64_t b) { return __longlong_as_double((long long)b); }

// ----------------------------------------------------- cache hints ----
// The CSR index stream is read once per sweep: load it through an L2
// evict-first access policy so the gathered rank vector keeps the L2
// (evict-last policy on the gathers).
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int ld_stream_i32(const int32_t* p, uint64_t pol) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int4 ld_stream_i32x4(const int32_t* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_gather_f64(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_gather_f32(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}

}  // namespace prdf
