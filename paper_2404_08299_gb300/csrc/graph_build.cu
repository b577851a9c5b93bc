// CSR construction on the device: the CSR of G and of its transpose G'
// (Section 4.1, 4.3 of arXiv 2404.08299) from an edge list, with duplicate
// edges merged and exactly one self-loop per vertex (Section 3.1, 5.1.3).
//
// Unweighted lists without skipped entries take the radix-sort build of
// radix_build.cu. This pipeline serves weighted lists (duplicates keep the
// largest weight) and lists with skipped entries (all hand-written kernels):
//   row histogram -> exclusive scan -> atomic scatter into row buckets ->
//   per-row sort + unique, by row-length class:
//     <= 8      one thread, 19-comparator sorting network in registers
//     <= 32     one warp, bitonic network over shuffles
//     <= 256    one warp, 8 keys per lane in registers, bitonic network
//               (in-lane exchanges below distance 8, shuffles above)
//     <= 2048   a 128-thread block, bitonic sort in 16 KB of shared memory
//     <= 16384  a 512-thread block, bitonic sort in 128 KB of shared memory
//     larger    one bit per possible column (bitmap), emitted in order
//   -> exclusive scan of unique counts -> compaction into the final CSR.
// Rows are sorted by 64-bit composite keys (column << 32 | ~weight bits), so
// the first entry of each run of equal columns carries the largest weight.
#include "internal.cuh"

namespace prdf {

namespace {

constexpr uint64_t kSent = ~0ull;
constexpr int kThrThread = 8;
constexpr int kThrWarp = 32;
constexpr int kThrWarp8 = 256;
constexpr int kThrSmallBlock = 2048;
constexpr int kThrBlock = 16384;
constexpr int kSmallBlockThreads = 128;
constexpr int kSmallBlockKeys = 16;  // keys per thread: kThrSmallBlock = 128 * 16
constexpr int kSortBlockThreads = 512;
constexpr int kSortBlockKeys = 32;   // kThrBlock = 512 * 32
static_assert(kSmallBlockThreads * kSmallBlockKeys == kThrSmallBlock, "one small-block row fits the block's keys");
static_assert(kSortBlockThreads * kSortBlockKeys == kThrBlock, "one block row fits the block's keys");
constexpr int64_t kBitmapBudget = 512ll << 20;  // bytes of row bitmaps per pass
constexpr int kHugeWordsPerThread = 32;
constexpr int kHugeChunkWords = 256 * kHugeWordsPerThread;

__device__ __forceinline__ bool entry_ok(int32_t r, int32_t c) { return r >= 0 && c >= 0; }

__device__ __forceinline__ uint64_t make_key(int32_t col, float w) {
  return ((uint64_t)(uint32_t)col << 32) | (uint64_t)(uint32_t)(~__float_as_uint(w));
}
__device__ __forceinline__ int32_t key_col(uint64_t k) { return (int32_t)(k >> 32); }
__device__ __forceinline__ float key_w(uint64_t k) { return __uint_as_float(~(uint32_t)(k & 0xFFFFFFFFull)); }

__device__ __forceinline__ void cswap(uint64_t& a, uint64_t& b) {
  const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
  a = lo;
  b = hi;
}

__global__ void k_validate(const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                           const float* __restrict__ w, int64_t m0, int32_t n, int allow_skip, int* bad) {
  int flag = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m0; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[i], c = cols[i];
    const bool skip = allow_skip && !entry_ok(r, c);
    if (!skip && (r < 0 || r >= n || c < 0 || c >= n)) flag |= 1;
    if (!skip && w) {
      const float x = w[i];
      if (!(x > 0.f) || !isfinite(x)) flag |= 2;
    }
  }
  flag = __reduce_or_sync(0xffffffffu, flag);
  if ((threadIdx.x & 31) == 0 && flag) atomicOr(bad, flag);
}

__global__ void k_fill_u32(uint32_t* a, int64_t n, uint32_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

__global__ void k_row_count(const int32_t* __restrict__ rows, const int32_t* __restrict__ cols, int64_t m0,
                            uint32_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m0; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[i], c = cols[i];
    if (entry_ok(r, c)) atomicAdd(&cnt[r], 1u);
  }
}

__global__ void k_init_rows(int32_t n, const int64_t* __restrict__ start, uint32_t* __restrict__ fill,
                            uint64_t* __restrict__ tmp) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    fill[v] = 1;
    tmp[start[v]] = make_key((int32_t)v, 0.f);  // self-loop; weight 0 marks "added"
  }
}

__global__ void k_scatter(const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                          const float* __restrict__ w, int64_t m0, const int64_t* __restrict__ start,
                          uint32_t* __restrict__ fill, uint64_t* __restrict__ tmp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m0; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[i], c = cols[i];
    if (!entry_ok(r, c)) continue;
    const int64_t pos = start[r] + atomicAdd(&fill[r], 1u);
    tmp[pos] = make_key(c, w ? w[i] : 0.f);
  }
}

// ---- rows of length <= 8: one thread, Batcher odd-even merge network ----
__global__ void k_sort_thread(const int32_t* __restrict__ list, int64_t count, const int64_t* __restrict__ start,
                              const uint64_t* __restrict__ tmp, uint64_t* __restrict__ out, uint32_t* __restrict__ ucnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = list[i];
    const int64_t b = start[v];
    const int L = (int)(start[v + 1] - b);
    uint64_t k[kThrThread];
#pragma unroll
    for (int j = 0; j < kThrThread; ++j) k[j] = j < L ? tmp[b + j] : kSent;
    cswap(k[0], k[1]); cswap(k[2], k[3]); cswap(k[4], k[5]); cswap(k[6], k[7]);
    cswap(k[0], k[2]); cswap(k[1], k[3]); cswap(k[4], k[6]); cswap(k[5], k[7]);
    cswap(k[1], k[2]); cswap(k[5], k[6]);
    cswap(k[0], k[4]); cswap(k[1], k[5]); cswap(k[2], k[6]); cswap(k[3], k[7]);
    cswap(k[2], k[4]); cswap(k[3], k[5]);
    cswap(k[1], k[2]); cswap(k[3], k[4]); cswap(k[5], k[6]);
    uint32_t u = 0;
#pragma unroll
    for (int j = 0; j < kThrThread; ++j) {
      const bool keep = k[j] != kSent && (j == 0 || key_col(k[j]) != key_col(k[j - 1]));
      if (keep) out[b + u++] = k[j];
    }
    ucnt[v] = u;
  }
}

// ---- rows of length <= 32: one warp, bitonic over shuffles ----
__global__ void k_sort_warp(const int32_t* __restrict__ list, int64_t count, const int64_t* __restrict__ start,
                            const uint64_t* __restrict__ tmp, uint64_t* __restrict__ out, uint32_t* __restrict__ ucnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < count; i += nwarps) {
    const int32_t v = list[i];
    const int64_t b = start[v];
    const int L = (int)(start[v + 1] - b);
    uint64_t key = lane < L ? tmp[b + lane] : kSent;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const uint64_t o = __shfl_xor_sync(0xffffffffu, key, j);
        const bool up = (lane & k) == 0;
        const bool lower = (lane & j) == 0;
        key = (lower == up) ? (key < o ? key : o) : (key < o ? o : key);
      }
    }
    const uint64_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool keep = key != kSent && (lane == 0 || key_col(prev) != key_col(key));
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) out[b + __popc(bal & ((1u << lane) - 1u))] = key;
    if (lane == 0) ucnt[v] = __popc(bal);
  }
}

// ---- rows of length <= 256: one warp, 8 keys per lane (element e = 8 * lane + q) ----
__global__ void k_sort_warp8(const int32_t* __restrict__ list, int64_t count, const int64_t* __restrict__ start,
                             const uint64_t* __restrict__ tmp, uint64_t* __restrict__ out,
                             uint32_t* __restrict__ ucnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < count; i += nwarps) {
    const int32_t v = list[i];
    const int64_t b = start[v];
    const int L = (int)(start[v + 1] - b);
    uint64_t k[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = 8 * lane + q;
      k[q] = e < L ? tmp[b + e] : kSent;
    }
#pragma unroll
    for (int kk = 2; kk <= 256; kk <<= 1) {
#pragma unroll
      for (int j = kk >> 1; j > 0; j >>= 1) {
        if (j >= 8) {
          // partner e ^ j lives in lane ^ (j / 8), same register
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const uint64_t o = __shfl_xor_sync(0xffffffffu, k[q], j >> 3);
            const int e = 8 * lane + q;
            const bool up = (e & kk) == 0;
            const bool lower = (e & j) == 0;
            k[q] = (lower == up) ? (k[q] < o ? k[q] : o) : (k[q] < o ? o : k[q]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int p = q ^ j;
            if (p > q) {
              const int e = 8 * lane + q;
              const bool up = (e & kk) == 0;
              if ((k[q] > k[p]) == up) {
                const uint64_t t = k[q];
                k[q] = k[p];
                k[p] = t;
              }
            }
          }
        }
      }
    }
    // first entry of each column run, written in order
    const uint64_t before = __shfl_up_sync(0xffffffffu, k[7], 1);
    uint32_t keep = 0, cnt = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint64_t prev = q > 0 ? k[q - 1] : before;
      const bool first = k[q] != kSent && ((lane == 0 && q == 0) || key_col(prev) != key_col(k[q]));
      keep |= first ? (1u << q) : 0u;
      cnt += first ? 1u : 0u;
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t pos = incl - cnt;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (keep & (1u << q)) out[b + pos++] = k[q];
    if (lane == 31) ucnt[v] = incl;
  }
}

// block-wide exclusive scan for NT threads (NT a multiple of 32, <= 1024)
template <int NT>
__device__ __forceinline__ uint32_t block_scan_u32(uint32_t v, uint32_t* total, uint32_t* sh /* NT/32 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) sh[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < NT / 32 ? sh[lane] : 0;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < NT / 32) sh[lane] = wi - w;
    if (lane == NT / 32 - 1) *total = wi;
  }
  __syncthreads();
  const uint32_t r = incl - v + sh[wid];
  __syncthreads();
  return r;
}

// ---- rows up to NT*E keys: one block per row, Batcher's bitonic sorting
// network with E consecutive keys per thread in registers. Stages whose
// partners lie E or more positions apart run in shared memory (one barrier
// each, every active thread owning E/2 pairs); the closer stages run in
// registers. A row of L keys is padded with sentinels to P2 = the power of
// two >= max(L, 32E) and handled by P2/E threads (whole warps); the others
// only meet the barriers. Shared memory keeps one pad slot per E keys so
// that a thread's E keys and a warp's pair accesses spread over the banks.
__device__ __forceinline__ void cswap_dir(uint64_t& a, uint64_t& b, bool up) {
  const bool sw = (a > b) == up;
  const uint64_t x = sw ? b : a, y = sw ? a : b;
  a = x;
  b = y;
}

template <int NT, int E>
__global__ void __launch_bounds__(NT) k_sort_block(const int32_t* __restrict__ list, int64_t count,
                                                   const int64_t* __restrict__ start, const uint64_t* __restrict__ tmp,
                                                   uint64_t* __restrict__ out, uint32_t* __restrict__ ucnt) {
  static_assert((E & (E - 1)) == 0 && E >= 2 && NT % 32 == 0, "E a power of two, NT whole warps");
  constexpr int LE = (E >= 32) ? 5 : (E >= 16) ? 4 : (E >= 8) ? 3 : (E >= 4) ? 2 : 1;
  static_assert((1 << LE) == E, "E up to 32");
  extern __shared__ uint64_t sk[];  // NT * (E + 1) keys
  __shared__ uint32_t scan_sh[NT / 32];
  __shared__ uint32_t total;
  const int tid = threadIdx.x;
  auto pad = [](int t) { return t + (t >> LE); };
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int32_t v = list[i];
    const int64_t b = start[v];
    const int L = (int)(start[v + 1] - b);
    int P2 = 32 * E;
    while (P2 < L) P2 <<= 1;
    const int A = P2 / E;  // active threads: a multiple of 32, <= NT
    const bool act = tid < A;
    for (int t = tid; t < P2; t += NT) sk[pad(t)] = t < L ? tmp[b + t] : kSent;
    __syncthreads();
    uint64_t r[E];
#pragma unroll
    for (int x = 0; x < E; ++x) r[x] = act ? sk[pad(tid * E + x)] : kSent;
    // sizes 2 .. E: within the thread
#pragma unroll
    for (int k = 2; k <= E; k <<= 1) {
      const bool up_hi = (tid & 1) == 0;  // direction bit of size E comes from the thread index
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
        for (int x = 0; x < E; ++x)
          if ((x & j) == 0) cswap_dir(r[x], r[x | j], k < E ? (x & k) == 0 : up_hi);
      }
    }
    // sizes 2E .. P2: far stages in shared memory, the last log2(E) in registers
    for (int k = 2 * E; k <= P2; k <<= 1) {
      __syncthreads();  // every thread has read its keys of the previous size
      if (act) {
#pragma unroll
        for (int x = 0; x < E; ++x) sk[pad(tid * E + x)] = r[x];
      }
      __syncthreads();
      for (int j = k >> 1; j >= E; j >>= 1) {
        if (act) {
          const int lj = __ffs(j) - 1;
          for (int q = tid; q < (P2 >> 1); q += A) {
            const int t = ((q >> lj) << (lj + 1)) | (q & (j - 1));
            const int p = t | j;
            uint64_t a = sk[pad(t)], c = sk[pad(p)];
            cswap_dir(a, c, (t & k) == 0);
            sk[pad(t)] = a;
            sk[pad(p)] = c;
          }
        }
        __syncthreads();
      }
      if (act) {
#pragma unroll
        for (int x = 0; x < E; ++x) r[x] = sk[pad(tid * E + x)];
        const bool up = ((tid * E) & k) == 0;
#pragma unroll
        for (int j = E >> 1; j > 0; j >>= 1) {
#pragma unroll
          for (int x = 0; x < E; ++x)
            if ((x & j) == 0) cswap_dir(r[x], r[x | j], up);
        }
      }
    }
    // keep the first key of each column run (the largest weight), in order
    __syncthreads();
    if (act) {
#pragma unroll
      for (int x = 0; x < E; ++x) sk[pad(tid * E + x)] = r[x];
    }
    __syncthreads();
    const uint64_t before = (act && tid > 0) ? sk[pad(tid * E - 1)] : kSent;
    uint32_t keep = 0, mine = 0;
    if (act) {
      uint64_t pv = before;
#pragma unroll
      for (int x = 0; x < E; ++x) {
        const bool k1 = r[x] != kSent && ((tid == 0 && x == 0) || key_col(r[x]) != key_col(pv));
        keep |= (k1 ? 1u : 0u) << x;
        mine += k1 ? 1u : 0u;
        pv = r[x];
      }
    }
    uint32_t pos = block_scan_u32<NT>(mine, &total, scan_sh);
    if (act) {
#pragma unroll
      for (int x = 0; x < E; ++x)
        if (keep & (1u << x)) out[b + pos++] = r[x];
    }
    if (tid == 0) ucnt[v] = total;
    __syncthreads();
  }
}

// ---- longer rows: one bit per column ----
__global__ void k_huge_set(const int32_t* __restrict__ rowlist, const int64_t* __restrict__ start,
                           const uint64_t* __restrict__ tmp, uint32_t* __restrict__ bm, int64_t words) {
  const int32_t v = rowlist[blockIdx.y];
  const int64_t b = start[v], e = start[v + 1];
  uint32_t* row = bm + (int64_t)blockIdx.y * words;
  for (int64_t j = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < e; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = key_col(tmp[j]);
    atomicOr(&row[c >> 5], 1u << (c & 31));
  }
}

__global__ void k_huge_count(const uint32_t* __restrict__ bm, int64_t words, int64_t nchunks, int64_t* __restrict__ cc) {
  const uint32_t* row = bm + (int64_t)blockIdx.y * words;
  const int64_t w0 = (int64_t)blockIdx.x * kHugeChunkWords + (int64_t)threadIdx.x * kHugeWordsPerThread;
  uint32_t s = 0;
#pragma unroll 8
  for (int k = 0; k < kHugeWordsPerThread; ++k)
    if (w0 + k < words) s += __popc(row[w0 + k]);
  __shared__ uint32_t sh[8];
  __shared__ uint32_t tot;
  block_scan_u32<256>(s, &tot, sh);
  if (threadIdx.x == 0) cc[(int64_t)blockIdx.y * nchunks + blockIdx.x] = tot;
}

__global__ void k_huge_emit(const int32_t* __restrict__ rowlist, const int64_t* __restrict__ start,
                            const uint32_t* __restrict__ bm, int64_t words, int64_t nchunks,
                            const int64_t* __restrict__ ccoff, uint64_t* __restrict__ out, uint32_t* __restrict__ ucnt) {
  const int32_t v = rowlist[blockIdx.y];
  const uint32_t* row = bm + (int64_t)blockIdx.y * words;
  const int64_t rowbase = ccoff[(int64_t)blockIdx.y * nchunks];
  const int64_t w0 = (int64_t)blockIdx.x * kHugeChunkWords + (int64_t)threadIdx.x * kHugeWordsPerThread;
  uint32_t s = 0;
  for (int k = 0; k < kHugeWordsPerThread; ++k)
    if (w0 + k < words) s += __popc(row[w0 + k]);
  __shared__ uint32_t sh[8];
  __shared__ uint32_t tot;
  uint32_t pos = block_scan_u32<256>(s, &tot, sh);
  int64_t o = start[v] + (ccoff[(int64_t)blockIdx.y * nchunks + blockIdx.x] - rowbase) + pos;
  for (int k = 0; k < kHugeWordsPerThread; ++k) {
    if (w0 + k >= words) break;
    uint32_t word = row[w0 + k];
    while (word) {
      const int bit = __ffs(word) - 1;
      word &= word - 1;
      out[o++] = make_key((int32_t)((w0 + k) * 32 + bit), 0.f);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ucnt[v] = (uint32_t)(ccoff[(int64_t)(blockIdx.y + 1) * nchunks] - rowbase);
}

// weights of bitmap rows: max over duplicates via integer max on positive float bits
__global__ void k_huge_weights(const int32_t* __restrict__ rowlist, const int64_t* __restrict__ start,
                               const uint64_t* __restrict__ tmp, const uint32_t* __restrict__ ucnt,
                               uint64_t* __restrict__ out) {
  const int32_t v = rowlist[blockIdx.y];
  const int64_t b = start[v], e = start[v + 1];
  const int64_t u = ucnt[v];
  for (int64_t j = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < e; j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = tmp[j];
    const int32_t c = key_col(k);
    int64_t lo = b, hi = b + u;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (key_col(out[mid]) < c) lo = mid + 1; else hi = mid;
    }
    // low 32 bits hold ~weight: the largest weight has the smallest low word
    atomicMin((unsigned long long*)&out[lo], (unsigned long long)k);
  }
}

// Final CSR from the sorted row buckets: row v's unique keys start at
// start[v] and go to off[v]. Balanced by entries, not rows: a warp takes
// kCompactChunk consecutive output entries (lane-strided), finds the row of
// the first one by binary search, and each lane walks rows forward (a few
// steps, then a binary search past runs of empty rows).
constexpr int64_t kCompactChunk = 1024;

__global__ void k_compact(int32_t n, int64_t m, const int64_t* __restrict__ start,
                          const uint64_t* __restrict__ sorted, const int64_t* __restrict__ off,
                          int32_t* __restrict__ adj, float* __restrict__ w) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p0 = warp * kCompactChunk; p0 < m; p0 += nwarps * kCompactChunk) {
    int64_t lo = 0, hi = n;  // the last row r with off[r] <= p0
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (off[mid] <= p0) lo = mid; else hi = mid;
    }
    int64_t r = lo, rs = off[r], re = off[r + 1], src = start[r];
    for (int64_t p = p0 + lane; p < p0 + kCompactChunk && p < m; p += 32) {
      if (p >= re) {
        // a few steps forward, then a binary search (CSRs of small batches are mostly empty rows)
        int steps = 0;
        do {
          ++r;
          re = off[r + 1];
        } while (p >= re && ++steps < 8);
        if (p >= re) {
          int64_t a = r, z = n;  // the last row with off[row] <= p
          while (z - a > 1) {
            const int64_t mid = (a + z) >> 1;
            if (off[mid] <= p) a = mid; else z = mid;
          }
          r = a;
          re = off[r + 1];
        }
        rs = off[r];
        src = start[r];
      }
      const uint64_t k = sorted[src + (p - rs)];
      adj[p] = key_col(k);
      if (w) {
        const float x = key_w(k);
        w[p] = x > 0.f ? x : 1.0f;  // an added self-loop carries weight 1
      }
    }
  }
}

}  // namespace

int build_csr(int32_t n, int64_t m0, const int32_t* rows, const int32_t* cols, const float* w, bool self_loops,
              bool allow_skip, Csr& out, Workspace& ws, cudaStream_t s) {
  if (n < 1 || m0 < 0 || m0 >= (1ll << 32)) {
    set_error("build_csr: n=%d m0=%lld out of range", n, (long long)m0);
    return PRDF_EINVAL;
  }
  const int T = 256;
  // validate ids (and weights)
  {
    DBuf<int> bad;
    PRDF_TRY(bad.alloc(1, s));
    PRDF_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    if (m0 > 0) {
      k_validate<<<grid_for(m0, T), T, 0, s>>>(rows, cols, w, m0, n, allow_skip ? 1 : 0, bad.p);
      PRDF_LAUNCH_CHECK();
    }
    int hb = 0;
    PRDF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PRDF_CUDA(cudaStreamSynchronize(s));
    if (hb & 1) {
      set_error("edge list has a vertex id outside [0, %d)", n);
      return PRDF_EINVAL;
    }
    if (hb & 2) {
      set_error("edge weights must be finite and > 0");
      return PRDF_EINVAL;
    }
  }
  if (radix_build_applies(n, m0, w, allow_skip, self_loops))
    return build_csr_radix(n, m0, rows, cols, self_loops, out, ws, s);
  const int64_t N = n;
  DBuf<uint32_t> cnt, fill, ucnt;
  DBuf<int64_t> start;
  PRDF_TRY(cnt.alloc(N, s));
  PRDF_TRY(fill.alloc(N, s));
  PRDF_TRY(ucnt.alloc(N, s));
  PRDF_TRY(start.alloc(N + 1, s));
  k_fill_u32<<<grid_for(N, T), T, 0, s>>>(cnt.p, N, self_loops ? 1u : 0u);
  if (m0 > 0) k_row_count<<<grid_for(m0, T), T, 0, s>>>(rows, cols, m0, cnt.p);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(exclusive_scan_u32(cnt.p, N, start.p, ws, s));
  int64_t M = 0;
  PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, start.p + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  M = ws.host_i64[0];
  DBuf<uint64_t> tmp, srt;
  PRDF_TRY(tmp.alloc(M > 0 ? M : 1, s));
  PRDF_TRY(srt.alloc(M > 0 ? M : 1, s));
  if (self_loops) {
    k_init_rows<<<grid_for(N, T), T, 0, s>>>(n, start.p, fill.p, tmp.p);
  } else {
    k_fill_u32<<<grid_for(N, T), T, 0, s>>>(fill.p, N, 0u);
  }
  if (m0 > 0) k_scatter<<<grid_for(m0, T), T, 0, s>>>(rows, cols, w, m0, start.p, fill.p, tmp.p);
  PRDF_LAUNCH_CHECK();

  // classify rows by raw length
  DBuf<int32_t> rowP;
  PRDF_TRY(rowP.alloc(N, s));
  PartThr t;
  t.n = 5;
  t.thr[0] = kThrThread;
  t.thr[1] = kThrWarp;
  t.thr[2] = kThrWarp8;
  t.thr[3] = kThrSmallBlock;
  t.thr[4] = kThrBlock;
  int64_t cls[6];
  PRDF_TRY(partition_by_degree(start.p, N, t, rowP.p, cls, ws, s));
  const int32_t* l0 = rowP.p;
  const int32_t* l1 = l0 + cls[0];
  const int32_t* l2 = l1 + cls[1];
  const int32_t* l3 = l2 + cls[2];
  const int32_t* l4 = l3 + cls[3];
  const int32_t* l5 = l4 + cls[4];
  if (cls[0]) k_sort_thread<<<grid_for(cls[0], T), T, 0, s>>>(l0, cls[0], start.p, tmp.p, srt.p, ucnt.p);
  if (cls[1]) k_sort_warp<<<grid_for(cls[1] * 32, T), T, 0, s>>>(l1, cls[1], start.p, tmp.p, srt.p, ucnt.p);
  if (cls[2]) k_sort_warp8<<<grid_for(cls[2] * 32, T), T, 0, s>>>(l2, cls[2], start.p, tmp.p, srt.p, ucnt.p);
  if (cls[3]) {
    const int smem = kSmallBlockThreads * (kSmallBlockKeys + 1) * (int)sizeof(uint64_t);
    k_sort_block<kSmallBlockThreads, kSmallBlockKeys><<<grid_for(cls[3], 1, kSMs * 16), kSmallBlockThreads, smem, s>>>(
        l3, cls[3], start.p, tmp.p, srt.p, ucnt.p);
  }
  if (cls[4]) {
    const int smem = kSortBlockThreads * (kSortBlockKeys + 1) * (int)sizeof(uint64_t);
    PRDF_CUDA(cudaFuncSetAttribute(k_sort_block<kSortBlockThreads, kSortBlockKeys>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int grid = (int)(cls[4] < kSMs * 2 ? cls[4] : kSMs * 2);
    k_sort_block<kSortBlockThreads, kSortBlockKeys><<<grid, kSortBlockThreads, smem, s>>>(l4, cls[4], start.p, tmp.p,
                                                                                       srt.p, ucnt.p);
  }
  PRDF_LAUNCH_CHECK();
  if (cls[5]) {
    const int64_t words = (N + 31) / 32;
    const int64_t nchunks = (words + kHugeChunkWords - 1) / kHugeChunkWords;
    int64_t per = kBitmapBudget / (words * 4);
    if (per < 1) per = 1;
    if (per > 65535) per = 65535;
    DBuf<uint32_t> bm;
    DBuf<int64_t> cc, ccoff;
    const int64_t rows_batch = cls[5] < per ? cls[5] : per;
    PRDF_TRY(bm.alloc(rows_batch * words, s));
    PRDF_TRY(cc.alloc(rows_batch * nchunks, s));
    PRDF_TRY(ccoff.alloc(rows_batch * nchunks + 1, s));
    for (int64_t h0 = 0; h0 < cls[5]; h0 += rows_batch) {
      const int64_t rb = (cls[5] - h0) < rows_batch ? (cls[5] - h0) : rows_batch;
      PRDF_CUDA(cudaMemsetAsync(bm.p, 0, (size_t)(rb * words) * 4, s));
      k_huge_set<<<dim3(64, (unsigned)rb), T, 0, s>>>(l5 + h0, start.p, tmp.p, bm.p, words);
      k_huge_count<<<dim3((unsigned)nchunks, (unsigned)rb), 256, 0, s>>>(bm.p, words, nchunks, cc.p);
      PRDF_LAUNCH_CHECK();
      PRDF_TRY(exclusive_scan_i64(cc.p, rb * nchunks, ccoff.p, ws, s));
      k_huge_emit<<<dim3((unsigned)nchunks, (unsigned)rb), 256, 0, s>>>(l5 + h0, start.p, bm.p, words, nchunks,
                                                                          ccoff.p, srt.p, ucnt.p);
      if (w) k_huge_weights<<<dim3(64, (unsigned)rb), T, 0, s>>>(l5 + h0, start.p, tmp.p, ucnt.p, srt.p);
      PRDF_LAUNCH_CHECK();
    }
  }
  // final offsets and compaction
  PRDF_TRY(out.off.alloc(N + 1, s));
  PRDF_TRY(exclusive_scan_u32(ucnt.p, N, out.off.p, ws, s));
  PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, out.off.p + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  out.m = ws.host_i64[0];
  PRDF_TRY(out.adj.alloc(out.m > 0 ? out.m : 1, s));
  if (w) PRDF_TRY(out.w.alloc(out.m > 0 ? out.m : 1, s));
  else out.w.release();
  if (out.m > 0)
    k_compact<<<grid_for((out.m + kCompactChunk - 1) / kCompactChunk * 32, T), T, 0, s>>>(
        n, out.m, start.p, srt.p, out.off.p, out.adj.p, w ? out.w.p : nullptr);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

}  // namespace prdf
