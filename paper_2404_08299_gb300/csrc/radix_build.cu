// CSR construction by a least-significant-digit radix sort of packed edge
// keys: the CSR of G or of G' (Section 4.1, 4.3 of arXiv 2404.08299) from an
// unweighted edge list, duplicates merged and one self-loop per vertex
// (Section 3.1, 5.1.3).
//
// Key of entry (r, c): r << B | c, B = bits of n - 1, so the key order is the
// CSR order (rows ascending, columns ascending inside a row). Eight key bits
// per pass, ceil(2B / 8) passes; each pass is
//   tile histograms -> one exclusive scan over [digit][tile] -> stable scatter
// with tiles of 4096 keys. The scatter ranks a tile's keys by digit in shared
// memory (warp-level match of equal digits, per-warp counters, in input
// order, so every pass is stable) and writes each digit's run of the tile to
// its global place from a staged copy, so the stores are contiguous runs
// rather than one random store per key. No global atomics, so the result
// and its timing do not depend on how skewed the rows are. The first pass
// reads the edge list and makes the keys (and the self-loop keys) on the
// fly. After the last pass, adjacent equal keys are merged: a count per warp,
// one scan, one emit pass that writes the columns and the row offsets (found
// row-parallel instead when the list is much shorter than n).
#include "internal.cuh"

namespace prdf {

namespace {

constexpr int kRT = 256;              // threads per tile
constexpr int kRK = 16;               // keys per thread
constexpr int kRTile = kRT * kRK;     // 4096 keys per tile
constexpr int kRWarps = kRT / 32;
constexpr int kRDigits = 256;
static_assert(kRT == kRDigits, "one digit per thread in the scatter's digit scan");
static_assert(kRTile <= 65536 && kRK % 2 == 0, "ranks are packed two to a word");

struct KeySrc {
  const uint64_t* keys;  // later passes
  const int32_t* rows;   // first pass: entry i < m0 is (rows[i], cols[i]),
  const int32_t* cols;   // entry m0 + v is the self-loop (v, v)
  int64_t m0;
  int B;
};

template <bool FIRST>
__device__ __forceinline__ uint64_t load_key(const KeySrc& s, int64_t i) {
  if (!FIRST) return __ldcs(reinterpret_cast<const unsigned long long*>(s.keys) + i);
  if (i < s.m0) return ((uint64_t)(uint32_t)__ldcs(s.rows + i) << s.B) | (uint64_t)(uint32_t)__ldcs(s.cols + i);
  const uint64_t v = (uint64_t)(i - s.m0);
  return (v << s.B) | v;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Lanes of the warp whose value d (BITS bits) equals this lane's: one ballot
// per bit. Bit 8 marks lanes without a key; full tiles match 8 bits.
template <int BITS>
__device__ __forceinline__ uint32_t match_digit(uint32_t d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < BITS; ++b) {
    const uint32_t m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
    peers &= ((d >> b) & 1u) ? m : ~m;
  }
  return peers;
}

// Exclusive scan of one value per thread over a block of kRT threads.
// wsum: kRWarps words of shared memory; the caller syncs before reusing it.
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t v, uint32_t* wsum, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  uint32_t add = 0, all = 0;
#pragma unroll
  for (int k = 0; k < kRWarps; ++k) {
    const uint32_t c = wsum[k];
    add += k < w ? c : 0u;
    all += c;
  }
  if (total) *total = all;
  return x - v + add;
}

// hist[d * ntiles + tile] = number of keys of the tile whose digit is d.
// Counting needs no ranks: a shared-memory atomic per key on the warp's own
// counters (equal digits within a warp are serialised by the hardware).
template <bool FIRST>
__global__ void __launch_bounds__(kRT) k_radix_hist(const KeySrc src, int64_t M, int shift, uint32_t* __restrict__ hist,
                                                     int64_t ntiles) {
  __shared__ uint32_t h[kRWarps][kRDigits];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kRWarps; ++k) h[k][threadIdx.x] = 0;
  const int64_t i0 = (int64_t)blockIdx.x * kRTile + (int64_t)w * (32 * kRK) + lane;
  const int nv = M <= i0 ? 0 : (M - i0 >= 32 * kRK ? kRK : (int)((M - i0 + 31) / 32));
  uint32_t d[kRK];
#pragma unroll
  for (int r = 0; r < kRK; ++r) d[r] = r < nv ? (uint32_t)(load_key<FIRST>(src, i0 + r * 32) >> shift) & 0xFFu : 0u;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRK; ++r)
    if (r < nv) atomicAdd(&h[w][d[r]], 1u);
  __syncthreads();
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < kRWarps; ++k) c += h[k][threadIdx.x];
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = c;
}

// Stable scatter of one tile by digit; goff = exclusive scan of hist.
template <bool FIRST>
__global__ void __launch_bounds__(kRT, 3) k_radix_scatter(const KeySrc src, int64_t M, int shift,
                                                          const int64_t* __restrict__ goff, int64_t ntiles,
                                                          uint64_t* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* buf = reinterpret_cast<uint64_t*>(smem_raw);          // kRTile keys
  int64_t* gbase = reinterpret_cast<int64_t*>(buf + kRTile);       // kRDigits
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(gbase + kRDigits);  // kRWarps x kRDigits
  uint32_t* lstart = wcnt + kRWarps * kRDigits;                    // kRDigits
  uint32_t* wsum = lstart + kRDigits;                              // kRWarps
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kRWarps; ++k) wcnt[k * kRDigits + threadIdx.x] = 0;
  const int64_t t0 = (int64_t)blockIdx.x * kRTile;
  const int64_t i0 = t0 + (int64_t)w * (32 * kRK) + lane;
  // rounds r < nv hold a key of this thread
  const int nv = M <= i0 ? 0 : (M - i0 >= 32 * kRK ? kRK : (int)((M - i0 + 31) / 32));
  uint64_t key[kRK];
#pragma unroll
  for (int r = 0; r < kRK; ++r) key[r] = r < nv ? load_key<FIRST>(src, i0 + r * 32) : 0ull;
  __syncthreads();
  // rank of each key among the equal digits before it: earlier rounds of this
  // warp (its counter), then lower lanes of the same round
  uint32_t* mine = wcnt + w * kRDigits;
  const uint32_t lt = lanemask_lt();
  const bool full = t0 + kRTile <= M;
  uint32_t rank[kRK / 2];  // two 16-bit ranks a word (a rank is below kRTile)
#pragma unroll
  for (int r = 0; r < kRK; ++r) {
    const bool ok = r < nv;
    const uint32_t d = ok ? (uint32_t)(key[r] >> shift) & 0xFFu : 0x100u;
    const uint32_t peers = full ? match_digit<8>(d) : match_digit<9>(d);
    const uint32_t before = (uint32_t)__popc(peers & lt);
    const uint32_t prev = ok ? mine[d] : 0u;
    __syncwarp();
    if (ok && before == 0) mine[d] = prev + (uint32_t)__popc(peers);
    __syncwarp();
    const uint32_t rk = prev + before;
    if (r & 1) rank[r >> 1] |= rk << 16;
    else rank[r >> 1] = rk;
  }
  __syncthreads();
  // digit d = this thread: warp bases (in warp order), the tile's count of d,
  // and the digit's start inside the tile
  {
    const int d = threadIdx.x;
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kRWarps; ++k) {
      const uint32_t c = wcnt[k * kRDigits + d];
      wcnt[k * kRDigits + d] = acc;
      acc += c;
    }
    const uint32_t ls = block_scan_excl(acc, wsum, nullptr);
    lstart[d] = ls;
    gbase[d] = goff[(int64_t)d * ntiles + blockIdx.x] - (int64_t)ls;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRK; ++r) {
    if (r < nv) {
      const uint32_t d = (uint32_t)(key[r] >> shift) & 0xFFu;
      buf[lstart[d] + mine[d] + ((rank[r >> 1] >> (16 * (r & 1))) & 0xFFFFu)] = key[r];
    }
  }
  __syncthreads();
  const int cnt = (int)(M - t0 < kRTile ? M - t0 : kRTile);
  for (int i = threadIdx.x; i < cnt; i += kRT) {
    const uint64_t k = buf[i];
    __stcs(reinterpret_cast<unsigned long long*>(out) + gbase[(k >> shift) & 0xFFu] + i, k);
  }
}

constexpr int kRScatterSmem = kRTile * 8 + kRDigits * 8 + kRWarps * kRDigits * 4 + kRDigits * 4 + kRWarps * 4;

// ---- merge of equal keys ----
// A warp takes 32 * kRK consecutive sorted keys, 32 per round (coalesced);
// key i is new when it differs from key i - 1, which is the lane below in the
// same round, lane 31 of the round before, or the previous warp's last key.

__device__ __forceinline__ bool new_key(int64_t i, uint64_t key, uint64_t& carry, int lane) {
  uint64_t prev = __shfl_up_sync(0xffffffffu, key, 1);
  if (lane == 0) prev = carry;
  carry = __shfl_sync(0xffffffffu, key, 31);
  return i == 0 || key != prev;
}

__device__ __forceinline__ uint64_t warp_carry_in(const uint64_t* __restrict__ k, int64_t i0) {
  return i0 > 0 ? k[i0 - 1] : ~0ull;  // i0: the warp's first key (lane 0)
}

// cnt[warp] = number of new keys among the warp's 32 * kRK
__global__ void __launch_bounds__(kRT) k_uniq_count(const uint64_t* __restrict__ k, int64_t M, uint32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kRT + threadIdx.x) >> 5;
  const int64_t base = gw * (32 * kRK);
  uint64_t key[kRK];
#pragma unroll
  for (int r = 0; r < kRK; ++r) {
    const int64_t i = base + r * 32 + lane;
    key[r] = i < M ? __ldcs(reinterpret_cast<const unsigned long long*>(k) + i) : ~0ull;
  }
  uint64_t carry = base < M ? warp_carry_in(k, base) : ~0ull;
  uint32_t c = 0;
#pragma unroll
  for (int r = 0; r < kRK; ++r) {
    const int64_t i = base + r * 32 + lane;
    const bool f = new_key(i, key[r], carry, lane) && i < M;
    c += (uint32_t)__popc(__ballot_sync(0xffffffffu, f));
  }
  if (lane == 0) cnt[gw] = c;
}

// Columns of the unique keys, and off[r] = position of row r's first unique
// key (rows without keys take the next row's start; off[n] = total).
// woff = exclusive scan of the per-warp counts, woff[nw] = total. With urow
// (lists much shorter than n) the row of each unique key goes to urow instead
// and k_offsets_from_rows fills off.
__global__ void __launch_bounds__(kRT) k_uniq_emit(const uint64_t* __restrict__ k, int64_t M, int B, int32_t n,
                                                   const int64_t* __restrict__ woff, int64_t nw,
                                                   int32_t* __restrict__ adj, int64_t* __restrict__ off,
                                                   int32_t* __restrict__ urow) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kRT + threadIdx.x) >> 5;
  const int64_t base = gw * (32 * kRK);
  const uint32_t lt = lanemask_lt();
  const uint64_t cmask = (1ull << B) - 1;
  uint64_t key[kRK];
#pragma unroll
  for (int r = 0; r < kRK; ++r) {
    const int64_t i = base + r * 32 + lane;
    key[r] = i < M ? __ldcs(reinterpret_cast<const unsigned long long*>(k) + i) : ~0ull;
  }
  uint64_t carry = base < M ? warp_carry_in(k, base) : ~0ull;
  int64_t pos = gw < nw ? woff[gw] : 0;
#pragma unroll
  for (int r = 0; r < kRK; ++r) {
    const int64_t i = base + r * 32 + lane;
    uint64_t prev = __shfl_up_sync(0xffffffffu, key[r], 1);
    if (lane == 0) prev = carry;
    carry = __shfl_sync(0xffffffffu, key[r], 31);
    const bool f = i < M && (i == 0 || key[r] != prev);
    const uint32_t bal = __ballot_sync(0xffffffffu, f);
    if (f) {
      const int64_t p = pos + __popc(bal & lt);
      const int64_t row = (int64_t)(key[r] >> B);
      adj[p] = (int32_t)(key[r] & cmask);
      if (urow) {
        urow[p] = (int32_t)row;
      } else {
        const int64_t first = i == 0 ? 0 : (int64_t)(prev >> B) + 1;  // rows after the previous key's
        for (int64_t q = first; q <= row; ++q) off[q] = p;
      }
    }
    if (!urow && i == M - 1) {
      const int64_t total = woff[nw];
      for (int64_t q = (int64_t)(key[r] >> B) + 1; q <= n; ++q) off[q] = total;
    }
    pos += __popc(bal);
  }
}

// off[r] = first position whose row is >= r (urow ascending, length mu): one
// binary search per row, for lists much shorter than n
__global__ void k_offsets_from_rows(const int32_t* __restrict__ urow, int64_t mu, int32_t n, int64_t* __restrict__ off) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= n; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = mu;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (urow[mid] < r) lo = mid + 1; else hi = mid;
    }
    off[r] = lo;
  }
}

template <bool FIRST>
int radix_pass(const KeySrc& src, int64_t M, int shift, uint64_t* out, DBuf<uint32_t>& hist, DBuf<int64_t>& goff,
               int64_t ntiles, Workspace& ws, cudaStream_t s) {
  k_radix_hist<FIRST><<<(unsigned)ntiles, kRT, 0, s>>>(src, M, shift, hist.p, ntiles);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(exclusive_scan_u32(hist.p, ntiles * kRDigits, goff.p, ws, s));
  k_radix_scatter<FIRST><<<(unsigned)ntiles, kRT, kRScatterSmem, s>>>(src, M, shift, goff.p, ntiles, out);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

}  // namespace

bool radix_build_applies(int32_t n, int64_t m0, const float* w, bool allow_skip, bool self_loops) {
  const int64_t M = m0 + (self_loops ? n : 0);
  return !w && !allow_skip && M > 0 && M < (1ll << 32);
}

int build_csr_radix(int32_t n, int64_t m0, const int32_t* rows, const int32_t* cols, bool self_loops, Csr& out,
                    Workspace& ws, cudaStream_t s) {
  const int64_t M = m0 + (self_loops ? n : 0);
  int B = 1;
  while (B < 31 && ((int64_t)1 << B) < (int64_t)n) ++B;  // ids < n <= 2^B
  const int passes = (2 * B + 7) / 8;
  const int64_t ntiles = (M + kRTile - 1) / kRTile;
  static bool smem_set = false;
  if (!smem_set) {
    PRDF_CUDA(cudaFuncSetAttribute(k_radix_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRScatterSmem));
    PRDF_CUDA(cudaFuncSetAttribute(k_radix_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRScatterSmem));
    smem_set = true;
  }
  DBuf<uint64_t> ka, kb;
  DBuf<uint32_t> hist;
  DBuf<int64_t> goff;
  PRDF_TRY(ka.alloc((size_t)M, s));
  PRDF_TRY(kb.alloc((size_t)M, s));
  PRDF_TRY(hist.alloc((size_t)(ntiles * kRDigits), s));
  PRDF_TRY(goff.alloc((size_t)(ntiles * kRDigits + 1), s));
  KeySrc src;
  src.keys = nullptr;
  src.rows = rows;
  src.cols = cols;
  src.m0 = m0;
  src.B = B;
  uint64_t* cur = ka.p;
  uint64_t* nxt = kb.p;
  PRDF_TRY(radix_pass<true>(src, M, 0, cur, hist, goff, ntiles, ws, s));
  for (int p = 1; p < passes; ++p) {
    src.keys = cur;
    PRDF_TRY(radix_pass<false>(src, M, 8 * p, nxt, hist, goff, ntiles, ws, s));
    uint64_t* t = cur;
    cur = nxt;
    nxt = t;
  }
  // merge equal keys
  const int64_t nw = ntiles * kRWarps;
  DBuf<uint32_t> wcnt;
  DBuf<int64_t> woff;
  PRDF_TRY(wcnt.alloc((size_t)nw, s));
  PRDF_TRY(woff.alloc((size_t)nw + 1, s));
  k_uniq_count<<<(unsigned)ntiles, kRT, 0, s>>>(cur, M, wcnt.p);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(exclusive_scan_u32(wcnt.p, nw, woff.p, ws, s));
  PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, woff.p + nw, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  out.m = ws.host_i64[0];
  PRDF_TRY(out.off.alloc((size_t)n + 1, s));
  PRDF_TRY(out.adj.alloc((size_t)(out.m > 0 ? out.m : 1), s));
  out.w.release();
  // a list much shorter than n leaves long runs of empty rows: their offsets
  // are found row-parallel instead of by the lanes that emit the keys
  const bool sparse = M * 16 < (int64_t)n;
  DBuf<int32_t> urow;
  if (sparse) PRDF_TRY(urow.alloc((size_t)(out.m > 0 ? out.m : 1), s));
  k_uniq_emit<<<(unsigned)ntiles, kRT, 0, s>>>(cur, M, B, n, woff.p, nw, out.adj.p, out.off.p,
                                               sparse ? urow.p : nullptr);
  if (sparse) k_offsets_from_rows<<<grid_for((int64_t)n + 1, kRT), kRT, 0, s>>>(urow.p, out.m, n, out.off.p);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

}  // namespace prdf
