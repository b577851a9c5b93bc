// Device-wide exclusive scan and the stable degree partition (Alg. partition,
// Appendix A.2 of arXiv 2404.08299), generalised to up to four classes.
#include <mutex>

#include "internal.cuh"

namespace prdf {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048 elements per block

// Exclusive scan of one value per thread across a block of kScanThreads.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total) {
  __shared__ T warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    T w = lane < kScanThreads / 32 ? warp_tot[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  T res = incl - v + warp_tot[wid];
  __syncthreads();
  return res;
}

template <class TIn>
__global__ void k_tile_sums(const TIn* __restrict__ in, int64_t n, int64_t* __restrict__ tile_sum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += (int64_t)in[base + k];
  __shared__ int64_t tot;
  block_exclusive_scan<int64_t>(s, &tot);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// In-place exclusive scan of tile sums by one block; writes the grand total to ts[ntiles].
__global__ void k_scan_tile_sums(int64_t* ts, int64_t ntiles) {
  __shared__ int64_t carry_s;
  __shared__ int64_t tot;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t c = 0; c < ntiles; c += kScanTile) {
    const int64_t base = c + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = (base + k < ntiles) ? ts[base + k] : 0;
      s += v[k];
    }
    int64_t ex = block_exclusive_scan<int64_t>(s, &tot) + carry_s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (base + k < ntiles) ts[base + k] = ex;
      ex += v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_s += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) ts[ntiles] = carry_s;
}

template <class TIn>
__global__ void k_scan_apply(const TIn* __restrict__ in, int64_t n, const int64_t* __restrict__ tile_off,
                             int64_t* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? (int64_t)in[base + k] : 0;
    s += v[k];
  }
  __shared__ int64_t tot;
  int64_t ex = block_exclusive_scan<int64_t>(s, &tot) + tile_off[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = tile_off[gridDim.x];
}

// ---------------------------------------------------------- partition ----

constexpr int kPartItems = 8;
constexpr int kPartTile = kScanThreads * kPartItems;

__device__ __forceinline__ int degree_class(int64_t d, const PartThr& t) {
  int c = 0;
#pragma unroll
  for (int k = 0; k < kMaxThr; ++k) c += (k < t.n && d > t.thr[k]) ? 1 : 0;
  return c;
}

// Class counts of a thread's vertices, packed as 16-bit fields: classes 0-3 in
// p[0], classes 4-7 in p[1] (a tile has at most 2048 vertices).
struct Packed2 {
  uint64_t p[2] = {0, 0};
  __device__ __forceinline__ void add(int c) { p[c >> 2] += 1ull << (16 * (c & 3)); }
  __device__ __forceinline__ int64_t get(int c) const { return (int64_t)((p[c >> 2] >> (16 * (c & 3))) & 0xFFFF); }
};

// Class of list entry i: vertex v = in[i] (in = NULL: v = i) classed by its
// degree; desc reverses the class order (highest degrees first).
__device__ __forceinline__ int entry_class(const int64_t* __restrict__ off, const int32_t* __restrict__ in, int64_t i,
                                           const PartThr& t, bool desc) {
  const int64_t v = in ? in[i] : i;
  const int c = degree_class(off[v + 1] - off[v], t);
  return desc ? t.n - c : c;
}

// count[c * ntiles + tile] = number of list entries of class c in the tile
__global__ void k_part_count(const int64_t* __restrict__ off, const int32_t* __restrict__ in, int64_t n, PartThr t,
                             bool desc, int64_t* __restrict__ count) {
  const int64_t base = (int64_t)blockIdx.x * kPartTile + (int64_t)threadIdx.x * kPartItems;
  Packed2 pk;
#pragma unroll
  for (int k = 0; k < kPartItems; ++k) {
    const int64_t i = base + k;
    if (i < n) pk.add(entry_class(off, in, i, t, desc));
  }
  __shared__ uint64_t tot0, tot1;
  block_exclusive_scan<uint64_t>(pk.p[0], &tot0);
  if (t.n >= 4) block_exclusive_scan<uint64_t>(pk.p[1], &tot1);
  if (threadIdx.x == 0) {
    Packed2 tot;
    tot.p[0] = tot0;
    tot.p[1] = t.n >= 4 ? tot1 : 0;
    for (int c = 0; c <= t.n; ++c) count[(int64_t)c * gridDim.x + blockIdx.x] = tot.get(c);
  }
}

// P[base[c][tile] + rank within tile] = entry, ranks in list order (stable).
__global__ void k_part_scatter(const int64_t* __restrict__ off, const int32_t* __restrict__ in, int64_t n, PartThr t,
                               bool desc, const int64_t* __restrict__ base, int32_t* __restrict__ P) {
  const int64_t first = (int64_t)blockIdx.x * kPartTile + (int64_t)threadIdx.x * kPartItems;
  int cls[kPartItems];
  Packed2 pk;
#pragma unroll
  for (int k = 0; k < kPartItems; ++k) {
    const int64_t i = first + k;
    cls[k] = i < n ? entry_class(off, in, i, t, desc) : -1;
    if (cls[k] >= 0) pk.add(cls[k]);
  }
  __shared__ uint64_t tot0, tot1;
  Packed2 ex;
  ex.p[0] = block_exclusive_scan<uint64_t>(pk.p[0], &tot0);
  if (t.n >= 4) ex.p[1] = block_exclusive_scan<uint64_t>(pk.p[1], &tot1);
#pragma unroll
  for (int k = 0; k < kPartItems; ++k) {
    if (cls[k] < 0) continue;
    const int c = cls[k];
    const int64_t pos = base[(int64_t)c * gridDim.x + blockIdx.x] + ex.get(c);
    P[pos] = in ? in[first + k] : (int32_t)(first + k);
    ex.add(c);
  }
}

}  // namespace

int exclusive_scan_u32(const uint32_t* in, int64_t n, int64_t* out, Workspace& ws, cudaStream_t s) {
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  if (nt == 0) {
    PRDF_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return PRDF_OK;
  }
  PRDF_TRY(ws.scan.reserve((size_t)nt + 1, s));
  k_tile_sums<uint32_t><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, ws.scan.p);
  k_scan_tile_sums<<<1, kScanThreads, 0, s>>>(ws.scan.p, nt);
  k_scan_apply<uint32_t><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, ws.scan.p, out);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int exclusive_scan_i64(const int64_t* in, int64_t n, int64_t* out, Workspace& ws, cudaStream_t s) {
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  if (nt == 0) {
    PRDF_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return PRDF_OK;
  }
  PRDF_TRY(ws.scan.reserve((size_t)nt + 1, s));
  k_tile_sums<int64_t><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, ws.scan.p);
  k_scan_tile_sums<<<1, kScanThreads, 0, s>>>(ws.scan.p, nt);
  k_scan_apply<int64_t><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, ws.scan.p, out);
  PRDF_LAUNCH_CHECK();
  return PRDF_OK;
}

int partition_by_degree(const int64_t* off, int64_t n, const PartThr& t, int32_t* P, int64_t* counts_host,
                        Workspace& ws, cudaStream_t s) {
  return partition_list(off, nullptr, n, t, false, P, counts_host, ws, s);
}

int partition_list(const int64_t* off, const int32_t* in, int64_t n, const PartThr& t, bool desc, int32_t* P,
                   int64_t* counts_host, Workspace& ws, cudaStream_t s) {
  const int64_t nt = (n + kPartTile - 1) / kPartTile;
  const int C = t.n + 1;
  if (nt == 0) {
    for (int c = 0; c < C; ++c) counts_host[c] = 0;
    return PRDF_OK;
  }
  PRDF_TRY(ws.part_cnt.reserve((size_t)C * nt, s));
  PRDF_TRY(ws.part_base.reserve((size_t)C * nt + 1, s));
  k_part_count<<<(unsigned)nt, kScanThreads, 0, s>>>(off, in, n, t, desc, ws.part_cnt.p);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(exclusive_scan_i64(ws.part_cnt.p, C * nt, ws.part_base.p, ws, s));
  k_part_scatter<<<(unsigned)nt, kScanThreads, 0, s>>>(off, in, n, t, desc, ws.part_base.p, P);
  PRDF_LAUNCH_CHECK();
  // class sizes from the class boundaries of the flattened scan
  int64_t* hb = ws.host_i64;
  for (int c = 0; c <= C; ++c)
    PRDF_CUDA(cudaMemcpyAsync(hb + c, ws.part_base.p + (int64_t)c * nt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; c < C; ++c) counts_host[c] = hb[c + 1] - hb[c];
  return PRDF_OK;
}

// ---------------------------------------------------------------------------
// Alg. partition for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or any allocator) at the point where
// they partition: their device memory is handed out up front by a pool that
// owns all of it, or they run on a path that must not take the allocator's
// device-wide synchronisation. prdf_partition_noalloc serves them: it runs
// the same kernels as prdf_partition, but its scratch (per-tile class counts,
// their scan, and the scan's tile sums) lives in the fixed file-scope device
// array below, sized for at most kNoAllocMaxN vertices. Every GPU that loads
// the library holds this array (about 512 KB) until the process exits.
//
// The array's name means nothing as a device address in host code, so the
// first call on each device (with that device current) looks its address up
// with cudaGetSymbolAddress and caches it for the life of the process. A
// reset of the device (cudaDeviceReset) would leave the cached address
// stale, so calls after one are not supported. All calls share the one array, which keeps the last call's
// contents: each call overwrites every entry it reads before reading it, so
// nothing needs clearing, but calls that overlap on the GPU (other streams,
// other threads) race on it and must be serialised by the caller.
namespace {

constexpr int64_t kNoAllocMaxN = 1ll << 24;
constexpr int64_t kNoAllocMaxTiles = (kNoAllocMaxN + kPartTile - 1) / kPartTile;
constexpr int kNoAllocMaxThr = 3;  // at most four classes
constexpr int64_t kNoAllocCnt = (int64_t)(kNoAllocMaxThr + 1) * kNoAllocMaxTiles;
constexpr int64_t kNoAllocScan = (kNoAllocCnt + kScanTile - 1) / kScanTile + 1;
constexpr int64_t kNoAllocWords = kNoAllocCnt + (kNoAllocCnt + 1) + kNoAllocScan;

static __device__ __align__(256) int64_t g_noalloc_scratch[kNoAllocWords];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
int64_t* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
int noalloc_scratch(int64_t** out) {
  int dev = 0;
  PRDF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("device ordinal %d beyond %d", dev, kNoAllocMaxDevices);
    return PRDF_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    PRDF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = (int64_t*)p;
  }
  *out = g_noalloc_addr[dev];
  return PRDF_OK;
}

}  // namespace

}  // namespace prdf

extern "C" int prdf_partition_noalloc(const int64_t* off, int32_t n, int n_thr, const int64_t* thr_host, int32_t* P,
                                      int64_t* counts_host, void* stream) {
  using namespace prdf;
  if (!off || !P || !counts_host || !thr_host || n < 1 || n_thr < 1 || n_thr > kNoAllocMaxThr) {
    set_error("prdf_partition_noalloc: bad arguments");
    return PRDF_EINVAL;
  }
  if ((int64_t)n > kNoAllocMaxN) {
    set_error("prdf_partition_noalloc: n = %d exceeds the fixed scratch limit of %lld vertices", n,
              (long long)kNoAllocMaxN);
    return PRDF_EINVAL;
  }
  PartThr t;
  t.n = n_thr;
  for (int i = 0; i < n_thr; ++i) {
    if (thr_host[i] < 0 || (i > 0 && thr_host[i] <= thr_host[i - 1])) {
      set_error("prdf_partition_noalloc: thresholds must be >= 0 and strictly increasing");
      return PRDF_EINVAL;
    }
    t.thr[i] = thr_host[i];
  }
  int64_t* scratch = nullptr;
  PRDF_TRY(noalloc_scratch(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nt = ((int64_t)n + kPartTile - 1) / kPartTile;
  const int C = n_thr + 1;
  const int64_t cn = (int64_t)C * nt;
  int64_t* cnt = scratch;
  int64_t* base = scratch + kNoAllocCnt;
  int64_t* sums = base + kNoAllocCnt + 1;
  const int64_t nt2 = (cn + kScanTile - 1) / kScanTile;
  k_part_count<<<(unsigned)nt, kScanThreads, 0, s>>>(off, nullptr, n, t, false, cnt);
  k_tile_sums<int64_t><<<(unsigned)nt2, kScanThreads, 0, s>>>(cnt, cn, sums);
  k_scan_tile_sums<<<1, kScanThreads, 0, s>>>(sums, nt2);
  k_scan_apply<int64_t><<<(unsigned)nt2, kScanThreads, 0, s>>>(cnt, cn, sums, base);
  k_part_scatter<<<(unsigned)nt, kScanThreads, 0, s>>>(off, nullptr, n, t, false, base, P);
  PRDF_LAUNCH_CHECK();
  int64_t hb[kNoAllocMaxThr + 2];
  for (int c = 0; c <= C; ++c)
    PRDF_CUDA(cudaMemcpyAsync(hb + c, base + (int64_t)c * nt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; c < C; ++c) counts_host[c] = hb[c + 1] - hb[c];
  return PRDF_OK;
}
