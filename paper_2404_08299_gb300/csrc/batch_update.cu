// Incremental batch update of one CSR (Sec. 3.3 set semantics): every row
// becomes (old \ D) u I, merged in column order without re-sorting the
// graph. The batch itself is turned into two small CSRs (D and I, sorted and
// deduplicated per row, I keeping the maximum weight of duplicates); then
//   - a D entry removes an element if it is in the old row;
//   - an I entry adds an element unless it is in the old row and not deleted
//     (then it only raises that edge's weight to the maximum);
//   - each surviving old entry moves to
//       new_off[u] + (j - off[u]) - #(D entries in old, col < c) + #(adding I entries, col < c),
//   - each adding I entry to
//       new_off[u] + #(old entries, col < c) - #(D entries in old, col < c) + #(adding I entries before it).
// Rows without batch entries are copied edge-parallel in contiguous segments
// between the changed rows, each with one shift. The result equals a rebuild
// of the whole edge list when every vertex already has its self-loop.
//
// Keyed form: the rows of a CSR in the sweep numbering hold renumbered ids in
// the order of the vertices' original ids. With key (renumbered -> original)
// every comparison with an old entry uses key[entry], the batch's columns are
// original ids, and store (original -> renumbered) maps an added column to the
// value stored; rows stay ordered by original id.
#include "internal.cuh"

namespace prdf {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* a, int64_t lo, int64_t hi, int32_t c) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool contains(const int64_t* off, const int32_t* adj, int32_t u, int32_t c) {
  const int64_t e = off[u + 1];
  const int64_t p = lower_bound_i32(adj, off[u], e, c);
  return p < e && adj[p] == c;
}

// the same on an old row compared through key (null: the entries themselves)
__device__ __forceinline__ int64_t lower_bound_key(const int32_t* a, const int32_t* key, int64_t lo, int64_t hi,
                                                   int32_t c) {
  if (!key) return lower_bound_i32(a, lo, hi, c);
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (key[a[mid]] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ bool contains_key(const int64_t* off, const int32_t* adj, const int32_t* key, int32_t u,
                                             int32_t c) {
  const int64_t e = off[u + 1];
  const int64_t p = lower_bound_key(adj, key, off[u], e, c);
  return p < e && (key ? key[adj[p]] : adj[p]) == c;
}

// row of CSR entry k: the last u with off[u] <= k
__device__ __forceinline__ int32_t row_of(const int64_t* off, int32_t n, int64_t k) {
  int32_t lo = 0, hi = n;  // off[lo] <= k < off[hi]
  while (hi - lo > 1) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    if (off[mid] <= k) lo = mid; else hi = mid;
  }
  return lo;
}

// flag[i] = deletion i is not a self-loop (self-loops are never deleted)
__global__ void k_not_self(const int32_t* __restrict__ r, const int32_t* __restrict__ c, int64_t cnt,
                           const int32_t* __restrict__ key, uint32_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (key ? key[r[i]] : r[i]) == c[i] ? 0u : 1u;
}

// the flagged pairs, in order, at their scanned positions
__global__ void k_keep_pairs(const int32_t* __restrict__ r, const int32_t* __restrict__ c, int64_t cnt,
                             const uint32_t* __restrict__ flag, const int64_t* __restrict__ pos,
                             int32_t* __restrict__ ro, int32_t* __restrict__ co) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) {
      ro[pos[i]] = r[i];
      co[pos[i]] = c[i];
    }
}

// dflag[k] = D entry k is in the old row; iflag[k] = I entry k adds an element
__global__ void k_batch_flags(int32_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                              const int32_t* __restrict__ key, const int64_t* __restrict__ d_off,
                              const int32_t* __restrict__ d_adj, int64_t nd, const int64_t* __restrict__ i_off,
                              const int32_t* __restrict__ i_adj, int64_t ni, uint32_t* __restrict__ dflag,
                              uint32_t* __restrict__ iflag) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nd + ni; k += (int64_t)gridDim.x * blockDim.x) {
    if (k < nd) {
      const int32_t u = row_of(d_off, n, k);
      dflag[k] = contains_key(off, adj, key, u, d_adj[k]) ? 1u : 0u;
    } else {
      const int64_t q = k - nd;
      const int32_t u = row_of(i_off, n, q);
      const int32_t c = i_adj[q];
      const bool surviving = contains_key(off, adj, key, u, c) && !contains(d_off, d_adj, u, c);
      iflag[q] = surviving ? 0u : 1u;
    }
  }
}

// new row lengths: old - removed + added (dpref, ipref: exclusive scans of the flags)
__global__ void k_new_len(int32_t n, const int64_t* __restrict__ off, const int64_t* __restrict__ d_off,
                          const int64_t* __restrict__ dpref, const int64_t* __restrict__ i_off,
                          const int64_t* __restrict__ ipref, int64_t* __restrict__ len) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t removed = dpref[d_off[u + 1]] - dpref[d_off[u]];
    const int64_t added = ipref[i_off[u + 1]] - ipref[i_off[u]];
    len[u] = (off[u + 1] - off[u]) - removed + added;
  }
}

// rows with batch entries, listed in ascending order (flag, exclusive scan, list)
__global__ void k_mark_changed(int32_t n, const int64_t* __restrict__ d_off, const int64_t* __restrict__ i_off,
                               uint32_t* __restrict__ flag) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    flag[u] = (d_off[u + 1] > d_off[u] || i_off[u + 1] > i_off[u]) ? 1u : 0u;
}

__global__ void k_list_changed(int32_t n, const uint32_t* __restrict__ flag, const int64_t* __restrict__ pos,
                               int32_t* __restrict__ changed) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    if (flag[u]) changed[pos[u]] = (int32_t)u;
}

// Old entries of unchanged rows. Between two changed rows every entry moves by
// the same amount: noff[c] - off[c] of the next changed row c (new_m - m after
// the last one). A warp takes 256 consecutive entries (8 per lane,
// lane-strided, so loads and stores stay coalesced) and finds its place in the
// changed-row list once.
__global__ void k_copy_unchanged(int32_t n, int64_t m, const int64_t* __restrict__ off,
                                 const int64_t* __restrict__ noff, const int32_t* __restrict__ changed, int64_t k,
                                 const int32_t* __restrict__ adj, const float* __restrict__ w,
                                 int32_t* __restrict__ nadj, float* __restrict__ nw) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t tail_shift = noff[n] - off[n];
  // a warp takes a contiguous run of 256-entry windows: one binary search for
  // its first window, then the changed-row cursor only moves forward
  const int64_t nwin = (m + 255) >> 8;
  const int64_t per = (nwin + nwarps - 1) / nwarps;
  const int64_t win_end = (warp + 1) * per < nwin ? (warp + 1) * per : nwin;
  int64_t t = 0;  // number of changed rows that start at or before the window's base
  if (warp * per < win_end) {
    const int64_t base0 = (warp * per) << 8;
    int64_t lo = 0, hi = k;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (off[changed[mid]] <= base0) lo = mid + 1; else hi = mid;
    }
    t = lo;
  }
  for (int64_t win = warp * per; win < win_end; ++win) {
    const int64_t base = win << 8;
    while (t < k && off[changed[t]] <= base) ++t;
    // the common case: the window [base, base + 256) lies between the end of changed row t - 1 and the start
    // of changed row t, so every entry moves by the same shift (no per-entry tests, all loads in flight)
    const int64_t seg_b = t > 0 ? off[changed[t - 1] + 1] : 0;
    const int64_t seg_e = t < k ? off[changed[t]] : m;
    if (seg_b <= base && base + 256 <= seg_e) {
      const int64_t shift = t < k ? noff[changed[t]] - off[changed[t]] : tail_shift;
      int32_t va[8];
      float vw[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        va[q] = adj[base + lane + 32 * q];
        if (nw) vw[q] = w[base + lane + 32 * q];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        nadj[base + lane + 32 * q + shift] = va[q];
        if (nw) nw[base + lane + 32 * q + shift] = vw[q];
      }
      continue;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t j = base + lane + 32 * q;
      if (j >= m) break;
      while (t < k && off[changed[t]] <= j) ++t;
      if (t > 0 && j < off[changed[t - 1] + 1]) continue;  // an entry of a changed row
      const int64_t to = j + (t < k ? noff[changed[t]] - off[changed[t]] : tail_shift);
      nadj[to] = adj[j];
      if (nw) nw[to] = w[j];
    }
  }
}

// length of each changed row (for the entry-parallel pass below)
__global__ void k_changed_len(const int32_t* __restrict__ changed, int64_t k, const int64_t* __restrict__ off,
                              int64_t* __restrict__ len) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < k; r += (int64_t)gridDim.x * blockDim.x)
    len[r] = off[changed[r] + 1] - off[changed[r]];
}

// Surviving old entries of the changed rows, entry-parallel over their
// concatenation (cpref: exclusive scan of the row lengths, total T), 256
// entries per warp so that long rows spread over many warps; a re-inserted
// surviving edge keeps the larger weight.
__global__ void k_move_changed(const int32_t* __restrict__ changed, int64_t k, const int64_t* __restrict__ cpref,
                               int64_t T, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                               const int32_t* __restrict__ key, const float* __restrict__ w,
                               const int64_t* __restrict__ d_off,
                               const int32_t* __restrict__ d_adj, const int64_t* __restrict__ dpref,
                               const int64_t* __restrict__ i_off, const int32_t* __restrict__ i_adj,
                               const float* __restrict__ i_w, const int64_t* __restrict__ ipref,
                               const int64_t* __restrict__ noff, int32_t* __restrict__ nadj, float* __restrict__ nw) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // a warp takes a contiguous run of 256-entry windows: one binary search for
  // its first window, then the row cursor only moves forward
  const int64_t nwin = (T + 255) >> 8;
  const int64_t per = (nwin + nwarps - 1) / nwarps;
  const int64_t win_end = (warp + 1) * per < nwin ? (warp + 1) * per : nwin;
  int64_t r = 0;  // the changed row holding the entry: the last r with cpref[r] <= entry
  if (warp * per < win_end) {
    const int64_t base0 = (warp * per) << 8;
    int64_t lo = 0, hi = k;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (cpref[mid] <= base0) lo = mid; else hi = mid;
    }
    r = lo;
  }
  for (int64_t win = warp * per; win < win_end; ++win) {
    const int64_t base = win << 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t x = base + lane + 32 * q;
      if (x >= T) break;
      while (cpref[r + 1] <= x) ++r;
      const int32_t u = changed[r];
      const int64_t b = off[u], j = b + (x - cpref[r]);
      const int64_t db = d_off[u], de = d_off[u + 1], ib = i_off[u], ie = i_off[u + 1];
      const int32_t c = adj[j];
      const int32_t ck = key ? key[c] : c;  // the batch lists hold keys
      const int64_t p = lower_bound_i32(d_adj, db, de, ck);
      if (p < de && d_adj[p] == ck) continue;  // deleted (a re-insertion is placed by k_place_new)
      const int64_t qq = lower_bound_i32(i_adj, ib, ie, ck);
      const int64_t pos = noff[u] + (j - b) - (dpref[p] - dpref[db]) + (ipref[qq] - ipref[ib]);
      nadj[pos] = c;
      if (nw) nw[pos] = (qq < ie && i_adj[qq] == ck) ? fmaxf(w[j], i_w[qq]) : w[j];
    }
  }
}

// adding I entries (thread per entry)
__global__ void k_place_new(int32_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            const int32_t* __restrict__ key, const int32_t* __restrict__ store,
                            const int64_t* __restrict__ d_off, const int32_t* __restrict__ d_adj,
                            const int64_t* __restrict__ dpref, const int64_t* __restrict__ i_off,
                            const int32_t* __restrict__ i_adj, const float* __restrict__ i_w,
                            const uint32_t* __restrict__ iflag, const int64_t* __restrict__ ipref, int64_t ni,
                            const int64_t* __restrict__ noff, int32_t* __restrict__ nadj, float* __restrict__ nw) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ni; k += (int64_t)gridDim.x * blockDim.x) {
    if (!iflag[k]) continue;
    const int32_t u = row_of(i_off, n, k);
    const int32_t c = i_adj[k];
    const int64_t old_before = lower_bound_key(adj, key, off[u], off[u + 1], c) - off[u];
    const int64_t db = d_off[u];
    const int64_t p = lower_bound_i32(d_adj, db, d_off[u + 1], c);
    const int64_t pos = noff[u] + old_before - (dpref[p] - dpref[db]) + (ipref[k] - ipref[i_off[u]]);
    nadj[pos] = store ? store[c] : c;
    if (nw) nw[pos] = i_w[k];
  }
}


// ---------------------------------------------------------------------------
// Small batches (at most kSmallBatch deletions and kSmallBatch insertions):
// the batch is prepared by one block in shared memory instead of being turned
// into two CSRs over all n rows, so the only O(n) pass left is the one that
// writes the new row offsets (and the O(m) copy of the unchanged rows).
constexpr int kSmallBatch = 4096;
constexpr int kPrepThreads = 1024;
constexpr uint64_t kNoKey = ~0ull;

__device__ __forceinline__ uint64_t rc_key(int32_t r, int32_t c) { return ((uint64_t)(uint32_t)r << 32) | (uint32_t)c; }

// bitonic sort of cnt (a power of two) keys in shared memory, payload p (nullable) moved along
__device__ void block_sort(uint64_t* k, int32_t* p, int cnt) {
  for (int size = 2; size <= cnt; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const uint64_t a = k[i], b = k[j];
          if ((a > b) == up) {
            k[i] = b;
            k[j] = a;
            if (p) {
              const int32_t t = p[i];
              p[i] = p[j];
              p[j] = t;
            }
          }
        }
      }
      __syncthreads();
    }
}

// exclusive scan of v[0..cnt) in shared memory, in place; returns the total (every thread);
// every thread of the block must call it
__device__ int64_t block_scan(int64_t* v, int cnt, int64_t* tmp /* blockDim.x + 1 */) {
  const int per = (cnt + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per, e = min(b + per, cnt);
  int64_t sum = 0;
  for (int i = b; i < e; ++i) sum += v[i];
  tmp[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int64_t x = tmp[t];
      tmp[t] = run;
      run += x;
    }
    tmp[blockDim.x] = run;
  }
  __syncthreads();
  int64_t run = tmp[threadIdx.x];
  for (int i = b; i < e; ++i) {
    const int64_t x = v[i];
    v[i] = run;
    run += x;
  }
  const int64_t total = tmp[blockDim.x];
  __syncthreads();
  return total;
}

__device__ __forceinline__ int lower_bound_u64(const uint64_t* a, int lo, int hi, uint64_t x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One block: sorts and deduplicates D (self-loops dropped) and I (duplicates
// keep the maximum weight), classifies every entry against the old rows (a
// deletion removes, an insertion adds unless the edge survives), and lists the
// changed rows with their ranges in the sorted lists and the prefix of their
// length changes. Outputs: d_cols, dpref (nd + 1), i_rows, i_cols, i_w, iflag,
// ipref (ni + 1), changed, c_db, c_de, c_ib, c_ie, c_shift (kc + 1),
// sizes = {nd, ni, kc, total length change}.
__global__ void __launch_bounds__(kPrepThreads) k_prep_small(
    const int64_t* __restrict__ off, const int32_t* __restrict__ adj, const int32_t* __restrict__ key,
    const int32_t* __restrict__ del_rows, const int32_t* __restrict__ del_cols, int64_t n_del,
    const int32_t* __restrict__ ins_rows, const int32_t* __restrict__ ins_cols, const float* __restrict__ ins_w,
    int64_t n_ins, int nd_pow, int ni_pow, int32_t* __restrict__ d_cols, int64_t* __restrict__ dpref,
    int32_t* __restrict__ i_rows, int32_t* __restrict__ i_cols, float* __restrict__ i_w,
    uint32_t* __restrict__ iflag, int64_t* __restrict__ ipref, int32_t* __restrict__ changed,
    int64_t* __restrict__ c_db, int64_t* __restrict__ c_de, int64_t* __restrict__ c_ib, int64_t* __restrict__ c_ie,
    int64_t* __restrict__ c_shift, int64_t* __restrict__ sizes) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* dk = reinterpret_cast<uint64_t*>(smem);  // D keys (nd_pow)
  uint64_t* ik = dk + nd_pow;                         // I keys (ni_pow)
  uint64_t* rk = ik + ni_pow;                         // changed rows (nd_pow + ni_pow)
  int64_t* cnt = reinterpret_cast<int64_t*>(rk + nd_pow + ni_pow);  // scratch counts (nd_pow + ni_pow)
  int32_t* ip = reinterpret_cast<int32_t*>(cnt + nd_pow + ni_pow);  // I payload (ni_pow)
  __shared__ int64_t tmp[kPrepThreads + 1];
  __shared__ int s_nd, s_ni, s_kc;
  for (int i = threadIdx.x; i < nd_pow; i += blockDim.x) {
    uint64_t kk = kNoKey;
    if (i < n_del) {
      const int32_t r = del_rows[i], c = del_cols[i];
      if ((key ? key[r] : r) != c) kk = rc_key(r, c);  // self-loops are never deleted
    }
    dk[i] = kk;
  }
  for (int i = threadIdx.x; i < ni_pow; i += blockDim.x) {
    ik[i] = i < n_ins ? rc_key(ins_rows[i], ins_cols[i]) : kNoKey;
    ip[i] = i;
  }
  __syncthreads();
  block_sort(dk, nullptr, nd_pow);
  block_sort(ik, ip, ni_pow);
  // first entries of equal-key runs survive the deduplication
  for (int i = threadIdx.x; i < nd_pow; i += blockDim.x) cnt[i] = (dk[i] != kNoKey && (i == 0 || dk[i] != dk[i - 1]));
  __syncthreads();
  const int64_t nd = block_scan(cnt, nd_pow, tmp);
  // compact D into rk (scratch), then back
  for (int i = threadIdx.x; i < nd_pow; i += blockDim.x)
    if (dk[i] != kNoKey && (i == 0 || dk[i] != dk[i - 1])) rk[cnt[i]] = dk[i];
  __syncthreads();
  for (int i = threadIdx.x; i < nd; i += blockDim.x) {
    dk[i] = rk[i];
    d_cols[i] = (int32_t)(uint32_t)rk[i];
  }
  __syncthreads();
  // I: the first of a run takes the run's maximum weight; its key and weight go to global memory
  for (int i = threadIdx.x; i < ni_pow; i += blockDim.x)
    cnt[nd_pow + i] = (ik[i] != kNoKey && (i == 0 || ik[i] != ik[i - 1]));
  __syncthreads();
  const int64_t ni = block_scan(cnt + nd_pow, ni_pow, tmp);
  for (int i = threadIdx.x; i < ni_pow; i += blockDim.x) {
    if (ik[i] == kNoKey || (i > 0 && ik[i] == ik[i - 1])) continue;
    const int64_t q = cnt[nd_pow + i];
    float wmax = ins_w ? ins_w[ip[i]] : 0.f;
    for (int j = i + 1; j < ni_pow && ik[j] == ik[i]; ++j)
      if (ins_w) wmax = fmaxf(wmax, ins_w[ip[j]]);
    i_rows[q] = (int32_t)(ik[i] >> 32);
    i_cols[q] = (int32_t)(uint32_t)ik[i];
    if (ins_w) i_w[q] = wmax;
    rk[nd_pow + q] = ik[i];  // compact I keys
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ni; i += blockDim.x) ik[i] = rk[nd_pow + i];
  __syncthreads();
  // classification against the old rows
  for (int i = threadIdx.x; i < nd; i += blockDim.x) {
    const int32_t r = (int32_t)(dk[i] >> 32), c = (int32_t)(uint32_t)dk[i];
    cnt[i] = contains_key(off, adj, key, r, c) ? 1 : 0;
  }
  for (int i = threadIdx.x; i < ni; i += blockDim.x) {
    const int32_t r = (int32_t)(ik[i] >> 32), c = (int32_t)(uint32_t)ik[i];
    const int pdel = lower_bound_u64(dk, 0, (int)nd, ik[i]);
    const bool deleted = pdel < nd && dk[pdel] == ik[i];
    const bool surviving = contains_key(off, adj, key, r, c) && !deleted;
    iflag[i] = surviving ? 0u : 1u;
    cnt[nd_pow + i] = surviving ? 0 : 1;
  }
  __syncthreads();
  const int64_t dtot = block_scan(cnt, (int)nd, tmp);
  const int64_t itot = block_scan(cnt + nd_pow, (int)ni, tmp);
  for (int i = threadIdx.x; i <= nd; i += blockDim.x) dpref[i] = i < nd ? cnt[i] : dtot;
  for (int i = threadIdx.x; i <= ni; i += blockDim.x) ipref[i] = i < ni ? cnt[nd_pow + i] : itot;
  // changed rows: the sorted union of the rows of D and I
  const int rcnt = nd_pow + ni_pow;
  for (int i = threadIdx.x; i < rcnt; i += blockDim.x) {
    uint64_t r = kNoKey;
    if (i < nd) r = dk[i] >> 32;
    else if (i >= nd_pow && i - nd_pow < ni) r = ik[i - nd_pow] >> 32;
    rk[i] = r;
  }
  __syncthreads();
  block_sort(rk, nullptr, rcnt);
  for (int i = threadIdx.x; i < rcnt; i += blockDim.x) cnt[i] = (rk[i] != kNoKey && (i == 0 || rk[i] != rk[i - 1]));
  __syncthreads();
  const int64_t kc = block_scan(cnt, rcnt, tmp);
  // the changed rows' ranges and length changes (the dpref / ipref prefixes are in global memory)
  __syncthreads();
  for (int i = threadIdx.x; i < rcnt; i += blockDim.x) {
    if (rk[i] == kNoKey || (i > 0 && rk[i] == rk[i - 1])) continue;
    const int64_t t = cnt[i];
    const int32_t r = (int32_t)rk[i];
    const int db = lower_bound_u64(dk, 0, (int)nd, rc_key(r, 0)), de = lower_bound_u64(dk, 0, (int)nd, rc_key(r + 1, 0));
    const int ib = lower_bound_u64(ik, 0, (int)ni, rc_key(r, 0)), ie = lower_bound_u64(ik, 0, (int)ni, rc_key(r + 1, 0));
    changed[t] = r;
    c_db[t] = db;
    c_de[t] = de;
    c_ib[t] = ib;
    c_ie[t] = ie;
    c_shift[t] = (ipref[ie] - ipref[ib]) - (dpref[de] - dpref[db]);
  }
  __syncthreads();
  // c_shift[t] becomes the total length change of the changed rows before t (a scan in shared memory,
  // over the space of dk and ik, which are no longer needed)
  int64_t* sh = reinterpret_cast<int64_t*>(dk);
  for (int t = threadIdx.x; t < kc; t += blockDim.x) sh[t] = c_shift[t];
  __syncthreads();
  const int64_t run = block_scan(sh, (int)kc, tmp);
  for (int t = threadIdx.x; t <= kc; t += blockDim.x) c_shift[t] = t < kc ? sh[t] : run;
  if (threadIdx.x == 0) {
    sizes[0] = nd;
    sizes[1] = ni;
    sizes[2] = kc;
    sizes[3] = run;
  }
}

// new row offsets: noff[u] = off[u] + the length change of the changed rows before u (u in [0, n])
__global__ void k_new_offsets(int32_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ changed,
                              int64_t kc, const int64_t* __restrict__ c_shift, int64_t* __restrict__ noff) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u <= n; u += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = kc;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (changed[mid] < u) lo = mid + 1; else hi = mid;
    }
    noff[u] = off[u] + c_shift[lo];
  }
}

// surviving old entries of the changed rows (as k_move_changed, with each changed row's batch ranges given)
__global__ void k_move_changed_t(const int32_t* __restrict__ changed, int64_t k, const int64_t* __restrict__ cpref,
                                 int64_t T, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                 const int32_t* __restrict__ key, const float* __restrict__ w,
                                 const int64_t* __restrict__ c_db, const int64_t* __restrict__ c_de,
                                 const int64_t* __restrict__ c_ib, const int64_t* __restrict__ c_ie,
                                 const int32_t* __restrict__ d_cols, const int64_t* __restrict__ dpref,
                                 const int32_t* __restrict__ i_cols, const float* __restrict__ i_w,
                                 const int64_t* __restrict__ ipref, const int64_t* __restrict__ noff,
                                 int32_t* __restrict__ nadj, float* __restrict__ nw) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp * 256; base < T; base += nwarps * 256) {
    int64_t lo = 0, hi = k;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (cpref[mid] <= base) lo = mid; else hi = mid;
    }
    int64_t r = lo;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t x = base + lane + 32 * q;
      if (x >= T) break;
      while (cpref[r + 1] <= x) ++r;
      const int32_t u = changed[r];
      const int64_t b = off[u], j = b + (x - cpref[r]);
      const int64_t db = c_db[r], de = c_de[r], ib = c_ib[r], ie = c_ie[r];
      const int32_t c = adj[j];
      const int32_t ck = key ? key[c] : c;
      const int64_t p = lower_bound_i32(d_cols, db, de, ck);
      if (p < de && d_cols[p] == ck) continue;  // deleted
      const int64_t qq = lower_bound_i32(i_cols, ib, ie, ck);
      const int64_t pos = noff[u] + (j - b) - (dpref[p] - dpref[db]) + (ipref[qq] - ipref[ib]);
      nadj[pos] = c;
      if (nw) nw[pos] = (qq < ie && i_cols[qq] == ck) ? fmaxf(w[j], i_w[qq]) : w[j];
    }
  }
}

// adding I entries of a small batch (thread per entry)
__global__ void k_place_new_t(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                              const int32_t* __restrict__ key, const int32_t* __restrict__ store,
                              const int32_t* __restrict__ changed, int64_t kc, const int64_t* __restrict__ c_db,
                              const int64_t* __restrict__ c_ib, const int32_t* __restrict__ d_cols,
                              const int64_t* __restrict__ c_de, const int64_t* __restrict__ dpref,
                              const int32_t* __restrict__ i_rows, const int32_t* __restrict__ i_cols,
                              const float* __restrict__ i_w, const uint32_t* __restrict__ iflag,
                              const int64_t* __restrict__ ipref, int64_t ni, const int64_t* __restrict__ noff,
                              int32_t* __restrict__ nadj, float* __restrict__ nw) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ni; q += (int64_t)gridDim.x * blockDim.x) {
    if (!iflag[q]) continue;
    const int32_t u = i_rows[q], c = i_cols[q];
    int64_t lo = 0, hi = kc;  // the changed-row index of u
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (changed[mid] < u) lo = mid + 1; else hi = mid;
    }
    const int64_t db = c_db[lo], de = c_de[lo], ib = c_ib[lo];
    const int64_t old_before = lower_bound_key(adj, key, off[u], off[u + 1], c) - off[u];
    const int64_t p = lower_bound_i32(d_cols, db, de, c);
    const int64_t pos = noff[u] + old_before - (dpref[p] - dpref[db]) + (ipref[q] - ipref[ib]);
    nadj[pos] = store ? store[c] : c;
    if (nw) nw[pos] = i_w[q];
  }
}

}  // namespace

namespace {

int pow2_at_least(int64_t x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

int update_csr_small(int32_t n, const Csr& old, const int32_t* del_rows, const int32_t* del_cols, int64_t n_del,
                     const int32_t* ins_rows, const int32_t* ins_cols, const float* ins_w, int64_t n_ins, Csr& out,
                     Workspace& ws, cudaStream_t s, const int32_t* key, const int32_t* store) {
  const bool weighted = old.w.p != nullptr;
  // both lists padded to one power of two P, so the union of their rows (2P keys) sorts as a power of two
  const int P = pow2_at_least(n_del > n_ins ? n_del : (n_ins > 0 ? n_ins : 1));
  const int nd_pow = P, ni_pow = P;
  const size_t smem = (size_t)(nd_pow + ni_pow) * (8 + 8 + 8) + (size_t)ni_pow * 4;
  static const bool smem_set = [] {
    // the largest case: kSmallBatch keys per list
    const int mx = (2 * kSmallBatch) * (8 + 8 + 8) + kSmallBatch * 4;
    if (cudaFuncSetAttribute(k_prep_small, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess)
      cudaGetLastError();
    return true;
  }();
  (void)smem_set;
  const size_t nb = (size_t)(n_del + n_ins > 0 ? n_del + n_ins : 1);
  DBuf<int32_t> i32;  // d_cols | i_rows | i_cols | changed
  DBuf<int64_t> i64;  // dpref | ipref | c_db | c_de | c_ib | c_ie | c_shift | sizes
  DBuf<float> iw;
  DBuf<uint32_t> iflag;
  PRDF_TRY(i32.alloc((size_t)n_del + 2 * (size_t)n_ins + nb + 4, s));
  PRDF_TRY(i64.alloc((size_t)n_del + 1 + (size_t)n_ins + 1 + 5 * (nb + 1) + 4, s));
  PRDF_TRY(iw.alloc((size_t)(n_ins > 0 ? n_ins : 1), s));
  PRDF_TRY(iflag.alloc((size_t)(n_ins > 0 ? n_ins : 1), s));
  int32_t* d_cols = i32.p;
  int32_t* i_rows = d_cols + n_del;
  int32_t* i_cols = i_rows + n_ins;
  int32_t* changed = i_cols + n_ins;
  int64_t* dpref = i64.p;
  int64_t* ipref = dpref + n_del + 1;
  int64_t* c_db = ipref + n_ins + 1;
  int64_t* c_de = c_db + (nb + 1);
  int64_t* c_ib = c_de + (nb + 1);
  int64_t* c_ie = c_ib + (nb + 1);
  int64_t* c_shift = c_ie + (nb + 1);
  int64_t* sizes = c_shift + (nb + 1);
  k_prep_small<<<1, kPrepThreads, smem, s>>>(old.off.p, old.adj.p, key, del_rows, del_cols, n_del, ins_rows, ins_cols,
                                             weighted ? ins_w : nullptr, n_ins, nd_pow, ni_pow, d_cols, dpref, i_rows,
                                             i_cols, iw.p, iflag.p, ipref, changed, c_db, c_de, c_ib, c_ie, c_shift,
                                             sizes);
  PRDF_LAUNCH_CHECK();
  PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, sizes, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  const int64_t ni = ws.host_i64[1], kc = ws.host_i64[2], dm = ws.host_i64[3];
  out.m = old.m + dm;
  PRDF_TRY(out.off.alloc((size_t)n + 1, s));
  PRDF_TRY(out.adj.alloc((size_t)(out.m > 0 ? out.m : 1), s));
  if (weighted) PRDF_TRY(out.w.alloc((size_t)(out.m > 0 ? out.m : 1), s));
  else out.w.release();
  k_new_offsets<<<grid_for((int64_t)n + 1, kThreads), kThreads, 0, s>>>(n, old.off.p, changed, kc, c_shift, out.off.p);
  PRDF_LAUNCH_CHECK();
  if (old.m > 0) {
    k_copy_unchanged<<<grid_for((old.m + 7) / 8, kThreads), kThreads, 0, s>>>(
        n, old.m, old.off.p, out.off.p, changed, kc, old.adj.p, old.w.p, out.adj.p, out.w.p);
    PRDF_LAUNCH_CHECK();
  }
  if (kc > 0) {
    DBuf<int64_t> clen, cpref;
    PRDF_TRY(clen.alloc((size_t)kc, s));
    PRDF_TRY(cpref.alloc((size_t)kc + 1, s));
    k_changed_len<<<grid_for(kc, kThreads), kThreads, 0, s>>>(changed, kc, old.off.p, clen.p);
    PRDF_LAUNCH_CHECK();
    PRDF_TRY(exclusive_scan_i64(clen.p, kc, cpref.p, ws, s));
    PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, cpref.p + kc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PRDF_CUDA(cudaStreamSynchronize(s));
    const int64_t T = ws.host_i64[0];
    if (T > 0) {
      k_move_changed_t<<<grid_for((T + 7) / 8, kThreads), kThreads, 0, s>>>(
          changed, kc, cpref.p, T, old.off.p, old.adj.p, key, old.w.p, c_db, c_de, c_ib, c_ie, d_cols, dpref, i_cols,
          weighted ? iw.p : nullptr, ipref, out.off.p, out.adj.p, out.w.p);
      PRDF_LAUNCH_CHECK();
    }
  }
  if (ni > 0) {
    k_place_new_t<<<grid_for(ni, kThreads), kThreads, 0, s>>>(old.off.p, old.adj.p, key, store, changed, kc, c_db, c_ib,
                                                              d_cols, c_de, dpref, i_rows, i_cols,
                                                              weighted ? iw.p : nullptr, iflag.p, ipref, ni, out.off.p,
                                                              out.adj.p, out.w.p);
    PRDF_LAUNCH_CHECK();
  }
  return PRDF_OK;
}

}  // namespace

int update_csr(int32_t n, const Csr& old, const int32_t* del_rows, const int32_t* del_cols, int64_t n_del,
               const int32_t* ins_rows, const int32_t* ins_cols, const float* ins_w, int64_t n_ins, Csr& out,
               Workspace& ws, cudaStream_t s, const int32_t* key, const int32_t* store) {
  if (n_del <= kSmallBatch && n_ins <= kSmallBatch)
    return update_csr_small(n, old, del_rows, del_cols, n_del, ins_rows, ins_cols, ins_w, n_ins, out, ws, s, key,
                            store);
  const bool weighted = old.w.p != nullptr;
  // the batch as two small CSRs over the same rows
  Csr D, I;
  {
    // self-loop deletions are dropped first, so that D is built from a plain
    // list (the radix-sort build)
    DBuf<uint32_t> keep;
    DBuf<int64_t> kpos;
    DBuf<int32_t> dr, dc;
    int64_t nk = 0;
    if (n_del > 0) {
      PRDF_TRY(keep.alloc((size_t)n_del, s));
      PRDF_TRY(kpos.alloc((size_t)n_del + 1, s));
      k_not_self<<<grid_for(n_del, kThreads), kThreads, 0, s>>>(del_rows, del_cols, n_del, key, keep.p);
      PRDF_LAUNCH_CHECK();
      PRDF_TRY(exclusive_scan_u32(keep.p, n_del, kpos.p, ws, s));
      PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, kpos.p + n_del, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      PRDF_CUDA(cudaStreamSynchronize(s));
      nk = ws.host_i64[0];
    }
    PRDF_TRY(dr.alloc((size_t)(nk > 0 ? nk : 1), s));
    PRDF_TRY(dc.alloc((size_t)(nk > 0 ? nk : 1), s));
    if (nk > 0) {
      k_keep_pairs<<<grid_for(n_del, kThreads), kThreads, 0, s>>>(del_rows, del_cols, n_del, keep.p, kpos.p, dr.p,
                                                                  dc.p);
      PRDF_LAUNCH_CHECK();
    }
    PRDF_TRY(build_csr(n, nk, dr.p, dc.p, nullptr, false, false, D, ws, s));
  }
  PRDF_TRY(build_csr(n, n_ins, ins_rows, ins_cols, weighted ? ins_w : nullptr, false, false, I, ws, s));
  const int64_t nd = D.m, ni = I.m;
  DBuf<uint32_t> dflag, iflag;
  DBuf<int64_t> dpref, ipref;
  PRDF_TRY(dflag.alloc((size_t)(nd > 0 ? nd : 1), s));
  PRDF_TRY(iflag.alloc((size_t)(ni > 0 ? ni : 1), s));
  PRDF_TRY(dpref.alloc((size_t)nd + 1, s));
  PRDF_TRY(ipref.alloc((size_t)ni + 1, s));
  if (nd + ni > 0) {
    k_batch_flags<<<grid_for(nd + ni, kThreads), kThreads, 0, s>>>(n, old.off.p, old.adj.p, key, D.off.p, D.adj.p,
                                                                   nd, I.off.p, I.adj.p, ni, dflag.p, iflag.p);
    PRDF_LAUNCH_CHECK();
  }
  PRDF_TRY(exclusive_scan_u32(dflag.p, nd, dpref.p, ws, s));
  PRDF_TRY(exclusive_scan_u32(iflag.p, ni, ipref.p, ws, s));
  DBuf<int64_t> len;
  PRDF_TRY(len.alloc((size_t)n, s));
  k_new_len<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, old.off.p, D.off.p, dpref.p, I.off.p, ipref.p, len.p);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(out.off.alloc((size_t)n + 1, s));
  PRDF_TRY(exclusive_scan_i64(len.p, n, out.off.p, ws, s));
  PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, out.off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  out.m = ws.host_i64[0];
  PRDF_TRY(out.adj.alloc((size_t)(out.m > 0 ? out.m : 1), s));
  if (weighted) PRDF_TRY(out.w.alloc((size_t)(out.m > 0 ? out.m : 1), s));
  else out.w.release();
  // the changed rows (those with batch entries), ascending
  DBuf<uint32_t> cflag;
  DBuf<int64_t> cpos;
  PRDF_TRY(cflag.alloc((size_t)n, s));
  PRDF_TRY(cpos.alloc((size_t)n + 1, s));
  k_mark_changed<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, D.off.p, I.off.p, cflag.p);
  PRDF_LAUNCH_CHECK();
  PRDF_TRY(exclusive_scan_u32(cflag.p, n, cpos.p, ws, s));
  PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, cpos.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PRDF_CUDA(cudaStreamSynchronize(s));
  const int64_t k = ws.host_i64[0];
  DBuf<int32_t> changed;
  PRDF_TRY(changed.alloc((size_t)(k > 0 ? k : 1), s));
  if (k > 0) {
    k_list_changed<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, cflag.p, cpos.p, changed.p);
    PRDF_LAUNCH_CHECK();
  }
  if (old.m > 0) {
    k_copy_unchanged<<<grid_for((old.m + 7) / 8, kThreads), kThreads, 0, s>>>(
        n, old.m, old.off.p, out.off.p, changed.p, k, old.adj.p, old.w.p, out.adj.p, out.w.p);
    PRDF_LAUNCH_CHECK();
  }
  if (k > 0) {
    DBuf<int64_t> clen, cpref;
    PRDF_TRY(clen.alloc((size_t)k, s));
    PRDF_TRY(cpref.alloc((size_t)k + 1, s));
    k_changed_len<<<grid_for(k, kThreads), kThreads, 0, s>>>(changed.p, k, old.off.p, clen.p);
    PRDF_LAUNCH_CHECK();
    PRDF_TRY(exclusive_scan_i64(clen.p, k, cpref.p, ws, s));
    PRDF_CUDA(cudaMemcpyAsync(ws.host_i64, cpref.p + k, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PRDF_CUDA(cudaStreamSynchronize(s));
    const int64_t T = ws.host_i64[0];
    if (T > 0) {
      k_move_changed<<<grid_for((T + 7) / 8, kThreads), kThreads, 0, s>>>(
          changed.p, k, cpref.p, T, old.off.p, old.adj.p, key, old.w.p, D.off.p, D.adj.p, dpref.p, I.off.p, I.adj.p,
          weighted ? I.w.p : nullptr, ipref.p, out.off.p, out.adj.p, out.w.p);
      PRDF_LAUNCH_CHECK();
    }
  }
  if (ni > 0) {
    k_place_new<<<grid_for(ni, kThreads), kThreads, 0, s>>>(n, old.off.p, old.adj.p, key, store, D.off.p, D.adj.p,
                                                            dpref.p,
                                                            I.off.p, I.adj.p, weighted ? I.w.p : nullptr, iflag.p,
                                                            ipref.p, ni, out.off.p, out.adj.p, out.w.p);
    PRDF_LAUNCH_CHECK();
  }
  return PRDF_OK;
}

}  // namespace prdf
