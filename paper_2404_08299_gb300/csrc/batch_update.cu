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

// deletion rows with self-loops masked out (self-loops are never deleted; a
// row id r is compared through key when the columns are original ids)
__global__ void k_mask_self(const int32_t* __restrict__ r, const int32_t* __restrict__ c, int64_t cnt,
                            const int32_t* __restrict__ key, int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (key ? key[r[i]] : r[i]) == c[i] ? -1 : r[i];
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
  for (int64_t base = warp * 256; base < m; base += nwarps * 256) {
    // t = number of changed rows that start at or before base
    int64_t lo = 0, hi = k;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (off[changed[mid]] <= base) lo = mid + 1; else hi = mid;
    }
    int64_t t = lo;
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
  for (int64_t base = warp * 256; base < T; base += nwarps * 256) {
    // r = the changed row holding entry base: the last r with cpref[r] <= base
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

}  // namespace

int update_csr(int32_t n, const Csr& old, const int32_t* del_rows, const int32_t* del_cols, int64_t n_del,
               const int32_t* ins_rows, const int32_t* ins_cols, const float* ins_w, int64_t n_ins, Csr& out,
               Workspace& ws, cudaStream_t s, const int32_t* key, const int32_t* store) {
  const bool weighted = old.w.p != nullptr;
  // the batch as two small CSRs over the same rows
  Csr D, I;
  {
    DBuf<int32_t> dr;
    PRDF_TRY(dr.alloc((size_t)(n_del > 0 ? n_del : 1), s));
    if (n_del > 0) {
      k_mask_self<<<grid_for(n_del, kThreads), kThreads, 0, s>>>(del_rows, del_cols, n_del, key, dr.p);
      PRDF_LAUNCH_CHECK();
    }
    PRDF_TRY(build_csr(n, n_del, dr.p, del_cols, nullptr, false, true, D, ws, s));
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
