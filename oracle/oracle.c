/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, sequential-order FP64 CPU implementation of what the GPU
 * library computes, written from the paper (Sahu, "Efficient GPU
 * Implementation of Static and Incrementally Expanding DF-P PageRank for
 * Dynamic Graphs", arXiv 2404.08299). Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does. It
 * shares no code, header or table with the CUDA library.
 *
 * Conventions: vertex ids int32, CSR offsets int64, ranks double, flags
 * uint8 (Section 5.1.2). Every vertex loop may run under OpenMP with
 * schedule(dynamic, 2048) as in Section 5.1.2; each vertex's neighbour sum is
 * a sequential loop in ascending neighbour order and every max-reduction is
 * exact, so results do not depend on the thread count.
 *
 * Readings where the paper is silent or inconsistent:
 *  R1 unaffected vertices are copied through: Rnew[v] = R[v];
 *  R2 updates are synchronous: read R, write Rnew; the prune/expand tests
 *     compare r with R[v] of the previous iteration;
 *  R3 the expand condition sets deltaN[v] = 1 (Alg. update prints 0);
 *  R4 in(v) comes from the transpose G^t', |out(.)| from G^t, including the
 *     self-loop;
 *  R5 deletions mark deltaN[u] and deltaV[v] as Alg. affected does;
 *  R6 Static is updateRanks with flags disabled: every vertex, Eq. 1, no
 *     prune/expand;
 *  R8 the relative change uses max(r, R[v]); prune on <= tau_p, expand on
 *     > tau_f;
 *  R9 the convergence test (L-inf <= tau) follows the swap and precedes the
 *     expand; the iteration count includes the final sweep;
 *  R10 duplicates are removed, then exactly one self-loop per vertex;
 *  R11 batch updates have set semantics: E^t = (E^{t-1} \ D) u I, self-loops
 *     are never deleted;
 *  R12 Dynamic Traversal closes the marked set under reachability along the
 *     out-edges of G^t (Alg. traversal passes G^t; a vertex reachable in
 *     G^{t-1} only through deleted edges is reached from their targets, which
 *     initialAffected marks).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Graph construction (Section 3.1 self-loops; Section 4.5 CSR of G and G')  */
/* ------------------------------------------------------------------------ */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/*
 * CSR with rows[] as row index and cols[] as column: the set
 * E = unique{(rows[i], cols[i])} u {(v, v) : v in V}, each row sorted
 * ascending (reading R10). Pass (src, dst) for the out-CSR of G and
 * (dst, src) for the in-CSR of the transpose G'. off has n+1 entries, adj
 * needs room for m0 + n entries. Returns m, or -1 on an id outside [0, n).
 */
int64_t oracle_csr_build(int32_t n, int64_t m0, const int32_t* rows, const int32_t* cols, int add_self_loops,
                         int64_t* off, int32_t* adj) {
  for (int64_t i = 0; i < m0; ++i)
    if (rows[i] < 0 || rows[i] >= n || cols[i] < 0 || cols[i] >= n) return -1;
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < m0; ++i) cnt[rows[i]]++;
  if (add_self_loops)
    for (int32_t v = 0; v < n; ++v) cnt[v]++;
  int64_t* start = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  start[0] = 0;
  for (int32_t v = 0; v < n; ++v) start[v + 1] = start[v] + cnt[v];
  int64_t* fill = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  memcpy(fill, start, ((size_t)n + 1) * sizeof(int64_t));
  int32_t* tmp = (int32_t*)malloc((size_t)(start[n] > 0 ? start[n] : 1) * sizeof(int32_t));
  for (int64_t i = 0; i < m0; ++i) tmp[fill[rows[i]]++] = cols[i];
  if (add_self_loops)
    for (int32_t v = 0; v < n; ++v) tmp[fill[v]++] = v;
  /* sort + unique each row */
#pragma omp parallel for schedule(dynamic, 2048)
  for (int32_t v = 0; v < n; ++v) {
    int64_t b = start[v], e = start[v + 1];
    qsort(tmp + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
    int64_t u = 0;
    for (int64_t j = b; j < e; ++j)
      if (j == b || tmp[j] != tmp[j - 1]) tmp[b + u++] = tmp[j];
    cnt[v] = u;
  }
  off[0] = 0;
  for (int32_t v = 0; v < n; ++v) off[v + 1] = off[v] + cnt[v];
#pragma omp parallel for schedule(dynamic, 2048)
  for (int32_t v = 0; v < n; ++v) memcpy(adj + off[v], tmp + start[v], (size_t)cnt[v] * sizeof(int32_t));
  int64_t m = off[n];
  free(cnt); free(start); free(fill); free(tmp);
  return m;
}

/* Is (u, v) an edge of the CSR (rows sorted)? Binary search. */
static int has_edge(const int64_t* off, const int32_t* adj, int32_t u, int32_t v) {
  int64_t lo = off[u], hi = off[u + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (adj[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo < off[u + 1] && adj[lo] == v;
}

/*
 * Batch update with set semantics (Section 3.3; reading R11):
 * E^t = (E^{t-1} \ D) u I with self-loops kept. The old graph is its out-CSR
 * (off, adj) with m edges. The new out-CSR goes to (noff, nadj), nadj with
 * room for m + n_ins entries; returns its edge count. del_eff[i] is 1 iff
 * deletion i is in E^{t-1} \ E^t, ins_eff[i] is 1 iff insertion i is in
 * E^t \ E^{t-1}: these define the effective Delta^{t-} and Delta^{t+}.
 */
int64_t oracle_apply_batch(int32_t n, const int64_t* off, const int32_t* adj,
                           const int32_t* del_src, const int32_t* del_dst, int64_t n_del,
                           const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins,
                           int64_t* noff, int32_t* nadj, uint8_t* del_eff, uint8_t* ins_eff) {
  const int64_t m = off[n];
  for (int64_t i = 0; i < n_del; ++i)
    if (del_src[i] < 0 || del_src[i] >= n || del_dst[i] < 0 || del_dst[i] >= n) return -1;
  for (int64_t i = 0; i < n_ins; ++i)
    if (ins_src[i] < 0 || ins_src[i] >= n || ins_dst[i] < 0 || ins_dst[i] >= n) return -1;
  /* deleted[j] marks old edge slots removed by D (self-loops never) */
  uint8_t* deleted = (uint8_t*)calloc((size_t)m + 1, 1);
  for (int64_t i = 0; i < n_del; ++i) {
    int32_t u = del_src[i], v = del_dst[i];
    if (u == v) continue;
    int64_t lo = off[u], hi = off[u + 1];
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (adj[mid] < v) lo = mid + 1; else hi = mid;
    }
    if (lo < off[u + 1] && adj[lo] == v) deleted[lo] = 1;
  }
  int64_t cap = m + n_ins;
  int32_t* rs = (int32_t*)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
  int32_t* cs = (int32_t*)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
  int64_t k = 0;
  for (int32_t u = 0; u < n; ++u)
    for (int64_t j = off[u]; j < off[u + 1]; ++j)
      if (!deleted[j]) { rs[k] = u; cs[k] = adj[j]; ++k; }
  for (int64_t i = 0; i < n_ins; ++i) { rs[k] = ins_src[i]; cs[k] = ins_dst[i]; ++k; }
  int64_t mn = oracle_csr_build(n, k, rs, cs, 1, noff, nadj);
  for (int64_t i = 0; i < n_del; ++i)
    del_eff[i] = (uint8_t)(has_edge(off, adj, del_src[i], del_dst[i]) && !has_edge(noff, nadj, del_src[i], del_dst[i]));
  for (int64_t i = 0; i < n_ins; ++i)
    ins_eff[i] = (uint8_t)(!has_edge(off, adj, ins_src[i], ins_dst[i]) && has_edge(noff, nadj, ins_src[i], ins_dst[i]));
  free(deleted); free(rs); free(cs);
  return mn;
}

/* ------------------------------------------------------------------------ */
/* Partition (Alg. partition, Appendix A.2)                                 */
/* ------------------------------------------------------------------------ */

/*
 * Stable partition of 0..n-1 by degree deg[v] = off[v+1] - off[v] into
 * n_thr+1 classes: class 0 holds deg <= thr[0], class c holds
 * thr[c-1] < deg <= thr[c], the last class deg > thr[n_thr-1]; each class in
 * ascending vertex order, classes concatenated. With one threshold D_P this is
 * exactly Alg. partition (low degree first, N_P = count[0]). count[c] receives
 * each class size.
 */
void oracle_partition(int32_t n, const int64_t* off, int n_thr, const int64_t* thr, int32_t* P, int64_t* count) {
  int64_t k = 0;
  for (int c = 0; c <= n_thr; ++c) {
    int64_t before = k;
    for (int32_t v = 0; v < n; ++v) {
      int64_t d = off[v + 1] - off[v];
      int cls = 0;
      while (cls < n_thr && d > thr[cls]) ++cls;
      if (cls == c) P[k++] = v;
    }
    count[c] = k - before;
  }
}

/* ------------------------------------------------------------------------ */
/* Affected-vertex marking (Alg. affected, Appendix A.3)                    */
/* ------------------------------------------------------------------------ */

/*
 * initialAffected: for each deletion (u, v) set deltaN[u] and deltaV[v]; for
 * each insertion (u, .) set deltaN[u] (reading R5). Entries whose mask byte
 * is 0 are skipped (mask may be NULL: all entries count). Flags are OR-ed
 * into the arrays, which the caller zeroes first.
 */
void oracle_initial_affected(int32_t n, const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask,
                             int64_t n_del, const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins,
                             uint8_t* dV, uint8_t* dN) {
  (void)n;
  for (int64_t i = 0; i < n_del; ++i) {
    if (del_mask && !del_mask[i]) continue;
    dN[del_src[i]] = 1;
    dV[del_dst[i]] = 1;
  }
  for (int64_t i = 0; i < n_ins; ++i) {
    if (ins_mask && !ins_mask[i]) continue;
    dN[ins_src[i]] = 1;
  }
}

/* expandAffected: deltaV[w] = 1 for every w in G^t.out(u) with deltaN[u]. */
void oracle_expand_affected(int32_t n, const int64_t* off, const int32_t* adj, const uint8_t* dN, uint8_t* dV) {
  for (int32_t u = 0; u < n; ++u)
    if (dN[u])
      for (int64_t j = off[u]; j < off[u + 1]; ++j) dV[adj[j]] = 1;
}

/* ------------------------------------------------------------------------ */
/* Rank iterations (Eq. 1, Eq. 2, Alg. static, Alg. frontier, Alg. update)   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int iterations;
  int converged;
  double final_delta;
} oracle_stats;

/* ||a - b||_inf, exact. */
static double linf_delta(int32_t n, const double* a, const double* b) {
  double m = 0;
#pragma omp parallel for schedule(dynamic, 2048) reduction(max : m)
  for (int32_t v = 0; v < n; ++v) {
    double d = fabs(a[v] - b[v]);
    if (d > m) m = d;
  }
  return m;
}

/*
 * Static PageRank (Alg. static; Eq. 1). in_off/in_adj is the in-CSR of G',
 * outdeg[u] = |G.out(u)| including the self-loop. R0 is the starting vector
 * (NULL: 1/|V| for every vertex, as Alg. static initialises; a previous rank
 * vector gives Naive-dynamic, Alg. naive). Iterates synchronously until the
 * L-inf change is <= tol or max_iter sweeps ran. The result goes to R.
 * max_sweeps_cap < 0 means no extra cap; otherwise at most that many sweeps
 * run (used to time a bounded sample).
 */
int oracle_pagerank_static(int32_t n, const int64_t* in_off, const int32_t* in_adj, const int64_t* outdeg,
                           double alpha, double tol, int max_iter, const double* R0, double* R,
                           oracle_stats* st) {
  double* Ra = (double*)malloc((size_t)n * sizeof(double));
  double* Rb = (double*)malloc((size_t)n * sizeof(double));
  for (int32_t v = 0; v < n; ++v) Ra[v] = Rb[v] = R0 ? R0[v] : 1.0 / (double)n;
  const double C0 = (1.0 - alpha) / (double)n;
  double* cur = Ra;
  double* nxt = Rb;
  int it = 0, conv = 0;
  double dR = 0;
  for (int i = 0; i < max_iter; ++i) {
#pragma omp parallel for schedule(dynamic, 2048)
    for (int32_t v = 0; v < n; ++v) {
      double c = 0;
      for (int64_t j = in_off[v]; j < in_off[v + 1]; ++j) {
        int32_t u = in_adj[j];
        c += cur[u] / (double)outdeg[u];
      }
      nxt[v] = C0 + alpha * c;
    }
    dR = linf_delta(n, nxt, cur);
    double* t = cur; cur = nxt; nxt = t;
    it = i + 1;
    if (dR <= tol) { conv = 1; break; }
  }
  memcpy(R, cur, (size_t)n * sizeof(double));
  if (st) { st->iterations = it; st->converged = conv; st->final_delta = dR; }
  free(Ra); free(Rb);
  return 0;
}

/*
 * Dynamic Frontier (prune = 0) and Dynamic Frontier with Pruning (prune = 1)
 * PageRank: Alg. frontier with Alg. update and Alg. affected, executed
 * sequentially in the paper's order (readings R1-R9).
 *   G^t:  out_off/out_adj (out-CSR), used for |out(.)| and for marking;
 *   G^t': in_off/in_adj (in-CSR), used for the in-neighbour sums;
 *   Delta: effective deletions (del_src, del_dst, del_mask) and insertions
 *          (ins_src, ins_mask); masks may be NULL;
 *   Rprev: R^{t-1}.
 * dV_out (may be NULL) receives the final deltaV; affected_trace (may be
 * NULL, room for max_iter entries) receives |deltaV| before each sweep.
 */
int oracle_pagerank_dfp(int32_t n, const int64_t* out_off, const int32_t* out_adj,
                        const int64_t* in_off, const int32_t* in_adj,
                        const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask, int64_t n_del,
                        const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins,
                        const double* Rprev, double alpha, double tol, double tau_f, double tau_p,
                        int max_iter, int prune, double* R, uint8_t* dV_out, int64_t* affected_trace,
                        oracle_stats* st) {
  double* Ra = (double*)malloc((size_t)n * sizeof(double));
  double* Rb = (double*)malloc((size_t)n * sizeof(double));
  uint8_t* dV = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* dN = (uint8_t*)calloc((size_t)n, 1);
  int64_t* deg = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) deg[v] = out_off[v + 1] - out_off[v];
  /* R <- Rnew <- R^{t-1} */
  for (int32_t v = 0; v < n; ++v) Ra[v] = Rb[v] = Rprev[v];
  /* initialAffected, then expandAffected */
  oracle_initial_affected(n, del_src, del_dst, del_mask, n_del, ins_src, ins_mask, n_ins, dV, dN);
  oracle_expand_affected(n, out_off, out_adj, dN, dV);
  const double C0 = (1.0 - alpha) / (double)n;
  double* cur = Ra;
  double* nxt = Rb;
  int it = 0, conv = 0;
  double dR = 0;
  for (int i = 0; i < max_iter; ++i) {
    if (affected_trace) {
      int64_t a = 0;
      for (int32_t v = 0; v < n; ++v) a += dV[v];
      affected_trace[i] = a;
    }
    memset(dN, 0, (size_t)n);
    /* updateRanks (Alg. update): every vertex of the partition lists, which
       together are all of V; the order of processing does not matter for a
       synchronous update. */
#pragma omp parallel for schedule(dynamic, 2048)
    for (int32_t v = 0; v < n; ++v) {
      if (!dV[v]) { nxt[v] = cur[v]; continue; }
      double c = 0;
      const double d = (double)deg[v];
      for (int64_t j = in_off[v]; j < in_off[v + 1]; ++j) {
        int32_t u = in_adj[j];
        c += cur[u] / (double)deg[u];
      }
      double r;
      if (prune) r = 1.0 / (1.0 - alpha / d) * (C0 + alpha * (c - cur[v] / d));  /* Eq. 2 */
      else r = C0 + alpha * c;                                                  /* Eq. 1 */
      double dr = fabs(r - cur[v]);
      double rel = dr / fmax(r, cur[v]);
      if (prune && rel <= tau_p) dV[v] = 0;
      if (rel > tau_f) dN[v] = 1;
      nxt[v] = r;
    }
    dR = linf_delta(n, nxt, cur);
    double* t = cur; cur = nxt; nxt = t;
    it = i + 1;
    if (dR <= tol) { conv = 1; break; }
    oracle_expand_affected(n, out_off, out_adj, dN, dV);
  }
  memcpy(R, cur, (size_t)n * sizeof(double));
  if (dV_out) memcpy(dV_out, dV, (size_t)n);
  if (st) { st->iterations = it; st->converged = conv; st->final_delta = dR; }
  free(Ra); free(Rb); free(dV); free(dN); free(deg);
  return 0;
}

/*
 * Dynamic Traversal (Alg. traversal). Marking: initialAffected over the batch
 * and one expandAffected, as in DF. Then the affected set is closed under
 * reachability along the out-edges of G^t: the frontier (at first every
 * affected vertex) is replaced by its out-neighbours, which join deltaV, until
 * countOnes(deltaV) stops changing. Iterations: Eq. 1 on the affected vertices
 * only (unaffected vertices keep R^{t-1}), no prune and no further expansion,
 * until the L-inf change is <= tol. n_affected (nullable): |deltaV| after the
 * closure; rounds (nullable): expansion rounds of the closure loop.
 */
int oracle_pagerank_dt(int32_t n, const int64_t* out_off, const int32_t* out_adj, const int64_t* in_off,
                       const int32_t* in_adj, const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask,
                       int64_t n_del, const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins,
                       const double* Rprev, double alpha, double tol, int max_iter, double* R, uint8_t* dV_out,
                       int64_t* n_affected, int64_t* rounds, oracle_stats* st) {
  double* Ra = (double*)malloc((size_t)n * sizeof(double));
  double* Rb = (double*)malloc((size_t)n * sizeof(double));
  uint8_t* dV = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* dN = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* dF = (uint8_t*)calloc((size_t)n, 1);
  int64_t* deg = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) deg[v] = out_off[v + 1] - out_off[v];
  for (int32_t v = 0; v < n; ++v) Ra[v] = Rb[v] = Rprev[v];
  /* mark */
  oracle_initial_affected(n, del_src, del_dst, del_mask, n_del, ins_src, ins_mask, n_ins, dV, dN);
  oracle_expand_affected(n, out_off, out_adj, dN, dV);
  int64_t na = 0;
  for (int32_t v = 0; v < n; ++v) na += dV[v];
  memcpy(dN, dV, (size_t)n);
  int64_t nr = 0;
  for (;;) {
    memset(dF, 0, (size_t)n);
    oracle_expand_affected(n, out_off, out_adj, dN, dF);
    for (int32_t v = 0; v < n; ++v) dV[v] |= dF[v];
    uint8_t* t = dN; dN = dF; dF = t;
    ++nr;
    int64_t na2 = 0;
    for (int32_t v = 0; v < n; ++v) na2 += dV[v];
    if (na2 == na) break;
    na = na2;
  }
  /* Eq. 1 over the affected vertices */
  const double C0 = (1.0 - alpha) / (double)n;
  double* cur = Ra;
  double* nxt = Rb;
  int it = 0, conv = 0;
  double dR = 0;
  for (int i = 0; i < max_iter; ++i) {
#pragma omp parallel for schedule(dynamic, 2048)
    for (int32_t v = 0; v < n; ++v) {
      if (!dV[v]) { nxt[v] = cur[v]; continue; }
      double c = 0;
      for (int64_t j = in_off[v]; j < in_off[v + 1]; ++j) {
        int32_t u = in_adj[j];
        c += cur[u] / (double)deg[u];
      }
      nxt[v] = C0 + alpha * c;
    }
    dR = linf_delta(n, nxt, cur);
    double* t = cur; cur = nxt; nxt = t;
    it = i + 1;
    if (dR <= tol) { conv = 1; break; }
  }
  memcpy(R, cur, (size_t)n * sizeof(double));
  if (dV_out) memcpy(dV_out, dV, (size_t)n);
  if (n_affected) *n_affected = na;
  if (rounds) *rounds = nr;
  if (st) { st->iterations = it; st->converged = conv; st->final_delta = dR; }
  free(Ra); free(Rb); free(dV); free(dN); free(dF); free(deg);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Weighted personalised PageRank and its adjoint (extensions beyond the    */
/* paper: the same Jacobi iteration with a row-stochastic weight matrix)    */
/* ------------------------------------------------------------------------ */

/*
 * Out-row weight sums W[u] = sum_k w_uk over the out-CSR (weights in out-CSR
 * slot order), and the transition probabilities P_uv = w_uv / W_u.
 */
void oracle_row_normalise(int32_t n, const int64_t* out_off, const double* w, double* P) {
  for (int32_t u = 0; u < n; ++u) {
    double W = 0;
    for (int64_t j = out_off[u]; j < out_off[u + 1]; ++j) W += w[j];
    for (int64_t j = out_off[u]; j < out_off[u + 1]; ++j) P[j] = w[j] / W;
  }
}

/*
 * K-column personalised PageRank: R[v, c] = alpha * sum_{u in in(v)} P_uv R[u, c]
 * + (1 - alpha) S[v, c], row-major [n, K]. Pin is the in-CSR weight array:
 * Pin[j] = P_{u v} for the in-edge slot j of v whose source is in_adj[j].
 * Starts from R = S (when R0 is NULL) and stops when the L-inf change over all
 * columns is <= tol or after max_iter sweeps.
 */
int oracle_ppr(int32_t n, int K, const int64_t* in_off, const int32_t* in_adj, const double* Pin,
               const double* S, double alpha, double tol, int max_iter, const double* R0, double* R,
               oracle_stats* st) {
  size_t nk = (size_t)n * K;
  double* cur = (double*)malloc(nk * sizeof(double));
  double* nxt = (double*)malloc(nk * sizeof(double));
  memcpy(cur, R0 ? R0 : S, nk * sizeof(double));
  int it = 0, conv = 0;
  double dR = 0;
  for (int i = 0; i < max_iter; ++i) {
    double m = 0;
#pragma omp parallel for schedule(dynamic, 2048) reduction(max : m)
    for (int32_t v = 0; v < n; ++v) {
      for (int c = 0; c < K; ++c) {
        double acc = 0;
        for (int64_t j = in_off[v]; j < in_off[v + 1]; ++j) acc += Pin[j] * cur[(size_t)in_adj[j] * K + c];
        double r = alpha * acc + (1.0 - alpha) * S[(size_t)v * K + c];
        nxt[(size_t)v * K + c] = r;
        double d = fabs(r - cur[(size_t)v * K + c]);
        if (d > m) m = d;
      }
    }
    dR = m;
    double* t = cur; cur = nxt; nxt = t;
    it = i + 1;
    if (dR <= tol) { conv = 1; break; }
  }
  memcpy(R, cur, nk * sizeof(double));
  if (st) { st->iterations = it; st->converged = conv; st->final_delta = dR; }
  free(cur); free(nxt);
  return 0;
}

/*
 * Adjoint of the K-column fixed point r = alpha P^T r + (1 - alpha) s for the
 * loss L = sum_c g_c . r_c. lambda solves (I - alpha P) lambda = g, i.e.
 * lambda[u] = g[u] + alpha * sum_{k in out(u)} P_uk lambda[k], by Jacobi sweeps
 * over the out-CSR (Pout in out-CSR slot order) until the L-inf change is
 * <= tol. Then dL/dS = (1 - alpha) lambda and, for the out-edge slot j = (u, v),
 * dL/dw_uv = sum_c (alpha r_c[u] / W_u) (lambda_c[v] - sum_k P_uk lambda_c[k]).
 * grad_S [n, K] and grad_w [m] may be NULL.
 */
int oracle_ppr_adjoint(int32_t n, int K, const int64_t* out_off, const int32_t* out_adj, const double* w,
                       const double* Pout, const double* Rk, const double* G, double alpha, double tol, int max_iter,
                       double* lambda_out, double* grad_S, double* grad_w, oracle_stats* st) {
  size_t nk = (size_t)n * K;
  double* cur = (double*)malloc(nk * sizeof(double));
  double* nxt = (double*)malloc(nk * sizeof(double));
  memcpy(cur, G, nk * sizeof(double));
  int it = 0, conv = 0;
  double dR = 0;
  for (int i = 0; i < max_iter; ++i) {
    double m = 0;
#pragma omp parallel for schedule(dynamic, 2048) reduction(max : m)
    for (int32_t u = 0; u < n; ++u) {
      for (int c = 0; c < K; ++c) {
        double acc = 0;
        for (int64_t j = out_off[u]; j < out_off[u + 1]; ++j) acc += Pout[j] * cur[(size_t)out_adj[j] * K + c];
        double l = G[(size_t)u * K + c] + alpha * acc;
        nxt[(size_t)u * K + c] = l;
        double d = fabs(l - cur[(size_t)u * K + c]);
        if (d > m) m = d;
      }
    }
    dR = m;
    double* t = cur; cur = nxt; nxt = t;
    it = i + 1;
    if (dR <= tol) { conv = 1; break; }
  }
  if (lambda_out) memcpy(lambda_out, cur, nk * sizeof(double));
  if (grad_S)
    for (size_t i = 0; i < nk; ++i) grad_S[i] = (1.0 - alpha) * cur[i];
  if (grad_w) {
    double* pl = (double*)malloc((size_t)K * sizeof(double));
    for (int32_t u = 0; u < n; ++u) {
      double W = 0;
      for (int64_t j = out_off[u]; j < out_off[u + 1]; ++j) W += w[j];
      /* pl[c] = sum_k P_uk lambda_c[k] */
      for (int c = 0; c < K; ++c) {
        pl[c] = 0;
        for (int64_t k = out_off[u]; k < out_off[u + 1]; ++k) pl[c] += Pout[k] * cur[(size_t)out_adj[k] * K + c];
      }
      for (int64_t j = out_off[u]; j < out_off[u + 1]; ++j) {
        int32_t v = out_adj[j];
        double gsum = 0;
        for (int c = 0; c < K; ++c) gsum += alpha * Rk[(size_t)u * K + c] / W * (cur[(size_t)v * K + c] - pl[c]);
        grad_w[j] = gsum;
      }
    }
    free(pl);
  }
  if (st) { st->iterations = it; st->converged = conv; st->final_delta = dR; }
  free(cur); free(nxt);
  return 0;
}

/* Set the OpenMP thread count of later calls (no effect without OpenMP). */
void oracle_set_threads(int k) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  if (k > 0) omp_set_num_threads(k);
#else
  (void)k;
#endif
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
