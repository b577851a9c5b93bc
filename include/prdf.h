/*
 * prdf -- Static and Dynamic Frontier with Pruning (DF-P) PageRank on one
 * NVIDIA GB300 (sm_103a).
 *
 * C ABI of libprdf.so. The operations follow the statement of the problem in
 * Sahu, "Efficient GPU Implementation of Static and Incrementally Expanding
 * DF-P PageRank for Dynamic Graphs" (arXiv 2404.08299):
 *   - PageRank, Eq. 1 (Section 3.1), with a self-loop on every vertex;
 *   - Static PageRank, Alg. static (Section 4.1-4.2);
 *   - DF / DF-P PageRank, Alg. frontier with the closed-loop update Eq. 2
 *     (Section 4.3, 4.5);
 *   - degree partitioning, Alg. partition (Appendix A.2);
 *   - affected-vertex marking, Alg. affected (Appendix A.3);
 *   - Dynamic Traversal, Alg. traversal (Section 3.3);
 *   - Naive-dynamic, Alg. naive (Static from the previous ranks);
 *   - batch updates Delta^{t-} = E^{t-1} \ E^t, Delta^{t+} = E^t \ E^{t-1}
 *     (Section 3.3).
 * Extensions beyond the paper: FP32 sweeps refined in FP64, K-column
 * weighted personalised PageRank, and its adjoint (gradients).
 *
 * Conventions for every entry point
 *   - Array arguments are DEVICE pointers (for example torch tensors'
 *     data_ptr) unless the name ends in _host. Work is issued on the
 *     cudaStream_t passed as `stream` (NULL = legacy default stream) and the
 *     call returns after the results are complete on that stream unless the
 *     comment says otherwise.
 *   - Vertex ids are int32 in [0, n); edge offsets are int64; ranks are
 *     double (FP64) unless stated; flags are uint8 (Section 5.1.2).
 *   - The caller owns every array it passes. A prdf_graph owns its device
 *     CSR of G and G', degree arrays, partitions and scratch; it is freed by
 *     prdf_graph_destroy.
 *   - Return value: PRDF_OK (0) or a negative PRDF_E* code; nothing is
 *     written to outputs on PRDF_EINVAL. prdf_last_error() gives a message
 *     for the calling thread's last failure. No entry point traps or asserts
 *     on the device. Reaching max_iter is not an error: stats->converged = 0.
 *   - Not reentrant on one graph: calls on the same prdf_graph must not
 *     overlap (they share its scratch).
 */
#ifndef PRDF_H
#define PRDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PRDF_OK 0
#define PRDF_EINVAL (-1)   /* bad argument: id >= n, size < 0, alpha not in (0,1), tol <= 0, K <= 0, ... */
#define PRDF_ENOMEM (-2)   /* device allocation failed */
#define PRDF_ECUDA (-3)    /* a CUDA runtime call or kernel failed */
#define PRDF_ETIMEOUT (-4) /* a bounded device-side wait ran out */
#define PRDF_ESTATE (-5)   /* call out of order (e.g. weights needed but graph unweighted) */

/* which CSR */
#define PRDF_OUT 0 /* G:  row u lists out-neighbours of u (targets) */
#define PRDF_IN 1  /* G': row v lists in-neighbours of v (sources)  */

/* precision of the rank iteration */
#define PRDF_FP64 0        /* FP64 ranks and sweeps (Section 5.1.2) */
#define PRDF_FP32_REFINE 1 /* FP32 ranks + compensated sums, then FP64 refinement sweeps */

/* accumulation of in-neighbour sums in FP64 sweeps */
#define PRDF_ACC_EXACT 0 /* exact fixed-point sum of the FP64 terms, rounded once */
#define PRDF_ACC_FP64 1  /* plain FP64 additions */

/* graph creation flags */
#define PRDF_ADD_SELF_LOOPS 1u /* give every vertex exactly one self-loop (Section 3.1) */

typedef struct prdf_graph prdf_graph;

typedef struct {
  double alpha;        /* damping factor, default 0.85 (Section 5.1.2) */
  double tol;          /* L-inf iteration tolerance tau, default 1e-10 */
  double tau_f;        /* DF frontier tolerance, default 1e-6 */
  double tau_p;        /* DF-P prune tolerance, default 1e-6 */
  int max_iter;        /* MAX_ITERATIONS, default 500 */
  int precision;       /* PRDF_FP64 (default) or PRDF_FP32_REFINE */
  double tol_fp32_rel; /* FP32 stage stops when ||dR||_inf <= tol_fp32_rel * ||R||_inf; default 1e-6 */
  int accumulate;      /* PRDF_ACC_EXACT (default) or PRDF_ACC_FP64 */
  int prune;           /* DF-P (1, default) or DF (0), for prdf_pagerank_dfp */
  int check_every;     /* sweeps launched between host convergence checks, default 8 */
  int time_sweeps;     /* 1: time every rank sweep with CUDA events (stats->ms_sweep) from a host-driven
                          loop (a residual read every check_every sweeps); 0 (default): every sweep
                          loop (Static, DF, DF-P, DT, and the FP32 stage of each) runs as one CUDA
                          graph with the convergence test on the device, no host round trips. Both
                          give identical results. */
  int tile;            /* K-column calls: columns per index fetch (8, 16, 32, 64); 0 = automatic */
  double expand_pull;  /* DF / DF-P: an expansion round after a sweep runs in pull form (each vertex
                          outside the affected set looks for a frontier in-neighbour in G') when the
                          frontier's out-edges exceed expand_pull * |E|, else in push form (Alg.
                          affected). Both mark the same set. Default 1/16; >= 1 keeps the push form;
                          must be >= 0. */
  int64_t expand_list; /* DF / DF-P / DT: a push-form round whose frontier holds at most this many
                          vertices lists them and expands them from the list, instead of scanning
                          every vertex's flag through the out-degree partition; the marks are the
                          same. -1 (default): min(32768, n / 8) on graphs of at least 2^22 vertices,
                          0 below that (where the scan is cheaper than the list's extra launches);
                          0: never; must be >= -1. */
  void* stream;        /* cudaStream_t for all work; NULL = legacy default stream */
} prdf_params;

typedef struct {
  int iterations;           /* sweeps run, including the final one (all stages) */
  int converged;            /* 1 if the final L-inf change was <= tol */
  double final_delta;       /* L-inf change of the final sweep */
  int iterations_fp32;      /* sweeps of the FP32 stage (PRDF_FP32_REFINE) */
  int sweeps_launched;      /* sweeps issued, including those that exited at once after convergence */
  float ms_total;           /* device time of the whole call (CUDA events) */
  float ms_partition;       /* initialisation + partitioning */
  float ms_mark;            /* initial marking (DF/DF-P) */
  float ms_iterate;         /* sweeps + residual + frontier expansion (incl. host convergence checks) */
  float ms_sweep;           /* device time of the first `iterations` rank sweeps (needs time_sweeps) */
  long long edges_processed;/* in-edges gathered over all sweeps (Static) */
  long long affected_initial; /* |deltaV| before the first sweep (DF/DF-P) */
  long long kernel_launches;  /* kernels launched by the call */
} prdf_stats;

/* Fill *p with the defaults above. */
void prdf_params_default(prdf_params* p);

/* Message for the calling thread's last failing call ("" if none). */
const char* prdf_last_error(void);
const char* prdf_strerror(int code);

/*
 * Device memory: the library allocates stream-ordered from its own memory
 * pool on the current device, and memory it frees stays reserved in that
 * pool for its later calls (no re-mapping of large buffers per build or
 * batch). This call gives every block of the reserve that no allocation or
 * pending free still uses back to the driver; synchronise the streams the
 * library used first. Returns PRDF_OK or PRDF_ECUDA.
 */
int prdf_release_cached_memory(void);

/* ---------------------------------------------------------------- graph -- */

/*
 * Build G (out-CSR) and G' (in-CSR) on the device from an edge list
 * (Section 4.1, 4.3: the CSR of G^t and of its transpose G^t').
 * src, dst: int32[m0] device arrays, ids in [0, n). Duplicate edges are
 * merged; with PRDF_ADD_SELF_LOOPS every vertex gets exactly one self-loop
 * (Section 3.1, 5.1.3). Rows are sorted by ascending neighbour id.
 * w: optional float32[m0] positive edge weights (NULL = unweighted); the
 * weight of merged duplicates is their maximum, an added self-loop gets 1.0.
 * n >= 1, 0 <= m0 < 2^32. Returns PRDF_EINVAL for ids out of range.
 */
int prdf_graph_create(int32_t n, const int32_t* src, const int32_t* dst, const float* w, int64_t m0,
                      unsigned flags, void* stream, prdf_graph** out);
void prdf_graph_destroy(prdf_graph* g);

/* n and the number of (unique, self-loop-including) edges m. Host outputs. */
int prdf_graph_size(const prdf_graph* g, int32_t* n_host, int64_t* m_host);

/*
 * Copy one CSR out: off int64[n+1], adj int32[m] (device). w (float32[m],
 * nullable) receives the edge weights in the same slot order (weighted
 * graphs only).
 */
int prdf_graph_export_csr(const prdf_graph* g, int which, int64_t* off, int32_t* adj, float* w, void* stream);

/*
 * Apply a batch update with set semantics (Section 3.3):
 * E^t = (E^{t-1} \ D) u I, self-loops never deleted (Section 5.1.3).
 * del_src/del_dst: int32[n_del], ins_src/ins_dst: int32[n_ins] (device).
 * Updates G and G' in place: when every vertex already has its self-loop,
 * each row becomes (old \ D) u I by an order-preserving merge (no re-sort of
 * the graph); otherwise the graph is rebuilt from its edge list, which gives
 * every vertex its self-loop. del_eff (uint8[n_del], nullable) gets 1 where
 * the deletion is in Delta^{t-} = E^{t-1} \ E^t; ins_eff (uint8[n_ins],
 * nullable) gets 1 where the insertion is in Delta^{t+} = E^t \ E^{t-1}.
 * Weighted graphs take new edges' weights from ins_w (float32[n_ins]), which
 * is then required; an edge inserted again keeps the larger of its weights,
 * duplicates in the batch take their maximum. Self-loop deletions and
 * deletions of missing edges are ignored. The sweep numbering and the
 * partitions are rebuilt for the new graph.
 */
int prdf_graph_apply_batch(prdf_graph* g, const int32_t* del_src, const int32_t* del_dst, int64_t n_del,
                           const int32_t* ins_src, const int32_t* ins_dst, const float* ins_w, int64_t n_ins,
                           uint8_t* del_eff, uint8_t* ins_eff, void* stream);

/*
 * Degree thresholds between the vertex classes of one CSR's kernels
 * (Alg. partition generalised to n_thr+1 classes). Class 0 holds
 * degree <= thr[0], class c holds thr[c-1] < degree <= thr[c], the last class
 * degree > thr[n_thr-1]; 1 <= n_thr <= 7. For PRDF_IN the classes select the
 * rank-sweep kernels (the last class one block per vertex, the one before it
 * one warp per vertex, lower classes 1, 4, 8 or 16 lanes per vertex by their
 * upper bound; default thresholds 1, 4, 16, 32, 128, 4096); for PRDF_OUT the
 * marking kernels (thread, 8 lanes, warp, block; default 8, 64, 2048).
 * thr_host: host int64[n_thr], strictly increasing, thr[0] >= 0.
 */
int prdf_graph_set_thresholds(prdf_graph* g, int which, int n_thr, const int64_t* thr_host);

/*
 * Alg. partition: stable partition of vertex ids by the degree of one CSR
 * into the classes above; P int32[n] (device) receives the ids, class by
 * class, each class in ascending id order; counts_host (host int64[n_thr+1],
 * at most 8) receives the class sizes (N_P = counts_host[0] for the paper's
 * two classes).
 */
int prdf_partition(prdf_graph* g, int which, int32_t* P, int64_t* counts_host, void* stream);

/*
 * Degree partition, the same result as prdf_partition, for callers that
 * cannot allocate device memory at this point (their memory is handed out up
 * front by a pool that owns all of it, or their path must not take the
 * device-wide synchronisation that cudaMalloc/cudaFree can imply). The paper
 * has no counterpart: this is a library service. It allocates nothing: its
 * scratch is a fixed device array inside the library (about 512 KB, held by
 * every GPU that loads the library until exit).
 * off: int64[n+1] device CSR offsets (degree = off[v+1] - off[v]);
 * thresholds as in prdf_graph_set_thresholds (n_thr in 1..3, host array);
 * P: int32[n] device output; counts_host: host int64[n_thr+1] output.
 * n must be in [1, 16777216]; larger n returns PRDF_EINVAL with a message.
 * The first call on each device looks the scratch's device address up and
 * keeps it for the life of the process, so calls after a reset of that
 * device (cudaDeviceReset) are not supported. Calls share the scratch: calls that overlap on the GPU race and
 * must be serialised by the caller. Returns after the results are complete
 * on `stream`.
 */
int prdf_partition_noalloc(const int64_t* off, int32_t n, int n_thr, const int64_t* thr_host, int32_t* P,
                           int64_t* counts_host, void* stream);

/* ------------------------------------------------------------- frontier -- */

/*
 * Alg. affected, initialAffected: for each deletion i with del_mask[i] != 0
 * (all if del_mask is NULL) set dN[del_src[i]] = 1 and dV[del_dst[i]] = 1; for
 * each insertion i with ins_mask[i] != 0 set dN[ins_src[i]] = 1. dV, dN:
 * uint8[n] device arrays, OR-ed into (not cleared).
 */
int prdf_initial_affected(prdf_graph* g, const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask,
                          int64_t n_del, const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins,
                          uint8_t* dV, uint8_t* dN, void* stream);

/*
 * Alg. affected, expandAffected: dV[w] = 1 for every w in G.out(u) with
 * dN[u] != 0, by the thread/warp/block-per-vertex kernels over the out-degree
 * partition. dV, dN: uint8[n] device; dV is OR-ed into.
 */
int prdf_expand_affected(prdf_graph* g, const uint8_t* dN, uint8_t* dV, void* stream);

/* ---------------------------------------------------------------- ranks -- */

/*
 * Static PageRank, Alg. static with Eq. 1: R = 1/n (or R0 if not NULL, which
 * is Naive-dynamic, Alg. naive), partition G' by in-degree, then synchronous
 * pull sweeps until ||R_new - R||_inf <= p->tol or p->max_iter sweeps.
 * ranks: double[n] device output. R0: double[n] device or NULL; its entries
 * must be finite and >= 0 and sum to at most 4 (a rank vector sums to 1; the
 * exact accumulator of the sweeps holds in-neighbour sums below 16), else
 * PRDF_EINVAL. p->precision = PRDF_FP32_REFINE: FP32 sweeps with compensated
 * sums until ||dR||_inf <= p->tol_fp32_rel * ||R||_inf, then FP64 sweeps from
 * their result to p->tol (stats->iterations_fp32 counts the FP32 sweeps).
 * stats may be NULL.
 */
int prdf_pagerank_static(prdf_graph* g, const prdf_params* p, const double* R0, double* ranks, prdf_stats* stats);

/*
 * DF-P (p->prune = 1) or DF (p->prune = 0) PageRank, Alg. frontier with
 * Alg. update and Alg. affected, on the graph's current G^t, G^t':
 * deletions (del_src, del_dst, del_mask) and insertions (ins_src, ins_mask)
 * as in prdf_initial_affected (pass the effectiveness masks from
 * prdf_graph_apply_batch to use the effective Delta^{t-}, Delta^{t+});
 * prev_ranks: R^{t-1}, double[n], in the domain given for R0 of
 * prdf_pagerank_static (else PRDF_EINVAL); ranks: double[n] output (may
 * alias prev_ranks). dV_out: optional uint8[n] receiving the final deltaV.
 * p->precision = PRDF_FP32_REFINE: DF / DF-P sweeps on FP32 ranks with
 * compensated sums, the prune and expand tests evaluated in FP32, until
 * ||dR||_inf <= p->tol_fp32_rel * ||R||_inf over the updated vertices; then
 * FP64 DF / DF-P sweeps to p->tol from that result, on the affected set the
 * FP32 stage left plus every vertex whose rank it changed (their prune tests
 * are then decided in FP64). Vertices the FP32 stage left unchanged keep
 * their FP64 value.
 */
int prdf_pagerank_dfp(prdf_graph* g, const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask,
                      int64_t n_del, const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins,
                      const double* prev_ranks, double* ranks, const prdf_params* p, uint8_t* dV_out,
                      prdf_stats* stats);

/*
 * Dynamic Traversal PageRank (Alg. traversal), the paper's traversal-based
 * baseline for dynamic graphs. Marking as in prdf_pagerank_dfp
 * (initialAffected over the batch, then expandAffected); then deltaV is
 * closed under reachability along the out-edges of G^t (rounds that mark the
 * not-yet-affected out-neighbours of the last round's new vertices, until a
 * round adds none, i.e. until the affected count stops changing); then Eq. 1
 * sweeps on the affected vertices only, with no prune and no expansion (p->prune
 * and p->tau_f are ignored), until ||R_new - R||_inf <= p->tol or p->max_iter.
 * Unaffected vertices keep prev_ranks. Arguments as for prdf_pagerank_dfp
 * (PRDF_FP32_REFINE: the Eq. 1 sweeps run in FP32 to the relative stop, then
 * in FP64 to p->tol); dV_out receives the closed affected set,
 * stats->affected_initial its size.
 */
int prdf_pagerank_dt(prdf_graph* g, const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask,
                     int64_t n_del, const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins,
                     const double* prev_ranks, double* ranks, const prdf_params* p, uint8_t* dV_out,
                     prdf_stats* stats);

/* ------------------------------------------------------------ tuning -- */

/*
 * Choose the in-degree class thresholds of the rank sweep for this graph
 * (the paper leaves D_P and the kernel shapes open, Appendix A.2): each of a
 * fixed list of candidates is applied, `sweeps` FP64 sweeps are timed with
 * CUDA events, and the fastest candidate stays applied. best_index (host,
 * nullable) receives the winner's index, best_ms_per_sweep (host, nullable)
 * its time per sweep. Uses p->alpha, p->accumulate and p->stream.
 */
int prdf_autotune(prdf_graph* g, const prdf_params* p, int sweeps, int* best_index, float* best_ms_per_sweep);

/*
 * Choose the column tile width (8, 16, 32 or 64) of the K-column calls for
 * this graph and K by timing `sweeps` FP64 sweeps of prdf_pagerank_ppr with
 * teleport S (double [n, K] device). best_tile: host output; pass it as
 * prdf_params.tile.
 */
int prdf_autotune_tile(prdf_graph* g, const double* S, int K, const prdf_params* p, int sweeps, int* best_tile);

/* ------------------------------------------------------ K columns ------ */

/*
 * Weighted personalised PageRank for K teleport columns at once (extension of
 * Eq. 1 and Alg. static): R[:, c] = alpha * P^T R[:, c] + (1 - alpha) * S[:, c]
 * with P_uv = w_uv / sum_k w_uk (the graph must have been created with
 * weights). S, R: double [n, K] row-major device arrays in vertex-id order;
 * the iteration starts from R = S.
 * p->precision = PRDF_FP32_REFINE: FP32 sweeps with compensated products and
 * sums until max|dR| <= tol_fp32_rel * max|R|, then iterative refinement: an
 * FP64 Jacobi step gives the residual, an FP32 solve the correction, until
 * the L-inf change of an FP64 Jacobi step is <= tol (the returned R is that
 * step's result). p->precision = PRDF_FP64: FP64 Jacobi sweeps until the
 * L-inf change is <= tol. p->tile: columns handled per index fetch.
 * stats->iterations counts FP64 steps plus FP32 sweeps (iterations_fp32).
 * Returns PRDF_ESTATE for an unweighted graph, PRDF_EINVAL for K < 1.
 */
int prdf_pagerank_ppr(prdf_graph* g, const double* S, int K, double* R, const prdf_params* p, prdf_stats* stats);

/*
 * Replace the edge weights: w is float32[m] in the slot order of the out-CSR
 * (prdf_graph_export_csr(PRDF_OUT)), every weight finite and > 0 (else
 * PRDF_EINVAL). Makes an unweighted graph weighted.
 */
int prdf_graph_set_weights(prdf_graph* g, const float* w, void* stream);

/*
 * Adjoint of prdf_pagerank_ppr for the loss L = sum_c G[:, c] . R[:, c]
 * (extension; gradients of the fixed point R = alpha P^T R + (1 - alpha) S):
 *   lambda solves lambda = alpha P lambda + G, a pull over the out-edges of G
 *   (the transposed fixed point; same solver and precision options as the
 *   forward call);
 *   grad_S = (1 - alpha) lambda                          (double [n, K]);
 *   grad_w[j] for out-slot j = (u, v):
 *     (1 / W_u) sum_c R[u, c] (alpha lambda[v, c] - lambda[u, c] + G[u, c]),
 *     W_u = sum_k w_uk                                   (double [m]).
 * R: the forward result (double [n, K], needed for grad_w); G: dL/dR
 * (double [n, K]); grad_S, grad_w may be NULL. Device arrays, vertex-id order.
 */
int prdf_pagerank_backward(prdf_graph* g, const double* R, const double* G, int K, double* grad_S, double* grad_w,
                           const prdf_params* p, prdf_stats* stats);

#ifdef __cplusplus
}
#endif
#endif /* PRDF_H */
