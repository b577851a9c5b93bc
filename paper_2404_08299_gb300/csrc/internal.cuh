// Internal declarations shared by the translation units of libprdf.
#pragma once

#include <vector>

#include "common.cuh"

namespace prdf {

constexpr int kMaxThr = 7;  // at most eight degree classes

struct PartThr {
  int n = 0;                    // number of thresholds (classes = n + 1)
  int64_t thr[kMaxThr] = {0, 0, 0, 0, 0, 0, 0};
};

// Scratch reused across calls on one graph. Calls on a graph do not overlap.
struct Workspace {
  DBuf<int64_t> scan;       // tile sums of the device-wide scan
  DBuf<int64_t> part_cnt;   // per-tile class counts of the partition
  DBuf<int64_t> part_base;  // their exclusive scan
  int64_t* host_i64 = nullptr;  // pinned host scratch, kHostSlots entries
  static constexpr int kHostSlots = 64;
  int init();
  ~Workspace();
};

// Exclusive prefix sums: out[i] = sum(in[0..i)), out[n] = total.
int exclusive_scan_u32(const uint32_t* in, int64_t n, int64_t* out, Workspace& ws, cudaStream_t s);
int exclusive_scan_i64(const int64_t* in, int64_t n, int64_t* out, Workspace& ws, cudaStream_t s);

// Alg. partition over the rows of a CSR (degree = off[v+1] - off[v]).
int partition_by_degree(const int64_t* off, int64_t n, const PartThr& t, int32_t* P, int64_t* counts_host,
                        Workspace& ws, cudaStream_t s);
// Stable partition of a list of vertex ids (in = NULL: 0..n-1) by the degree
// classes of off; desc puts the highest class first. P may not alias in.
int partition_list(const int64_t* off, const int32_t* in, int64_t n, const PartThr& t, bool desc, int32_t* P,
                   int64_t* counts_host, Workspace& ws, cudaStream_t s);

// A device CSR with optional float weights.
struct Csr {
  DBuf<int64_t> off;  // n + 1
  DBuf<int32_t> adj;  // m
  DBuf<float> w;      // m or empty
  int64_t m = 0;
};

// Build a CSR of unique{(rows[i], cols[i])} (plus one self-loop per row if
// self_loops), rows sorted ascending. Entries with a negative row or column
// are skipped when allow_skip is set, otherwise they are an error. Weights
// (optional) of merged duplicates: maximum; added self-loops: 1.0.
int build_csr(int32_t n, int64_t m0, const int32_t* rows, const int32_t* cols, const float* w, bool self_loops,
              bool allow_skip, Csr& out, Workspace& ws, cudaStream_t s);
// The same CSR by a radix sort of packed (row, column) keys (radix_build.cu):
// unweighted lists without skipped entries, m0 + n < 2^32; ids already checked.
bool radix_build_applies(int32_t n, int64_t m0, const float* w, bool allow_skip, bool self_loops);
int build_csr_radix(int32_t n, int64_t m0, const int32_t* rows, const int32_t* cols, bool self_loops, Csr& out,
                    Workspace& ws, cudaStream_t s);

// Batch update of one CSR with set semantics (Sec. 3.3): out gets rows
// (old \ D) u I in column order, merged without re-sorting (batch_update.cu).
// D: (del_rows[i], del_cols[i]), self-loops ignored; I: (ins_rows[i],
// ins_cols[i]) with weights ins_w when old is weighted (duplicates and
// re-inserted surviving edges keep the maximum). Equal to a rebuild when
// every row of old holds its own vertex. Keyed form (key, store not null):
// old's entries are ordered by key[entry], the batch's columns are keys, an
// added column c is stored as store[c], and a deletion (r, c) is a self-loop
// when key[r] == c.
int update_csr(int32_t n, const Csr& old, const int32_t* del_rows, const int32_t* del_cols, int64_t n_del,
               const int32_t* ins_rows, const int32_t* ins_cols, const float* ins_w, int64_t n_ins, Csr& out,
               Workspace& ws, cudaStream_t s, const int32_t* key = nullptr, const int32_t* store = nullptr);

// The graph renumbered so that each in-degree class is a contiguous id range
// (new id i = vertex perm[i], perm being the in-degree partition).
struct Relabel {
  bool valid = false;
  PartThr thr;                       // in-degree classes the numbering follows
  int64_t count[kMaxThr + 1] = {};   // class sizes; class c is ids [sum(count[<c]), +count[c])
  DBuf<int32_t> perm;                // new -> old
  DBuf<int32_t> inv;                 // old -> new
  Csr in, out;                       // G' and G in the new numbering
  DBuf<double> degd, inv_deg;        // |out(i)| and 1/|out(i)| in the new numbering
  DBuf<double> kf;                   // Eq. 2 factor 1 / (1 - alpha / |out(i)|) for kf_alpha
  double kf_alpha = -1;              // alpha kf was made for (< 0: none)
  DBuf<int32_t> pout;                // out-degree partition of `out` (new ids), for marking
  int64_t pout_count[kMaxThr + 1] = {};
  bool pout_valid = false;
  uint64_t version = 0;              // bumped on every rebuild and every batch update
  // Batch updates keep the numbering: in and out are updated in place (rows
  // stay ordered by original id), so a vertex's degree may leave its class
  // bounds. Every kernel handles rows of any length; the one exception is the
  // class of in-degree <= 1, whose kernel reads no row: a vertex of that class
  // that gains an in-edge gets its bit in multi (one bit per vertex, cleared by
  // the next renumbering) and takes the general path.
  DBuf<uint32_t> multi;
  int64_t multi_count = 0;           // vertices with their bit set
  int64_t drift = 0;                 // batch entries applied since the numbering was made
};

// Rows of the highest in-degree class are cut into chunks of kHubChunk edges
// (used by the K-column calls and by the Static sweep): chunk c covers edges
// [chunk_j0[c], +kHubChunk) of vertex begin + chunk_hub[c]; the chunks of
// hub i are [hub_first[i], hub_first[i + 1]) in row order.
constexpr int64_t kHubChunk = 1024;
struct PprHub {
  int64_t begin, nhub, nchunk;
  const int32_t* chunk_hub;
  const int64_t* chunk_j0;
  const int64_t* hub_first;
};
// Per-sweep arguments of the pull rank kernels (Alg. update).
struct SweepArgs {
  const int64_t* off;      // in-CSR offsets of G'
  const int32_t* adj;      // in-CSR sources
  const double* x;         // x[u] = R[u] / |out(u)| of the previous iteration
  double* xn;              // next x
  const double* degd;      // |out(v)| (self-loop included), as a double
  const double* inv_deg;   // 1 / |out(v)|
  const double* kf;        // DF-P: 1 / (1 - alpha / |out(v)|) (Eq. 2's self-loop factor)
  double alpha, c0;        // damping, (1 - alpha) / n
  int self_loops;          // every vertex has exactly one self-loop (graph built with PRDF_ADD_SELF_LOOPS)
  const uint32_t* multi;   // null, or a bit per vertex: set for the in-degree <= 1 classes' vertices that
                           // gained in-edges since the numbering was made (they read their row)
  uint64_t* resid;         // L-inf change of this sweep (bits of a non-negative double), atomic max
  const uint64_t* prev;    // L-inf change of the previous sweep, or null on the first sweep
  double tol;              // the sweep exits at once if *prev <= tol (already converged)
  // DF / DF-P only
  // device-driven iteration (CUDA graph): when ctl is set the kernel takes
  // x/xn/resid/prev for iteration it = ctl[0] from xa/xb/resid_base instead
  const int* ctl;
  const double* xa;
  double* xb;
  uint64_t* resid_base;
  uint8_t* dV;             // affected flags (read; cleared on prune)
  uint8_t* dN;             // expand flags (set when the change exceeds tau_f)
  uint8_t* wrote;          // 1 where this vertex's slot in xn was written by the previous sweep
  double tau_f, tau_p;
  int prune;               // DF-P (Eq. 2, prune) or DF (Eq. 1)
  unsigned long long* fw;  // null, or: += out-edges of the vertices this sweep puts into deltaN
  unsigned long long* fw_base;  // graph-driven loop: fw of iteration it is fw_base + it
  // Static: chunks of the highest in-degree class's rows (nchunk = 0: none)
  // and one partial sum per chunk (4 words)
  PprHub hub;
  uint4* hub_part;
};

// FP32 stage of the mixed-precision sweeps (sweep32.cu): Static (Eq. 1 on
// every vertex) or DF / DF-P (Eq. 1 / Eq. 2 on the affected vertices, with
// the prune and expand flags of Alg. update).
struct Sweep32Args {
  const int64_t* off;      // in-CSR offsets of G' (class-contiguous numbering)
  const int32_t* adj;      // in-CSR sources
  const float* y;          // y[u] = R[u] / |out(u)| in FP32
  float* yn;               // next y
  const float* degf;       // |out(v)| as float
  const float* invf;       // 1 / |out(v)| as float
  float alpha, c0;
  int self_loops;
  const uint32_t* multi;   // as in SweepArgs
  uint32_t* resid;         // [0]: max |r - R[v]|, [1]: max r of this sweep (FP32 bits, atomic max)
  const uint32_t* prev;    // previous sweep's pair, or null
  float tol_rel;           // the sweep exits at once if prev[0] <= tol_rel * prev[1]
  // device-driven iteration (CUDA graph): when ctl is set the kernel takes
  // y/yn/resid/prev for iteration it = ctl[0] from ya/yb/resid_base instead
  const int* ctl;
  const float* ya;
  float* yb;
  uint32_t* resid_base;
  // DF / DF-P only (same meaning as in SweepArgs)
  const float* kf;         // Eq. 2 factor 1 / (1 - alpha / |out(v)|) as float
  uint8_t* dV;
  uint8_t* dN;
  uint8_t* wrote;
  float tau_f, tau_p;
  int prune;
  unsigned long long* fw;       // as in SweepArgs
  unsigned long long* fw_base;
  // chunks of the highest in-degree class's rows (nchunk = 0: a block per row)
  // and one compensated partial sum (s, e) per chunk
  PprHub hub;
  float2* hub_part;
};
int launch_sweep32(const Sweep32Args& a, const PartThr& t, const int64_t* class_begin, bool dynamic, cudaStream_t s);
// One-thread check of the graph-driven FP32 loop: it = ctl[0]; stop when
// r32[2 it] <= tol_rel * r32[2 it + 1] or it + 1 >= max_iter; ctl[0] = it + 1.
int launch_iter_check32(int* ctl, const uint32_t* resid_base, float tol_rel, int max_iter,
                        cudaGraphConditionalHandle h, cudaStream_t s);

// K-column personalised PageRank (ppr.cu), row-major [n, K] in the class-contiguous numbering.
struct Ppr32Args {
  const int64_t* off;      // in-CSR of G'
  const int32_t* adj;
  const float* P;          // P_uv for the in-edge slot (u -> v)
  const float* R;          // current [n, K]
  float* Rn;               // next [n, K]
  const float* S;          // right-hand side [n, K] (teleport, or residual / (1 - alpha))
  const int32_t* srow;     // null: S is dense; else S holds compact rows and row v is S[srow[v]] (-1: zero)
  int K;
  float alpha, beta;       // alpha, 1 - alpha
  uint32_t* resid;         // [0] max |R_new - R|, [1] max |R_new| (FP32 bits, atomic max)
  const uint32_t* prev;    // previous sweep's pair or null
  float tol_rel;
  // device-driven iteration (CUDA graph): when ctl is set, iteration it = ctl[0]
  // reads R from Ra (even it) or Rb (odd it), writes the other, and uses the
  // pair resid_base + 2 it (previous: resid_base + 2 (it - 1))
  const int* ctl;
  const float* Ra;
  float* Rb;
  uint32_t* resid_base;
};
struct Ppr64Args {
  const int64_t* off;
  const int32_t* adj;
  const double* P;
  const double* R;
  double* Rn;              // T(R)
  const double* S;         // right-hand side, dense or compact rows as in Ppr32Args
  const int32_t* srow;
  float* res32;            // (T(R) - R) / (1 - alpha) in FP32, or null
  int K;
  double alpha, beta, inv_beta;
  uint64_t* dmax;          // max |T(R) - R| (FP64 bits, atomic max)
  // device-driven iteration (CUDA graph): when ctl is set, step it = ctl[0]
  // reads R from Ra (even it) or Rb (odd it), writes the other, and puts its
  // maximum in dmax_base + it
  const int* ctl;
  const double* Ra;
  double* Rb;
  uint64_t* dmax_base;
};

// Owner of a chunk table (PprHub above) of one CSR of the sweep numbering.
struct PprHubTable {
  int64_t begin = 0, nhub = 0, nchunk = 0;
  DBuf<int32_t> chunk_hub;
  DBuf<int64_t> chunk_j0, hub_first;
  uint64_t version = 0;  // numbering version it was built for
  bool valid = false;
  PprHub view() const { return PprHub{begin, nhub, nchunk, chunk_hub.p, chunk_j0.p, hub_first.p}; }
};
int build_ppr_hub(const int64_t* off, int64_t begin, int64_t n, PprHubTable& t, Workspace& ws, cudaStream_t s);

// FP32 sweep over tiles of `tile` columns: vertices [0, hub_begin) one per
// slot, [hub_begin, h.begin) a warp each, the hub rows in chunks (part:
// h.nchunk * tile float2 scratch).
int launch_ppr32_sweep(const Ppr32Args& a, int tile, int64_t n, int64_t hub_begin, const PprHub& h, float2* part,
                       cudaStream_t s);
// FP64 Jacobi step over tiles of `tile` columns, same ranges as the FP32
// sweep (part: h.nchunk * tile doubles of scratch).
int launch_ppr64_step(const Ppr64Args& a, int tile, int64_t n, int64_t hub_begin, const PprHub& h, double* part,
                      cudaStream_t s);
// Sparse teleport: the rows of S (double [n, K]) with a non-zero entry. When
// at most n / 4 rows are non-zero, srow[v] gets v's compact row (-1 for none),
// Sc64 / Sc32 the rows in FP64 / FP32, R32 (float [n, K]) the FP32 matrix
// (the iteration's start R = S) and rows their count; otherwise rows = 0 and
// the dense form is kept. Sweeps then read 4 bytes per vertex instead of the
// vertex's whole teleport row.
struct PprSparseRhs {
  int64_t rows = 0;
  DBuf<int32_t> srow;
  DBuf<double> Sc64;
  DBuf<float> Sc32;
};
int ppr_sparse_rhs(const double* S, int64_t n, int K, Workspace& ws, PprSparseRhs* out, float* R32, cudaStream_t s);
int ppr_add_correction(double* R, const float* E, int64_t cnt, cudaStream_t s);
int launch_grad_w(const int64_t* off, const int32_t* adj, const int32_t* perm, const int64_t* orig_off,
                  const double* lam, const double* Gs, double g_scale, const double* Rr, const double* W, int32_t n,
                  int K, double alpha, double* grad_w, cudaStream_t s);
int ppr_narrow(const double* x, int64_t cnt, float* y, cudaStream_t s);
int ppr_widen(const float* y, int64_t cnt, double* x, cudaStream_t s);

// One-thread iteration check of the graph-driven loop: it = ctl[0]; stop when
// resid[it] <= tol or it + 1 >= max_iter; ctl[0] = it + 1; sets the while condition.
int launch_iter_check(int* ctl, const uint64_t* resid_base, double tol, int max_iter,
                      cudaGraphConditionalHandle h, cudaStream_t s);

// Launch one rank sweep (all degree classes) for Static (dynamic = false) or DF/DF-P.
int launch_sweep(const SweepArgs& a, const PartThr& t, const int64_t* class_begin, bool exact, bool dynamic,
                 cudaStream_t s);

// Stop rule of the loop an expansion round belongs to, read on the device so
// that rounds launched after the converged sweep do nothing. FP64 loops:
// r64[it] <= tol; FP32 stage: r32[2 it] <= tol_rel * r32[2 it + 1]; neither
// set: the round always runs. it = ctl[0] in the graph-driven loop, else 0
// (r64 / r32 then point at this sweep's slot).
struct Stop {
  const uint64_t* r64 = nullptr;
  double tol = 0;
  const uint32_t* r32 = nullptr;
  float tol_rel = 0;
  const int* ctl = nullptr;
};

// Alg. affected kernels (frontier.cu). map (nullable): vertex id -> flag index.
int launch_initial_affected(const int32_t* del_src, const int32_t* del_dst, const uint8_t* del_mask, int64_t n_del,
                            const int32_t* ins_src, const uint8_t* ins_mask, int64_t n_ins, const int32_t* map,
                            uint8_t* dV, uint8_t* dN, cudaStream_t s);
// expandAffected over the out-degree partition; skipped on the device when the
// stop rule st holds, and when fw (nullable; this round's counter, indexed by
// st.ctl in the graph-driven loop) is given, also when *fw > fthr (the pull
// form runs instead). dF (nullable): also mark in dF every vertex that was not
// yet in dV (one round of Dynamic Traversal's reachability closure).
// fl (optional scratch): a frontier of at most fl.cap vertices is listed and
// expanded from the list, without the partition kernels' scan of every vertex.
struct FrontList {
  int32_t* list = nullptr;      // cap entries
  unsigned int* cnt = nullptr;  // one counter
  unsigned int cap = 0;
};
int launch_expand(const int64_t* off, const int32_t* adj, const int32_t* P, const int64_t* cb, int nclass,
                  const uint8_t* dN, uint8_t* dV, uint8_t* dF, const Stop& st, cudaStream_t s,
                  const unsigned long long* fw = nullptr, unsigned long long fthr = 0,
                  const FrontList& fl = FrontList());
// The same round in pull form over G' (in_off/in_adj; rows from warp_begin on
// take a warp each): marks only if *fw, the frontier's out-edges (counted by
// the sweep before it), exceeds fthr.
int launch_expand_pull(const int64_t* in_off, const int32_t* in_adj, int64_t n, int64_t warp_begin,
                       const uint8_t* dN, uint8_t* dV, const unsigned long long* fw, unsigned long long fthr,
                       const Stop& st, cudaStream_t s);
int count_flags(const uint8_t* f, int64_t n, unsigned long long* dev_out, cudaStream_t s);

}  // namespace prdf

// The graph handle of the C ABI.
struct prdf_graph {
  int32_t n = 0;
  bool weighted = false;
  bool self_loops = true;           // every vertex has exactly one self-loop
  cudaStream_t stream = nullptr;
  prdf::Csr csr[2];                  // [PRDF_OUT] = G, [PRDF_IN] = G' in original ids (see orig_valid)
  bool orig_valid = true;            // false after a batch update until ensure_orig()
  int64_t m = 0;                     // edges of G (self-loops included)
  prdf::PartThr thr[2];              // class thresholds per CSR
  prdf::DBuf<int32_t> P[2];          // partitions
  int64_t pcount[2][prdf::kMaxThr + 1] = {};
  bool pvalid[2] = {false, false};
  prdf::Workspace ws;
  // solver scratch
  prdf::DBuf<double> xa, xb;
  prdf::PprHubTable hub_in, hub_out;  // chunk tables of G' (Static sweep, K-column forward) and G (adjoint)
  prdf::DBuf<uint4> sweep_hub_part;   // FP64 sweeps: one exact partial sum per chunk of G's hub rows
  prdf::DBuf<float2> sweep_hub_part32;  // FP32 sweeps: one compensated partial sum per chunk
  prdf::DBuf<float2> ppr_part;        // chunk partial sums of one column tile (FP32 sweeps)
  prdf::DBuf<double> ppr_part64;      // chunk partial sums of one column tile (FP64 steps)
  prdf::DBuf<float> ya, yb, degf, invf;  // FP32 stage state and degrees (class-contiguous numbering)
  prdf::DBuf<float> kf32;                // FP32 stage of DF-P: Eq. 2 factor
  prdf::DBuf<uint32_t> resid32;
  prdf::DBuf<uint64_t> resid;
  prdf::DBuf<uint8_t> dV, dN, wrote;
  prdf::DBuf<uint8_t> dF;  // Dynamic Traversal: next frontier of the closure
  prdf::DBuf<unsigned long long> counter;
  prdf::DBuf<unsigned long long> chk;  // input checks: bad-id flag, bad-rank flag, rank sum (double bits)
  prdf::DBuf<unsigned long long> fwork;  // frontier out-edges of each expansion round
  prdf::DBuf<int32_t> flist;             // a small frontier listed for its expansion round (frontier.cu)
  prdf::DBuf<unsigned int> fcnt;         // its size
  prdf::DBuf<int> ctl;               // device iteration counter of the graph-driven loop
  cudaStream_t cap_stream = nullptr; // private stream used to capture graph bodies
  // instantiated loops (CUDA graphs), one per kind of loop, each with the
  // arguments and buffers it was captured for: sweep loops at fp32 * 4 +
  // dynamic * 2 + expand; K-column loops from 8 on
  cudaGraphExec_t loop_exec[16] = {};
  std::vector<uint64_t> loop_key[16];
  prdf::Relabel rl;                  // class-contiguous copy used by the sweeps
  // weighted graphs: transition probabilities P_uv = w_uv / sum_k w_uk
  bool ppr_valid = false;
  prdf::DBuf<double> wsum;           // sum of out-weights per vertex (sweep numbering)
  prdf::DBuf<double> pin64;          // P on the in-edge slots of rl.in
  prdf::DBuf<float> pin32;
  prdf::DBuf<double> pout64;         // P on the out-edge slots of rl.out (adjoint)
  prdf::DBuf<float> pout32;
  // K-column scratch
  prdf::DBuf<double> S64, R64a, R64b;
  prdf::PprSparseRhs ppr_rhs;        // compact teleport rows of the last forward call (rows = 0: dense)
  prdf::DBuf<float> S32, R32a, R32b;
};

namespace prdf {
int build_relabelled(prdf_graph* g, cudaStream_t s);
int build_ppr_weights(prdf_graph* g, cudaStream_t s);
// The CSRs of G and G' in original ids, derived from the sweep numbering's
// copies when a batch update has changed those (rows come out sorted, as the
// numbering keeps each row in original-id order).
int ensure_orig(prdf_graph* g, cudaStream_t s);
// |out(i)| and 1 / |out(i)| of the sweep numbering from its out-CSR (drops the cached Eq. 2 factor)
int update_degrees(prdf_graph* g, cudaStream_t s);
// the same, and the cached Eq. 2 factor, for the rows of the cnt vertices a[] (original ids) only
int update_degrees_of(prdf_graph* g, const int32_t* a, int64_t cnt, cudaStream_t s);
}
