/*
 * Seeded synthetic inputs for the Static / DF-P PageRank workloads.
 *
 * This module only draws inputs: graphs, batch updates, personalisation
 * vectors and loss weights. It holds none of the PageRank arithmetic and is
 * shared, unchanged, by the CPU oracle tests and by the GPU tests / benchmark.
 *
 * Random numbers come from SplitMix64 used as a counter-based generator: the
 * k-th output (k = 0, 1, ...) of the stream with initial state `key` is
 * mix(key + (k + 1) * GOLDEN), where GOLDEN = 0x9E3779B97F4A7C15 and mix() is
 * SplitMix64's output function (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014). Stream keys are derived from
 * (seed, s1, s2, s3) by chaining the same mix. Because every draw is a pure
 * function of its counter, the OpenMP loops below give identical output for
 * any thread count.
 *
 * Workload shapes follow Section 5.1 of the paper (batch generation: 80/20
 * insertions/deletions, insertions are uniform vertex pairs, deletions are
 * uniformly chosen existing edges, no new vertices) with R-MAT and grid graphs
 * standing in for the web/social and road-network graphs of its datasets.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t synth_key(uint64_t seed, uint64_t s1, uint64_t s2, uint64_t s3) {
  uint64_t k = sm64_mix(seed + GOLDEN);
  k = sm64_mix(k + (s1 + 1) * GOLDEN);
  k = sm64_mix(k + (s2 + 1) * GOLDEN);
  k = sm64_mix(k + (s3 + 1) * GOLDEN);
  return k;
}

/* k-th draw (0-based) of the stream with initial state key. */
static inline uint64_t draw(uint64_t key, uint64_t k) { return sm64_mix(key + (k + 1) * GOLDEN); }

uint64_t synth_draw(uint64_t key, uint64_t k) { return draw(key, k); }

/* Uniform integer in [0, bound) from a 64-bit draw (multiply-high). */
static inline uint64_t below(uint64_t r, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/*
 * R-MAT edge sampler (Chakrabarti, Zhan, Faloutsos, SDM 2004). Edge i draws
 * ceil(scale/2) 64-bit numbers; each supplies two 32-bit uniforms (low half
 * first), one per recursion level, most significant bit first. A uniform u
 * selects quadrant a (no bit), b (target bit), c (source bit) or d (both) by
 * comparison with the integer thresholds floor(a*2^32), floor((a+b)*2^32),
 * floor((a+b+c)*2^32).
 */
void synth_rmat(int scale, int64_t nedges, double a, double b, double c, uint64_t seed,
                int32_t* src, int32_t* dst) {
  const uint64_t key = synth_key(seed, 0x524d4154ULL /* "RMAT" */, (uint64_t)scale, 0);
  const uint64_t ta = (uint64_t)floor(a * 4294967296.0);
  const uint64_t tb = (uint64_t)floor((a + b) * 4294967296.0);
  const uint64_t tc = (uint64_t)floor((a + b + c) * 4294967296.0);
  const int per_edge = (scale + 1) / 2;
#pragma omp parallel for schedule(static, 65536)
  for (int64_t i = 0; i < nedges; ++i) {
    uint32_t u = 0, v = 0;
    for (int l = 0; l < scale; ++l) {
      uint64_t r = draw(key, (uint64_t)i * per_edge + (uint64_t)(l >> 1));
      uint64_t x = (l & 1) ? (r >> 32) : (r & 0xFFFFFFFFULL);
      uint32_t sb = 0, db = 0;
      if (x < ta) { }
      else if (x < tb) { db = 1; }
      else if (x < tc) { sb = 1; }
      else { sb = 1; db = 1; }
      u = (u << 1) | sb;
      v = (v << 1) | db;
    }
    src[i] = (int32_t)u;
    dst[i] = (int32_t)v;
  }
}

/*
 * side x side 4-neighbour grid, both directions, each directed edge kept with
 * probability 1 - p_drop. Vertex (r, c) has id r*side + c. Directed edges are
 * enumerated per source vertex in the order up, down, left, right; edge slot
 * 4*id + dir uses draw number 4*id + dir. Returns the number of kept edges;
 * src/dst must hold 4*side*side entries.
 */
int64_t synth_grid(int side, double p_drop, uint64_t seed, int32_t* src, int32_t* dst) {
  const uint64_t key = synth_key(seed, 0x47524944ULL /* "GRID" */, (uint64_t)side, 0);
  const double keep_lim = (1.0 - p_drop) * 18446744073709551616.0;
  const uint64_t keep = keep_lim >= 18446744073709551615.0 ? UINT64_MAX : (uint64_t)keep_lim;
  int64_t m = 0;
  const int dr[4] = {-1, 1, 0, 0}, dc[4] = {0, 0, -1, 1};
  for (int r = 0; r < side; ++r)
    for (int c = 0; c < side; ++c) {
      int64_t id = (int64_t)r * side + c;
      for (int d = 0; d < 4; ++d) {
        int rr = r + dr[d], cc = c + dc[d];
        if (rr < 0 || rr >= side || cc < 0 || cc >= side) continue;
        uint64_t x = draw(key, (uint64_t)id * 4 + d);
        if (x < keep) {
          src[m] = (int32_t)id;
          dst[m] = (int32_t)((int64_t)rr * side + cc);
          ++m;
        }
      }
    }
  return m;
}

/*
 * Random batch update on the graph whose out-CSR is (off, adj):
 * n_del deletions drawn without replacement from the existing edges that are
 * not self-loops (uniform over edge slots, rejection of self-loops and of
 * slots already drawn), and n_ins insertions of uniform vertex pairs
 * (u, v) in [0, n)^2 (Section 5.1, batch generation). The deletion stream is
 * key(seed, s1, s2, 1) and the insertion stream key(seed, s1, s2, 2).
 * Returns the number of deletions actually drawn (fewer than n_del only if
 * the graph has fewer non-self-loop edges).
 */
int64_t synth_batch(int32_t n, const int64_t* off, const int32_t* adj, int64_t n_del, int64_t n_ins,
                    uint64_t seed, uint64_t s1, uint64_t s2,
                    int32_t* del_src, int32_t* del_dst, int32_t* ins_src, int32_t* ins_dst) {
  const int64_t m = off[n];
  int64_t nonself = 0;
  for (int32_t u = 0; u < n; ++u)
    for (int64_t j = off[u]; j < off[u + 1]; ++j) nonself += (adj[j] != u);
  if (n_del > nonself) n_del = nonself;
  const uint64_t kd = synth_key(seed, s1, s2, 1), ki = synth_key(seed, s1, s2, 2);
  uint8_t* taken = (uint8_t*)calloc((size_t)(m + 7) / 8 + 1, 1);
  int64_t got = 0;
  uint64_t k = 0;
  while (got < n_del) {
    int64_t j = (int64_t)below(draw(kd, k++), (uint64_t)m);
    if (taken[j >> 3] & (1u << (j & 7))) continue;
    /* row of slot j: last u with off[u] <= j */
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
      int32_t mid = lo + (hi - lo + 1) / 2;
      if (off[mid] <= j) lo = mid; else hi = mid - 1;
    }
    if (adj[j] == lo) continue;
    taken[j >> 3] |= (uint8_t)(1u << (j & 7));
    del_src[got] = lo;
    del_dst[got] = adj[j];
    ++got;
  }
  free(taken);
#pragma omp parallel for schedule(static, 65536)
  for (int64_t i = 0; i < n_ins; ++i) {
    ins_src[i] = (int32_t)below(draw(ki, 2 * (uint64_t)i), (uint64_t)n);
    ins_dst[i] = (int32_t)below(draw(ki, 2 * (uint64_t)i + 1), (uint64_t)n);
  }
  return got;
}

/*
 * Edge weights uniform in [lo, hi), a pure function of (seed, u, v) so that
 * duplicate edges carry equal weights.
 */
void synth_edge_weights(int64_t m, const int32_t* src, const int32_t* dst, uint64_t seed,
                        double lo, double hi, float* w) {
  const uint64_t key = synth_key(seed, 0x57474854ULL /* "WGHT" */, 0, 0);
#pragma omp parallel for schedule(static, 65536)
  for (int64_t i = 0; i < m; ++i) {
    uint64_t pair = ((uint64_t)(uint32_t)src[i] << 32) | (uint32_t)dst[i];
    w[i] = (float)(lo + (hi - lo) * unit(draw(key, pair)));
  }
}

/*
 * K personalisation columns, row-major S[v*K + c]. Column c puts mass on
 * n_seed distinct uniform vertices with Dirichlet(1) weights, i.e. Exp(1)
 * variates -log(1 - U) normalised to sum 1 (in double, then stored). Column c
 * uses the stream key(seed, "PPRS", c).
 */
void synth_ppr_seeds(int32_t n, int K, int n_seed, uint64_t seed, double* S) {
  memset(S, 0, sizeof(double) * (size_t)n * K);
  int32_t* pick = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_seed);
  double* e = (double*)malloc(sizeof(double) * (size_t)n_seed);
  for (int c = 0; c < K; ++c) {
    const uint64_t key = synth_key(seed, 0x50505253ULL /* "PPRS" */, (uint64_t)c, 0);
    uint64_t k = 0;
    int got = 0;
    while (got < n_seed && got < n) {
      int32_t v = (int32_t)below(draw(key, k++), (uint64_t)n);
      int dup = 0;
      for (int j = 0; j < got; ++j) dup |= (pick[j] == v);
      if (!dup) pick[got++] = v;
    }
    double tot = 0;
    for (int j = 0; j < got; ++j) {
      e[j] = -log(1.0 - unit(draw(key, k++)));
      tot += e[j];
    }
    for (int j = 0; j < got; ++j) S[(size_t)pick[j] * K + c] = e[j] / tot;
  }
  free(pick);
  free(e);
}

/* Standard normal variates by Box-Muller on pairs of draws. */
void synth_normal(int64_t count, uint64_t seed, double* out) {
  const uint64_t key = synth_key(seed, 0x4e524d4cULL /* "NRML" */, 0, 0);
#pragma omp parallel for schedule(static, 65536)
  for (int64_t i = 0; i < count; ++i) {
    double u1 = 1.0 - unit(draw(key, 2 * (uint64_t)i));
    double u2 = unit(draw(key, 2 * (uint64_t)i + 1));
    out[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  }
}

/* Uniform doubles in [0, 1): used for random starting vectors in tests. */
void synth_uniform(int64_t count, uint64_t seed, double* out) {
  const uint64_t key = synth_key(seed, 0x554e4946ULL /* "UNIF" */, 0, 0);
#pragma omp parallel for schedule(static, 65536)
  for (int64_t i = 0; i < count; ++i) out[i] = unit(draw(key, (uint64_t)i));
}

/* Uniform int32 in [0, bound): used for random edge lists and flag patterns in tests. */
void synth_randint(int64_t count, int64_t bound, uint64_t seed, int32_t* out) {
  const uint64_t key = synth_key(seed, 0x52494e54ULL /* "RINT" */, 0, 0);
#pragma omp parallel for schedule(static, 65536)
  for (int64_t i = 0; i < count; ++i) out[i] = (int32_t)below(draw(key, (uint64_t)i), (uint64_t)bound);
}
