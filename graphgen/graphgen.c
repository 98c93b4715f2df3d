/*
 * graphgen.c -- seeded synthetic directed graphs in CSR form.
 *
 * This module only draws graphs. It holds no trimming arithmetic: it never
 * looks at degrees-to-zero, frontiers or levels. Both the CPU oracle and the
 * CUDA trimming path take their inputs from here.
 *
 * Randomness: every random word is a pure function of (seed, stream, index),
 * the "SplitMix64" mixing function of Steele, Lea & Flood (OOPSLA 2014) used
 * as a counter-based generator:
 *     mix64(z): z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
 *               z *= 0x94D049BB133111EB; z ^= z>>31
 *     key      = mix64(seed ^ mix64(stream + GAMMA))
 *     word(i)  = mix64(key + (i+1) * GAMMA),  GAMMA = 0x9E3779B97F4A7C15
 * so generation order (threads, chunking) never changes the graph.
 * A uniform integer in [0,k) is Lemire's multiply-shift: floor(word * k / 2^64)
 * (no rejection; bias <= k / 2^64).
 *
 * Graph shapes follow the workloads of Guo & Sekerinski, "Efficient Parallel
 * Graph Trimming by Arc-Consistency" (Section 9, Table 10): R-MAT graphs with
 * skewed degrees, graphs with a large trimmable share and deep peeling depth.
 *
 * All rows of the produced CSR are sorted ascending with duplicates removed.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA 0x9E3779B97F4A7C15ull

static inline uint64_t mix64(uint64_t z) {
  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27; z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(seed ^ mix64(stream + GAMMA));
}
static inline uint64_t word_at(uint64_t key, uint64_t i) {
  return mix64(key + (i + 1) * GAMMA);
}
static inline uint64_t below(uint64_t w, uint64_t k) { /* uniform in [0,k) */
  return (uint64_t)(((unsigned __int128)w * k) >> 64);
}

uint64_t gg_word(uint64_t seed, uint64_t stream, uint64_t i) {
  return word_at(stream_key(seed, stream), i);
}

/* ---------- bijections (pseudo-random permutations) ---------- */

/* A bijection on [0, 2^k): rounds of (multiply by odd) (xor-shift) (add);
 * the round constants are words 0..7 of the key's stream. */
typedef struct { uint64_t a[4], c[4], mask; int s; } perm_consts;
static inline void perm_setup(perm_consts* P, int k, uint64_t pkey) {
  P->mask = (k >= 64) ? ~0ull : ((1ull << k) - 1);
  P->s = (k + 1) / 2 > 0 ? (k + 1) / 2 : 1;
  for (int r = 0; r < 4; ++r) {
    P->a[r] = word_at(pkey, 2 * r) | 1ull;
    P->c[r] = word_at(pkey, 2 * r + 1);
  }
}
static inline uint64_t perm_apply(const perm_consts* P, uint64_t x) {
  for (int r = 0; r < 4; ++r) {
    x = (x * P->a[r]) & P->mask;
    x ^= x >> P->s;
    x = (x + P->c[r]) & P->mask;
  }
  return x;
}
static inline uint64_t perm_pow2(uint64_t x, int k, uint64_t pkey) {
  perm_consts P;
  perm_setup(&P, k, pkey);
  return perm_apply(&P, x);
}
static int ceil_log2(uint64_t n) { int k = 0; while ((1ull << k) < n) ++k; return k; }
/* Bijection on [0,n) by cycle-walking the power-of-two bijection. */
static inline uint64_t perm_n(uint64_t x, uint64_t n, int k, uint64_t pkey) {
  perm_consts P;
  perm_setup(&P, k, pkey);
  do { x = perm_apply(&P, x); } while (x >= n);
  return x;
}

uint32_t gg_perm(uint64_t seed, uint64_t salt, uint32_t n, uint32_t x) {
  if (n <= 1) return 0;
  return (uint32_t)perm_n(x, n, ceil_log2(n), stream_key(seed, salt));
}

/* ---------- row sort + dedup ---------- */

static int cmp_u32(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return (x > y) - (x < y);
}
/* sorts row[0..len) ascending, removes duplicates, returns the new length */
static uint32_t sort_unique(uint32_t* row, uint32_t len) {
  if (len <= 1) return len;
  if (len <= 32) {
    for (uint32_t i = 1; i < len; ++i) {
      uint32_t x = row[i]; int64_t j = (int64_t)i - 1;
      while (j >= 0 && row[j] > x) { row[j + 1] = row[j]; --j; }
      row[j + 1] = x;
    }
  } else {
    qsort(row, len, sizeof(uint32_t), cmp_u32);
  }
  uint32_t w = 1;
  for (uint32_t i = 1; i < len; ++i) if (row[i] != row[w - 1]) row[w++] = row[i];
  return w;
}

/* Compacts rows that live at cap_off[v].. with lengths len[v] into off/tgt
 * (tgt may alias the row storage: compaction moves data only leftwards). */
static uint64_t compact_rows(uint32_t n, const uint64_t* cap_off, const uint32_t* len,
                             uint32_t* tgt, uint32_t* off) {
  uint64_t pos = 0;
  for (uint32_t v = 0; v < n; ++v) {
    off[v] = (uint32_t)pos;
    if (pos != cap_off[v]) memmove(tgt + pos, tgt + cap_off[v], (size_t)len[v] * 4);
    pos += len[v];
  }
  off[n] = (uint32_t)pos;
  return pos;
}

/* ---------- planted-trim graphs ---------- */

/* Layout of a planted graph (ids relative to the block):
 *   C = [0,nC)              core: each vertex draws k in [c_kmin,c_kmax] targets in C
 *   R = [nC, nC+nR)          reaching set: k in [r_kmin,r_kmax]; the first target is
 *                            uniform in C, the rest uniform in R u C
 *   T = [nC+nR, n)           trimmable set, ranked 0..nT-1 by id
 *     rank mode (n_chains==0): rank < t_sinks has no out-edge; every other rank
 *                            draws k in [t_kmin,t_kmax] targets among lower ranks
 *     chain mode (n_chains>0): rank = pos*n_chains + chain; pos 0 has no out-edge;
 *                            pos>=1 has one edge to (pos-1, same chain) plus
 *                            k in [t_kmin,t_kmax] extra targets uniform over ranks
 *                            at strictly lower positions.
 * Self-loops in C are allowed; duplicates are removed. */
typedef struct {
  uint32_t nC, nR, nT;
  uint32_t c_kmin, c_kmax;
  uint32_t r_kmin, r_kmax;
  uint32_t t_sinks;
  uint32_t t_kmin, t_kmax;
  uint32_t n_chains;
} gg_planted_params;

static inline uint32_t draw_k(uint64_t key, uint32_t kmin, uint32_t kmax) {
  return kmin + (uint32_t)below(word_at(key, 0), (uint64_t)kmax - kmin + 1);
}

/* number of raw draws (before dedup) of vertex v; 0 for sinks */
static inline uint32_t planted_k(const gg_planted_params* p, uint64_t key, uint32_t v) {
  const uint32_t nCR = p->nC + p->nR;
  if (v < p->nC) return draw_k(key, p->c_kmin, p->c_kmax);
  if (v < nCR) return draw_k(key, p->r_kmin, p->r_kmax);
  uint32_t rank = v - nCR;
  if (p->n_chains == 0) {
    if (rank < p->t_sinks) return 0;
    return draw_k(key, p->t_kmin, p->t_kmax);
  }
  if (rank < p->n_chains) return 0;             /* position 0 */
  return 1 + draw_k(key, p->t_kmin, p->t_kmax);
}

static inline uint32_t planted_target(const gg_planted_params* p, uint64_t key, uint32_t v,
                                      uint32_t j) {
  const uint32_t nCR = p->nC + p->nR;
  uint64_t w = word_at(key, 1 + j);
  if (v < p->nC) return (uint32_t)below(w, p->nC);
  if (v < nCR) return (uint32_t)(j == 0 ? below(w, p->nC) : below(w, nCR));
  uint32_t rank = v - nCR;
  if (p->n_chains == 0) return nCR + (uint32_t)below(w, rank);
  uint32_t pos = rank / p->n_chains;
  if (j == 0) return nCR + rank - p->n_chains;  /* predecessor in the chain */
  return nCR + (uint32_t)below(w, (uint64_t)pos * p->n_chains);
}

/* Returns m. off must hold n+1 entries, tgt must hold gg_planted_maxm() entries.
 * Vertex v uses stream (salt + v), so distinct salts give independent blocks. */
uint64_t gg_planted_maxm(uint64_t seed, uint64_t salt, const gg_planted_params* p) {
  const uint32_t n = p->nC + p->nR + p->nT;
  uint64_t total = 0;
  #pragma omp parallel for schedule(static) reduction(+ : total)
  for (int64_t v = 0; v < (int64_t)n; ++v)
    total += planted_k(p, stream_key(seed, salt + (uint64_t)v), (uint32_t)v);
  return total;
}

uint64_t gg_planted(uint64_t seed, uint64_t salt, const gg_planted_params* p,
                    uint32_t* off, uint32_t* tgt) {
  const uint32_t n = p->nC + p->nR + p->nT;
  uint64_t* cap = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
  uint32_t* len = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
  if (!cap || !len) { free(cap); free(len); return UINT64_MAX; }
  #pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < (int64_t)n; ++v)
    len[v] = planted_k(p, stream_key(seed, salt + (uint64_t)v), (uint32_t)v);
  uint64_t acc = 0;
  for (uint32_t v = 0; v < n; ++v) { cap[v] = acc; acc += len[v]; }
  cap[n] = acc;
  #pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < (int64_t)n; ++v) {
    uint64_t key = stream_key(seed, salt + (uint64_t)v);
    uint32_t* row = tgt + cap[v];
    for (uint32_t j = 0; j < len[v]; ++j) row[j] = planted_target(p, key, (uint32_t)v, j);
    len[v] = sort_unique(row, len[v]);
  }
  uint64_t m = compact_rows(n, cap, len, tgt, off);
  free(cap); free(len);
  return m;
}

/* ---------- R-MAT ---------- */

/* Chakrabarti, Zhan & Faloutsos, "R-MAT" (SDM 2004): each draw descends `scale`
 * levels of the adjacency matrix choosing quadrant a (0,0), b (0,1), c (1,0) or
 * d (1,1); probabilities are quantised to 1/65536. Ids are then mapped through a
 * pseudo-random bijection of [0, 2^scale), self-loops dropped, duplicates
 * removed, and the out-edges of exactly floor(sink_frac * n) vertices (chosen by
 * a second bijection) are deleted. */
typedef struct {
  int scale;
  uint64_t ndraws;
  double a, b, c;
  double sink_frac;
} gg_rmat_params;

static inline void rmat_draw(uint64_t key, int scale, uint32_t ta, uint32_t tab, uint32_t tabc,
                             uint32_t* s, uint32_t* d) {
  uint32_t src = 0, dst = 0;
  uint64_t w = 0;
  for (int l = 0; l < scale; ++l) {
    if ((l & 3) == 0) w = word_at(key, (uint64_t)(l >> 2));
    uint32_t u = (uint32_t)(w & 0xFFFF); w >>= 16;
    uint32_t sb, db;
    if (u < ta) { sb = 0; db = 0; }
    else if (u < tab) { sb = 0; db = 1; }
    else if (u < tabc) { sb = 1; db = 0; }
    else { sb = 1; db = 1; }
    src = (src << 1) | sb; dst = (dst << 1) | db;
  }
  *s = src; *d = dst;
}

typedef struct {
  uint64_t seed, pkey, skey;
  perm_consts pid, psink;
  int scale;
  uint32_t n, nsinks, ta, tab, tabc;
} rmat_ctx;

static void rmat_setup(uint64_t seed, const gg_rmat_params* p, rmat_ctx* c) {
  c->seed = seed; c->scale = p->scale; c->n = 1u << p->scale;
  c->pkey = stream_key(seed, 0xA11CEull);
  c->skey = stream_key(seed, 0x5111Cull);
  perm_setup(&c->pid, p->scale, c->pkey);
  perm_setup(&c->psink, p->scale, c->skey);
  c->nsinks = (uint32_t)(p->sink_frac * (double)c->n);
  c->ta = (uint32_t)(p->a * 65536.0 + 0.5);
  c->tab = (uint32_t)((p->a + p->b) * 65536.0 + 0.5);
  c->tabc = (uint32_t)((p->a + p->b + p->c) * 65536.0 + 0.5);
}
/* 1 if draw i yields a kept edge (s,d) */
static inline int rmat_edge(const rmat_ctx* c, uint64_t i, uint32_t* s, uint32_t* d) {
  uint32_t s0, d0;
  rmat_draw(stream_key(c->seed, (1ull << 62) + i), c->scale, c->ta, c->tab, c->tabc, &s0, &d0);
  uint32_t s1 = (uint32_t)perm_apply(&c->pid, s0);
  uint32_t d1 = (uint32_t)perm_apply(&c->pid, d0);
  if (s1 == d1) return 0;
  if (perm_apply(&c->psink, s1) < c->nsinks) return 0;
  *s = s1; *d = d1;
  return 1;
}

/* Returns m; off holds n+1 = 2^scale+1 entries, tgt holds ndraws entries. */
uint64_t gg_rmat(uint64_t seed, const gg_rmat_params* p, uint32_t* off, uint32_t* tgt) {
  rmat_ctx c; rmat_setup(seed, p, &c);
  const uint32_t n = c.n;
  uint64_t* cap = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
  uint32_t* len = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
  if (!cap || !len) { free(cap); free(len); return UINT64_MAX; }
  /* pass 1: count kept draws per source */
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)p->ndraws; ++i) {
    uint32_t s, d;
    if (rmat_edge(&c, (uint64_t)i, &s, &d)) {
      #pragma omp atomic
      len[s]++;
    }
  }
  uint64_t acc = 0;
  for (uint32_t v = 0; v < n; ++v) { cap[v] = acc; acc += len[v]; len[v] = 0; }
  cap[n] = acc;
  /* pass 2: scatter (order inside a row does not matter: rows are sorted next) */
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)p->ndraws; ++i) {
    uint32_t s, d;
    if (rmat_edge(&c, (uint64_t)i, &s, &d)) {
      uint32_t slot;
      #pragma omp atomic capture
      slot = len[s]++;
      tgt[cap[s] + slot] = d;
    }
  }
  #pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < (int64_t)n; ++v) len[v] = sort_unique(tgt + cap[v], len[v]);
  uint64_t m = compact_rows(n, cap, len, tgt, off);
  free(cap); free(len);
  return m;
}

/* ---------- Erdos-Renyi G(n, m) ---------- */

/* m_draws uniform ordered pairs (u,v), u != v, duplicates removed (so m is
 * m_draws minus the few collisions), as SNAP's random-graph generator used for
 * the ER workload of Table 10. Returns m; tgt holds m_draws entries. */
uint64_t gg_er(uint64_t seed, uint32_t n, uint64_t m_draws, uint32_t* off, uint32_t* tgt) {
  uint64_t* cap = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
  uint32_t* len = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
  if (!cap || !len || n < 2) { free(cap); free(len); return UINT64_MAX; }
  const uint64_t key = stream_key(seed, 0xE7ull);
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)m_draws; ++i) {
    uint64_t w = word_at(key, (uint64_t)i);
    uint32_t s = (uint32_t)below(w, n);
    #pragma omp atomic
    len[s]++;
  }
  uint64_t acc = 0;
  for (uint32_t v = 0; v < n; ++v) { cap[v] = acc; acc += len[v]; len[v] = 0; }
  cap[n] = acc;
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)m_draws; ++i) {
    uint64_t w = word_at(key, (uint64_t)i);
    uint32_t s = (uint32_t)below(w, n);
    /* target uniform over the n-1 vertices other than s */
    uint32_t d = (uint32_t)below(word_at(key ^ 0x5DEECE66Dull, (uint64_t)i), (uint64_t)n - 1);
    if (d >= s) d++;
    uint32_t slot;
    #pragma omp atomic capture
    slot = len[s]++;
    tgt[cap[s] + slot] = d;
  }
  #pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < (int64_t)n; ++v) len[v] = sort_unique(tgt + cap[v], len[v]);
  uint64_t m = compact_rows(n, cap, len, tgt, off);
  free(cap); free(len);
  return m;
}

/* ---------- relabelling ---------- */

/* new id of old vertex v is perm(v); writes the relabelled CSR to (off2,tgt2)
 * with rows sorted. perm must be a bijection on [0,n). */
void gg_relabel(uint32_t n, const uint32_t* off, const uint32_t* tgt, const uint32_t* perm,
                uint32_t* off2, uint32_t* tgt2) {
  uint32_t* inv = (uint32_t*)malloc((size_t)n * 4);
  for (uint32_t v = 0; v < n; ++v) inv[perm[v]] = v;
  uint64_t pos = 0;
  for (uint32_t nv = 0; nv < n; ++nv) {
    uint32_t v = inv[nv];
    off2[nv] = (uint32_t)pos;
    for (uint32_t e = off[v]; e < off[v + 1]; ++e) tgt2[pos++] = perm[tgt[e]];
  }
  off2[n] = (uint32_t)pos;
  #pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < (int64_t)n; ++v)
    sort_unique(tgt2 + off2[v], off2[v + 1] - off2[v]);
  free(inv);
}

/* ---------- transposed graph (input preparation) ---------- */

/* sorts row[0..len) ascending, keeping duplicates */
static void sort_row(uint32_t* row, uint32_t len) {
  if (len <= 32) {
    for (uint32_t i = 1; i < len; ++i) {
      uint32_t x = row[i]; int64_t j = (int64_t)i - 1;
      while (j >= 0 && row[j] > x) { row[j + 1] = row[j]; --j; }
      row[j + 1] = x;
    }
  } else {
    qsort(row, len, sizeof(uint32_t), cmp_u32);
  }
}

/* G^T of a CSR graph: off_in[v]..off_in[v+1] lists the sources of the edges into
 * v, in ascending order (a parallel counting sort by target, then each row
 * sorted, so the result does not depend on the thread count). Parallel edges
 * appear once per copy. Returns 0, -1 if a target is >= n, -2 without memory. */
int gg_transpose(uint32_t n, const uint32_t* off, const uint32_t* tgt, uint32_t* off_in,
                 uint32_t* tgt_in) {
  const uint64_t m = off[n];
  uint32_t* fill = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
  if (!fill) return -2;
  int bad = 0;
  #pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t e = 0; e < (int64_t)m; ++e) {
    const uint32_t t = tgt[e];
    if (t >= n) { bad = 1; continue; }
    #pragma omp atomic
    fill[t]++;
  }
  if (bad) { free(fill); return -1; }
  uint64_t acc = 0;
  for (uint32_t v = 0; v < n; ++v) { off_in[v] = (uint32_t)acc; acc += fill[v]; fill[v] = 0; }
  off_in[n] = (uint32_t)acc;
  #pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t u = 0; u < (int64_t)n; ++u)
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
      const uint32_t t = tgt[e];
      uint32_t slot;
      #pragma omp atomic capture
      slot = fill[t]++;
      tgt_in[off_in[t] + slot] = (uint32_t)u;
    }
  #pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < (int64_t)n; ++v) sort_row(tgt_in + off_in[v], off_in[v + 1] - off_in[v]);
  free(fill);
  return 0;
}

/* ---------- deterministic real helpers (no libm: identical on every host) ---------- */

/* e^x by range reduction x = k ln2 + r, |r| <= ln2/2, and a degree-16 Taylor
 * polynomial; compiled with -ffp-contract=off so every host rounds alike. */
double gg_exp(double x) {
  const double LN2 = 0.69314718055994530942;
  double kf = x / LN2;
  long k = (long)(kf < 0 ? kf - 0.5 : kf + 0.5);
  double r = x - (double)k * LN2;
  double term = 1.0, sum = 1.0;
  for (int i = 1; i <= 16; ++i) { term = term * r / (double)i; sum = sum + term; }
  double p = 1.0;
  if (k > 0) for (long i = 0; i < k; ++i) p = p * 2.0;
  else for (long i = 0; i < -k; ++i) p = p * 0.5;
  return sum * p;
}
/* uniform double in [0,1) with 53 random bits */
double gg_unit(uint64_t seed, uint64_t stream, uint64_t i) {
  return (double)(gg_word(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}
/* Standard normal approximated by the Irwin-Hall sum of 12 uniforms minus 6. */
double gg_normal12(uint64_t seed, uint64_t stream) {
  double s = 0.0;
  for (int i = 0; i < 12; ++i) s = s + gg_unit(seed, stream, (uint64_t)i);
  return s - 6.0;
}
