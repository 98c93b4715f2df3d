/*
 * oracle.c -- the CPU oracle for graph trimming (TEST INFRASTRUCTURE ONLY).
 *
 * Plain, sequential, obviously-correct C written from Guo & Sekerinski,
 * "Efficient Parallel Graph Trimming by Arc-Consistency" (arXiv 2107.12720).
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file; the product path never does. It shares no
 * code with the CUDA path.
 *
 * Result definition (Definition 1, Definition 2 of the paper):
 *   status[v] = 1 (LIVE) iff v belongs to the maximal subgraph in which every
 *   vertex keeps at least one out-edge; otherwise 0 (DEAD).
 *   level[v]  = the peeling step in which the synchronous process of
 *   Definition 2 removes v, counted from 0 (a vertex without out-edges has
 *   level 0; otherwise 1 + the largest level among its successors), and
 *   0xFFFFFFFF for LIVE vertices.
 *
 * Functions:
 *   or_transpose   G -> G^T (Section 2, "transposed graph")
 *   or_peel        O1: sequential AC-4-based trimming (Algorithm 5) run one
 *                  peeling step at a time so that each removal carries its step
 *   or_ac6         O2: sequential AC-6-based trimming (Algorithm 7) with the
 *                  edge_index jump of Section 8, then levels in removal order
 *   or_ac3         O3: AC-3-based trimming (Algorithm 4) with one snapshot per
 *                  repetition (every repetition reads the previous one's status)
 *   or_certificate local conditions that hold for exactly one assignment
 *   or_peel_inout  in+out trimming (the in-degree check of Section 4's remark on
 *                  AC-3 with G^T loaded): removal on no live successor OR no
 *                  live predecessor, one peeling step at a time
 *   or_certificate_inout  its local conditions (exactly one assignment)
 *   or_peel_masked vertex-sampled inputs (Section 9, scalability experiment):
 *                  unsampled vertices are DEAD from the start
 *   or_scc         strongly connected components (Section 1: the decomposition
 *                  trimming feeds), Tarjan's algorithm, labelled canonically
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LIVE 0xFFFFFFFFu

/* G^T: off_in[v]..off_in[v+1] lists the predecessors of v, in increasing
 * source order (a counting sort by target). Returns 0, or -1 on bad input. */
int or_transpose(uint32_t n, const uint32_t* off, const uint32_t* tgt,
                 uint32_t* off_in, uint32_t* tgt_in) {
  uint64_t m = off[n];
  memset(off_in, 0, ((size_t)n + 1) * sizeof(uint32_t));
  for (uint64_t e = 0; e < m; ++e) {
    if (tgt[e] >= n) return -1;
    off_in[tgt[e] + 1]++;
  }
  for (uint32_t v = 0; v < n; ++v) off_in[v + 1] += off_in[v];
  uint32_t* fill = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
  if (!fill) return -2;
  memcpy(fill, off_in, ((size_t)n + 1) * sizeof(uint32_t));
  for (uint32_t u = 0; u < n; ++u)
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) tgt_in[fill[tgt[e]]++] = u;
  free(fill);
  return 0;
}

/* O1. Algorithm 5 (sequential AC-4-based trimming): counters deg_out(v) start at
 * |v.post| (taken as the CSR offset difference, the "AC4Trim*" reading of
 * Section 9.3), and every removed vertex w decrements the counter of each
 * predecessor v' in w(G^T).post (one decrement per parallel edge). Here the
 * waiting set is processed one peeling step at a time: `cur` holds the vertices
 * removed in step r-1, `nxt` collects those whose counter reaches zero while
 * `cur` is propagated; they are removed in step r. Returns alpha (the number of
 * peeling steps, 0 if nothing is removed). */
uint32_t or_peel(uint32_t n, const uint32_t* off, const uint32_t* off_in, const uint32_t* tgt_in,
                 uint32_t* level, uint8_t* status) {
  uint32_t* cnt = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* cur = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* nxt = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t ncur = 0, alpha = 0;
  for (uint32_t v = 0; v < n; ++v) {
    cnt[v] = off[v + 1] - off[v];
    level[v] = LIVE;
    if (cnt[v] == 0) { level[v] = 0; cur[ncur++] = v; }
  }
  for (uint32_t r = 1; ncur > 0; ++r) {
    alpha = r;
    uint32_t nnxt = 0;
    for (uint32_t i = 0; i < ncur; ++i) {
      uint32_t w = cur[i];
      for (uint32_t e = off_in[w]; e < off_in[w + 1]; ++e) {
        uint32_t u = tgt_in[e];
        cnt[u] -= 1;
        if (cnt[u] == 0) { level[u] = r; nxt[nnxt++] = u; }
      }
    }
    uint32_t* t = cur; cur = nxt; nxt = t; ncur = nnxt;
  }
  for (uint32_t v = 0; v < n; ++v) status[v] = (level[v] == LIVE);
  free(cnt); free(cur); free(nxt);
  return alpha;
}

/* O2. Algorithm 7 (sequential AC-6-based trimming). Each vertex v keeps one
 * support: the first LIVE successor found by scanning v.post from its
 * edge_index; v is recorded in that successor's supporting set S (Definition 3,
 * an intrusive list s_head/s_next here). When a vertex w is removed, every
 * member of w.S resumes its scan after the edge it had chosen; a member whose
 * scan runs off the end is removed and queued in turn. Each edge is inspected
 * at most once (Section 8, "Traverse Edges"); *edges_scanned returns that count.
 * Levels follow in removal order, which lists every removed vertex after all of
 * its successors (a vertex is removed only once its successors are removed):
 * level = 0 without out-edges, else 1 + max over successors. Returns alpha. */
uint32_t or_ac6(uint32_t n, const uint32_t* off, const uint32_t* tgt, uint32_t* level,
                uint8_t* status, uint64_t* edges_scanned) {
  const uint32_t NIL = LIVE;
  uint8_t* dead = (uint8_t*)calloc((size_t)n + 1, 1);
  uint32_t* edge_index = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* s_head = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* s_next = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* queue = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* order = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t qh = 0, qt = 0, nord = 0;
  uint64_t scanned = 0;
  for (uint32_t v = 0; v < n; ++v) { edge_index[v] = off[v]; s_head[v] = NIL; }
  for (uint32_t v0 = 0; v0 < n; ++v0) {
    uint32_t pending = v0;  /* DoPost(v0), then propagate the waiting set */
    for (;;) {
      if (pending != NIL) {
        uint32_t v = pending;
        int found = 0;
        while (edge_index[v] < off[v + 1]) {
          uint32_t w = tgt[edge_index[v]++];
          scanned++;
          if (!dead[w]) { s_next[v] = s_head[w]; s_head[w] = v; found = 1; break; }
        }
        if (!found) { dead[v] = 1; queue[qt++] = v; order[nord++] = v; }
        pending = NIL;
      }
      if (qh == qt) break;
      uint32_t w = queue[qh];
      if (s_head[w] == NIL) { qh++; continue; }
      pending = s_head[w];          /* remove one member v' from w.S ... */
      s_head[w] = s_next[pending];  /* ... and DoPost(v') on the next pass */
    }
  }
  for (uint32_t v = 0; v < n; ++v) level[v] = LIVE;
  uint32_t alpha = 0;
  for (uint32_t i = 0; i < nord; ++i) {
    uint32_t v = order[i], lv = 0;
    for (uint32_t e = off[v]; e < off[v + 1]; ++e) {
      uint32_t lw = level[tgt[e]];
      if (lw + 1 > lv) lv = lw + 1;
    }
    level[v] = lv;
    if (lv + 1 > alpha) alpha = lv + 1;
  }
  for (uint32_t v = 0; v < n; ++v) status[v] = !dead[v];
  if (edges_scanned) *edges_scanned = scanned;
  free(dead); free(edge_index); free(s_head); free(s_next); free(queue); free(order);
  return alpha;
}

/* O3. Algorithm 4 (AC-3-based trimming): repeat a sweep over all LIVE vertices,
 * removing each one for which ZeroOutDegree holds (no LIVE successor), until a
 * sweep changes nothing. Every sweep r reads the status left by sweep r-1 and
 * vertices removed in sweep r get level r. Returns alpha (= the number of
 * sweeps that removed something). */
uint32_t or_ac3(uint32_t n, const uint32_t* off, const uint32_t* tgt, uint32_t* level,
                uint8_t* status) {
  uint8_t* live = (uint8_t*)malloc((size_t)n + 1);
  uint8_t* live_next = (uint8_t*)malloc((size_t)n + 1);
  for (uint32_t v = 0; v < n; ++v) { live[v] = 1; level[v] = LIVE; }
  uint32_t r = 0;
  for (;;) {
    int change = 0;
    memcpy(live_next, live, n);
    for (uint32_t v = 0; v < n; ++v) {
      if (!live[v]) continue;
      int zero_out = 1;
      for (uint32_t e = off[v]; e < off[v + 1]; ++e)
        if (live[tgt[e]]) { zero_out = 0; break; }
      if (zero_out) { live_next[v] = 0; level[v] = r; change = 1; }
    }
    uint8_t* t = live; live = live_next; live_next = t;
    if (!change) break;
    ++r;
  }
  for (uint32_t v = 0; v < n; ++v) status[v] = live[v];
  free(live); free(live_next);
  return r;
}

/* Certificate check. Conditions:
 *  (i)  every LIVE v (status 1, level LIVE) has a LIVE successor;
 *  (ii) every DEAD v has only DEAD successors and level[v] = 0 if it has no
 *       out-edge, else 1 + max level over its successors;
 *  (iii) status and level agree (status 1 <=> level == LIVE).
 * (ii) makes levels strictly decrease along edges between DEAD vertices, so no
 * DEAD vertex reaches a cycle; (i) gives every LIVE vertex an infinite walk,
 * hence a cycle: the LIVE set is exactly the vertices that reach a cycle (the
 * maximal subgraph of Definition 1) and the levels are the Definition 2 steps.
 * Returns -1 if all hold, else the first violating vertex. */
int64_t or_certificate(uint32_t n, const uint32_t* off, const uint32_t* tgt,
                       const uint32_t* level, const uint8_t* status) {
  for (uint32_t v = 0; v < n; ++v) {
    int is_live = status[v] != 0;
    if (is_live != (level[v] == LIVE)) return v;
    if (is_live) {
      int ok = 0;
      for (uint32_t e = off[v]; e < off[v + 1]; ++e)
        if (level[tgt[e]] == LIVE) { ok = 1; break; }
      if (!ok) return v;
    } else {
      uint32_t want = 0;
      for (uint32_t e = off[v]; e < off[v + 1]; ++e) {
        uint32_t lw = level[tgt[e]];
        if (lw == LIVE) return v;
        if (lw + 1 > want) want = lw + 1;
      }
      if (level[v] != want) return v;
    }
  }
  return -1;
}

/* In+out trimming. Section 4 remarks that with G^T in memory each vertex must
 * also keep at least one available incoming edge, which trims more size-1 SCCs
 * (the form FW-BW and ISPAN use, Section 1). The process is Definition 2's with
 * both conditions: step 0 removes every vertex without out-edges or without
 * in-edges; step r removes every vertex still present with no successor or no
 * predecessor among the vertices present after step r-1. Here, as in or_peel,
 * two counters per vertex count its successors and predecessors still present;
 * every vertex removed in step r-1 decrements the out-counter of each
 * predecessor and the in-counter of each successor (once per parallel edge),
 * and a present vertex whose counter reaches zero is removed in step r.
 * Returns alpha (the number of steps that removed something). */
uint32_t or_peel_inout(uint32_t n, const uint32_t* off, const uint32_t* tgt,
                       const uint32_t* off_in, const uint32_t* tgt_in, uint32_t* level,
                       uint8_t* status) {
  uint32_t* cnt_out = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* cnt_in = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* cur = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* nxt = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t ncur = 0, alpha = 0;
  for (uint32_t v = 0; v < n; ++v) {
    cnt_out[v] = off[v + 1] - off[v];
    cnt_in[v] = off_in[v + 1] - off_in[v];
    level[v] = LIVE;
    if (cnt_out[v] == 0 || cnt_in[v] == 0) { level[v] = 0; cur[ncur++] = v; }
  }
  for (uint32_t r = 1; ncur > 0; ++r) {
    alpha = r;
    uint32_t nnxt = 0;
    for (uint32_t i = 0; i < ncur; ++i) {
      uint32_t w = cur[i];
      for (uint32_t e = off_in[w]; e < off_in[w + 1]; ++e) {  /* w's predecessors */
        uint32_t u = tgt_in[e];
        if (level[u] != LIVE) continue;
        cnt_out[u] -= 1;
        if (cnt_out[u] == 0) { level[u] = r; nxt[nnxt++] = u; }
      }
      for (uint32_t e = off[w]; e < off[w + 1]; ++e) {  /* w's successors */
        uint32_t s = tgt[e];
        if (level[s] != LIVE) continue;
        cnt_in[s] -= 1;
        if (cnt_in[s] == 0) { level[s] = r; nxt[nnxt++] = s; }
      }
    }
    uint32_t* t = cur; cur = nxt; nxt = t; ncur = nnxt;
  }
  for (uint32_t v = 0; v < n; ++v) status[v] = (level[v] == LIVE);
  free(cnt_out); free(cnt_in); free(cur); free(nxt);
  return alpha;
}

/* Certificate of in+out trimming. With t_out(v) = 0 if v has no successor, else
 * 1 + the largest successor level if every successor is DEAD, else infinity;
 * and t_in(v) the same over predecessors:
 *  (i)  every LIVE v has a LIVE successor and a LIVE predecessor;
 *  (ii) every DEAD v has level[v] = min(t_out(v), t_in(v)) (finite);
 *  (iii) status and level agree.
 * (i) makes the LIVE set a subgraph in which every vertex keeps an in- and an
 * out-edge; by (ii), induction on the level shows that no DEAD vertex belongs
 * to such a subgraph and that the vertices of each level are exactly those the
 * process removes in that step. Returns -1 if all hold, else the first
 * violating vertex. */
int64_t or_certificate_inout(uint32_t n, const uint32_t* off, const uint32_t* tgt,
                             const uint32_t* off_in, const uint32_t* tgt_in,
                             const uint32_t* level, const uint8_t* status) {
  const uint64_t INF = 0xFFFFFFFFFFull;
  for (uint32_t v = 0; v < n; ++v) {
    int is_live = status[v] != 0;
    if (is_live != (level[v] == LIVE)) return v;
    int live_succ = 0, live_pred = 0;
    uint64_t t_out = 0, t_in = 0;
    for (uint32_t e = off[v]; e < off[v + 1]; ++e) {
      uint32_t lw = level[tgt[e]];
      if (lw == LIVE) live_succ = 1;
      else if ((uint64_t)lw + 1 > t_out) t_out = (uint64_t)lw + 1;
    }
    for (uint32_t e = off_in[v]; e < off_in[v + 1]; ++e) {
      uint32_t lu = level[tgt_in[e]];
      if (lu == LIVE) live_pred = 1;
      else if ((uint64_t)lu + 1 > t_in) t_in = (uint64_t)lu + 1;
    }
    if (live_succ) t_out = INF;
    if (live_pred) t_in = INF;
    if (is_live) {
      if (!live_succ || !live_pred) return v;
    } else {
      uint64_t want = t_out < t_in ? t_out : t_in;
      if (want == INF || level[v] != want) return v;
    }
  }
  return -1;
}

/* Vertex-sampled inputs. Section 9's scalability experiment samples vertices by
 * setting the unsampled ones DEAD before trimming (and notes that AC-4 still
 * computes their out-degree counters). Here mask[v] != 0 marks an unsampled
 * vertex: it is DEAD from the start and gets level MASKED = 0xFFFFFFFE; it is
 * not removed by any step and not counted in alpha. As in or_peel, counters
 * start at |v.post|; the unsampled vertices first decrement the counter of each
 * of their predecessors (they are dead before step 0), then step 0 removes
 * every sampled vertex whose counter is zero, and the layer-synchronous
 * peeling goes on from there. Returns alpha. */
uint32_t or_peel_masked(uint32_t n, const uint32_t* off, const uint32_t* off_in,
                        const uint32_t* tgt_in, const uint8_t* mask, uint32_t* level,
                        uint8_t* status) {
  const uint32_t MASKED = 0xFFFFFFFEu;
  uint32_t* cnt = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* cur = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* nxt = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t ncur = 0, alpha = 0;
  for (uint32_t v = 0; v < n; ++v) {
    cnt[v] = off[v + 1] - off[v];
    level[v] = mask[v] ? MASKED : LIVE;
  }
  for (uint32_t w = 0; w < n; ++w) {  /* the unsampled vertices are dead before step 0 */
    if (!mask[w]) continue;
    for (uint32_t e = off_in[w]; e < off_in[w + 1]; ++e) cnt[tgt_in[e]] -= 1;
  }
  for (uint32_t v = 0; v < n; ++v)
    if (!mask[v] && cnt[v] == 0) { level[v] = 0; cur[ncur++] = v; }
  for (uint32_t r = 1; ncur > 0; ++r) {
    alpha = r;
    uint32_t nnxt = 0;
    for (uint32_t i = 0; i < ncur; ++i) {
      uint32_t w = cur[i];
      for (uint32_t e = off_in[w]; e < off_in[w + 1]; ++e) {
        uint32_t u = tgt_in[e];
        if (mask[u]) continue;
        cnt[u] -= 1;
        if (cnt[u] == 0) { level[u] = r; nxt[nnxt++] = u; }
      }
    }
    uint32_t* t = cur; cur = nxt; nxt = t; ncur = nnxt;
  }
  for (uint32_t v = 0; v < n; ++v) status[v] = (level[v] == LIVE);
  free(cnt); free(cur); free(nxt);
  return alpha;
}

/* Strongly connected components (Section 1: FW-BW with trimming computes this
 * decomposition; size-1 SCCs are the trimmable vertices). Tarjan's algorithm
 * (one depth-first search; a vertex whose lowlink equals its own index roots a
 * component made of the vertices above it on the component stack), written
 * with an explicit call stack. comp[v] receives the smallest vertex id of v's
 * component, which labels every decomposition the same way. Returns the number
 * of components, or UINT32_MAX without memory. */
uint32_t or_scc(uint32_t n, const uint32_t* off, const uint32_t* tgt, uint32_t* comp) {
  const uint32_t NONE = 0xFFFFFFFFu;
  uint32_t* index = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint32_t* low = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4);
  uint8_t* on_stack = (uint8_t*)calloc((size_t)n + 1, 1);
  uint32_t* cstack = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4); /* component stack */
  uint32_t* call_v = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4); /* DFS call stack */
  uint32_t* call_e = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 4); /* next edge */
  if (!index || !low || !on_stack || !cstack || !call_v || !call_e) {
    free(index); free(low); free(on_stack); free(cstack); free(call_v); free(call_e);
    return 0xFFFFFFFFu;
  }
  for (uint32_t v = 0; v < n; ++v) index[v] = NONE;
  uint32_t next_index = 0, csp = 0, ncomp = 0;
  for (uint32_t root = 0; root < n; ++root) {
    if (index[root] != NONE) continue;
    uint32_t depth = 0;
    call_v[0] = root; call_e[0] = off[root];
    index[root] = low[root] = next_index++;
    cstack[csp++] = root; on_stack[root] = 1;
    while (1) {
      uint32_t v = call_v[depth];
      if (call_e[depth] < off[v + 1]) {          /* visit the next successor */
        uint32_t w = tgt[call_e[depth]++];
        if (index[w] == NONE) {
          index[w] = low[w] = next_index++;
          cstack[csp++] = w; on_stack[w] = 1;
          ++depth; call_v[depth] = w; call_e[depth] = off[w];
        } else if (on_stack[w] && index[w] < low[v]) {
          low[v] = index[w];
        }
        continue;
      }
      if (low[v] == index[v]) {                   /* v roots a component */
        uint32_t start = csp, lo = v;
        do { start--; if (cstack[start] < lo) lo = cstack[start]; } while (cstack[start] != v);
        for (uint32_t i = start; i < csp; ++i) { comp[cstack[i]] = lo; on_stack[cstack[i]] = 0; }
        csp = start;
        ncomp++;
      }
      if (depth == 0) break;                      /* return to the caller */
      --depth;
      uint32_t u = call_v[depth];
      if (low[v] < low[u]) low[u] = low[v];
    }
  }
  free(index); free(low); free(on_stack); free(cstack); free(call_v); free(call_e);
  return ncomp;
}
