// trim_scc.cu -- kernels of the SCC decomposition that trimming feeds
// (Section 1: FW-BW with trimming, as in ISPAN): size-2 SCC trimming and the
// steps of a colour-partitioned forward-backward search. The host driver is
// trim_run_scc in trim_api.cu; size-1 SCCs come from in+out trimming.
//
// State: comp[v] = the smallest vertex id of v's component once known, else
// SCC_OPEN. A step works on every open vertex at once: its forward part labels
// each open vertex with the smallest open vertex that reaches it (label
// propagation along G, i.e. forward searches from every vertex at once, each
// vertex keeping the smallest source); a vertex r whose label is r itself is
// reached by no smaller open vertex, and the backward search from r inside
// label r (through G^T) collects exactly r's component: every member reaches r
// and is reached from r, so it carries label r, and r, reached by no smaller
// vertex, is its smallest member. Each step closes at least the component of
// the smallest open vertex, and disconnected parts of the graph (separate
// graphs of a batch) progress together.
#include "trim_internal.cuh"

using namespace trimk;

namespace {
constexpr uint32_t SCC_OPEN = 0xFFFFFFFFu;
constexpr uint32_t NONE = 0xFFFFFFFFu;
__device__ __forceinline__ uint32_t gtid() { return blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ uint32_t gsize() { return gridDim.x * blockDim.x; }
}  // namespace

// After in+out trimming: removed vertices are size-1 components; the others
// are open, all in partition 0.
__global__ void scc_init_kernel(const uint32_t* level, uint32_t n, uint32_t* comp, uint32_t* color) {
  for (uint32_t v = gtid(); v < n; v += gsize()) {
    const bool open = level[v] == LIVE;
    comp[v] = open ? SCC_OPEN : v;
    color[v] = 0u;
  }
}

// Warp-collective row probe: for the lanes with want, counts (up to cap) the
// entries of row [s, s+d) whose vertex is open, skipping `self`, and returns
// the first such vertex (NONE if none). Rows of up to 32 entries are probed by
// their own lane; longer ones by the whole warp, 32 entries per step, stopping
// once cap open entries are seen.
__device__ __forceinline__ uint32_t probe_row(const uint32_t* rowtgt, uint32_t s, uint32_t d,
                                              bool want, uint32_t self, const uint32_t* comp,
                                              uint32_t cap, uint32_t& count) {
  const unsigned lane = lane_id();
  uint32_t first = NONE;
  count = 0;
  const bool own = want && d <= 32u;
  for (uint32_t k = 0; own && k < d && count < cap; ++k) {
    const uint32_t w = rowtgt[s + k];
    if (w != self && ldcg(&comp[w]) == SCC_OPEN) {
      if (first == NONE) first = w;
      ++count;
    }
  }
  unsigned big = __ballot_sync(0xFFFFFFFFu, want && d > 32u);
  while (big) {
    const int j = __ffs(big) - 1;
    big &= big - 1u;
    const uint32_t sj = __shfl_sync(0xFFFFFFFFu, s, j), dj = __shfl_sync(0xFFFFFFFFu, d, j);
    const uint32_t self_j = __shfl_sync(0xFFFFFFFFu, self, j);
    uint32_t cnt = 0, fst = NONE;
    for (uint32_t k0 = 0; k0 < dj && cnt < cap; k0 += 32u) {  // warp-uniform
      const uint32_t k = k0 + lane;
      bool hit = false;
      uint32_t w = 0;
      if (k < dj) {
        w = rowtgt[sj + k];
        hit = w != self_j && ldcg(&comp[w]) == SCC_OPEN;
      }
      const unsigned hm = __ballot_sync(0xFFFFFFFFu, hit);
      if (hm && fst == NONE) fst = __shfl_sync(0xFFFFFFFFu, w, __ffs(hm) - 1);
      cnt += __popc(hm);
    }
    if ((int)lane == j) {
      first = fst;
      count = min(cnt, cap);
    }
  }
  return first;
}

// Size-2 trimming, pass 1: for every open vertex, its only open successor
// other than itself (out1) and its only open predecessor other than itself
// (in1), counting parallel edges separately, or NONE when there is none or
// more than one. A self-loop makes v a component of its own, so such a vertex
// is never paired (NONE).
__global__ void scc_trim2_single_kernel(const uint32_t* off, const uint32_t* tgt,
                                        const uint32_t* ioff, const uint32_t* itgt, uint32_t n,
                                        const uint32_t* comp, uint32_t* out1, uint32_t* in1) {
  for (uint32_t w0 = gtid() & ~31u; w0 < n; w0 += gsize()) {  // warp-uniform
    const uint32_t v = w0 + lane_id();
    const bool open = v < n && comp[v] == SCC_OPEN;
    const uint32_t s = open ? off[v] : 0u, d = open ? off[v + 1] - s : 0u;
    const uint32_t is = open ? ioff[v] : 0u, id = open ? ioff[v + 1] - is : 0u;
    uint32_t oc = 0, ic = 0, lc = 0;
    // a self-loop: counted as the one "open entry equal to v" of its row
    const uint32_t o = probe_row(tgt, s, d, open, v, comp, 2u, oc);
    const uint32_t i = probe_row(itgt, is, id, open, v, comp, 2u, ic);
    const uint32_t all_out = probe_row(tgt, s, d, open, NONE, comp, 3u, lc);
    const bool loop = open && lc > oc;  // more open entries with v itself than without
    (void)all_out;
    if (v < n) {
      out1[v] = (open && !loop && oc == 1u) ? o : NONE;
      in1[v] = (open && !loop && ic == 1u) ? i : NONE;
    }
  }
}

// Size-2 trimming, pass 2: v and u = out1[v] with out1[u] = v are each other's
// only open successors, so {u, v} is a component (a closed 2-cycle); the same
// with predecessors. Both members write the same label. Counts the pairs.
__global__ void scc_trim2_pair_kernel(uint32_t n, const uint32_t* out1, const uint32_t* in1,
                                      uint32_t* comp, unsigned long long* pairs) {
  unsigned long long k = 0;
  for (uint32_t v = gtid(); v < n; v += gsize()) {
    const uint32_t o = out1[v], i = in1[v];
    uint32_t u = NONE;
    if (o != NONE && out1[o] == v) u = o;
    else if (i != NONE && in1[i] == v) u = i;
    if (u != NONE) {
      comp[v] = min(u, v);
      k += (v < u) ? 1u : 0u;
    }
  }
  k = warp_sum(k);
  if (lane_id() == 0 && k) atomicAdd(pairs, k);
}

// One trimming pass: an open vertex without an open successor, or without an
// open predecessor, is a component of its own (its other neighbours are in
// components already complete, so no cycle through it remains). Counts what
// it removed (0: nothing left to trim).
__global__ void scc_trim1_kernel(const uint32_t* off, const uint32_t* tgt, const uint32_t* ioff,
                                 const uint32_t* itgt, uint32_t n, uint32_t* comp,
                                 unsigned long long* removed) {
  unsigned long long k = 0;
  for (uint32_t w0 = gtid() & ~31u; w0 < n; w0 += gsize()) {  // warp-uniform
    const uint32_t v = w0 + lane_id();
    const bool open = v < n && ldcg(&comp[v]) == SCC_OPEN;
    const uint32_t s = open ? off[v] : 0u, d = open ? off[v + 1] - s : 0u;
    uint32_t oc = 0, ic = 0;
    probe_row(tgt, s, d, open, NONE, comp, 1u, oc);
    const bool need_in = open && oc > 0u;
    const uint32_t is = need_in ? ioff[v] : 0u, id = need_in ? ioff[v + 1] - is : 0u;
    probe_row(itgt, is, id, need_in, NONE, comp, 1u, ic);
    if (open && (oc == 0u || ic == 0u)) {
      comp[v] = v;
      ++k;
    }
  }
  k = warp_sum(k);
  if (lane_id() == 0 && k) atomicAdd(removed, k);
}

// Labels: every open vertex starts with its own id and joins the first frontier.
__global__ void scc_label_start_kernel(uint32_t n, const uint32_t* comp, uint32_t* label,
                                       uint32_t* frontier, uint32_t* count,
                                       unsigned long long* open) {
  unsigned long long k = 0;
  for (uint32_t w0 = gtid() & ~31u; w0 < n; w0 += gsize()) {  // warp-uniform
    const uint32_t v = w0 + lane_id();
    const bool o = v < n && comp[v] == SCC_OPEN;
    if (v < n) label[v] = o ? v : NONE;
    const unsigned bm = __ballot_sync(0xFFFFFFFFu, o);
    if (!bm) continue;
    uint32_t at = 0;
    if (lane_id() == (unsigned)(__ffs(bm) - 1)) at = atomicAdd(count, (uint32_t)__popc(bm));
    at = __shfl_sync(0xFFFFFFFFu, at, __ffs(bm) - 1);
    if (o) frontier[at + __popc(bm & ((1u << lane_id()) - 1u))] = v;
    k += o ? 1u : 0u;
  }
  k = warp_sum(k);
  if (lane_id() == 0 && k) atomicAdd(open, k);
}

// One level of label propagation along G: every frontier vertex offers its
// label to its open successors; a successor whose label drops joins the next
// frontier (once per level: inq holds the level's stamp).
__global__ void scc_label_level_kernel(const uint32_t* off, const uint32_t* tgt,
                                       const uint32_t* comp, uint32_t* label, uint32_t* inq,
                                       uint32_t stamp, const uint32_t* frontier, uint32_t count,
                                       uint32_t* next, uint32_t* next_count) {
  const uint32_t lane = lane_id();
  const uint32_t warps = gsize() >> 5;
  for (uint32_t i = gtid() >> 5; i < count; i += warps) {
    const uint32_t u = frontier[i];
    const uint32_t lu = ldcg(&label[u]);
    const uint32_t s = off[u], e = off[u + 1];
    for (uint32_t k0 = s; k0 < e; k0 += 32u) {
      const uint32_t k = k0 + lane;
      bool take = false;
      uint32_t w = 0;
      if (k < e) {
        w = tgt[k];
        if (comp[w] == SCC_OPEN && ldcg(&label[w]) > lu && atomicMin(&label[w], lu) > lu)
          take = atomicExch(&inq[w], stamp) != stamp;
      }
      const unsigned bm = __ballot_sync(0xFFFFFFFFu, take);
      if (!bm) continue;
      uint32_t at = 0;
      if (lane == 0) at = atomicAdd(next_count, (uint32_t)__popc(bm));
      at = __shfl_sync(0xFFFFFFFFu, at, 0);
      if (take) next[at + __popc(bm & ((1u << lane) - 1u))] = w;
    }
  }
}

// Roots: open vertices that kept their own label start the backward searches.
__global__ void scc_roots_start_kernel(uint32_t n, const uint32_t* comp, const uint32_t* label,
                                       uint32_t* mark, uint32_t stamp, uint32_t* frontier,
                                       uint32_t* count) {
  for (uint32_t w0 = gtid() & ~31u; w0 < n; w0 += gsize()) {  // warp-uniform
    const uint32_t v = w0 + lane_id();
    const bool root = v < n && comp[v] == SCC_OPEN && label[v] == v;
    const unsigned bm = __ballot_sync(0xFFFFFFFFu, root);
    if (!bm) continue;
    uint32_t at = 0;
    if (lane_id() == (unsigned)(__ffs(bm) - 1)) at = atomicAdd(count, (uint32_t)__popc(bm));
    at = __shfl_sync(0xFFFFFFFFu, at, __ffs(bm) - 1);
    if (root) {
      mark[v] = stamp;
      frontier[at + __popc(bm & ((1u << lane_id()) - 1u))] = v;
    }
  }
}

// One level of the backward searches (through G^T): each warp takes frontier
// vertices, its lanes walk the row; an open neighbour with the same label not
// yet marked with this stamp is marked (the atomic exchange that sees an older
// stamp wins) and joins the next frontier.
__global__ void scc_search_level_kernel(const uint32_t* rowoff, const uint32_t* rowtgt,
                                        const uint32_t* comp, const uint32_t* color,
                                        uint32_t* mark, uint32_t stamp, const uint32_t* frontier,
                                        uint32_t count, uint32_t* next, uint32_t* next_count) {
  const uint32_t lane = lane_id();
  const uint32_t warps = gsize() >> 5;
  for (uint32_t i = gtid() >> 5; i < count; i += warps) {
    const uint32_t u = frontier[i];
    const uint32_t c = color[u];
    const uint32_t s = rowoff[u], e = rowoff[u + 1];
    for (uint32_t k0 = s; k0 < e; k0 += 32u) {
      const uint32_t k = k0 + lane;
      bool take = false;
      uint32_t w = 0;
      if (k < e) {
        w = rowtgt[k];
        take = comp[w] == SCC_OPEN && color[w] == c && ldcg(&mark[w]) != stamp &&
               atomicExch(&mark[w], stamp) != stamp;
      }
      const unsigned bm = __ballot_sync(0xFFFFFFFFu, take);
      if (!bm) continue;
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(next_count, (uint32_t)__popc(bm));
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if (take) next[base + __popc(bm & ((1u << lane) - 1u))] = w;
    }
  }
}

// Close: every open vertex the backward search from its label's root reached
// belongs to that root's component. Counts the vertices placed.
__global__ void scc_close_kernel(uint32_t n, uint32_t* comp, const uint32_t* label,
                                 const uint32_t* mark, uint32_t stamp,
                                 unsigned long long* placed) {
  unsigned long long k = 0;
  for (uint32_t v = gtid(); v < n; v += gsize()) {
    if (comp[v] == SCC_OPEN && mark[v] == stamp) {
      comp[v] = label[v];
      ++k;
    }
  }
  k = warp_sum(k);
  if (lane_id() == 0 && k) atomicAdd(placed, k);
}

// Number of components: vertices that label their own component.
__global__ void scc_count_kernel(uint32_t n, const uint32_t* comp, unsigned long long* count) {
  unsigned long long k = 0;
  for (uint32_t v = gtid(); v < n; v += gsize()) k += comp[v] == v ? 1u : 0u;
  k = warp_sum(k);
  if (lane_id() == 0 && k) atomicAdd(count, k);
}
