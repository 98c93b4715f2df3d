// trim_kernels.cu -- the persistent round-synchronous trimming kernel.
//
// One cooperative launch runs every round of the trimming of Guo & Sekerinski
// (arXiv 2107.12720): round 0 removes the vertices without out-edges, round r
// the vertices whose successors were all removed in rounds < r (Definition 2).
// Each round runs one of three kernels, chosen per round:
//
//   AC-4 push   (Section 5, Algorithm 6): each removed vertex w decrements the
//               out-degree counter of every predecessor through G^T; the atomic
//               decrement that returns 1 removes the predecessor (it is unique,
//               so no CAS on the status is needed).
//   AC-6 support (Section 6, Algorithms 7/8, Definition 3): every live vertex
//               keeps one support (edge_index) and sits in that support's
//               supporting set S; when a support is removed, the members of its
//               S re-scan forward for the next live successor. Rounds replace the
//               paper's spin locks: a set is only read after the round in which
//               its owner was removed, and no vertex joins the S of a vertex
//               removed in an earlier round.
//   AC-3 pull   (Section 4, Algorithm 4 with the edge_index jump of Section 8):
//               a sweep over a compacted list of the vertices still live.
//
// All three read "u removed before round r" as level[u] < r, so mixing them
// round by round yields the same levels.
//
// Rounds end at a grid-wide barrier (a monotone arrival counter, bounded spin).
// No CTA hands anything to another between rounds: every CTA advances its own
// copy of the schedule state (Sched, in shared memory) from the same global
// inputs, so the copies agree. Appends to the dead log, the AC-4 work list and
// the AC-3 live list go to per-warp shared-memory slices and reach global
// memory with one atomic per counter per CTA per round.
//
// A scheduled run may span several launches (segments): at the start of a
// round every CTA can decide from the same state to stop (the kernel lacks the
// variant the scheduler chose); CTA 0 then saves the schedule state in the
// control block, and the next launch resumes from it at the same round. A
// scheduler that commits to its choice stays in the same kernel: the rounds
// of a committed stretch skip the scheduler and its features (and in the AC-4
// + schedulers flavour may run as local rounds).
#include "trim_internal.cuh"

// This file is compiled once per kernel flavour: TRIM_MODES is a bit set of the
// variants the kernel can run (1 AC-4, 2 AC-6, 4 AC-3) plus 8 for the
// per-round schedulers (features, heuristic, MLP, scripted lists), or 17 for
// in+out trimming. A fixed variant gets a kernel with only its own path,
// hence fewer registers.
#ifndef TRIM_MODES
#define TRIM_MODES 15
#endif
#define TRIM_CAT2(a, b) a##b
#define TRIM_CAT(a, b) TRIM_CAT2(a, b)
#ifdef TRIM_KERNEL_SUFFIX
#define TRIM_KERNEL TRIM_CAT(trim_persistent_kernel_m, TRIM_KERNEL_SUFFIX)
#else
#define TRIM_KERNEL TRIM_CAT(trim_persistent_kernel_m, TRIM_MODES)
#endif

using namespace trimk;

namespace {

constexpr int MODES = TRIM_MODES;
// In the all-variant flavour each round function keeps its own register
// allocation, so the heavier AC-6 code cannot push the AC-4 loop into spills.
#if TRIM_MODES == 15
#define ROUND_FN __noinline__
#else
#define ROUND_FN __forceinline__
#endif
constexpr int M_AC4 = 1, M_AC6 = 2, M_AC3 = 4, M_SCHED = 8;
// in+out trimming: AC-4 pushes on both G^T (out-degree counters) and G
// (in-degree counters); its own flavour, with no other variant
constexpr int M_INOUT = 16;
// implicit graph (Section 2.1, on-the-fly): successors computed, no CSR; with
// AC-6 (34) or AC-3 (36) only
constexpr int M_IMPLICIT = 32;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int MAX_WARPS = 16;   // blockDim.x <= 512
constexpr int WBUF = 64;        // per-warp staging of supporting-set members

// Work counters (TRIM_FLAG_STATS). Each round function keeps its own in
// registers and adds them to the global totals when it returns.
struct Counters {
  unsigned edges = 0, pushed = 0, cand = 0, swept = 0;  // one round: each at most m < 2^32
};

// Per-warp append slices. Each warp buffers what it removes (and, in AC-3
// rounds, what survives) in its own slice of shared memory; no shared atomics
// and no CTA-wide synchronisation inside the variant loops. A full slice is
// flushed by its warp alone; at the end of a round one CTA-wide flush moves
// all slices with one global atomic per counter.
constexpr uint32_t LW = 256;  // entries per warp slice (per buffer)
struct WarpSlice {
  uint32_t nlog, nw4, nedge, nlive;   // entries in the slices; edges of the w4 entries
  uint32_t ncount;                    // removals counted in the log but not written to it
  uint32_t log_base, w4_base, edge_base, live_base;  // global bases at the CTA flush
  uint32_t sum_in, sum_out;  // feature sums (distinct removed vertices: at most m < 2^32)
  uint32_t hist[3];
  uint32_t max_din;          // largest in-degree among this warp's work-list entries
};

// Local AC-4 rounds (the AC-4-only flavour, and the AC-4 + schedulers flavour
// inside committed stretches): while the pending work is small,
// each CTA keeps the vertices it removes in a shared-memory queue together with
// their predecessors (their G^T rows, loaded when they are removed) and
// decrements those predecessors' counters itself in the next round. A round then
// needs neither the dead log nor the work list in global memory, nor space
// reservations, nor a read of the control block: it ends at a barrier that
// carries the round's totals (see local_barrier). A removal that does not fit
// the queue goes to the global lists, and the run returns to ordinary rounds.
#if TRIM_MODES == 1 || TRIM_MODES == 9
#define TRIM_LOCAL 1
#else
#define TRIM_LOCAL 0
#endif
#if TRIM_LOCAL
constexpr uint32_t LQ_EDGES = 1024;   // predecessors queued per CTA per round
constexpr uint32_t LQ_ENTRIES = 256;  // removed vertices queued per CTA per round
constexpr uint32_t LQ_DMAX = 64;      // larger in-degrees always go to the global work list
// asynchronous AC-4 tail (see async_tail)
constexpr uint32_t ASYNC_MIN_ROUND = 128;  // rounds before the tail may take over
constexpr uint32_t AQ_LOCAL_DMAX = 1024; // larger in-degrees always go to the shared queue
#endif

// Per-CTA shared state.
struct Cta {
  Sched S;
  WarpSlice ws[MAX_WARPS];
  unsigned epoch;     // grid barriers passed by this kernel
  unsigned bar_base;  // barrier counter when this kernel started
  unsigned resume;    // this launch continues a run a segment handed over
  unsigned skip;      // continuation launch of a run that needs none: return at once
  unsigned mode;      // trim_variant_t of the run
  unsigned err;
  unsigned w4_wide;   // initial pass: the work-list slices take all four buffers
  unsigned lq_scratch;  // initial pass with a dead mask: deferred heavy rows
  unsigned long long kstat[4];  // TRIM_FLAG_STATS totals of this CTA (see stats_flush)
  uint32_t wbuf[MAX_WARPS][WBUF];
#if TRIM_LOCAL
  // local queues, double-buffered by local-round parity: buffer b is filled in
  // the round whose lround parity is b and read in the next one
  uint32_t lq_ids[2][LQ_EDGES];       // predecessors to decrement
  uint32_t lq_row[2][LQ_ENTRIES];     // the queued vertices' G^T rows ...
  uint32_t lq_din[2][LQ_ENTRIES];     // ... and in-degrees
  unsigned long long lq_cnt[2];       // reserved: entries (low 32) | predecessors (high 32)
  uint32_t lq_vend[2];                // end of the reservations that fit (entries)
  uint32_t lq_k;                      // this round's removals kept local
  uint32_t lq_ovf;                    // 1: a removal of this round went to the global lists
  uint32_t lq_pushed;                 // predecessors decremented from the queue this round
  uint32_t lq_next;                   // how the stretch goes on after the local barrier
  // asynchronous tail: predecessors queued per buffer (dynamic shared memory):
  // reserved, and the end of the reservations that fit; the share of the last
  // rebalance (global entries [sh_elo, sh_ehi), pieces [sh_plo, sh_phi)); this
  // CTA's removals and top level since it last released its token; whether it
  // holds a token; steps run; whether it asks for a rebalance; rebalances
  // passed; start of the pieces written since the last one; average share
  // (entries) at the last one; its entry-list slot; what the next step does
  uint32_t aq_res[2];
  uint32_t aq_end[2];
  uint32_t sh_elo, sh_ehi, sh_plo, sh_phi;
  uint32_t a_removed, a_maxlev;
  uint32_t a_token;
  uint32_t a_steps;
  uint32_t a_want;
  uint32_t a_gen;
  uint32_t a_plo;
  uint32_t a_avg;
  uint32_t a_base;
  uint32_t a_next;
#endif
};

// Are scheduler features gathered in round S.round? The learned scheduler (and
// a round log of a scheduled run) reads them after every round in which it is
// consulted, i.e. every round outside a committed stretch.
__device__ __forceinline__ bool feats_on(const Dev& D, const Sched& S) {
  return (MODES & M_SCHED) && (D.flags & F_NEED_FEATURES) &&
         !(S.cstop != 0u && S.round < S.cstop);
}

// dynamic shared memory: per warp w, 4 slices of LW words at w * 4 * LW:
// dead-log entries | work-list rows | work-list edge offsets (warp-local) | live-list entries
extern __shared__ uint32_t dyn_smem[];
__device__ __forceinline__ uint32_t* slice(unsigned warp, int which) {
  return dyn_smem + (warp * 4u + (unsigned)which) * LW;
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void red_relaxed_add(unsigned* p, unsigned v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ------------------------------------------------------------------ rows

#if TRIM_MODES & 32
// The implicit planted graph of trim_create_implicit (include/trim.h gives the
// definition): SplitMix64 (Steele, Lea & Flood) as a counter-based generator,
// key(v) = mix(seed ^ mix(salt + v + GAMMA)), word(v, i) = mix(key + (i+1) GAMMA),
// and Lemire's multiply-shift for a uniform integer below k.
constexpr uint64_t IG_GAMMA = 0x9E3779B97F4A7C15ull;
__device__ __forceinline__ uint64_t ig_mix(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t ig_word(const Dev& D, uint32_t v, uint64_t i) {
  const uint64_t key = ig_mix(D.ig.seed ^ ig_mix(D.ig.salt + v + IG_GAMMA));
  return ig_mix(key + (i + 1ull) * IG_GAMMA);
}
__device__ __forceinline__ uint32_t ig_below(uint64_t w, uint64_t k) {
  return (uint32_t)__umul64hi(w, k);
}
// number of successors of v
__device__ uint32_t ig_degree(const Dev& D, uint32_t v) {
  const trim_implicit_graph_t& g = D.ig;
  const uint64_t w0 = ig_word(D, v, 0);
  const uint32_t nCR = g.nC + g.nR;
  if (v < g.nC) return g.c_kmin + ig_below(w0, (uint64_t)g.c_kmax - g.c_kmin + 1u);
  if (v < nCR) return g.r_kmin + ig_below(w0, (uint64_t)g.r_kmax - g.r_kmin + 1u);
  const uint32_t rank = v - nCR;
  const uint32_t k = g.t_kmin + ig_below(w0, (uint64_t)g.t_kmax - g.t_kmin + 1u);
  if (g.n_chains == 0u) return rank < g.t_sinks ? 0u : k;
  return rank < g.n_chains ? 0u : 1u + k;
}
// successor j of v (j below its degree)
__device__ uint32_t ig_successor(const Dev& D, uint32_t v, uint32_t j) {
  const trim_implicit_graph_t& g = D.ig;
  const uint64_t w = ig_word(D, v, 1ull + j);
  const uint32_t nCR = g.nC + g.nR;
  if (v < g.nC) return ig_below(w, g.nC);
  if (v < nCR) return ig_below(w, j == 0u ? g.nC : nCR);
  const uint32_t rank = v - nCR;
  if (g.n_chains == 0u) return nCR + ig_below(w, rank);
  if (j == 0u) return v - g.n_chains;
  return nCR + ig_below(w, (uint64_t)(rank / g.n_chains) * g.n_chains);
}
#endif

// Row access of the scans: out-CSR loads, or computed successors on an
// implicit graph (where s is unused).
__device__ __forceinline__ void row_bounds(const Dev& D, uint32_t v, uint32_t& s, uint32_t& d) {
#if TRIM_MODES & 32
  s = 0u;
  d = ig_degree(D, v);
#else
  s = __ldg(&D.off[v]);
  d = __ldg(&D.off[v + 1]) - s;
#endif
}
__device__ __forceinline__ uint32_t row_target(const Dev& D, uint32_t v, uint32_t s, uint32_t j) {
#if TRIM_MODES & 32
  (void)s;
  return ig_successor(D, v, j);
#else
  (void)v;
  return __ldg(&D.tgt[s + j]);
#endif
}

// ------------------------------------------------------------------ appends

// Warp-collective: writes the chunk-owner index of the work-list entries the
// lanes hold: every chunk start 32c inside an entry's edge range [es, ee) is
// owned by that entry (pos). An entry with at most two chunk starts marks them
// itself; a longer one (a hub) is marked by the whole warp, so one lane never
// serialises thousands of stores.
__device__ __forceinline__ void mark_chunks(const Dev& D, bool has, uint32_t pos, uint32_t es,
                                            uint32_t ee) {
  const uint32_t c0 = (es + 31u) >> 5, c1 = (ee + 31u) >> 5;  // chunk starts in [es, ee)
  const bool big = has && c1 > c0 + 2u;
  if (has && !big) {
    if (c0 < c1) D.chunk_first[c0] = pos;
    if (c0 + 1u < c1) D.chunk_first[c0 + 1u] = pos;
  }
  unsigned bm = __ballot_sync(FULL, big);
  while (bm) {
    const int j = __ffs(bm) - 1;
    bm &= bm - 1u;
    const uint32_t p = __shfl_sync(FULL, pos, j), a = __shfl_sync(FULL, c0, j),
                   z = __shfl_sync(FULL, c1, j);
    for (uint32_t c = a + lane_id(); c < z; c += 32u) D.chunk_first[c] = p;
  }
}

// AC-4 work-list slices of a warp: G^T row starts and in-edge offsets. The
// initial pass writes no dead log and no live list, so there they span two
// buffers each (rows over buffers 0-1, offsets over 2-3): fewer warp flushes.
__device__ __forceinline__ uint32_t* w4_rows(const Cta& B, unsigned warp) {
  return slice(warp, B.w4_wide ? 0 : 1);
}
__device__ __forceinline__ uint32_t w4_cap(const Cta& B) { return B.w4_wide ? 2u * LW : LW; }

// Warp-collective: copies this warp's slices to global memory at the given bases.
__device__ __forceinline__ void copy_slices(const Dev& D, const Cta& B, const WarpSlice& w,
                                            unsigned warp, uint32_t* live_out) {
  const unsigned lane = lane_id();
  const uint32_t* sl = slice(warp, 0);
  const uint32_t* sr = w4_rows(B, warp);
  const uint32_t* se = slice(warp, 2);
  const uint32_t* sv = slice(warp, 3);
  for (uint32_t i = lane; i < w.nlog; i += 32) D.log[w.log_base + i] = sl[i];
  for (uint32_t i0 = 0; i0 < w.nw4; i0 += 32) {  // warp-uniform loop: mark_chunks is collective
    const uint32_t i = i0 + lane;
    const bool has = i < w.nw4;
    uint32_t eo = 0, ee = 0;
    if (has) {
      eo = w.edge_base + se[i];
      ee = w.edge_base + (i + 1 < w.nw4 ? se[i + 1] : w.nedge);
      D.w4_row[w.w4_base + i] = sr[i];
      D.w4_eoff[w.w4_base + i] = eo;
      if (MODES & M_INOUT) {  // in+out entries: in-degree in slice 0, G row in slice 3
        D.w4_din[w.w4_base + i] = sl[i];
        D.w4_orow[w.w4_base + i] = sv[i];
      }
    }
    mark_chunks(D, has, w.w4_base + i, eo, ee);
  }
  for (uint32_t i = lane; i < w.nlive; i += 32) live_out[w.live_base + i] = sv[i];
}

// Warp-collective: a slice is full; the warp reserves global space on its own.
__device__ __noinline__ void warp_flush(const Dev& D, Cta& B, uint32_t r, uint32_t* live_out) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  WarpSlice& w = B.ws[warp];
  // three lanes reserve at once; removals that are only counted (nlog = 0)
  // wait for the CTA flush
  if (lane == 0 && w.nlog) {
    w.log_base = atomicAdd(&D.C->log_len, w.nlog + w.ncount);
    if (w.log_base + w.nlog + w.ncount > D.n) { set_error(D, TRIM_ERR_STATE, 0xD1); w.nlog = 0; }
    w.ncount = 0;
  }
  if (lane == 1 && w.nw4) {
    const unsigned long long o = atomicAdd(
        &D.C->w4, (unsigned long long)w.nw4 | ((unsigned long long)w.nedge << 32));
    w.w4_base = (uint32_t)o;
    w.edge_base = (uint32_t)(o >> 32);
  }
  if (lane == 2 && w.nlive) {
    w.live_base = atomicAdd(&D.C->rs[r & 3].live_count, w.nlive);
    if (w.live_base + w.nlive > D.n) { set_error(D, TRIM_ERR_STATE, 0xD3); w.nlive = 0; }
  }
  __syncwarp();
  const WarpSlice c = w;
  copy_slices(D, B, c, warp, live_out);
  __syncwarp();
  if (lane == 0) w.nlog = w.nw4 = w.nedge = w.nlive = 0;
  __syncwarp();
}

// Warp-collective: lanes with pred are removed in round r: level[u] = r and u
// joins F_r in the dead log; if it has in-edges (and AC-4 may run) it also
// joins the AC-4 work list with its G^T row and in-degree. With pre, the caller
// has already loaded u's G^T row start (prow) and in-degree (pdin). dout is u's
// out-degree where the caller knows it (AC-3/AC-6 scans; 0 for AC-4, which
// never loads it): it only feeds the scheduler's live-edge count without G^T.
__device__ __forceinline__ void append_dead(const Dev& D, Cta& B, bool pred, uint32_t u,
                                            uint32_t r, uint32_t* live_out,
                                            bool initial = false, bool pre = false,
                                            uint32_t prow = 0, uint32_t pdin = 0,
                                            uint32_t dout = 0) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned mask = __ballot_sync(FULL, pred);
  if (mask == 0u) return;
  const bool feats = feats_on(D, B.S);
  const bool live_edges = feats || (D.flags & F_LIVE_EDGES);
  // whenever the run may use AC-4, every flavour keeps its work list complete
  const bool track = D.ioff != nullptr && ((D.flags & F_AC4_POSSIBLE) || feats);
  uint32_t row = 0, din = 0;
  if (!pred) dout = 0;
  if (pred && track) {
    if (pre) {
      row = prow;
      din = pdin;
    } else {
      row = __ldg(&D.ioff[u]);
      din = __ldg(&D.ioff[u + 1]) - row;
    }
  }
  const bool w = pred && din > 0u && (D.flags & F_AC4_POSSIBLE);
  const unsigned wmask = __ballot_sync(FULL, w);
  const unsigned lt = (1u << lane) - 1u;
  const unsigned k = __popc(mask), kw = __popc(wmask);
  const unsigned ew = w ? din : 0u;
  const unsigned eincl = warp_incl_scan(ew);
  const unsigned esum = __shfl_sync(FULL, eincl, 31);
  WarpSlice& ws = B.ws[warp];
  const unsigned kl = initial ? 0u : k;  // F_0 is only counted: no variant reads it back
  if (ws.nlog + kl > LW || ws.nw4 + kw > w4_cap(B)) warp_flush(D, B, r, live_out);
  const uint32_t pl = ws.nlog, pw = ws.nw4, pe = ws.nedge;
  if (pred && !initial) {
    slice(warp, 0)[pl + __popc(mask & lt)] = u;
    D.level[u] = r;
  }
  unsigned mdin = 0;
  if (wmask) {
    mdin = __reduce_max_sync(FULL, ew);
    if (w) {
      const unsigned at = pw + __popc(wmask & lt);
      w4_rows(B, warp)[at] = row;
      slice(warp, 2)[at] = pe + eincl - ew;
    }
  }
  unsigned s_in = 0, s_out = 0;
  unsigned h0 = 0, h1 = 0;
  if (live_edges) s_out = __reduce_add_sync(FULL, dout);
  if (feats) {
    s_in = __reduce_add_sync(FULL, din);
    h0 = __popc(__ballot_sync(FULL, pred && din < 8u));
    h1 = __popc(__ballot_sync(FULL, pred && din >= 8u && din < 256u));
  }
  __syncwarp();
  if (lane == 0) {
    ws.nlog = pl + kl;
    ws.ncount += k - kl;
    ws.nw4 = pw + kw;
    ws.nedge = pe + esum;
    ws.max_din = max(ws.max_din, mdin);
    if (live_edges) ws.sum_out += s_out;
    if (feats) {
      ws.sum_in += s_in;
      ws.hist[0] += h0;
      ws.hist[1] += h1;
      ws.hist[2] += k - h0 - h1;
    }
  }
  __syncwarp();
}

#if TRIM_MODES & 16
// Warp-collective, in+out trimming: lanes with pred were removed in round r
// (their level is already set). Each joins the work list with one entry whose
// edge range covers its G^T row (row, din edges: the predecessors whose
// out-degree counters it decrements) and then its G row (orow, dout edges: the
// successors whose in-degree counters it decrements). Removals are only
// counted in the dead log, never written: no variant of this flavour reads it.
__device__ __forceinline__ void append_dead_io(const Dev& D, Cta& B, bool pred, uint32_t u,
                                               uint32_t r, bool pre, uint32_t prow,
                                               uint32_t pdin, uint32_t porow, uint32_t pdout) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned mask = __ballot_sync(FULL, pred);
  if (mask == 0u) return;
  uint32_t row = 0, din = 0, orow = 0, dout = 0;
  if (pred) {
    if (pre) {
      row = prow; din = pdin; orow = porow; dout = pdout;
    } else {
      row = __ldg(&D.ioff[u]);
      din = __ldg(&D.ioff[u + 1]) - row;
      orow = __ldg(&D.off[u]);
      dout = __ldg(&D.off[u + 1]) - orow;
    }
  }
  const bool w = pred && din + dout > 0u;
  const unsigned wmask = __ballot_sync(FULL, w);
  const unsigned k = __popc(mask), kw = __popc(wmask);
  const unsigned ew = w ? din + dout : 0u;
  const unsigned eincl = warp_incl_scan(ew);
  const unsigned esum = __shfl_sync(FULL, eincl, 31);
  WarpSlice& ws = B.ws[warp];
  if (ws.nw4 + kw > w4_cap(B)) warp_flush(D, B, r, D.live0);
  const uint32_t pw = ws.nw4, pe = ws.nedge;
  const unsigned mdin = __reduce_max_sync(FULL, ew);
  if (w) {
    const unsigned at = pw + __popc(wmask & ((1u << lane) - 1u));
    w4_rows(B, warp)[at] = row;
    slice(warp, 2)[at] = pe + eincl - ew;
    slice(warp, 0)[at] = din;
    slice(warp, 3)[at] = orow;
  }
  __syncwarp();
  if (lane == 0) {
    ws.ncount += k;
    ws.nw4 = pw + kw;
    ws.nedge = pe + esum;
    ws.max_din = max(ws.max_din, mdin);
  }
  __syncwarp();
}
#endif

// Warp-collective append of survivors to the AC-3 output live list.
__device__ __forceinline__ void append_live(const Dev& D, Cta& B, bool pred, uint32_t v,
                                            uint32_t r, uint32_t* out_list) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned mask = __ballot_sync(FULL, pred);
  if (mask == 0u) return;
  const unsigned k = __popc(mask);
  WarpSlice& ws = B.ws[warp];
  if (ws.nlive + k > LW) warp_flush(D, B, r, out_list);
  const uint32_t pv = ws.nlive;
  if (pred) slice(warp, 3)[pv + __popc(mask & ((1u << lane) - 1u))] = v;
  __syncwarp();
  if (lane == 0) ws.nlive = pv + k;
  __syncwarp();
}

#if TRIM_LOCAL
// Warp-collective: lanes with pred add a work-list entry (G^T row start, in-degree)
// of a vertex that is already removed and counted (local queue entries handed
// to the global work list when local rounds end).
__device__ __forceinline__ void append_w4(const Dev& D, Cta& B, bool pred, uint32_t row,
                                          uint32_t din, uint32_t r) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const bool w = pred && din > 0u;
  const unsigned wmask = __ballot_sync(FULL, w);
  if (wmask == 0u) return;
  const unsigned kw = __popc(wmask);
  const unsigned ew = w ? din : 0u;
  const unsigned eincl = warp_incl_scan(ew);
  const unsigned esum = __shfl_sync(FULL, eincl, 31);
  WarpSlice& ws = B.ws[warp];
  if (ws.nw4 + kw > w4_cap(B)) warp_flush(D, B, r, D.live0);
  const uint32_t pw = ws.nw4, pe = ws.nedge;
  const unsigned mdin = __reduce_max_sync(FULL, ew);
  if (w) {
    const unsigned at = pw + __popc(wmask & ((1u << lane) - 1u));
    w4_rows(B, warp)[at] = row;
    slice(warp, 2)[at] = pe + eincl - ew;
  }
  __syncwarp();
  if (lane == 0) {
    ws.nw4 = pw + kw;
    ws.nedge = pe + esum;
    ws.max_din = max(ws.max_din, mdin);
  }
  __syncwarp();
}

// Warp-collective, local rounds: lanes with pred remove u in round r (its G^T
// row start and in-degree already loaded). A removal with at most LQ_DMAX
// in-edges that fits this CTA's queue (buffer b) stays local: its G^T row is
// copied into the queue now, all of the warp's rows at once (each lane loads
// entries of the flattened rows, so the loads overlap). Everything else takes
// the global path of an ordinary round (dead log, work list) and marks the
// round as overflowing.
__device__ __forceinline__ void local_append(const Dev& D, Cta& B, bool pred, uint32_t u,
                                             uint32_t r, uint32_t row, uint32_t din,
                                             uint32_t b) {
  const unsigned lane = lane_id();
  const unsigned mask = __ballot_sync(FULL, pred);
  if (mask == 0u) return;
  if (pred) D.level[u] = r;
  const bool want = pred && din > 0u && din <= LQ_DMAX;
  const unsigned wm = __ballot_sync(FULL, want);
  bool ovf = pred && din > LQ_DMAX;
  if (wm) {
    const unsigned ew = want ? din : 0u;
    const unsigned eincl = warp_incl_scan(ew);
    const unsigned esum = __shfl_sync(FULL, eincl, 31);
    const unsigned excl = eincl - ew;
    const unsigned k = __popc(wm);
    unsigned long long old = 0;
    if (lane == 0)
      old = atomicAdd(&B.lq_cnt[b], (unsigned long long)k | ((unsigned long long)esum << 32));
    old = __shfl_sync(FULL, old, 0);
    const uint32_t be = (uint32_t)old, bd = (uint32_t)(old >> 32);
    if (be + k <= LQ_ENTRIES && bd + esum <= LQ_EDGES) {  // warp-uniform
      if (lane == 0) atomicMax(&B.lq_vend[b], be + k);
      if (want) {
        const uint32_t slot = be + __popc(wm & ((1u << lane) - 1u));
        B.lq_row[b][slot] = row;
        B.lq_din[b][slot] = din;
      }
      // predecessors: element j of the flattened rows belongs to the lane with
      // the largest exclusive prefix <= j; four loads in flight per lane
      for (uint32_t j0 = 0; j0 < esum; j0 += 128u) {
        uint32_t t[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t j = j0 + (uint32_t)q * 32u + lane;
          const unsigned o = owner_of(excl, j);
          const uint32_t ro = __shfl_sync(FULL, row, o), xo = __shfl_sync(FULL, excl, o);
          t[q] = j < esum ? __ldg(&D.itgt[ro + (j - xo)]) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t j = j0 + (uint32_t)q * 32u + lane;
          if (j < esum) B.lq_ids[b][bd + j] = t[q];
        }
      }
    } else {
      ovf = ovf || want;
    }
  }
  const unsigned om = __ballot_sync(FULL, ovf);
  if (lane == 0) {
    atomicAdd(&B.lq_k, (unsigned)__popc(mask & ~om));
    if (om) B.lq_ovf = 1u;
  }
  append_dead(D, B, ovf, u, r, D.live0, false, true, row, din);
}
#endif

// End of round r: moves every warp slice of the CTA to global memory with one
// global atomic per counter (all threads of the CTA). The (up to three) space
// reservations are issued by three lanes at once, so they cost one round trip.
__device__ void flush_round(const Dev& D, Cta& B, uint32_t r, uint32_t* live_out) {
  __syncthreads();
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (warp == 0) {
    // exclusive prefix of the per-warp counts (lane i holds warp i)
    const bool has = lane < nw;
    const uint32_t a = has ? B.ws[lane].nlog + B.ws[lane].ncount : 0u,
                   b = has ? B.ws[lane].nw4 : 0u, c = has ? B.ws[lane].nedge : 0u,
                   d = has ? B.ws[lane].nlive : 0u;
    const uint32_t ia = warp_incl_scan(a), ib = warp_incl_scan(b), ic = warp_incl_scan(c),
                   id = warp_incl_scan(d);
    const uint32_t ta = __shfl_sync(FULL, ia, 31), tb = __shfl_sync(FULL, ib, 31),
                   tc = __shfl_sync(FULL, ic, 31), td = __shfl_sync(FULL, id, 31);
    RoundStat* rs = &D.C->rs[r & 3];
    unsigned long long got = 0;
    if (lane == 0 && ta) got = atomicAdd(&D.C->log_len, ta);
    if (lane == 1 && tb)
      got = atomicAdd(&D.C->w4, (unsigned long long)tb | ((unsigned long long)tc << 32));
    if (lane == 2 && td) got = atomicAdd(&rs->live_count, td);
    uint32_t lb = (uint32_t)__shfl_sync(FULL, got, 0);
    const unsigned long long w4o = __shfl_sync(FULL, got, 1);
    uint32_t vb = (uint32_t)__shfl_sync(FULL, got, 2);
    const uint32_t wb = (uint32_t)w4o, eb = (uint32_t)(w4o >> 32);
    if (ta && lb + ta > D.n) {
      if (lane == 0) set_error(D, TRIM_ERR_STATE, 0xD5);
      lb = 0xFFFFFFFFu;
    }
    if (td && vb + td > D.n) {
      if (lane == 0) set_error(D, TRIM_ERR_STATE, 0xD6);
      vb = 0xFFFFFFFFu;
    }
    const bool feats = feats_on(D, B.S);
    if (feats || (D.flags & F_LIVE_EDGES)) {
      const uint32_t s_out = __reduce_add_sync(FULL, has ? B.ws[lane].sum_out : 0u);
      if (lane == 4 && s_out) atomicAdd(&rs->sum_out, (unsigned long long)s_out);
    }
    {
      const uint32_t md = __reduce_max_sync(FULL, has ? B.ws[lane].max_din : 0u);
      if (lane == 8 && md) atomicMax(&rs->max_din, md);
    }
    if (feats) {
      const uint32_t s_in = __reduce_add_sync(FULL, has ? B.ws[lane].sum_in : 0u);
      uint32_t h[3];
      for (int i = 0; i < 3; ++i) h[i] = __reduce_add_sync(FULL, has ? B.ws[lane].hist[i] : 0u);
      // independent reductions from separate lanes (no return value: no wait)
      if (lane == 3 && s_in) atomicAdd(&rs->sum_in, (unsigned long long)s_in);
      if (lane >= 5 && lane < 8 && h[lane - 5]) atomicAdd(&rs->hist[lane - 5], h[lane - 5]);
    }
    if (has) {
      WarpSlice& w = B.ws[lane];
      w.log_base = lb + ia - a;
      w.w4_base = wb + ib - b;
      w.edge_base = eb + ic - c;
      w.live_base = vb + id - d;
      if (lb == 0xFFFFFFFFu) w.nlog = 0;
      if (vb == 0xFFFFFFFFu) w.nlive = 0;
    }
  }
  __syncthreads();
  const WarpSlice c = B.ws[warp];
  copy_slices(D, B, c, warp, live_out);
  __syncwarp();
  if (lane == 0) {
    WarpSlice& w = B.ws[warp];
    w.nlog = w.nw4 = w.nedge = w.nlive = w.ncount = 0;
    w.sum_in = w.sum_out = 0;
    w.hist[0] = w.hist[1] = w.hist[2] = 0;
    w.max_din = 0;
  }
}

// ------------------------------------------------------------------ grid barrier

// Grid-wide barrier: each CTA adds one arrival to a monotone counter and waits
// until all gridDim.x arrivals of this epoch are in (counted from the value the
// counter had when this kernel started: a resumed segment continues it). The
// wait is bounded by spin_limit_ns; past it the run stops with
// TRIM_ERR_TIMEOUT. Returns false if the run must stop (any error flag).
// With read_err false the error flag is not read here: the round loop reads it
// in advance(), together with the round's counters (one memory round trip less).
__device__ bool grid_barrier(const Dev& D, Cta& B, bool read_err = true) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = B.bar_base + (++B.epoch) * gridDim.x;
    fence_acq_rel();
    red_relaxed_add(&D.C->bar, 1u);
    const uint64_t t0 = globaltimer();
    // relaxed polls, then one acquiring load once every arrival is in (an
    // acquiring load per poll would invalidate this SM's L1 every time)
    while ((int)(ld_relaxed(&D.C->bar) - target) < 0) {
      if (globaltimer() - t0 > D.spin_limit_ns) {
        set_error(D, TRIM_ERR_TIMEOUT, 1);
        B.err = TRIM_ERR_TIMEOUT;
        break;
      }
    }
    (void)ld_acquire(&D.C->bar);
    if (read_err) B.err = ld_relaxed(&D.C->err);
  }
  __syncthreads();
  return B.err == 0u;
}

// Warp-collective: adds this warp's counters to the run totals (stats runs only).
// The CTA's totals stay in shared memory for the whole launch and reach the
// global counters once, when the kernel ends (stats_publish): no global
// atomics per warp and round.
__device__ __forceinline__ void stats_flush(const Dev& D, Cta& B, const Counters& K) {
  if (!(D.flags & F_STATS)) return;
  // a round's counts of a whole warp are counts of distinct edges or vertices
  const unsigned e = __reduce_add_sync(FULL, K.edges), p = __reduce_add_sync(FULL, K.pushed),
                 c = __reduce_add_sync(FULL, K.cand), s = __reduce_add_sync(FULL, K.swept);
  if (lane_id() == 0) {
    if (e) atomicAdd(&B.kstat[0], (unsigned long long)e);
    if (p) atomicAdd(&B.kstat[1], (unsigned long long)p);
    if (c) atomicAdd(&B.kstat[2], (unsigned long long)c);
    if (s) atomicAdd(&B.kstat[3], (unsigned long long)s);
  }
}

__device__ __forceinline__ void stats_publish(const Dev& D, Cta& B) {
  if (!(D.flags & F_STATS)) return;
  __syncthreads();
  if (threadIdx.x < 4 && B.kstat[threadIdx.x]) atomicAdd(&D.C->stats[threadIdx.x], B.kstat[threadIdx.x]);
}

// ------------------------------------------------------------------ scans

// Thread-level forward scan of v's successors from position i (row start s,
// length d): returns the first position whose target is not removed before
// round r, or d. At most `batches` x 4 edges; *resolved tells whether it ended.
__device__ __forceinline__ uint32_t scan_thread(const Dev& D, uint32_t v, uint32_t s, uint32_t d,
                                                uint32_t i, uint32_t r, int batches,
                                                bool& resolved, Counters& K) {
  for (int b = 0; b < batches; ++b) {
    if (i >= d) { resolved = true; return d; }
    const uint32_t nb = min(4u, d - i);
    uint32_t t[4], lv[4];
#if TRIM_MODES & 32
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = (q < (int)nb) ? row_target(D, v, s, i + q) : 0u;
#else
    // four targets on a 16-byte boundary (of the address: a caller's array may
    // start anywhere) come with one load
    if (nb == 4u && (reinterpret_cast<uintptr_t>(D.tgt + s + i) & 15u) == 0u) {
      const uint4 x = __ldg(reinterpret_cast<const uint4*>(D.tgt + s + i));
      t[0] = x.x; t[1] = x.y; t[2] = x.z; t[3] = x.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) t[q] = (q < (int)nb) ? __ldg(&D.tgt[s + i + q]) : 0u;
    }
#endif
#pragma unroll
    for (int q = 0; q < 4; ++q) lv[q] = (q < (int)nb) ? ldcg(&D.level[t[q]]) : 0u;
    K.edges += nb;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < (int)nb && lv[q] >= r) { resolved = true; return i + q; }
    i += nb;
  }
  resolved = (i >= d);
  return i;
}

// Warp-collective: finishes the scans of lanes with !resolved, one lane at a
// time, 32 successors per step (ballot picks the first live one).
__device__ __forceinline__ void scan_warp_finish(const Dev& D, bool& resolved, uint32_t v,
                                                 uint32_t s, uint32_t d, uint32_t& i, uint32_t r,
                                                 Counters& K) {
  const unsigned lane = lane_id();
  unsigned pend = __ballot_sync(FULL, !resolved);
  while (pend) {
    const int src = __ffs(pend) - 1;
    pend &= pend - 1;
    const uint32_t ss = __shfl_sync(FULL, s, src), dd = __shfl_sync(FULL, d, src);
    const uint32_t vv = __shfl_sync(FULL, v, src);
    uint32_t ii = __shfl_sync(FULL, i, src);
    uint32_t found = dd;
    while (ii < dd) {
      const uint32_t k = ii + lane;
      bool live = false;
      if (k < dd) live = ldcg(&D.level[row_target(D, vv, ss, k)]) >= r;
      const unsigned b = __ballot_sync(FULL, live);
      if (lane == 0) K.edges += min(32u, dd - ii);
      if (b) { found = ii + __ffs(b) - 1; break; }
      ii += 32;
    }
    if ((int)lane == src) { i = found; resolved = true; }
  }
}

// ------------------------------------------------------------------ scheduler

__device__ __forceinline__ float log2p1(float x) { return log2f(1.0f + x); }

// Cost rule of TRIM_SCHED_HEURISTIC: the work each variant would do in round
// r+1, in units of one random memory access, with one-time entry costs spread
// over a horizon of H rounds (a greedy rule that charged them to one round
// would never leave a variant whose cost recurs every round).
//   AC-4: pushes every in-edge of the removed vertices it has not processed yet
//         (the backlog beyond the newest frontier is a one-time cost).
//   AC-3: sweeps its live list (all n vertices the first time), every round.
//   AC-6: while it runs, re-scans about one supporting-set member per removed
//         vertex; entering it rebuilds the sets of all live vertices.
__device__ uint32_t heuristic_choice(const Dev& D, const Sched& L, uint32_t nF, uint32_t n_live,
                                     uint32_t w_end, uint32_t e_end) {
  constexpr float H = 4.0f;
  const float inf = 3.0e38f;
  const float eF = (float)(e_end - L.e_end);          // in-edges of the newest frontier
  const float backlog = (float)(e_end - L.e_c4);      // in-edges not yet pushed
  const float items = (float)(w_end - L.c4w);
  float c4 = (L.variant == TRIM_AC4_PUSH) ? eF + 0.25f * items
                                           : (backlog - eF) / H + eF + 0.25f * items;
  const float sweep = (L.ac3_list == NIL) ? (float)D.n : (float)L.live_in_len;
  float c3 = 2.0f * sweep;
  float c6 = (L.variant == TRIM_AC6_SUPPORT)
                 ? 4.0f * (float)nF
                 : (3.0f * (float)n_live + (float)D.n) / H + 4.0f * (float)nF;
  c4 *= D.heur_push_ratio;
  c6 *= D.heur_ac6_ratio;
  if (!(D.flags & F_AC4_POSSIBLE) || D.ioff == nullptr) c4 = inf;
  if (!(D.flags & F_AC6_POSSIBLE)) c6 = inf;
  if (!(D.flags & F_AC3_POSSIBLE)) c3 = inf;
  if (c4 <= c3 && c4 <= c6) return TRIM_AC4_PUSH;
  if (c6 <= c3) return TRIM_AC6_SUPPORT;
  return TRIM_AC3_PULL;
}

// Warp-collective MLP 12 -> 32 -> 32 -> 3 (ReLU) read from the model blob in
// global memory (W1[32][12] b1[32] W2[32][32] b2[32] W3[3][32] b3[3] mean[12]
// istd[12] lo[12] hi[12]; 16-byte aligned): lane j computes hidden unit j of
// each layer from row j of W1 and W2 (float4 loads). It runs only in rounds
// after which the scheduler is consulted, so the model stays out of shared
// memory. Returns the argmax class among the available variants, its softmax
// probability, and whether every feature lies in the model's training range.
__device__ uint32_t mlp_choice(const Dev& D, const float* f, bool* in_range,
                               float* confidence) {
  const unsigned lane = lane_id();
  const float* M = D.model;
  bool ok = true;
  float x[NFEAT];
#pragma unroll
  for (int i = 0; i < NFEAT; ++i) {
    const float mean = __ldg(M + 1571 + i), istd = __ldg(M + 1583 + i);
    const float lo = __ldg(M + 1595 + i), hi = __ldg(M + 1607 + i);
    ok = ok && f[i] >= lo && f[i] <= hi;
    x[i] = (f[i] - mean) * istd;
  }
  const float4* w1 = reinterpret_cast<const float4*>(M + lane * NFEAT);
  float h1 = __ldg(M + 384 + lane);
#pragma unroll
  for (int q = 0; q < NFEAT / 4; ++q) {
    const float4 w = __ldg(w1 + q);
    h1 = fmaf(w.x, x[4 * q], h1);
    h1 = fmaf(w.y, x[4 * q + 1], h1);
    h1 = fmaf(w.z, x[4 * q + 2], h1);
    h1 = fmaf(w.w, x[4 * q + 3], h1);
  }
  h1 = fmaxf(h1, 0.0f);
  const float4* w2 = reinterpret_cast<const float4*>(M + 416 + lane * 32);
  float acc[4] = {__ldg(M + 1440 + lane), 0.0f, 0.0f, 0.0f};  // four independent chains
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 w = __ldg(w2 + q);
    acc[0] = fmaf(w.x, __shfl_sync(FULL, h1, 4 * q), acc[0]);
    acc[1] = fmaf(w.y, __shfl_sync(FULL, h1, 4 * q + 1), acc[1]);
    acc[2] = fmaf(w.z, __shfl_sync(FULL, h1, 4 * q + 2), acc[2]);
    acc[3] = fmaf(w.w, __shfl_sync(FULL, h1, 4 * q + 3), acc[3]);
  }
  const float h2 = fmaxf((acc[0] + acc[1]) + (acc[2] + acc[3]), 0.0f);
  float z[3];
#pragma unroll
  for (int o = 0; o < 3; ++o)
    z[o] = warp_sum(__ldg(M + 1472 + o * 32 + lane) * h2) + __ldg(M + 1568 + o);
  if (D.ioff == nullptr || !(D.flags & F_AC4_POSSIBLE)) z[TRIM_AC4_PUSH] = -3.0e38f;
  if (!(D.flags & F_AC6_POSSIBLE)) z[TRIM_AC6_SUPPORT] = -3.0e38f;
  if (!(D.flags & F_AC3_POSSIBLE)) z[TRIM_AC3_PULL] = -3.0e38f;
  uint32_t best = 0;
  if (z[1] > z[best]) best = 1;
  if (z[2] > z[best]) best = 2;
  // softmax probability of the choice among the available variants
  float den = 0.0f;
#pragma unroll
  for (int o = 0; o < 3; ++o) den += expf(z[o] - z[best]);
  *confidence = 1.0f / den;
  *in_range = ok;
  return best;
}

// Warp 0 of every CTA, after the barrier that ends round r (r = 0: the initial
// sink pass): closes round r in the CTA's copy of the schedule and prepares
// round r+1. Reads only values that are final for every CTA at this point, so
// all copies take the same decisions. CTA 0 also publishes results and logs.
__device__ ROUND_FN void advance(const Dev& D, Cta& B) {
  const unsigned lane = lane_id();
  Ctrl* C = D.C;
  Sched L = B.S;
  const uint32_t r = L.round;
  const RoundStat* rs = &C->rs[r & 3];
  // the scheduler chooses round r+1 unless a committed stretch covers it
  const bool consult = (MODES & M_SCHED) && B.mode > TRIM_AC3_PULL &&
                       !(L.cstop != 0u && r < L.cstop);
  const bool feats = feats_on(D, L);
  const bool logged = (D.flags & F_ROUND_LOG) && D.rlog != nullptr && r >= 1 && r - 1 < D.rlog_cap;
  // every value this step reads from the control block, issued together
  const uint32_t err = ld_relaxed(&C->err);
  // removals so far: logged ones plus those counted only by local rounds
  const uint32_t len = ld_relaxed(&C->log_len) + L.skew;
  const unsigned long long w4 = ld_relaxed64(&C->w4);
  const uint32_t live_count = ld_relaxed(&rs->live_count);
  const uint32_t max_din = ld_relaxed(&rs->max_din);
  unsigned long long sum_in = 0, sum_out = 0, t_r = 0, t_rm1 = 0, local_edges = 0;
  uint32_t h0 = 0, h1 = 0, h2 = 0;
  const bool live_edges = feats || (D.flags & F_LIVE_EDGES);
  // with G^T and a complete AC-4 work list the live-edge count follows from
  // running totals (the scheduler flavours keep it without F_LIVE_EDGES)
  const bool by_counts = D.ioff != nullptr && (D.flags & F_AC4_POSSIBLE) &&
                         ((MODES & M_SCHED) || live_edges);
  if (live_edges) sum_out = ld_relaxed64(&rs->sum_out);
  if (by_counts) local_edges = ld_relaxed64(&C->local_edges);
  if (feats) {
    sum_in = ld_relaxed64(&rs->sum_in);
    h0 = ld_relaxed(&rs->hist[0]);
    h1 = ld_relaxed(&rs->hist[1]);
    h2 = ld_relaxed(&rs->hist[2]);
    t_rm1 = ld_relaxed64(&C->t_round[(r - 1) & 3]);
  }
  if (feats || logged) t_r = ld_relaxed64(&C->t_round[r & 3]);
  const uint32_t w_end = (uint32_t)w4, e_end = (uint32_t)(w4 >> 32);
  const uint32_t nF = len - L.fe;  // |F_r|
  const bool cta0 = blockIdx.x == 0 && lane == 0;
  if (r >= 1) {
    if (L.variant <= 2u) L.vcount[L.variant] += 1;
    if (cta0) {
      if (L.variant <= 2u) C->vcount[L.variant] = L.vcount[L.variant];
      if (logged) {
        trim_round_rec_t* rec = &D.rlog[r - 1];
        rec->round = r;
        rec->variant = L.variant;
        rec->frontier = L.fe - L.fb;
        rec->removed = nF;
        rec->t_start_ns = t_r;
        rec->t_end_ns = globaltimer();
        rec->t_work_ns = ld_relaxed64(&C->t_work[r & 3]);
        rec->t_flush_ns = ld_relaxed64(&C->t_flush[r & 3]);
        for (int i = 0; i < NFEAT; ++i) rec->features[i] = L.feat[i];
        C->rlog_len = r;
      }
    }
    if (L.variant == TRIM_AC4_PUSH) {  // pushed every work-list entry that existed before round r
      L.c4w = L.w_end;
      L.e_c4 = L.e_end;
      L.bmax = 0;
    }
    if (L.variant == TRIM_AC3_PULL) {
      L.ac3_list = L.live_out;
      L.live_in_len = live_count;
    }
    // the first AC-6 or AC-3 round wrote the support position of every vertex
    // still live (both sweep all live vertices when they first run)
    if (L.variant == TRIM_AC6_SUPPORT || L.variant == TRIM_AC3_PULL) L.supp_valid = 1u;
  }
  L.bmax = max(L.bmax, max_din);  // the entries of F_r join the AC-4 backlog
  if (cta0) {
    D.roff[r] = L.fe;
    D.roff[r + 1] = len;
    C->rounds = nF ? r + 1 : r;
    C->n_dead = len;
  }
  // live-edge count. With G^T and a complete AC-4 work list: edges between live
  // vertices = m minus the in-edges of removed vertices (a removed vertex has
  // only removed successors, so every edge that touches one ends in one).
  // Otherwise: with G^T, the same from the in-degree sums; without it, out-edges
  // of live vertices (AC-3/AC-6 know each removed vertex's degree).
  // (in-edges pushed from local queues belong to removed vertices without
  // work-list entries)
  if (by_counts) L.m_live = (unsigned long long)D.m - e_end - local_edges;
  else if (live_edges) L.m_live -= (D.ioff != nullptr) ? sum_in : sum_out;
  if (nF == 0) {
    L.done = 1;
  } else {
    const uint32_t n_live = D.n - len;
    float f[NFEAT];
    for (int i = 0; i < NFEAT; ++i) f[i] = 0.0f;
    if (feats) {
      f[0] = log2p1((float)nF);
      f[1] = log2p1((float)sum_in);
      f[2] = log2p1((float)(e_end - L.e_c4));  // in-edges AC-4 has not pushed yet
      f[3] = log2p1((float)n_live);
      f[4] = log2p1((float)L.m_live);
      f[5] = (float)nF / (float)max(1u, n_live);
      f[6] = (float)sum_in / (float)max(1ull, L.m_live);
      f[7] = (float)h0 / (float)nF;
      f[8] = (float)h1 / (float)nF;
      f[9] = (float)h2 / (float)nF;
      // time of round r-1 per vertex of its frontier (CTA 0's clock, published to all)
      f[10] = (r >= 2) ? log2p1((float)(t_r - t_rm1) / (float)max(1u, L.fprev)) : 0.0f;
      f[11] = (r >= 1) ? (float)L.variant : -1.0f;  // the variant whose state is current
    }
    uint32_t next;
    bool confident = false;  // the learned scheduler may commit at once
    if (!(MODES & M_SCHED) || B.mode <= TRIM_AC3_PULL) {
      next = B.mode;
    } else if (!consult) {
      next = L.variant;  // inside a committed stretch
    } else if (B.mode == TRIM_SCHED_SCRIPTED) {
      next = D.script_len ? D.script[r % D.script_len] : 0u;
      if (next > 2u) next = TRIM_AC3_PULL;
      if (next == TRIM_AC4_PUSH && D.ioff == nullptr) next = TRIM_AC3_PULL;
    } else {
      next = heuristic_choice(D, L, nF, n_live, w_end, e_end);
      if (B.mode == TRIM_SCHED_LEARNED && D.model != nullptr) {
        bool in_range = false;
        float conf = 0.0f;
#if TRIM_MODES & 8
        const uint32_t learned = mlp_choice(D, f, &in_range, &conf);
#else
        const uint32_t learned = next;
#endif
        if (in_range) {
          next = learned;
          confident = D.commit_confidence > 0.0f && conf >= D.commit_confidence;
        }
      }
    }
    // rounds in a row with an unchanged choice. After commit_after of them
    // (or a learned choice at or above commit_confidence) the run commits: the
    // next recheck_rounds rounds (doubling while the same commit repeats) run
    // the variant without consulting the scheduler or gathering features, and
    // the count stays one short of a commit, so that the first consulted round
    // after the stretch re-commits if the scheduler keeps the variant.
    if (!consult) {
      L.stable = D.commit_after ? D.commit_after - 1u : 0u;
    } else {
      L.stable = (r >= 1 && next == L.variant) ? L.stable + 1u : 1u;
      if (confident) L.stable = max(L.stable, D.commit_after);
      L.cstop = 0u;
      if (D.commit_after != 0u && L.stable >= D.commit_after) {
        const uint32_t p0 = D.recheck_rounds ? D.recheck_rounds : 1u;
        const uint32_t p = (next == L.clast && L.cperiod) ? min(L.cperiod * 2u, 1u << 30) : p0;
        L.cperiod = p;
        L.clast = next;
        const unsigned long long stop = (unsigned long long)r + 1u + p;
        L.cstop = stop > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)stop;
        L.stable = D.commit_after - 1u;
        if (cta0 && r == 0u) C->commit_round0 = 1u;
      }
      if (cta0) C->consults += 1u;
    }
    L.prev_variant = (r >= 1) ? L.variant : NIL;
    L.fprev = L.fe - L.fb;  // frontier of round r, for the timing feature two rounds on
    L.variant = next;
    if (next != TRIM_AC4_PUSH) L.mixed = 1;
    L.round = r + 1;
    L.fb = L.fe;
    L.fe = len;
    L.w_end = w_end;
    L.e_end = e_end;
    if (next == TRIM_AC3_PULL) L.live_out = (L.ac3_list == NIL) ? 0u : (L.ac3_list ^ 1u);
    for (int i = 0; i < NFEAT; ++i) L.feat[i] = f[i];
  }
  __syncwarp();
  if (lane == 0) {
    B.S = L;
    B.err = err;
  }
}

// CTA 0, start of round k: timestamp, and zero the accumulator slot of round k+2.
__device__ __forceinline__ void start_round(const Dev& D, uint32_t k) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    D.C->t_round[k & 3] = globaltimer();
    RoundStat* z = &D.C->rs[(k + 2) & 3];
    z->sum_in = 0; z->sum_out = 0;
    z->hist[0] = z->hist[1] = z->hist[2] = 0;
    z->live_count = 0;
    z->max_din = 0;
  }
}

// ------------------------------------------------------------------ AC-4

// AC-4 push: decrement the counters of the predecessors of every removed vertex
// not yet pushed, i.e. the in-edges [e_c4, e_end) of the work list. The edges are
// cut into 32-edge chunks and each warp takes an equal run of chunks, so a hub's
// in-edges spread over many warps. The owner of a chunk's first edge comes from
// chunk_first; the next 31 work-list entries own the rest of the chunk (every
// entry has at least one edge), and a shuffle search finds each lane's owner.
__device__ ROUND_FN void ac4_round(const Dev& D, Cta& B, const Sched& S, uint32_t gwarp,
                                   uint32_t nwarps) {
  constexpr int U = 4;  // chunks in flight per warp
  Counters K;
  const unsigned lane = lane_id();
  const uint32_t r = S.round;
  // a vertex whose counter reaches zero is still live unless another variant
  // ran (also in the AC-4-only flavour: a committed stretch of a scheduled run
  // may follow AC-6 or AC-3 rounds, whose removals AC-4 has not yet pushed)
  const bool check = S.mixed;
  const uint32_t ea = S.e_c4, eb = S.e_end, ia = S.c4w, ib = S.w_end;
  if (eb <= ea) return;
  // A small round (at most one entry and one 32-edge chunk per warp) whose
  // entries all have few in-edges gives each warp one work-list entry: its row
  // and edge range come with one load, no chunk-owner lookup, and the warp
  // walks the entry's in-edges 32 at a time (at most 8 steps).
  if (ib - ia <= nwarps && eb - ea <= 32u * nwarps && S.bmax <= 256u) {
    // warp w of CTA c takes entry w * grid + c: a small round's entries (and
    // the memory requests they cause) spread over every SM
    const uint32_t j = ia + (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    if (j < ib) {
      const uint32_t row = ldcg(&D.w4_row[j]);
      const uint32_t eo = ldcg(&D.w4_eoff[j]);
      const uint32_t ee = (j + 1u < ib) ? ldcg(&D.w4_eoff[j + 1u]) : eb;
      for (uint32_t k0 = eo; k0 < ee; k0 += 32u) {
        const uint32_t e = k0 + lane;
        const bool valid = e < ee;
        const uint32_t u = valid ? __ldg(&D.itgt[row + (e - eo)]) : 0u;
        const uint32_t old = valid ? atomicSub(&D.cnt[u], 1u) : 0u;
        K.pushed += valid ? 1 : 0;
        bool pred = valid && old == 1u;
        if (pred && check) pred = ldcg(&D.level[u]) == LIVE;
        append_dead(D, B, pred, u, r, D.live0);
      }
    }
    stats_flush(D, B, K);
    return;
  }
  const uint32_t c0 = ea >> 5, c1 = (eb + 31u) >> 5;
  const uint32_t per = (c1 - c0 + nwarps - 1) / nwarps;
  const uint32_t cb = c0 + gwarp * per, ce = min(c1, cb + per);
  uint32_t cfb = 0;
  for (uint32_t c = cb; c < ce; c += U) {
    const uint32_t k = (c - cb) & 31u;
    if (k == 0u) cfb = (c + lane < ce) ? ldcg(&D.chunk_first[c + lane]) : 0u;
    uint32_t wrow[U], weo[U], u[U], old[U];
    bool valid[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const uint32_t first = max(__shfl_sync(FULL, cfb, (k + q) & 31u), ia);
      const uint32_t ii = first + lane;
      const bool in = c + q < ce && ii < ib;
      wrow[q] = in ? ldcg(&D.w4_row[ii]) : 0u;
      weo[q] = in ? ldcg(&D.w4_eoff[ii]) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const uint32_t e = ((c + q) << 5) + lane;
      valid[q] = c + q < ce && e >= ea && e < eb;
      const unsigned j = owner_of(weo[q], e);
      const uint32_t idx = __shfl_sync(FULL, wrow[q], j) + (e - __shfl_sync(FULL, weo[q], j));
      u[q] = valid[q] ? __ldg(&D.itgt[idx]) : 0u;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) old[q] = valid[q] ? atomicSub(&D.cnt[u[q]], 1u) : 0u;
#pragma unroll
    for (int q = 0; q < U; ++q) {
      K.pushed += valid[q] ? 1 : 0;
      bool pred = valid[q] && old[q] == 1u;
      if (pred && check) pred = ldcg(&D.level[u[q]]) == LIVE;
      append_dead(D, B, pred, u[q], r, D.live0);
    }
  }
  stats_flush(D, B, K);
}

#if TRIM_LOCAL
// ------------------------------------------------------------------ local AC-4 rounds

// End of a local stretch that returns to ordinary rounds (all threads): the
// queued vertices of round r (buffer b) become work-list entries, and the round
// ends like an ordinary one (flush, grid barrier, advance). A rare path, out of
// line in the scheduler flavour so that its flush and scheduler code add no
// registers to the local rounds.
#if TRIM_MODES & 8
__device__ __noinline__
#else
__device__ __forceinline__
#endif
void local_leave(const Dev& D, Cta& B, uint32_t b, uint32_t r) {
  const unsigned lane = lane_id();
  const uint32_t ne = B.lq_vend[b];
  for (uint32_t i0 = (threadIdx.x >> 5) * 32u; i0 < ne; i0 += blockDim.x) {
    const uint32_t i = i0 + lane;
    const bool has = i < ne;
    append_w4(D, B, has, has ? B.lq_row[b][i] : 0u, has ? B.lq_din[b][i] : 0u, r);
  }
  flush_round(D, B, r, D.live0);
  if ((D.flags & F_ROUND_LOG) && blockIdx.x == 0 && threadIdx.x == 0)
    D.C->t_flush[r & 3] = globaltimer();
  if (!grid_barrier(D, B, false)) return;
  if (threadIdx.x < 32) advance(D, B);
  __syncthreads();
}

// Does round S.round start a stretch of local rounds? Its pending work-list
// entries (the stretch's first round gives each warp whole entries) must have
// at most local_edges_max in-edges in all, none more than 256.
__device__ __forceinline__ bool local_start(const Dev& D, const Sched& S) {
  if (D.local_edges_max == 0u || S.variant != TRIM_AC4_PUSH) return false;
  // with the schedulers: inside a committed stretch only, whose last round
  // (the one the scheduler reads features of) runs as an ordinary round
  if ((MODES & M_SCHED) && !(S.cstop != 0u && S.round + 1u < S.cstop)) return false;
  const uint32_t edges = S.e_end - S.e_c4;
  return edges <= D.local_edges_max && S.bmax <= 256u;
}

// Thread 0: closes local round L.round, in which nF vertices were removed, all
// of them counted only by the local barrier (the schedule step of advance()
// for a round of the AC-4-only flavour, without reading the control block).
__device__ void local_close(const Dev& D, Cta& B, uint32_t nF) {
  Sched& L = B.S;
  const uint32_t r = L.round;
  L.vcount[TRIM_AC4_PUSH] += 1u;
  L.c4w = L.w_end;  // the stretch's first round pushed every pending entry
  L.e_c4 = L.e_end;
  L.bmax = 0u;
  L.skew += nF;
  if (blockIdx.x == 0) {
    Ctrl* C = D.C;
    C->vcount[TRIM_AC4_PUSH] = L.vcount[TRIM_AC4_PUSH];
    C->rounds = nF ? r + 1u : r;
    C->n_dead = L.fe + nF;
    C->local_rounds = L.lround;
    if ((D.flags & F_ROUND_LOG) && D.rlog != nullptr && r >= 1u && r - 1u < D.rlog_cap) {
      trim_round_rec_t* rec = &D.rlog[r - 1u];
      rec->round = r;
      rec->variant = TRIM_AC4_PUSH;
      rec->frontier = L.fe - L.fb;
      rec->removed = nF;
      rec->t_start_ns = C->t_round[r & 3];
      rec->t_end_ns = globaltimer();
      rec->t_work_ns = C->t_work[r & 3];
      rec->t_flush_ns = rec->t_work_ns;  // a local round moves nothing to global lists
      for (int i = 0; i < NFEAT; ++i) rec->features[i] = L.feat[i];  // that chose round r
      C->rlog_len = r;
    }
  }
  // round r+1 is chosen without the scheduler (a committed or fixed variant;
  // a flavour without the schedulers never sets features)
  if (MODES & M_SCHED)
    for (int i = 0; i < NFEAT; ++i) L.feat[i] = 0.0f;
  if (nF == 0u) {
    L.done = 1u;
    return;
  }
  L.stable = D.commit_after ? D.commit_after - 1u : 0u;  // as advance() in this flavour
  L.prev_variant = TRIM_AC4_PUSH;
  L.fprev = L.fe - L.fb;
  L.round = r + 1u;
  L.fb = L.fe;
  L.fe += nF;
}

// End of local round r (all threads): one arrival per CTA on the barrier word
// of this round's parity, carrying 2^48 + 2^32 * (overflowed) + the CTA's local
// removals; the wait ends when the word has grown by gridDim.x arrivals since
// its value after its previous round (lbase), and that growth is the round's
// totals. A slot is reused two rounds later, when every CTA has read it. The
// wait is bounded like grid_barrier's. Thread 0 then decides how the stretch
// goes on (B.lq_next: LQ_GO on, LQ_DONE the run is over, both after closing
// the round; LQ_LEAVE back to ordinary rounds). Returns false on a timeout.
constexpr uint32_t LQ_GO = 0, LQ_DONE = 1, LQ_LEAVE = 2;
__device__ bool local_barrier(const Dev& D, Cta& B, uint32_t b, uint32_t r) {
  __syncthreads();
  if (threadIdx.x == 0) {
    Sched& S = B.S;
    const uint32_t slot = S.lround & 1u;
    if (((MODES & M_SCHED) || (D.flags & F_LIVE_EDGES)) && B.lq_pushed)
      atomicAdd(&D.C->local_edges, (unsigned long long)B.lq_pushed);
    const unsigned long long add =
        (1ull << 48) | ((unsigned long long)B.lq_ovf << 32) | (unsigned long long)B.lq_k;
    const unsigned long long base = S.lbase[slot];
    // No fence before the arrival: across a local barrier CTAs exchange nothing
    // through plain memory, only counter decrements, and every decrement of
    // this round has returned its value (it is performed at L2) before this
    // arrival is issued. Levels written here are read after the kernel or
    // after an ordinary (fenced) barrier.
    red_relaxed_add64(&D.C->lbar[slot], add);
    const uint64_t t0 = globaltimer();
    // relaxed polls: an acquiring load would also invalidate this SM's L1 on
    // every iteration, and nothing read after this barrier needs it
    unsigned long long cur = ld_relaxed64(&D.C->lbar[slot]);
    while ((uint32_t)((cur - base) >> 48) != gridDim.x) {
      if (globaltimer() - t0 > D.spin_limit_ns) {
        set_error(D, TRIM_ERR_TIMEOUT, 2);
        B.err = TRIM_ERR_TIMEOUT;
        break;
      }
      cur = ld_relaxed64(&D.C->lbar[slot]);
    }
    const unsigned long long d = cur - base;
    S.lbase[slot] = cur;
    S.lround += 1u;
    const uint32_t nF = (uint32_t)d, n_ovf = (uint32_t)(d >> 32) & 0xFFFFu;
    // the stretch ends before the last round of a committed stretch (the
    // scheduler reads its features) and, where the asynchronous tail may take
    // over, before round ASYNC_MIN_ROUND (it starts from the work list)
    const bool stop = ((MODES & M_SCHED) && r + 1u >= S.cstop) ||
                      (D.async_edges_max != 0u && !(D.flags & F_ROUND_LOG) && !S.mixed &&
                       r + 1u == ASYNC_MIN_ROUND);
    if (n_ovf == 0u && (nF == 0u || !stop)) {
      local_close(D, B, nF);  // every removal of the round is in the queues
      B.lq_next = nF ? LQ_GO : LQ_DONE;
    } else {
      S.skew += nF;  // advance() closes the round after the work-list handover
      if (blockIdx.x == 0) D.C->local_rounds = S.lround;
      B.lq_next = LQ_LEAVE;
    }
    // the next round fills the buffer this round read
    B.lq_cnt[b ^ 1u] = 0ull;
    B.lq_vend[b ^ 1u] = 0u;
    B.lq_k = 0u;
    B.lq_ovf = 0u;
    B.lq_pushed = 0u;
  }
  __syncthreads();
  return B.err == 0u;
}

// Runs local rounds from round B.S.round on: the first pushes the pending
// work-list entries (one per warp), later ones the predecessors in the CTA's
// queue; every decrement loads the G^T row bounds of its vertex alongside the
// atomic, so a removal costs no further dependent load before its row is
// queued. The stretch ends when a round removes nothing (the run is done),
// when a round overflowed the queues, or (with the schedulers) before the last
// round of the committed stretch; in the last
// two cases the queued vertices join the global work list and the round ends
// like an ordinary one (flush, grid barrier, advance). Returns false on a
// timeout.
__device__ __noinline__ bool local_stretch(const Dev& D, Cta& B) {
  Counters K;
  const unsigned lane = lane_id();
  bool first = true;
  while (true) {
    const uint32_t r = B.S.round;
    const uint32_t b = B.S.lround & 1u;
    const bool check = B.S.mixed;
    start_round(D, r);
    if (first) {
      const uint32_t ia = B.S.c4w, ib = B.S.w_end, eb = B.S.e_end;
      const uint32_t nw = gridDim.x * (blockDim.x >> 5);
      for (uint32_t j = ia + (threadIdx.x >> 5) * gridDim.x + blockIdx.x; j < ib; j += nw) {
        const uint32_t row = ldcg(&D.w4_row[j]);
        const uint32_t eo = ldcg(&D.w4_eoff[j]);
        const uint32_t ee = (j + 1u < ib) ? ldcg(&D.w4_eoff[j + 1u]) : eb;
        for (uint32_t k0 = eo; k0 < ee; k0 += 32u) {
          const uint32_t e = k0 + lane;
          const bool valid = e < ee;
          const uint32_t u = valid ? __ldg(&D.itgt[row + (e - eo)]) : 0u;
          const uint32_t p0 = valid ? __ldg(&D.ioff[u]) : 0u;
          const uint32_t p1 = valid ? __ldg(&D.ioff[u + 1u]) : 0u;
          const uint32_t old = valid ? atomicSub(&D.cnt[u], 1u) : 0u;
          K.pushed += valid ? 1u : 0u;
          bool pred = valid && old == 1u;
          if (pred && check) pred = ldcg(&D.level[u]) == LIVE;
          local_append(D, B, pred, u, r, p0, p1 - p0, b);
        }
      }
    } else {
      const uint32_t qb = b ^ 1u;
      const uint32_t qe = (uint32_t)(B.lq_cnt[qb] >> 32);
      for (uint32_t base = 0; base < qe; base += 2u * blockDim.x) {  // CTA-uniform
        uint32_t u[2], p0[2], p1[2], old[2];
        bool valid[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const uint32_t k = base + (uint32_t)q * blockDim.x + threadIdx.x;
          valid[q] = k < qe;
          u[q] = valid[q] ? B.lq_ids[qb][k] : 0u;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          p0[q] = valid[q] ? __ldg(&D.ioff[u[q]]) : 0u;
          p1[q] = valid[q] ? __ldg(&D.ioff[u[q] + 1u]) : 0u;
          old[q] = valid[q] ? atomicSub(&D.cnt[u[q]], 1u) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          K.pushed += valid[q] ? 1u : 0u;
          bool pred = valid[q] && old[q] == 1u;
          if (pred && check) pred = ldcg(&D.level[u[q]]) == LIVE;
          local_append(D, B, pred, u[q], r, p0[q], p1[q] - p0[q], b);
        }
      }
      if (threadIdx.x == 0) B.lq_pushed = qe;
    }
    if ((D.flags & F_ROUND_LOG) && blockIdx.x == 0) {
      __syncthreads();
      if (threadIdx.x == 0) D.C->t_work[r & 3] = globaltimer();
    }
    if (!local_barrier(D, B, b, r)) break;
    const uint32_t next = B.lq_next;
    if (next == LQ_DONE) break;
    if (next == LQ_GO) {
      first = false;
      continue;
    }
    local_leave(D, B, b, r);
    break;
  }
  stats_flush(D, B, K);
  return B.err == 0u;
}

// ------------------------------------------------------- asynchronous AC-4 tail
//
// A vertex's level is one more than the top level among its successors
// (Definition 2: round r removes the vertices whose successors were all
// removed before round r, the last of them in round r - 1). The pushes can
// carry that maximum, and then the rest of an AC-4 run needs no rounds at all.
// Every vertex gets one 64-bit word, (top level pushed so far << 32 |
// live-successor counter); the push from a removed vertex of level l replaces
// it by (max(top, l) << 32 | counter - 1) in one compare-and-swap, and the
// push that takes the counter to zero removes the vertex with level
// max(top, l) + 1: every successor has pushed by then, so the maximum is over
// all of them, whatever the order of the pushes. No CTA waits for another:
// each runs steps of its own. A step pushes the predecessors queued in the
// CTA's shared memory (the G^T rows of the vertices it removed in its previous
// step, each with its vertex's level) and queues those of the vertices it
// removes now.
//
// A removed vertex's row stays with the CTA whose push removed it, and that
// CTA is one of its successors' CTAs: over many levels the work drifts onto
// fewer and fewer CTAs. A CTA whose queue holds far more than its share, or
// whose removals do not fit its queue (those rows go to a global list of
// pieces of at most kAsyncPiece in-edges), asks for a rebalance: every CTA
// joins at its next step boundary, writes its queued entries to a global list,
// and after a grid barrier each takes an even slice of those entries and of
// the pieces written since the last rebalance, then a second barrier closes
// the rebalance (counts published, the lists' counters ready for the next).
// The tail ends when no CTA has work: a token count holds one token per CTA
// with work; a CTA releases its token when its queue runs empty, and a count
// of zero (with no rebalance asked for) ends the run.
//
// It takes over at the start of an AC-4 round r (r >= ASYNC_MIN_ROUND) whose
// pending work-list entries are exactly the vertices removed in round r - 1,
// at most async_edges_max in-edges, and runs the rest of the run (with the
// schedulers: only inside a committed stretch, as the scheduler is not
// consulted again). Rounds before ASYNC_MIN_ROUND stay rounds (local ones
// where they can): on graphs that peel in fewer rounds they were faster.
__device__ __forceinline__ bool async_start(const Dev& D, const Sched& S) {
  if (D.async_edges_max == 0u || S.variant != TRIM_AC4_PUSH || S.mixed) return false;
  if ((D.flags & F_ROUND_LOG) || S.round < ASYNC_MIN_ROUND) return false;
  if (S.prev_variant != TRIM_AC4_PUSH) return false;
  if ((MODES & M_SCHED) && D.mode > TRIM_AC3_PULL && !(S.cstop != 0u && S.round < S.cstop))
    return false;
  return S.e_end - S.e_c4 <= D.async_edges_max && S.bmax <= 256u;
}

// Warp-collective: lanes with ovf set removed a vertex (G^T row start row,
// in-degree din, level lev) whose row goes to the global list of pieces, cut
// into pieces of at most kAsyncPiece in-edges; the CTA then asks for a
// rebalance. The pieces are read only after the rebalance's grid barrier.
__device__ __noinline__ void async_spill(const Dev& D, Cta& B, bool ovf, uint32_t row,
                                         uint32_t din, uint32_t lev) {
  const unsigned lane = lane_id();
  const uint32_t np = ovf ? (din + kAsyncPiece - 1u) / kAsyncPiece : 0u;
  const uint32_t incl = warp_incl_scan(np);
  const uint32_t tot = __shfl_sync(FULL, incl, 31);
  uint32_t s = 0;
  if (lane == 0) {
    s = atomicAdd(&D.C->oq_res, tot);
    B.a_want = 1u;
  }
  s = __shfl_sync(FULL, s, 0);
  // (cannot fail: every removal adds at most ceil(din / kAsyncPiece) pieces)
  if ((uint64_t)s + tot > D.oq_cap) {
    if (lane == 0) set_error(D, TRIM_ERR_STATE, 5);
    return;
  }
  if (ovf) {
    const uint32_t at = s + incl - np;
    for (uint32_t i = 0; i < np; ++i) {
      D.oq_row[at + i] = row + i * kAsyncPiece;
      D.oq_len[at + i] = min(kAsyncPiece, din - i * kAsyncPiece);
      D.oq_lev[at + i] = lev;
    }
  }
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Warp-collective: lanes with `removed` set removed vertex p with level lev
// (G^T row start row, in-degree din). The level is written and the
// predecessors are queued in buffer nxt with that level, all of the warp's
// rows at once (each lane loads entries of the flattened rows), each
// predecessor's word and row bounds prefetched into L2 for the step that
// pushes it; a row longer than AQ_LOCAL_DMAX, or one that does not fit, goes
// to the global pieces.
__device__ __forceinline__ void async_append(const Dev& D, Cta& B, bool removed, uint32_t p,
                                             uint32_t lev, uint32_t row, uint32_t din,
                                             uint32_t nxt, uint32_t QA) {
  const unsigned lane = lane_id();
  const unsigned mask = __ballot_sync(FULL, removed);
  if (mask == 0u) return;
  if (removed) D.level[p] = lev;
  const uint32_t top = __reduce_max_sync(FULL, removed ? lev : 0u);
  if (lane == 0) {
    atomicAdd(&B.a_removed, (unsigned)__popc(mask));
    atomicMax(&B.a_maxlev, top);
  }
  const bool want = removed && din > 0u && din <= AQ_LOCAL_DMAX;
  bool ovf = removed && din > AQ_LOCAL_DMAX;
  const unsigned wm = __ballot_sync(FULL, want);
  if (wm) {
    const unsigned ew = want ? din : 0u;
    const unsigned eincl = warp_incl_scan(ew);
    const unsigned esum = __shfl_sync(FULL, eincl, 31);
    const unsigned excl = eincl - ew;
    uint32_t be = 0;
    if (lane == 0) be = atomicAdd(&B.aq_res[nxt], esum);
    be = __shfl_sync(FULL, be, 0);
    if ((uint64_t)be + esum <= QA) {  // warp-uniform
      if (lane == 0) atomicMax(&B.aq_end[nxt], be + esum);
      uint32_t* ids = dyn_smem + nxt * QA;
      uint32_t* lv = dyn_smem + (2u + nxt) * QA;
      for (uint32_t j0 = 0; j0 < esum; j0 += 128u) {
        uint32_t t[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t j = j0 + (uint32_t)q * 32u + lane;
          const unsigned o = owner_of(excl, j);
          const uint32_t ro = __shfl_sync(FULL, row, o), xo = __shfl_sync(FULL, excl, o);
          l[q] = __shfl_sync(FULL, lev, o);
          t[q] = j < esum ? __ldg(&D.itgt[ro + (j - xo)]) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t j = j0 + (uint32_t)q * 32u + lane;
          if (j < esum) {
            ids[be + j] = t[q];
            lv[be + j] = l[q];
            prefetch_l2(&D.aw[t[q]]);  // for the step that pushes it
            prefetch_l2(&D.ioff[t[q]]);
          }
        }
      }
    } else {
      ovf = ovf || want;
    }
  }
  if (__ballot_sync(FULL, ovf)) async_spill(D, B, ovf, row, din, lev);
}

// Warp-collective: pushes from removed vertices to their predecessors p[q]
// (lanes with valid[q] set), each carrying its removed vertex's level l[q],
// by compare-and-swap on the predecessors' words; the row bounds of every
// predecessor load alongside its word, so a removal costs no further
// dependent load before its row is queued. A word whose counter is zero
// belongs to a vertex that is not live (masked): it is left alone.
template <int Q>
__device__ __forceinline__ void async_push(const Dev& D, Cta& B, const bool (&valid)[Q],
                                           const uint32_t (&p)[Q], const uint32_t (&l)[Q],
                                           uint32_t nxt, uint32_t QA, Counters& K) {
  unsigned long long w[Q];
  uint32_t p0[Q], p1[Q], lev[Q];
  bool pend[Q], removed[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    w[q] = valid[q] ? ld_relaxed64(&D.aw[p[q]]) : 0ull;
    p0[q] = valid[q] ? __ldg(&D.ioff[p[q]]) : 0u;
    p1[q] = valid[q] ? __ldg(&D.ioff[p[q] + 1u]) : 0u;
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    pend[q] = valid[q] && (uint32_t)w[q] != 0u;
    removed[q] = false;
    lev[q] = 0u;
    K.pushed += valid[q] ? 1u : 0u;
  }
  // a failed compare-and-swap means another push on the same word succeeded,
  // so the loop ends; the bound only guards against a broken invariant
  for (uint32_t it = 0;; ++it) {
    bool any = false;
#pragma unroll
    for (int q = 0; q < Q; ++q) any = any || pend[q];
    if (!__any_sync(FULL, any)) break;
    if (it == (1u << 22)) {
      if (lane_id() == 0) set_error(D, TRIM_ERR_TIMEOUT, 6);
      break;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (!pend[q]) continue;
      const uint32_t top = max((uint32_t)(w[q] >> 32), l[q]);
      const uint32_t cnt = (uint32_t)w[q];
      const unsigned long long nw = ((unsigned long long)top << 32) | (cnt - 1u);
      const unsigned long long prev = atomicCAS(&D.aw[p[q]], w[q], nw);
      if (prev == w[q]) {
        pend[q] = false;
        removed[q] = cnt == 1u;
        lev[q] = top + 1u;
      } else {
        w[q] = prev;
        if ((uint32_t)prev == 0u) pend[q] = false;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q)
    async_append(D, B, removed[q], p[q], lev[q], p0[q], p1[q] - p0[q], nxt, QA);
}

// Warp-collective: pushes the in-edges [row, row + len) of G^T, all carrying level l.
__device__ __forceinline__ void async_piece(const Dev& D, Cta& B, uint32_t row, uint32_t len,
                                            uint32_t l, uint32_t nxt, uint32_t QA,
                                            Counters& K) {
  const unsigned lane = lane_id();
  for (uint32_t k0 = 0; k0 < len; k0 += 64u) {
    bool valid[2];
    uint32_t p[2], lv[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint32_t e = k0 + (uint32_t)q * 32u + lane;
      valid[q] = e < len;
      p[q] = valid[q] ? __ldg(&D.itgt[row + e]) : 0u;
      lv[q] = l;
    }
    async_push<2>(D, B, valid, p, lv, nxt, QA, K);
  }
}

// All threads: pushes the entries [lo, hi) of a list of (predecessor, level)
// pairs, two per thread at a time (warps past the end skip the pass).
__device__ __forceinline__ void async_entries(const Dev& D, Cta& B, const uint32_t* ids,
                                              const uint32_t* lv, uint32_t lo, uint32_t hi,
                                              bool global, uint32_t nxt, uint32_t QA,
                                              Counters& K) {
  for (uint32_t base = lo; base < hi; base += 2u * blockDim.x) {  // CTA-uniform
    if (base + (threadIdx.x & ~31u) >= hi) break;  // (warp-uniform: later bases are larger)
    bool valid[2];
    uint32_t p[2], l[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint32_t k = base + (uint32_t)q * blockDim.x + threadIdx.x;
      valid[q] = k < hi;
      p[q] = valid[q] ? (global ? ldcg(&ids[k]) : ids[k]) : 0u;
      l[q] = valid[q] ? (global ? ldcg(&lv[k]) : lv[k]) : 0u;
    }
    async_push<2>(D, B, valid, p, l, nxt, QA, K);
  }
}

constexpr uint32_t AS_STEP = 0, AS_DONE = 1, AS_REBALANCE = 2;

// Thread 0: releases this CTA's token, after publishing its removals and top
// level (CTA 0 reads the totals once the token count is zero).
__device__ __forceinline__ void async_release(const Dev& D, Cta& B) {
  Ctrl* C = D.C;
  if (B.a_removed) {
    atomicAdd(&C->a_removed, B.a_removed);
    atomicMax(&C->a_maxlev, B.a_maxlev);
    B.a_removed = 0u;
    B.a_maxlev = 0u;
  }
  fence_acq_rel();  // the counts before the release
  atomicSub(&C->a_tokens, 1u);
  B.a_token = 0u;
}

// Thread 0, before each step: buffer cur holds the predecessors the next step
// pushes. A CTA with work asks for a rebalance when its removals did not fit
// its queue or its queue holds more than max(half its threads, 2 x the
// average share at the last rebalance): steps stay short (a step takes as long
// as its CTA's slowest chain of loads, and one push per thread or less keeps
// that to a single pass), and joins one when the hints (the requested
// generation and the error flag, loaded during the previous step) show one. A
// CTA without work publishes its counts, releases its token, and waits until
// a rebalance is asked for or the token count is zero (the run is over). The
// wait is bounded: spin_limit_ns without a heartbeat from a working CTA
// (every 256 of its steps) ends the run with TRIM_ERR_TIMEOUT.
__device__ void async_decide(const Dev& D, Cta& B, uint32_t cur, uint32_t h_req,
                             uint32_t h_err) {
  Ctrl* C = D.C;
  B.aq_res[cur ^ 1u] = 0u;  // read by the previous step: the next one fills it
  B.aq_end[cur ^ 1u] = 0u;
  B.sh_elo = B.sh_ehi = B.sh_plo = B.sh_phi = 0u;  // the last rebalance's share is pushed
  B.a_next = AS_STEP;
  const uint32_t qe = B.aq_end[cur];
  const bool over = qe > max(blockDim.x / 2u, 2u * B.a_avg);
  if (qe != 0u || B.a_want) {
    if ((++B.a_steps & 255u) == 0u) red_relaxed_add(&C->a_beat, 1u);
    if (h_err != 0u) {
      B.err = h_err;
      B.a_next = AS_DONE;
    } else if (B.a_want || over) {
      atomicMax(&C->a_req, B.a_gen + 1u);
      B.a_next = AS_REBALANCE;
    } else if ((int)(h_req - B.a_gen) > 0) {
      B.a_next = AS_REBALANCE;
    }
    return;
  }
  if (B.a_token) async_release(D, B);
  uint64_t t0 = globaltimer();
  uint32_t beat = ld_relaxed(&C->a_beat);
  while (true) {
    const uint32_t err = ld_relaxed(&C->err);
    const uint32_t req = ld_relaxed(&C->a_req);
    const uint32_t tok = ld_relaxed(&C->a_tokens);
    const uint32_t bt = ld_relaxed(&C->a_beat);
    if (err != 0u) {
      B.err = err;
      B.a_next = AS_DONE;
      return;
    }
    if ((int)(req - B.a_gen) > 0) {
      B.a_next = AS_REBALANCE;
      return;
    }
    // (a CTA that asks for a rebalance holds its token until the rebalance,
    // so a zero count means no rebalance can come)
    if (tok == 0u) {
      B.a_next = AS_DONE;
      return;
    }
    const uint64_t now = globaltimer();
    if (bt != beat) {
      beat = bt;
      t0 = now;
    } else if (now - t0 > D.spin_limit_ns) {
      set_error(D, TRIM_ERR_TIMEOUT, 4);
      B.err = TRIM_ERR_TIMEOUT;
      B.a_next = AS_DONE;
      return;
    }
    __nanosleep(256);
  }
}

// All threads, every CTA (generation g = B.a_gen): writes the entries of
// buffer cur to the global entry list of parity g & 1; after a grid barrier
// every CTA takes an even slice of those entries and of the pieces written
// since the last rebalance; tokens follow the new shares and CTA 0 clears the
// other parity's list (last read after rebalance g - 1, by every CTA before
// this rebalance's first barrier); a second barrier publishes both before any
// CTA writes to the lists again. Returns false on an error.
__device__ __noinline__ bool async_rebalance(const Dev& D, Cta& B, uint32_t cur, uint32_t QA) {
  Ctrl* C = D.C;
  const uint32_t par = B.a_gen & 1u;
  const uint32_t qe = B.aq_end[cur];
  uint32_t* eid = D.ae_id + (size_t)par * D.ae_cap;
  uint32_t* elv = D.ae_lev + (size_t)par * D.ae_cap;
  if (threadIdx.x == 0) {
    B.a_base = qe ? atomicAdd(&C->e_n[par], qe) : 0u;
    // (cannot fail: a list holds every CTA's whole queue)
    if ((uint64_t)B.a_base + qe > D.ae_cap) set_error(D, TRIM_ERR_STATE, 7);
  }
  __syncthreads();
  const uint32_t base = B.a_base;
  if ((uint64_t)base + qe <= D.ae_cap) {
    const uint32_t* ids = dyn_smem + cur * QA;
    const uint32_t* lv = dyn_smem + (2u + cur) * QA;
    for (uint32_t k = threadIdx.x; k < qe; k += blockDim.x) {
      eid[base + k] = ids[k];
      elv[base + k] = lv[k];
    }
  }
  if (!grid_barrier(D, B)) return false;
  if (threadIdx.x == 0) {
    const uint64_t G = gridDim.x, b = blockIdx.x;
    const uint64_t tE = ld_relaxed(&C->e_n[par]);
    const uint32_t p_hi = ld_relaxed(&C->oq_res);
    const uint64_t tP = p_hi - B.a_plo;
    B.sh_elo = (uint32_t)(b * tE / G);
    B.sh_ehi = (uint32_t)((b + 1u) * tE / G);
    B.sh_plo = B.a_plo + (uint32_t)(b * tP / G);
    B.sh_phi = B.a_plo + (uint32_t)((b + 1u) * tP / G);
    B.a_plo = p_hi;
    const uint64_t avg = (tE + tP * kAsyncPiece) / G;
    B.a_avg = avg < (1u << 24) ? (uint32_t)avg : (1u << 24);
    B.aq_res[cur] = 0u;  // the queue went to the list
    B.aq_end[cur] = 0u;
    B.a_want = 0u;
    B.a_gen += 1u;
    const uint32_t busy = (B.sh_ehi > B.sh_elo || B.sh_phi > B.sh_plo) ? 1u : 0u;
    if (busy && !B.a_token) {
      atomicAdd(&C->a_tokens, 1u);
      B.a_token = 1u;
    } else if (!busy && B.a_token) {
      async_release(D, B);
    }
    if (blockIdx.x == 0) {
      C->e_n[par ^ 1u] = 0u;
      C->a_rebalances = B.a_gen;
    }
  }
  return grid_barrier(D, B);
}

// Runs the rest of the run asynchronously from round B.S.round = r0 (all
// threads): every vertex's word is set from its counter, the pending
// work-list entries (level r0 - 1) are pushed, one per warp, and then the
// CTA runs steps (and rebalances) until the token count is zero. CTA 0 then
// publishes the run's totals: alpha = top level + 1 (r0 if the tail removed
// nothing), and one AC-4 round for each of rounds r0 .. alpha. Returns false
// on an error.
__device__ __noinline__ bool async_tail(const Dev& D, Cta& B) {
  Counters K;
  Ctrl* C = D.C;
  const unsigned warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t QA = nw * D.sbuf_cap;  // entries per buffer: the four slices' space
  const uint32_t r0 = B.S.round;
  {
    // four counters per 16-byte load where both arrays allow it
    const bool vec = ((reinterpret_cast<uintptr_t>(D.cnt) | reinterpret_cast<uintptr_t>(D.aw)) & 15u) == 0u;
    const uint32_t n4 = vec ? D.n >> 2 : 0u, stride = gridDim.x * blockDim.x;
    const uint4* c4 = reinterpret_cast<const uint4*>(D.cnt);
    ulonglong2* w2 = reinterpret_cast<ulonglong2*>(D.aw);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const uint4 c = __ldcg(&c4[i]);
      w2[2u * i] = make_ulonglong2(c.x, c.y);
      w2[2u * i + 1u] = make_ulonglong2(c.z, c.w);
    }
    for (uint32_t v = (n4 << 2) + blockIdx.x * blockDim.x + threadIdx.x; v < D.n; v += stride)
      D.aw[v] = (unsigned long long)ldcg(&D.cnt[v]);
  }
  if (threadIdx.x == 0) {
    B.aq_res[0] = B.aq_res[1] = 0u;
    B.aq_end[0] = B.aq_end[1] = 0u;
    B.sh_elo = B.sh_ehi = B.sh_plo = B.sh_phi = 0u;
    B.a_removed = 0u;
    B.a_maxlev = 0u;
    B.a_token = 1u;
    B.a_steps = 0u;
    B.a_want = 0u;
    B.a_gen = 0u;
    B.a_plo = 0u;
    B.a_avg = (B.S.e_end - B.S.e_c4) / gridDim.x;
    if (blockIdx.x == 0) {
      C->a_tokens = gridDim.x;
      C->a_round = r0;
    }
  }
  if (!grid_barrier(D, B, false)) return false;
  {
    const uint32_t ia = B.S.c4w, ib = B.S.w_end, eb = B.S.e_end;
    for (uint32_t j = ia + warp * gridDim.x + blockIdx.x; j < ib; j += gridDim.x * nw) {
      const uint32_t row = ldcg(&D.w4_row[j]);
      const uint32_t eo = ldcg(&D.w4_eoff[j]);
      const uint32_t ee = (j + 1u < ib) ? ldcg(&D.w4_eoff[j + 1u]) : eb;
      async_piece(D, B, row, ee - eo, r0 - 1u, 0u, QA, K);
    }
  }
  uint32_t cur = 0, h_req = 0, h_err = 0;
  bool ok = true;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) async_decide(D, B, cur, h_req, h_err);
    __syncthreads();
    const uint32_t next = B.a_next;
    if (next == AS_DONE) break;
    if (next == AS_REBALANCE && !async_rebalance(D, B, cur, QA)) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0) {  // hints for the next decision, in flight during the step
      h_req = ld_relaxed(&C->a_req);
      h_err = ld_relaxed(&C->err);
    }
    const uint32_t nxt = cur ^ 1u;
    // a rebalance's share: entries of the global list, then pieces (one per warp)
    if (B.sh_ehi > B.sh_elo) {
      const size_t o = (size_t)((B.a_gen - 1u) & 1u) * D.ae_cap;
      async_entries(D, B, D.ae_id + o, D.ae_lev + o, B.sh_elo, B.sh_ehi, true, nxt, QA, K);
    }
    for (uint32_t i = B.sh_plo + warp; i < B.sh_phi; i += nw)
      async_piece(D, B, ldcg(&D.oq_row[i]), ldcg(&D.oq_len[i]), ldcg(&D.oq_lev[i]), nxt, QA, K);
    async_entries(D, B, dyn_smem + cur * QA, dyn_smem + (2u + cur) * QA, 0u, B.aq_end[cur],
                  false, nxt, QA, K);
    cur = nxt;
  }
  stats_flush(D, B, K);
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0 && ok && B.err == 0u) {
      fence_acq_rel();  // every CTA published its counts before its last release
      const uint32_t removed = ld_relaxed(&C->a_removed);
      const uint32_t top = ld_relaxed(&C->a_maxlev);
      Sched& S = B.S;
      const uint32_t alpha = removed ? max(r0, top + 1u) : r0;
      S.vcount[TRIM_AC4_PUSH] += alpha - r0 + 1u;
      C->vcount[TRIM_AC4_PUSH] = S.vcount[TRIM_AC4_PUSH];
      C->rounds = alpha;
      C->n_dead = S.fe + removed;
    }
    B.S.done = 1u;
  }
  __syncthreads();
  return ok && B.err == 0u;
}
#endif

#if TRIM_MODES & 16
// ------------------------------------------------------------------ in+out

// In+out round r (Section 4's remark: with G^T loaded a vertex also needs a
// live incoming edge): every vertex removed before round r and not yet pushed
// decrements the out-degree counter of each predecessor (its G^T row) and the
// in-degree counter of each successor (its G row). A counter that reaches zero
// removes its vertex in round r unless the vertex is already removed; when
// both of a vertex's counters reach zero in the same round, the first
// compare-and-swap of its level wins. Edges are balanced over the warps in
// 32-edge chunks as in ac4_round.
__device__ ROUND_FN void inout_round(const Dev& D, Cta& B, const Sched& S, uint32_t gwarp,
                                     uint32_t nwarps) {
  constexpr int U = 4;
  Counters K;
  const unsigned lane = lane_id();
  const uint32_t r = S.round;
  const uint32_t ea = S.e_c4, eb = S.e_end, ia = S.c4w, ib = S.w_end;
  if (eb <= ea) return;
  const uint32_t c0 = ea >> 5, c1 = (eb + 31u) >> 5;
  const uint32_t per = (c1 - c0 + nwarps - 1) / nwarps;
  const uint32_t cb = c0 + gwarp * per, ce = min(c1, cb + per);
  uint32_t cfb = 0;
  for (uint32_t c = cb; c < ce; c += U) {
    const uint32_t k = (c - cb) & 31u;
    if (k == 0u) cfb = (c + lane < ce) ? ldcg(&D.chunk_first[c + lane]) : 0u;
    uint32_t wrow[U], weo[U], worow[U], wdin[U], u[U], old[U];
    bool valid[U], pred_in[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const uint32_t first = max(__shfl_sync(FULL, cfb, (k + q) & 31u), ia);
      const uint32_t ii = first + lane;
      const bool in = c + q < ce && ii < ib;
      wrow[q] = in ? ldcg(&D.w4_row[ii]) : 0u;
      weo[q] = in ? ldcg(&D.w4_eoff[ii]) : 0xFFFFFFFFu;
      worow[q] = in ? ldcg(&D.w4_orow[ii]) : 0u;
      wdin[q] = in ? ldcg(&D.w4_din[ii]) : 0u;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const uint32_t e = ((c + q) << 5) + lane;
      valid[q] = c + q < ce && e >= ea && e < eb;
      const unsigned j = owner_of(weo[q], e);
      const uint32_t kk = e - __shfl_sync(FULL, weo[q], j);
      const uint32_t dj = __shfl_sync(FULL, wdin[q], j);
      const uint32_t rj = __shfl_sync(FULL, wrow[q], j), oj = __shfl_sync(FULL, worow[q], j);
      pred_in[q] = kk < dj;  // the edge lies in the entry's G^T row
      u[q] = !valid[q] ? 0u : pred_in[q] ? __ldg(&D.itgt[rj + kk]) : __ldg(&D.tgt[oj + (kk - dj)]);
    }
#pragma unroll
    for (int q = 0; q < U; ++q)
      old[q] = valid[q] ? atomicSub(pred_in[q] ? &D.cnt[u[q]] : &D.cnt_in[u[q]], 1u) : 0u;
#pragma unroll
    for (int q = 0; q < U; ++q) {
      K.pushed += (valid[q] && pred_in[q]) ? 1 : 0;
      K.edges += (valid[q] && !pred_in[q]) ? 1 : 0;
      const bool pred = valid[q] && old[q] == 1u && atomicCAS(&D.level[u[q]], LIVE, r) == LIVE;
      append_dead_io(D, B, pred, u[q], r, false, 0u, 0u, 0u, 0u);
    }
  }
  stats_flush(D, B, K);
}
#endif

// ------------------------------------------------------------------ AC-3

__device__ ROUND_FN void ac3_round(const Dev& D, Cta& B, const Sched& S, uint32_t gwarp,
                                   uint32_t nwarps) {
  Counters K;
  const unsigned lane = lane_id();
  const uint32_t r = S.round;
  const bool all = (S.ac3_list == NIL);
  const uint32_t* Lin = (S.ac3_list == 1u) ? D.live1 : D.live0;
  uint32_t* Lout = S.live_out ? D.live1 : D.live0;
  const uint32_t N = all ? D.n : S.live_in_len;
  for (uint32_t base = gwarp * 32; base < N; base += nwarps * 32) {
    const uint32_t idx = base + lane;
    const bool has = idx < N;
    const uint32_t v = has ? (all ? idx : ldcg(&Lin[idx])) : 0u;
    const bool alive = has && ldcg(&D.level[v]) == LIVE;
    uint32_t s = 0, d = 0, i0 = 0, i = 0;
    bool resolved = true;
    if (alive) {
      row_bounds(D, v, s, d);
      i0 = S.supp_valid ? ldcg(&D.supp[v]) : 0u;  // no support position yet: the row start
      i = scan_thread(D, v, s, d, i0, r, 2, resolved, K);
    }
    scan_warp_finish(D, resolved, v, s, d, i, r, K);
    const bool dies = alive && i >= d;
    const bool stays = alive && !dies;
    if (stays && (i != i0 || !S.supp_valid)) D.supp[v] = i;
    K.swept += has ? 1 : 0;
    append_dead(D, B, dies, v, r, Lout, false, false, 0, 0, d);
    append_live(D, B, stays, v, r, Lout);
  }
  stats_flush(D, B, K);
}

// ------------------------------------------------------------------ AC-6

// Warp-collective re-scan of members of a supporting set whose owner was
// removed in round r-1: scan forward from the position after the lost support;
// on success join the new support's set (intrusive list), else remove.
__device__ __forceinline__ void ac6_rescan(const Dev& D, Cta& B, bool valid, uint32_t v,
                                           uint32_t r, Counters& K) {
  const bool alive = valid && ldcg(&D.level[v]) == LIVE;
  uint32_t s = 0, d = 0, i = 0;
  bool resolved = true;
  if (alive) {
    row_bounds(D, v, s, d);
    i = scan_thread(D, v, s, d, ldcg(&D.supp[v]) + 1u, r, 2, resolved, K);
  }
  scan_warp_finish(D, resolved, v, s, d, i, r, K);
  const bool dies = alive && i >= d;
  if (alive && !dies) {
    D.supp[v] = i;
    const uint32_t t = row_target(D, v, s, i);
    D.s_next[v] = atomicExch(&D.s_head[t], v);
  }
  K.cand += valid ? 1 : 0;
  append_dead(D, B, dies, v, r, D.live0, false, false, 0, 0, d);
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024).
__device__ unsigned block_excl_scan(unsigned x, unsigned* total) {
  __shared__ unsigned wsum[33];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned incl = warp_incl_scan(x);
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned t = lane < nw ? wsum[lane] : 0u;
    const unsigned ti = warp_incl_scan(t);
    wsum[lane] = ti - t;
    if (lane == 31) wsum[32] = ti;
  }
  __syncthreads();
  const unsigned res = incl - x + wsum[warp];
  *total = wsum[32];
  __syncthreads();
  return res;
}

__device__ unsigned block_sum(unsigned x) {
  __shared__ unsigned ws[32];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  x = warp_sum(x);
  if (lane == 0) ws[warp] = x;
  __syncthreads();
  unsigned t = 0;
  if (warp == 0) {
    t = lane < nw ? ws[lane] : 0u;
    t = warp_sum(t);
    if (lane == 0) ws[0] = t;
  }
  __syncthreads();
  t = ws[0];
  __syncthreads();
  return t;
}

// AC-6 entry (the first AC-6 round, or the first after another variant ran):
// every live vertex re-checks its support position, joins the bulk supporting
// set of the support it keeps (a counting sort by support: count, grid-wide
// scan, scatter), or is removed. Three internal grid barriers.
__device__ ROUND_FN bool ac6_entry(const Dev& D, Cta& B, const Sched& S, uint32_t gwarp,
                                   uint32_t nwarps) {
  Counters K;
  const unsigned lane = lane_id();
  const uint32_t r = S.round, n = D.n;
  for (uint32_t base = gwarp * 32; base < n; base += nwarps * 32) {
    const uint32_t v = base + lane;
    const bool has = v < n;
    if (has) D.s_head[v] = NIL;
    const bool alive = has && ldcg(&D.level[v]) == LIVE;
    uint32_t s = 0, d = 0, i0 = 0, i = 0;
    bool resolved = true;
    if (alive) {
      row_bounds(D, v, s, d);
      i0 = S.supp_valid ? ldcg(&D.supp[v]) : 0u;  // no support position yet: the row start
      i = scan_thread(D, v, s, d, i0, r, 2, resolved, K);
    }
    scan_warp_finish(D, resolved, v, s, d, i, r, K);
    const bool dies = alive && i >= d;
    if (alive && !dies) {
      if (i != i0 || !S.supp_valid) D.supp[v] = i;
      const uint32_t t = row_target(D, v, s, i);
      D.s_next[v] = t;  // parked here until the scatter below
      atomicAdd(&D.s_cnt[t], 1u);
    }
    K.swept += has ? 1 : 0;
    append_dead(D, B, dies, v, r, D.live0, false, false, 0, 0, d);
  }
  stats_flush(D, B, K);
  if (!grid_barrier(D, B)) return false;
  // grid-wide exclusive scan of s_cnt into s_off
  const uint32_t chunk = ((n + gridDim.x - 1) / gridDim.x + 31) & ~31u;
  const uint32_t c0 = min(n, blockIdx.x * chunk), c1 = min(n, c0 + chunk);
  {
    unsigned acc = 0;
    for (uint32_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) acc += ldcg(&D.s_cnt[i]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) D.bsum[blockIdx.x] = acc;
  }
  if (!grid_barrier(D, B)) return false;
  {
    unsigned pre = 0;
    for (uint32_t j = threadIdx.x; j < blockIdx.x; j += blockDim.x) pre += ldcg(&D.bsum[j]);
    pre = block_sum(pre);
    for (uint32_t t0 = c0; t0 < c1; t0 += blockDim.x) {
      const uint32_t i = t0 + threadIdx.x;
      const unsigned x = i < c1 ? ldcg(&D.s_cnt[i]) : 0u;
      unsigned tot;
      const unsigned ex = block_excl_scan(x, &tot);
      if (i < c1) D.s_off[i] = pre + ex;
      pre += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
      unsigned all = 0;
      for (uint32_t j = 0; j < gridDim.x; ++j) all += ldcg(&D.bsum[j]);
      D.s_off[n] = all;
    }
  }
  if (!grid_barrier(D, B)) return false;
  for (uint32_t base = gwarp * 32; base < n; base += nwarps * 32) {
    const uint32_t v = base + lane;
    if (v < n && ldcg(&D.level[v]) == LIVE) {
      const uint32_t t = ldcg(&D.s_next[v]);
      const uint32_t left = atomicSub(&D.s_cnt[t], 1u);
      const uint32_t pos = ldcg(&D.s_off[t]) + left - 1u;
      if (left == 0u || pos >= n) set_error(D, TRIM_ERR_STATE, 0xD2);  // counts out of step
      else D.s_list[pos] = v;
    }
  }
  return true;
}

__device__ ROUND_FN bool ac6_round(const Dev& D, Cta& B, const Sched& S, uint32_t gwarp,
                                   uint32_t nwarps) {
  if (S.prev_variant != TRIM_AC6_SUPPORT) return ac6_entry(D, B, S, gwarp, nwarps);
  Counters K;
  const unsigned lane = lane_id();
  const uint32_t r = S.round;
  const uint32_t N = S.fe - S.fb;
  const uint32_t G = min(32u, max(1u, (N + nwarps - 1) / nwarps));
  uint32_t* wb = B.wbuf[threadIdx.x >> 5];
  for (uint32_t base = S.fb + gwarp * G; base < S.fe; base += nwarps * G) {
    const uint32_t item = base + lane;
    const bool has = lane < G && item < S.fe;
    // F_{r-1} was logged by an AC-6 round: its entries sit `skew` positions
    // below their counts (removals counted only by local rounds are not logged)
    const uint32_t w = has ? ldcg(&D.log[item - S.skew]) : 0u;
    uint32_t cur = has ? ldcg(&D.s_head[w]) : NIL;
    // bulk members of S(w): contiguous, spread over the lanes
    uint32_t ss = 0, sd = 0;
    if (has) {
      ss = ldcg(&D.s_off[w]);
      sd = ldcg(&D.s_off[w + 1]) - ss;
    }
    const unsigned incl = warp_incl_scan(sd);
    const unsigned total = __shfl_sync(FULL, incl, 31);
    const unsigned excl = incl - sd;
    for (unsigned k0 = 0; k0 < total; k0 += 32) {
      const unsigned k = k0 + lane;
      const bool valid = k < total;
      const unsigned j = G == 1 ? 0u : owner_of(excl, k);
      const unsigned sj = __shfl_sync(FULL, ss, j), ej = __shfl_sync(FULL, excl, j);
      const uint32_t v = valid ? ldcg(&D.s_list[sj + (k - ej)]) : 0u;
      ac6_rescan(D, B, valid, v, r, K);
    }
    // members that joined S(w) during the epoch (intrusive lists): all walkers
    // hop in step and stage the members; re-scans run 32 at a time. A member's
    // next pointer is read before it can be re-scanned (and move to another set).
    unsigned nbuf = 0, steps = 0;
    while (true) {
      const bool walking = cur != NIL;
      const unsigned wm = __ballot_sync(FULL, walking);
      if (wm == 0u && nbuf == 0u) break;
      if (wm) {
        if (++steps > D.n) {  // a set holds at most n members: longer means a broken list
          if (lane == 0) set_error(D, TRIM_ERR_STATE, 0xD4);
          break;
        }
        if (walking) {
          const uint32_t v = cur;
          cur = ldcg(&D.s_next[v]);
          wb[nbuf + __popc(wm & ((1u << lane) - 1u))] = v;
        }
        nbuf += __popc(wm);
        __syncwarp();
      }
      const bool more = __any_sync(FULL, cur != NIL);
      while (nbuf >= 32u || (!more && nbuf > 0u)) {
        const unsigned take = min(32u, nbuf);
        const bool valid = lane < take;
        const uint32_t v = valid ? wb[nbuf - take + lane] : 0u;
        __syncwarp();
        nbuf -= take;
        ac6_rescan(D, B, valid, v, r, K);
      }
    }
  }
  stats_flush(D, B, K);
  return true;
}

// ------------------------------------------------------------------ init (round 0)

// Each warp takes U blocks of 32 consecutive vertices at a time and issues all
// their offset loads (and G^T offsets, needed for the sinks' work-list entries)
// before using any: the pass is bound by memory parallelism, not by bandwidth.
__device__ ROUND_FN void init_round(const Dev& D, Cta& B, uint32_t gwarp, uint32_t nwarps) {
  constexpr int U = 4;
  const unsigned lane = lane_id();
  const uint32_t n = D.n;
  const bool w4 = (D.flags & F_AC4_POSSIBLE) != 0;
  const bool rows = D.ioff != nullptr;
  for (uint32_t base = gwarp * (32u * U); base < n; base += nwarps * (32u * U)) {
    uint32_t o0[U], o1[U], i0[U], i1[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const uint32_t v = base + q * 32u + lane;
      const bool has = v < n;
#if TRIM_MODES & 32
      o0[q] = 0u;
      o1[q] = has ? ig_degree(D, v) : 0u;
#else
      o0[q] = has ? __ldg(&D.off[v]) : 0u;
      o1[q] = has ? __ldg(&D.off[v + 1]) : 0u;
#endif
#if TRIM_MODES & 16
      // in+out needs every vertex's in-degree
      i0[q] = (has && rows) ? __ldg(&D.ioff[v]) : 0u;
      i1[q] = (has && rows) ? __ldg(&D.ioff[v + 1]) : 0u;
#endif
    }
#if !(TRIM_MODES & 16)
    // one-sided: only the vertices removed here (no out-edge) need their G^T
    // row, for their work-list entry; the loads of all four blocks go out together
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const bool sink = base + q * 32u + lane < n && o1[q] == o0[q];
      i0[q] = (sink && rows) ? __ldg(&D.ioff[base + q * 32u + lane]) : 0u;
      i1[q] = (sink && rows) ? __ldg(&D.ioff[base + q * 32u + lane + 1]) : 0u;
    }
#endif
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const uint32_t v = base + q * 32u + lane;
      const bool has = v < n;
      const uint32_t d = o1[q] - o0[q];
#if TRIM_MODES & 16
      // in+out: no out-edge or no in-edge removes the vertex in round 0
      const uint32_t din = i1[q] - i0[q];
      if (has) {
        D.level[v] = (d && din) ? LIVE : 0u;
        D.cnt[v] = d;
        D.cnt_in[v] = din;
      }
      append_dead_io(D, B, has && (d == 0u || din == 0u), v, 0u, true, i0[q], din, o0[q], d);
#else
      if (has) {
        D.level[v] = d ? LIVE : 0u;
        if (w4) D.cnt[v] = d;
      }
      append_dead(D, B, has && d == 0u, v, 0u, D.live0, true, true, i0[q], i1[q] - i0[q]);
#endif
    }
  }
}

#if !(TRIM_MODES & 48)
// Initial pass with a dead mask (vertex sampling, Section 9): a masked vertex
// is DEAD from the start: level 0 (removed before round 1 for every variant),
// counter 0 (a decrement can never return 1), never on the work list, not
// counted. An unmasked vertex counts its unmasked successors: with none it is
// removed in round 0, else it is LIVE with that count as its AC-4 counter.
// With AC-4 every edge of an unmasked vertex is counted: each warp takes 32
// vertices and walks their edges laid end to end, 32 per step with four
// steps' loads in flight; a vertex's count in a step is the popcount of the
// step's unmasked-target ballot over the lanes that hold its edges. Rows with
// more than kMaskHeavy edges are left to the whole CTA afterwards (one warp
// would walk a skewed graph's longest row alone). A run
// without AC-4 needs only whether one unmasked successor exists, so each lane
// scans its own row and stops at the first one (rows longer than 32: the
// whole warp).
__device__ __forceinline__ uint32_t lane_range(uint32_t a, uint32_t b) {  // bits [a, b), b <= 32
  const uint32_t hi = b >= 32u ? 0xFFFFFFFFu : ((1u << b) - 1u);
  const uint32_t lo = a >= 32u ? 0xFFFFFFFFu : ((1u << a) - 1u);
  return hi & ~lo;
}

constexpr uint32_t kMaskHeavy = 1024;
constexpr uint32_t kMaskHeavyCap = LW - MAX_WARPS;  // list + per-warp sums in one slice

__device__ ROUND_FN void init_round_masked(const Dev& D, Cta& B, uint32_t gwarp,
                                           uint32_t nwarps) {
  const unsigned lane = lane_id();
  const uint32_t n = D.n;
  const bool w4 = (D.flags & F_AC4_POSSIBLE) != 0;
  // the CTA's deferred heavy rows and its reduction scratch: warp 0's live-list
  // slice, which no append of this pass uses (its work-list slices stay in
  // buffers 1 and 2: w4_wide is 0 here)
  uint32_t* heavy = slice(0, 3);
  uint32_t* wsum = heavy + kMaskHeavyCap;
  if (threadIdx.x == 0) B.lq_scratch = 0u;
  __syncthreads();
  for (uint32_t base = gwarp * 32u; base < n; base += nwarps * 32u) {
    const uint32_t v = base + lane;
    const bool has = v < n;
    const bool masked = has && D.mask[v] != 0;
    const uint32_t s = has ? __ldg(&D.off[v]) : 0u;
    const uint32_t d = has ? __ldg(&D.off[v + 1]) - s : 0u;
    uint32_t c = 0;
    bool deferred = false;
    if (w4 && !masked && d > kMaskHeavy) {
      const uint32_t at = atomicAdd(&B.lq_scratch, 1u);
      if (at < kMaskHeavyCap) {
        heavy[at] = v;
        deferred = true;
      }
    }
    if (w4) {
      const uint32_t dd = (masked || deferred) ? 0u : d;
      const uint32_t incl = warp_incl_scan(dd), excl = incl - dd;
      const uint32_t total = __shfl_sync(FULL, incl, 31);
      for (uint32_t k0 = 0; k0 < total; k0 += 128u) {  // warp-uniform
        uint32_t t[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t k = k0 + (uint32_t)q * 32u + lane;
          const unsigned o = owner_of(excl, k);
          const uint32_t so = __shfl_sync(FULL, s, o), xo = __shfl_sync(FULL, excl, o);
          t[q] = k < total ? __ldg(&D.tgt[so + (k - xo)]) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t cs = k0 + (uint32_t)q * 32u;  // flattened index of lane 0
          const bool live = cs + lane < total && D.mask[t[q]] == 0;
          const uint32_t bal = __ballot_sync(FULL, live);
          const uint32_t a = excl <= cs ? 0u : min(excl - cs, 32u);
          const uint32_t e = excl + dd;
          const uint32_t b = e <= cs ? 0u : min(e - cs, 32u);
          c += __popc(bal & lane_range(a, b));
        }
      }
    } else {
      const bool own = has && !masked && d <= 32u;  // scanned by its own lane
      for (uint32_t k0 = 0; k0 < (own ? d : 0u) && c == 0u; k0 += 4u) {
        uint32_t tq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) tq[q] = (k0 + q < d) ? __ldg(&D.tgt[s + k0 + q]) : 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) c += (k0 + q < d && D.mask[tq[q]] == 0) ? 1u : 0u;
      }
      unsigned big = __ballot_sync(FULL, has && !masked && d > 32u);
      while (big) {
        const int j = __ffs(big) - 1;
        big &= big - 1u;
        const uint32_t sj = __shfl_sync(FULL, s, j), dj = __shfl_sync(FULL, d, j);
        uint32_t part = 0;
        for (uint32_t k0 = 0; k0 < dj; k0 += 128u) {  // warp-uniform
          uint32_t tq[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t k = k0 + (uint32_t)q * 32u + lane;
            tq[q] = k < dj ? __ldg(&D.tgt[sj + k]) : 0u;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t k = k0 + (uint32_t)q * 32u + lane;
            part += (k < dj && D.mask[tq[q]] == 0) ? 1u : 0u;
          }
          if (__any_sync(FULL, part != 0u)) break;
        }
        part = __reduce_add_sync(FULL, part);
        if ((int)lane == j) c = part;
      }
    }
    // (a deferred row is counted below; every lane takes part in append_dead,
    // a warp-collective call)
    if (has && !deferred) {
      D.level[v] = (masked || c == 0u) ? 0u : LIVE;
      if (w4) D.cnt[v] = masked ? 0u : c;
    }
    append_dead(D, B, has && !masked && !deferred && c == 0u, v, 0u, D.live0, true);
  }
  __syncthreads();
  const uint32_t nh = min(B.lq_scratch, kMaskHeavyCap);
  const unsigned warp = threadIdx.x >> 5;
  for (uint32_t h = 0; h < nh; ++h) {  // block-uniform
    const uint32_t v = heavy[h];
    const uint32_t s = __ldg(&D.off[v]), e = __ldg(&D.off[v + 1]);
    uint32_t part = 0;
    for (uint32_t k0 = s; k0 < e; k0 += 4u * blockDim.x) {
      uint32_t tq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t k = k0 + (uint32_t)q * blockDim.x + threadIdx.x;
        tq[q] = k < e ? __ldg(&D.tgt[k]) : 0u;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t k = k0 + (uint32_t)q * blockDim.x + threadIdx.x;
        part += (k < e && D.mask[tq[q]] == 0) ? 1u : 0u;
      }
    }
    part = __reduce_add_sync(FULL, part);
    if (lane == 0) wsum[warp] = part;
    __syncthreads();
    if (warp == 0) {
      uint32_t c = lane < (blockDim.x >> 5) ? wsum[lane] : 0u;
      c = __reduce_add_sync(FULL, c);
      if (lane == 0) {
        D.level[v] = c ? LIVE : 0u;
        D.cnt[v] = c;
      }
      append_dead(D, B, lane == 0 && c == 0u, v, 0u, D.live0, true);
    }
    __syncthreads();
  }
}
#endif

}  // namespace

#ifndef TRIM_MIN_BLOCKS
#define TRIM_MIN_BLOCKS 2
#endif
__global__ void __launch_bounds__(512, TRIM_MIN_BLOCKS) TRIM_KERNEL(Dev D) {
  __shared__ Cta B;
  const uint32_t wpb = blockDim.x >> 5;
  const uint32_t nwarps = gridDim.x * wpb;
  const uint32_t gwarp = blockIdx.x * wpb + (threadIdx.x >> 5);
  if (D.flags & F_CONTINUE) {
    // enqueued behind a run's first segment: resume the run if that segment
    // handed it over; else (the run is over or failed) return at once
    if (threadIdx.x == 0) {
      const volatile Ctrl* C = D.C;
      B.skip = (C->err == 0u && C->resume != 0u) ? 0u : 1u;
    }
    __syncthreads();
    if (B.skip) return;  // every CTA read the same control block: all return
  }
  if (threadIdx.x == 0) {
    Sched& S = B.S;
    if (D.flags & F_CONTINUE) {
      B.resume = 1u;
      B.bar_base = ((const volatile Ctrl*)D.C)->bar;
    } else {
      B.resume = D.resume;
      B.bar_base = D.bar_base;
    }
    B.mode = D.mode;
    if (blockIdx.x == 0) D.C->segments += 1u;
    S.round = 0; S.fb = 0; S.fe = 0;
    S.variant = NIL; S.prev_variant = NIL;
    S.c4w = 0; S.e_c4 = 0; S.w_end = 0; S.e_end = 0;
    S.ac3_list = NIL; S.live_in_len = 0; S.live_out = 0;
    S.done = 0; S.fprev = 0; S.mixed = 0;
    S.vcount[0] = S.vcount[1] = S.vcount[2] = 0;
    S.stable = 0;
    S.cstop = 0; S.cperiod = 0; S.clast = NIL;
    S.bmax = 0;
    S.m_live = D.m;
    for (int i = 0; i < NFEAT; ++i) S.feat[i] = 0.0f;
    S.skew = 0;
    S.supp_valid = 0;
    S.lround = 0;
    S.lbase[0] = S.lbase[1] = 0;

    for (int w = 0; w < MAX_WARPS; ++w) {
      WarpSlice& x = B.ws[w];
      x.nlog = x.nw4 = x.nedge = x.nlive = x.ncount = 0;
      x.sum_in = x.sum_out = 0;
      x.max_din = 0;
      x.hist[0] = x.hist[1] = x.hist[2] = 0;
    }
    B.epoch = 0;
    B.err = 0;
    B.w4_wide = 0;
    B.kstat[0] = B.kstat[1] = B.kstat[2] = B.kstat[3] = 0;
#if TRIM_LOCAL
    B.lq_cnt[0] = B.lq_cnt[1] = 0;
    B.lq_vend[0] = B.lq_vend[1] = 0;
    B.lq_k = B.lq_ovf = B.lq_pushed = 0;
#endif
  }
  if (threadIdx.x == 0 && B.resume) {
    // continue a run that an earlier segment left at the start of round saved.round
    const volatile uint32_t* w = reinterpret_cast<const volatile uint32_t*>(&D.C->saved);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&B.S);
    for (unsigned i = 0; i < sizeof(Sched) / 4; ++i) dst[i] = w[i];
  }
  __syncthreads();
  bool ok = true;
  if (!B.resume) {
    start_round(D, 0);
    // (the initial pass with a dead mask keeps buffer 3 for its heavy rows)
    if (threadIdx.x == 0) B.w4_wide = ((MODES & M_INOUT) || D.mask != nullptr) ? 0u : 1u;
    __syncthreads();
#if !(TRIM_MODES & 48)
    if (D.mask != nullptr) init_round_masked(D, B, gwarp, nwarps);
    else
#endif
      init_round(D, B, gwarp, nwarps);
    flush_round(D, B, 0, D.live0);
    ok = grid_barrier(D, B, false);
    // every warp's copy finished before the barrier; the __syncthreads after
    // advance() publishes this before any work-list append
    if (threadIdx.x == 0) B.w4_wide = 0;
  }
  bool fresh = !B.resume;  // a resumed segment starts with its round already chosen
  while (ok) {
    if (fresh && threadIdx.x < 32) advance(D, B);  // also reads the error flag
    fresh = true;
    __syncthreads();
    if (B.err) break;
    const Sched& S = B.S;  // changes only in advance(), between barriers
    if (S.done) {
      if (blockIdx.x == 0 && threadIdx.x == 0) D.C->resume = 0;
      break;
    }
    const bool have = (S.variant == TRIM_AC4_PUSH && (MODES & M_AC4)) ||
                      (S.variant == TRIM_AC6_SUPPORT && (MODES & M_AC6)) ||
                      (S.variant == TRIM_AC3_PULL && (MODES & M_AC3));
    // This kernel lacks the variant chosen for this round: it saves the
    // schedule state and hands the run over at the start of the round (every
    // CTA takes the decision from the same state, so all stop here); the
    // kernel that has the variant resumes it.
    if (!have) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        volatile uint32_t* w = reinterpret_cast<volatile uint32_t*>(&D.C->saved);
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&B.S);
        for (unsigned i = 0; i < sizeof(Sched) / 4; ++i) w[i] = src[i];
        D.C->resume_variant = S.variant;
        if (D.C->first_exit_round == 0u) D.C->first_exit_round = S.round;
        __threadfence();
        D.C->resume = 1;
      }
      break;
    }
#if TRIM_LOCAL
    if (async_start(D, S)) {
      if (!async_tail(D, B)) break;
      fresh = false;  // done: the tail ran the rest of the run
      continue;
    }
    if (local_start(D, S)) {
      if (!local_stretch(D, B)) break;
      fresh = false;  // done, or the stretch's last round already ran advance()
      continue;
    }
#endif
    start_round(D, S.round);
#if TRIM_MODES & 16
    inout_round(D, B, S, gwarp, nwarps);
#else
    if ((MODES & M_AC4) && S.variant == TRIM_AC4_PUSH) {
      ac4_round(D, B, S, gwarp, nwarps);
    } else if ((MODES & M_AC6) && S.variant == TRIM_AC6_SUPPORT) {
      if (!ac6_round(D, B, S, gwarp, nwarps)) break;
    } else if (MODES & M_AC3) {
      ac3_round(D, B, S, gwarp, nwarps);
    }
#endif
    const bool stamp = (D.flags & F_ROUND_LOG) && blockIdx.x == 0 && threadIdx.x == 0;
    if (stamp) D.C->t_work[S.round & 3] = globaltimer();
    flush_round(D, B, S.round, S.live_out ? D.live1 : D.live0);
    if (stamp) D.C->t_flush[S.round & 3] = globaltimer();
    ok = grid_barrier(D, B, false);
  }
  stats_publish(D, B);  // every exit of the loop is taken by the whole CTA
}

// ---------------------------------------------------------------- helpers


#if TRIM_MODES == 34
// Edge count of an implicit graph: the sum of its degrees (one pass, n draws).
__global__ void trim_implicit_degree_sum_kernel(Dev D, unsigned long long* m) {
  unsigned long long acc = 0;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < D.n; v += gridDim.x * blockDim.x)
    acc += ig_degree(D, v);
  acc = warp_sum(acc);
  if (lane_id() == 0 && acc) atomicAdd(m, acc);
}
#endif
