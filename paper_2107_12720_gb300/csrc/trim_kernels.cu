// trim_kernels.cu -- the persistent round-synchronous trimming kernel.
//
// One cooperative launch runs every round of the trimming of Guo & Sekerinski
// (arXiv 2107.12720): round 0 removes the vertices without out-edges, round r
// the vertices whose successors were all removed in rounds < r (Definition 2).
// Between rounds a grid-wide barrier (bounded spin) hands control to one warp
// that closes the round's books and picks the variant of the next round:
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
#include "trim_internal.cuh"

using namespace trimk;

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

struct RoundInfo {
  uint32_t round, fb, fe, variant, prev_variant, c4, ac3_list, live_fill, done, npieces_prev,
      live_in_len;
};

// ------------------------------------------------------------------ counters
struct Counters {
  unsigned long long edges = 0, pushed = 0, cand = 0, swept = 0;
};

// ------------------------------------------------------------------ appends

__device__ __forceinline__ void reserve_pieces(const Dev& D, uint32_t u, uint32_t din,
                                               uint32_t r) {
  const uint32_t np = (din + D.piece_edges - 1) / D.piece_edges;
  const uint32_t pb = atomicAdd(&D.C->rs[r & 3].npieces, np);
  if (pb + np > D.piece_cap) {
    set_error(D, TRIM_ERR_STATE, 0xA4);
    return;
  }
  uint2* P = (r & 1) ? D.pieces1 : D.pieces0;
  for (uint32_t q = 0; q < np; ++q) P[pb + q] = make_uint2(u, q);
}

// Warp-collective: lanes with pred append u to the dead log as a member of F_r
// and set level[u] = r. One atomic per warp (warp-aggregated).
__device__ __forceinline__ void append_dead(const Dev& D, bool pred, uint32_t u, uint32_t r) {
  const unsigned lane = lane_id();
  const unsigned mask = __ballot_sync(FULL, pred);
  if (mask == 0u) return;
  const unsigned leader = __ffs(mask) - 1;
  unsigned base = 0;
  if (lane == leader) {
    base = atomicAdd(&D.C->log_len, (unsigned)__popc(mask));
    if (base + (unsigned)__popc(mask) > D.n) set_error(D, TRIM_ERR_STATE, 0xD1);  // never: each
  }                                                                           // vertex dies once
  base = __shfl_sync(FULL, base, leader);
  if (base + (unsigned)__popc(mask) > D.n) return;
  const bool feats = (D.flags & F_NEED_FEATURES) != 0;
  unsigned din = 0, dout = 0;
  if (pred) {
    D.log[base + __popc(mask & ((1u << lane) - 1u))] = u;
    D.level[u] = r;
    if (D.ioff != nullptr && (feats || (D.flags & F_AC4_POSSIBLE))) {
      din = __ldg(&D.ioff[u + 1]) - __ldg(&D.ioff[u]);
      if ((D.flags & F_AC4_POSSIBLE) && din > D.big_degree) reserve_pieces(D, u, din, r);
    }
    if (feats) dout = __ldg(&D.off[u + 1]) - __ldg(&D.off[u]);
  }
  if (feats) {
    const unsigned long long s_in = warp_sum<unsigned long long>(din);
    const unsigned long long s_out = warp_sum<unsigned long long>(dout);
    const unsigned h0 = __popc(__ballot_sync(FULL, pred && din < 8u));
    const unsigned h1 = __popc(__ballot_sync(FULL, pred && din >= 8u && din < 256u));
    const unsigned h2 = __popc(mask) - h0 - h1;
    if (lane == leader) {
      RoundStat* rs = &D.C->rs[r & 3];
      if (s_in) atomicAdd(&rs->sum_in, s_in);
      if (s_out) atomicAdd(&rs->sum_out, s_out);
      if (h0) atomicAdd(&rs->hist[0], h0);
      if (h1) atomicAdd(&rs->hist[1], h1);
      if (h2) atomicAdd(&rs->hist[2], h2);
    }
  }
}

// Warp-collective append to an AC-3 live list.
__device__ __forceinline__ void append_live(const Dev& D, bool pred, uint32_t v, uint32_t list) {
  const unsigned lane = lane_id();
  const unsigned mask = __ballot_sync(FULL, pred);
  if (mask == 0u) return;
  const unsigned leader = __ffs(mask) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(&D.C->live_len[list], (unsigned)__popc(mask));
  base = __shfl_sync(FULL, base, leader);
  if (base + (unsigned)__popc(mask) > D.n) {
    if (lane == leader) set_error(D, TRIM_ERR_STATE, 0xD3);
    return;
  }
  if (pred) (list ? D.live1 : D.live0)[base + __popc(mask & ((1u << lane) - 1u))] = v;
}

// ------------------------------------------------------------------ scans

// Thread-level forward scan of v's successors from position i (row start s,
// length d): returns the first position whose target is not removed before
// round r, or d. At most `batches` x 4 edges; *resolved tells whether it ended.
__device__ __forceinline__ uint32_t scan_thread(const Dev& D, uint32_t s, uint32_t d, uint32_t i,
                                                uint32_t r, int batches, bool& resolved,
                                                Counters& K) {
  for (int b = 0; b < batches; ++b) {
    if (i >= d) { resolved = true; return d; }
    const uint32_t nb = min(4u, d - i);
    uint32_t t[4], lv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = (q < (int)nb) ? __ldg(&D.tgt[s + i + q]) : 0u;
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
__device__ __forceinline__ void scan_warp_finish(const Dev& D, bool& resolved, uint32_t s,
                                                 uint32_t d, uint32_t& i, uint32_t r,
                                                 Counters& K) {
  const unsigned lane = lane_id();
  unsigned pend = __ballot_sync(FULL, !resolved);
  while (pend) {
    const int src = __ffs(pend) - 1;
    pend &= pend - 1;
    const uint32_t ss = __shfl_sync(FULL, s, src), dd = __shfl_sync(FULL, d, src);
    uint32_t ii = __shfl_sync(FULL, i, src);
    uint32_t found = dd;
    while (ii < dd) {
      const uint32_t k = ii + lane;
      bool live = false;
      if (k < dd) live = ldcg(&D.level[__ldg(&D.tgt[ss + k])]) >= r;
      const unsigned b = __ballot_sync(FULL, live);
      if (lane == 0) K.edges += min(32u, dd - ii);
      if (b) { found = ii + __ffs(b) - 1; break; }
      ii += 32;
    }
    if ((int)lane == src) { i = found; resolved = true; }
  }
}

// Warp-collective search: owner lane j of element k, i.e. the largest j with
// excl_j <= k (lanes that own nothing carry excl = total and are never picked).
__device__ __forceinline__ unsigned owner_of(unsigned excl, unsigned k) {
  unsigned lo = 0;
#pragma unroll
  for (unsigned step = 16; step >= 1; step >>= 1) {
    const unsigned cand = lo + step;
    const unsigned ex = __shfl_sync(FULL, excl, cand & 31u);
    if (cand < 32u && ex <= k) lo = cand;
  }
  return lo;
}

// ------------------------------------------------------------------ grid barrier

__device__ void round_hook(const Dev& D);

// Grid-wide barrier with a bounded spin. The last CTA to arrive runs the round
// hook (one warp) before it releases the others. Returns false if the run must
// stop (error flag set, including a timed-out wait).
__device__ bool grid_sync(const Dev& D, bool with_hook) {
  __shared__ unsigned s_err;
  __syncthreads();
  if (threadIdx.x < 32) {
    const unsigned lane = lane_id();
    unsigned gen = 0, last = 0;
    if (lane == 0) {
      gen = ld_relaxed(&D.C->bar_gen);
      __threadfence();
      last = (atom_add_acqrel(&D.C->bar_count, 1u) == gridDim.x - 1) ? 1u : 0u;
    }
    last = __shfl_sync(FULL, last, 0);
    if (last) {
      __threadfence();
      if (with_hook) round_hook(D);
      __syncwarp();
      if (lane == 0) {
        D.C->bar_count = 0;
        __threadfence();
        red_release_add(&D.C->bar_gen, 1u);
      }
    } else if (lane == 0) {
      const uint64_t t0 = globaltimer();
      while (ld_acquire(&D.C->bar_gen) == gen) {
        if (globaltimer() - t0 > D.spin_limit_ns) {
          set_error(D, TRIM_ERR_TIMEOUT, 1);
          break;
        }
      }
    }
    if (lane == 0) {
      __threadfence();
      s_err = ld_relaxed(&D.C->err);
    }
  }
  __syncthreads();
  return s_err == 0u;
}

// ------------------------------------------------------------------ scheduler

__device__ float log2p1(double x) { return (float)log2(1.0 + x); }

// Cost rule of TRIM_SCHED_HEURISTIC (work each variant would do next round, in
// rough units of one random 32-byte access): AC-4 walks the in-edges of every
// removed vertex it has not yet processed; AC-3 sweeps its live list (or all n
// the first time); AC-6 re-scans the supporting sets of the last frontier
// (about one member per removed vertex) or, on entry, rebuilds the sets of all
// live vertices.
__device__ uint32_t heuristic_choice(const Dev& D, volatile const Ctrl* C, uint32_t nF,
                                     unsigned long long backlog_in, uint32_t backlog_items,
                                     uint32_t n_live, uint32_t cur_variant) {
  const bool has4 = D.ioff != nullptr && (D.flags & F_AC4_POSSIBLE);
  const float inf = 3.0e38f;
  float c4 = has4 ? (float)backlog_in + 0.5f * (float)backlog_items : inf;
  const uint32_t list = C->ac3_list;
  const float sweep = (list == NIL) ? (float)D.n : (float)C->live_len[list];
  float c3 = 0.35f * sweep + 0.5f * (float)nF;
  float c6 = (cur_variant == TRIM_AC6_SUPPORT) ? 2.0f * (float)nF
                                               : 1.5f * (float)n_live + 0.25f * (float)D.n;
  c4 *= D.heur_push_ratio;
  c6 *= D.heur_ac6_ratio;
  if (!(D.flags & F_AC4_POSSIBLE)) c4 = inf;
  if (!(D.flags & F_AC6_POSSIBLE)) c6 = inf;
  if (!(D.flags & F_AC3_POSSIBLE)) c3 = inf;
  if (c4 <= c3 && c4 <= c6) return TRIM_AC4_PUSH;
  if (c6 <= c3) return TRIM_AC6_SUPPORT;
  return TRIM_AC3_PULL;
}

// Warp-collective MLP 12 -> 32 -> 32 -> 3 (ReLU); returns the argmax class
// among the available variants; *in_range = all features inside [lo, hi].
__device__ uint32_t mlp_choice(const Dev& D, const float* f, bool* in_range) {
  const unsigned lane = lane_id();
  const float* B = D.model;
  const float *W1 = B, *b1 = B + 384, *W2 = B + 416, *b2 = B + 1440, *W3 = B + 1472,
              *b3 = B + 1568, *mean = B + 1571, *istd = B + 1583, *lo = B + 1595,
              *hi = B + 1607;
  bool ok = true;
  float x[NFEAT];
#pragma unroll
  for (int i = 0; i < NFEAT; ++i) {
    ok = ok && f[i] >= __ldg(&lo[i]) && f[i] <= __ldg(&hi[i]);
    x[i] = (f[i] - __ldg(&mean[i])) * __ldg(&istd[i]);
  }
  float h1 = __ldg(&b1[lane]);
#pragma unroll
  for (int i = 0; i < NFEAT; ++i) h1 = fmaf(__ldg(&W1[lane * NFEAT + i]), x[i], h1);
  h1 = fmaxf(h1, 0.0f);
  float h2 = __ldg(&b2[lane]);
#pragma unroll
  for (int k = 0; k < 32; ++k) h2 = fmaf(__ldg(&W2[lane * 32 + k]), __shfl_sync(FULL, h1, k), h2);
  h2 = fmaxf(h2, 0.0f);
  float z[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) z[o] = warp_sum(__ldg(&W3[o * 32 + lane]) * h2) + __ldg(&b3[o]);
  if (D.ioff == nullptr || !(D.flags & F_AC4_POSSIBLE)) z[TRIM_AC4_PUSH] = -3.0e38f;
  if (!(D.flags & F_AC6_POSSIBLE)) z[TRIM_AC6_SUPPORT] = -3.0e38f;
  if (!(D.flags & F_AC3_POSSIBLE)) z[TRIM_AC3_PULL] = -3.0e38f;
  uint32_t best = 0;
  if (z[1] > z[best]) best = 1;
  if (z[2] > z[best]) best = 2;
  *in_range = ok;
  return best;
}

// Closes round r (r = 0 is the initial sink pass) and prepares round r+1.
// Runs on one warp of the last CTA to reach the barrier, before it releases.
__device__ void round_hook(const Dev& D) {
  volatile Ctrl* C = D.C;  // every word may have been written by another SM
  const unsigned lane = lane_id();
  const uint32_t r = C->round;
  const uint32_t len = C->log_len;
  const uint32_t fs = C->f_end;  // F_r = log[fs, len)
  const uint32_t nF = len - fs;
  const uint64_t now = globaltimer();
  const uint32_t var = C->variant;
  RoundStat rsr;
  rsr.sum_in = C->rs[r & 3].sum_in;
  rsr.sum_out = C->rs[r & 3].sum_out;
  for (int i = 0; i < 3; ++i) rsr.hist[i] = C->rs[r & 3].hist[i];
  const uint32_t frontier_prev = fs - C->f_begin;
  __syncwarp();
  if (lane == 0) {
    D.roff[r] = fs;
    D.roff[r + 1] = len;
    if (r >= 1) {
      if (var <= 2u) C->vcount[var] += 1;
      if ((D.flags & F_ROUND_LOG) && D.rlog != nullptr && r - 1 < D.rlog_cap) {
        trim_round_rec_t* rec = &D.rlog[r - 1];
        rec->round = r;
        rec->variant = var;
        rec->frontier = frontier_prev;
        rec->removed = nF;
        rec->t_start_ns = C->t_release;
        rec->t_end_ns = now;
        for (int i = 0; i < NFEAT; ++i) rec->features[i] = C->feat[i];
        C->rlog_len = r;
      }
      if (var == TRIM_AC4_PUSH) {
        C->c4 = fs;
        C->cum_in_c4 = C->cum_in;
      }
      if (var == TRIM_AC3_PULL) C->ac3_list = C->live_fill;
    }
    C->last_round_ns = now - C->t_release;
    C->cum_in += rsr.sum_in;
    C->m_live -= rsr.sum_out;
    if (nF) C->rounds = r + 1;
    if (nF == 0) C->done = 1;
  }
  __syncwarp();
  if (nF != 0) {
    const uint32_t n_live = D.n - len;
    const unsigned long long m_live = C->m_live;
    float f[NFEAT];
    f[0] = log2p1(nF);
    f[1] = log2p1((double)rsr.sum_in);
    f[2] = log2p1((double)rsr.sum_out);
    f[3] = log2p1(n_live);
    f[4] = log2p1((double)m_live);
    f[5] = (float)nF / (float)max(1u, n_live);
    f[6] = (float)((double)rsr.sum_in / (double)max(1ull, m_live));
    f[7] = (float)rsr.hist[0] / (float)nF;
    f[8] = (float)rsr.hist[1] / (float)nF;
    f[9] = (float)rsr.hist[2] / (float)nF;
    f[10] = log2p1((double)C->last_round_ns / (double)max(1u, r >= 1 ? frontier_prev : D.n));
    f[11] = (float)(r + 1) / (float)(r + 1 + 64);
    const uint32_t cur = (r >= 1) ? var : NIL;
    uint32_t next;
    if (D.mode <= TRIM_AC3_PULL) {
      next = D.mode;
    } else if (D.mode == TRIM_SCHED_SCRIPTED) {
      next = D.script_len ? D.script[r % D.script_len] : 0u;
      if (next > 2u) next = TRIM_AC3_PULL;
      if (next == TRIM_AC4_PUSH && D.ioff == nullptr) next = TRIM_AC3_PULL;
    } else {
      const unsigned long long backlog_in = C->cum_in - C->cum_in_c4;
      const uint32_t backlog_items = len - C->c4;
      next = heuristic_choice(D, C, nF, backlog_in, backlog_items, n_live, cur);
      if (D.mode == TRIM_SCHED_LEARNED && D.model != nullptr) {
        bool in_range = false;
        const uint32_t learned = mlp_choice(D, f, &in_range);
        if (in_range) next = learned;
      }
    }
    if (lane == 0) {
      C->prev_variant = cur;
      C->variant = next;
      C->round = r + 1;
      C->f_begin = fs;
      C->f_end = len;
      volatile RoundStat* nx = &C->rs[(r + 1) & 3];
      nx->sum_in = 0; nx->sum_out = 0;
      nx->hist[0] = nx->hist[1] = nx->hist[2] = 0;
      nx->npieces = 0;
      for (int i = 0; i < NFEAT; ++i) C->feat[i] = f[i];
      if (next == TRIM_AC3_PULL) {
        const uint32_t out = (C->ac3_list == NIL) ? 0u : (C->ac3_list ^ 1u);
        C->live_fill = out;
        C->live_len[out] = 0;
      }
    }
  }
  if (lane == 0) C->t_release = globaltimer();
}

// ------------------------------------------------------------------ AC-4

// Warp-balanced in-edge walk over the removed vertices log[a, b): every warp
// takes G consecutive entries and spreads their in-edges over its lanes
// (a warp prefix sum of the degrees plus a shuffle search for the owner).
// Vertices above big_degree are skipped when skip_big (they come as pieces).
__device__ void ac4_items(const Dev& D, uint32_t a, uint32_t b, uint32_t r, bool skip_big,
                          uint32_t gwarp, uint32_t nwarps, Counters& K) {
  const unsigned lane = lane_id();
  const uint32_t N = b - a;
  const uint32_t G = min(32u, max(1u, (N + nwarps - 1) / nwarps));
  for (uint32_t base = a + gwarp * G; base < b; base += nwarps * G) {
    const uint32_t item = base + lane;
    const bool has = lane < G && item < b;
    uint32_t s = 0, d = 0;
    if (has) {
      const uint32_t w = ldcg(&D.log[item]);
      s = __ldg(&D.ioff[w]);
      d = __ldg(&D.ioff[w + 1]) - s;
      if (skip_big && d > D.big_degree) d = 0;
    }
    const unsigned incl = warp_incl_scan(d);
    const unsigned total = __shfl_sync(FULL, incl, 31);
    const unsigned excl = incl - d;
    for (unsigned k0 = 0; k0 < total; k0 += 64) {
      uint32_t u[2], old[2];
      bool v[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const unsigned k = k0 + q * 32 + lane;
        v[q] = k < total;
        const unsigned j = owner_of(excl, k);
        const unsigned sj = __shfl_sync(FULL, s, j), ej = __shfl_sync(FULL, excl, j);
        u[q] = v[q] ? __ldg(&D.itgt[sj + (k - ej)]) : 0u;
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) old[q] = v[q] ? atomicSub(&D.cnt[u[q]], 1u) : 0u;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        K.pushed += v[q] ? 1 : 0;
        const bool pred = v[q] && old[q] == 1u && ldcg(&D.level[u[q]]) == LIVE;
        append_dead(D, pred, u[q], r);
      }
    }
  }
}

__device__ void ac4_round(const Dev& D, const RoundInfo& R, uint32_t gwarp, uint32_t nwarps,
                          Counters& K) {
  const unsigned lane = lane_id();
  const uint32_t r = R.round;
  if (R.c4 < R.fb) ac4_items(D, R.c4, R.fb, r, false, gwarp, nwarps, K);  // catch-up
  ac4_items(D, R.fb, R.fe, r, true, gwarp, nwarps, K);
  // pieces of the big vertices of F_{r-1}, reserved when they were appended
  const uint2* P = ((r - 1) & 1) ? D.pieces1 : D.pieces0;
  const uint32_t PE = D.piece_edges;
  for (uint32_t p = gwarp; p < R.npieces_prev; p += nwarps) {
    const uint32_t w = ldcg(&P[p].x), q = ldcg(&P[p].y);
    const uint32_t s0 = __ldg(&D.ioff[w]), e0 = __ldg(&D.ioff[w + 1]);
    const uint32_t s = s0 + q * PE, e = min(e0, s + PE);
    for (uint32_t k0 = s; k0 < e; k0 += 64) {
      uint32_t u[2], old[2];
      bool v[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const uint32_t k = k0 + t * 32 + lane;
        v[t] = k < e;
        u[t] = v[t] ? __ldg(&D.itgt[k]) : 0u;
      }
#pragma unroll
      for (int t = 0; t < 2; ++t) old[t] = v[t] ? atomicSub(&D.cnt[u[t]], 1u) : 0u;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        K.pushed += v[t] ? 1 : 0;
        const bool pred = v[t] && old[t] == 1u && ldcg(&D.level[u[t]]) == LIVE;
        append_dead(D, pred, u[t], r);
      }
    }
  }
}

// ------------------------------------------------------------------ AC-3

__device__ void ac3_round(const Dev& D, const RoundInfo& R, uint32_t gwarp, uint32_t nwarps,
                          Counters& K) {
  const unsigned lane = lane_id();
  const uint32_t r = R.round;
  const bool all = (R.ac3_list == NIL);
  const uint32_t* Lin = (R.ac3_list == 1u) ? D.live1 : D.live0;
  const uint32_t N = all ? D.n : R.live_in_len;
  for (uint32_t base = gwarp * 32; base < N; base += nwarps * 32) {
    const uint32_t idx = base + lane;
    const bool has = idx < N;
    const uint32_t v = has ? (all ? idx : ldcg(&Lin[idx])) : 0u;
    const bool alive = has && ldcg(&D.level[v]) == LIVE;
    uint32_t s = 0, d = 0, i0 = 0, i = 0;
    bool resolved = true;
    if (alive) {
      s = __ldg(&D.off[v]);
      d = __ldg(&D.off[v + 1]) - s;
      i0 = ldcg(&D.supp[v]);
      i = scan_thread(D, s, d, i0, r, 2, resolved, K);
    }
    scan_warp_finish(D, resolved, s, d, i, r, K);
    const bool dies = alive && i >= d;
    const bool stays = alive && !dies;
    if (stays && i != i0) D.supp[v] = i;
    K.swept += has ? 1 : 0;
    append_dead(D, dies, v, r);
    append_live(D, stays, v, R.live_fill);
  }
}

// ------------------------------------------------------------------ AC-6

// Warp-collective re-scan of members of a supporting set whose owner was
// removed in round r-1: scan forward from the position after the lost support;
// on success join the new support's set (intrusive list), else remove.
__device__ __forceinline__ void ac6_rescan(const Dev& D, bool valid, uint32_t v, uint32_t r,
                                           Counters& K) {
  const bool alive = valid && ldcg(&D.level[v]) == LIVE;
  uint32_t s = 0, d = 0, i = 0;
  bool resolved = true;
  if (alive) {
    s = __ldg(&D.off[v]);
    d = __ldg(&D.off[v + 1]) - s;
    i = scan_thread(D, s, d, ldcg(&D.supp[v]) + 1u, r, 2, resolved, K);
  }
  scan_warp_finish(D, resolved, s, d, i, r, K);
  const bool dies = alive && i >= d;
  if (alive && !dies) {
    D.supp[v] = i;
    const uint32_t t = __ldg(&D.tgt[s + i]);
    D.s_next[v] = atomicExch(&D.s_head[t], v);
  }
  K.cand += valid ? 1 : 0;
  append_dead(D, dies, v, r);
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
__device__ bool ac6_entry(const Dev& D, const RoundInfo& R, uint32_t gwarp, uint32_t nwarps,
                          Counters& K) {
  const unsigned lane = lane_id();
  const uint32_t r = R.round, n = D.n;
  for (uint32_t base = gwarp * 32; base < n; base += nwarps * 32) {
    const uint32_t v = base + lane;
    const bool has = v < n;
    if (has) D.s_head[v] = NIL;
    const bool alive = has && ldcg(&D.level[v]) == LIVE;
    uint32_t s = 0, d = 0, i0 = 0, i = 0;
    bool resolved = true;
    if (alive) {
      s = __ldg(&D.off[v]);
      d = __ldg(&D.off[v + 1]) - s;
      i0 = ldcg(&D.supp[v]);
      i = scan_thread(D, s, d, i0, r, 2, resolved, K);
    }
    scan_warp_finish(D, resolved, s, d, i, r, K);
    const bool dies = alive && i >= d;
    if (alive && !dies) {
      if (i != i0) D.supp[v] = i;
      const uint32_t t = __ldg(&D.tgt[s + i]);
      D.s_next[v] = t;  // parked here until the scatter below
      atomicAdd(&D.s_cnt[t], 1u);
    }
    K.swept += has ? 1 : 0;
    append_dead(D, dies, v, r);
  }
  if (!grid_sync(D, false)) return false;
  // grid-wide exclusive scan of s_cnt into s_off
  const uint32_t chunk = ((n + gridDim.x - 1) / gridDim.x + 31) & ~31u;
  const uint32_t c0 = min(n, blockIdx.x * chunk), c1 = min(n, c0 + chunk);
  {
    unsigned acc = 0;
    for (uint32_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) acc += ldcg(&D.s_cnt[i]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) D.bsum[blockIdx.x] = acc;
  }
  if (!grid_sync(D, false)) return false;
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
  if (!grid_sync(D, false)) return false;
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

__device__ bool ac6_round(const Dev& D, const RoundInfo& R, uint32_t gwarp, uint32_t nwarps,
                          Counters& K) {
  if (R.prev_variant != TRIM_AC6_SUPPORT) return ac6_entry(D, R, gwarp, nwarps, K);
  const unsigned lane = lane_id();
  const uint32_t r = R.round;
  const uint32_t N = R.fe - R.fb;
  const uint32_t G = min(32u, max(1u, (N + nwarps - 1) / nwarps));
  for (uint32_t base = R.fb + gwarp * G; base < R.fe; base += nwarps * G) {
    const uint32_t item = base + lane;
    const bool has = lane < G && item < R.fe;
    const uint32_t w = has ? ldcg(&D.log[item]) : 0u;
    // bulk members of S(w): contiguous
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
      const unsigned j = owner_of(excl, k);
      const unsigned sj = __shfl_sync(FULL, ss, j), ej = __shfl_sync(FULL, excl, j);
      const uint32_t v = valid ? ldcg(&D.s_list[sj + (k - ej)]) : 0u;
      ac6_rescan(D, valid, v, r, K);
    }
    // members that joined S(w) during the epoch: walk the lists, all lanes in step
    uint32_t cur = has ? ldcg(&D.s_head[w]) : NIL;
    uint32_t steps = 0;
    while (__any_sync(FULL, cur != NIL)) {
      if (++steps > D.n) {  // a set holds at most n members: a longer walk means a broken list
        if (lane == 0) set_error(D, TRIM_ERR_STATE, 0xD4);
        break;
      }
      const bool valid = cur != NIL;
      const uint32_t v = cur;
      if (valid) cur = ldcg(&D.s_next[v]);  // read before v can move to another set
      ac6_rescan(D, valid, v, r, K);
    }
  }
  return true;
}

// ------------------------------------------------------------------ init (round 0)

__device__ void init_round(const Dev& D, uint32_t gwarp, uint32_t nwarps) {
  const unsigned lane = lane_id();
  const uint32_t n = D.n;
  const bool w4 = (D.flags & F_AC4_POSSIBLE) != 0;
  const bool w6 = (D.flags & (F_AC6_POSSIBLE | F_AC3_POSSIBLE)) != 0;
  for (uint32_t base = gwarp * 32; base < n; base += nwarps * 32) {
    const uint32_t v = base + lane;
    const bool has = v < n;
    uint32_t d = 0;
    if (has) {
      d = __ldg(&D.off[v + 1]) - __ldg(&D.off[v]);
      D.level[v] = d ? LIVE : 0u;
      if (w4) D.cnt[v] = d;
      if (w6) D.supp[v] = 0u;
    }
    append_dead(D, has && d == 0u, v, 0u);
  }
}

}  // namespace

__global__ void __launch_bounds__(512, 2) trim_persistent_kernel(Dev D) {
  __shared__ RoundInfo sR;
  const uint32_t wpb = blockDim.x >> 5;
  const uint32_t nwarps = gridDim.x * wpb;
  const uint32_t gwarp = blockIdx.x * wpb + (threadIdx.x >> 5);
  Counters K;
  init_round(D, gwarp, nwarps);
  bool ok = grid_sync(D, true);
  while (ok) {
    if (threadIdx.x == 0) {
      const Ctrl* C = D.C;
      sR.done = ld_relaxed(&C->done);
      sR.round = ld_relaxed(&C->round);
      sR.fb = ld_relaxed(&C->f_begin);
      sR.fe = ld_relaxed(&C->f_end);
      sR.variant = ld_relaxed(&C->variant);
      sR.prev_variant = ld_relaxed(&C->prev_variant);
      sR.c4 = ld_relaxed(&C->c4);
      sR.ac3_list = ld_relaxed(&C->ac3_list);
      sR.live_fill = ld_relaxed(&C->live_fill);
      sR.npieces_prev = ld_relaxed(&C->rs[(sR.round - 1) & 3].npieces);
      sR.live_in_len = sR.ac3_list == NIL ? 0u : ld_relaxed(&C->live_len[sR.ac3_list]);
    }
    __syncthreads();
    const RoundInfo R = sR;
    __syncthreads();
    if (R.done) break;
    if (R.variant == TRIM_AC4_PUSH) {
      ac4_round(D, R, gwarp, nwarps, K);
    } else if (R.variant == TRIM_AC6_SUPPORT) {
      if (!ac6_round(D, R, gwarp, nwarps, K)) break;
    } else {
      ac3_round(D, R, gwarp, nwarps, K);
    }
    ok = grid_sync(D, true);
  }
  if (D.flags & F_STATS) {
    const unsigned long long e = warp_sum(K.edges), p = warp_sum(K.pushed),
                             c = warp_sum(K.cand), s = warp_sum(K.swept);
    if (lane_id() == 0) {
      if (e) atomicAdd(&D.C->stats[0], e);
      if (p) atomicAdd(&D.C->stats[1], p);
      if (c) atomicAdd(&D.C->stats[2], c);
      if (s) atomicAdd(&D.C->stats[3], s);
    }
  }
}

// ---------------------------------------------------------------- helpers

// Control block reset before every run (one thread).
__global__ void trim_reset_ctrl_kernel(Ctrl* C, uint64_t m) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned* w = reinterpret_cast<unsigned*>(C);
    for (size_t i = 0; i < sizeof(Ctrl) / 4; ++i) w[i] = 0u;
    C->prev_variant = NIL;
    C->variant = NIL;
    C->ac3_list = NIL;
    C->m_live = m;
    C->t_release = globaltimer();
  }
}

__global__ void trim_status_kernel(const uint32_t* level, uint32_t n, uint8_t* status) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    status[v] = level[v] == LIVE ? 1 : 0;
}

// in-degree histogram of the targets (and a check that every target is < n)
__global__ void trim_indeg_kernel(const uint32_t* tgt, uint64_t m, uint32_t n, uint32_t* cnt,
                                  uint32_t* bad) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t t = tgt[e];
    if (t < n) atomicAdd(&cnt[t], 1u);
    else atomicOr(bad, 1u);
  }
}

// exclusive scan, pass 1: each block scans `chunk` elements and writes its total
__global__ void trim_scan_blocks_kernel(const uint32_t* in, uint32_t n, uint32_t* out,
                                        uint32_t* block_sums, uint32_t chunk) {
  const uint32_t c0 = min(n, blockIdx.x * chunk), c1 = min(n, c0 + chunk);
  unsigned pre = 0;
  for (uint32_t t0 = c0; t0 < c1; t0 += blockDim.x) {
    const uint32_t i = t0 + threadIdx.x;
    const unsigned x = i < c1 ? in[i] : 0u;
    unsigned tot;
    const unsigned ex = block_excl_scan(x, &tot);
    if (i < c1) out[i] = pre + ex;
    pre += tot;
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = pre;
}

// exclusive scan, pass 2: add the prefix of the block totals; out[n] = total
__global__ void trim_scan_apply_kernel(uint32_t* out, uint32_t n, const uint32_t* block_sums,
                                       uint32_t nblocks, uint32_t chunk) {
  unsigned pre = 0;
  for (uint32_t j = threadIdx.x; j < blockIdx.x; j += blockDim.x) pre += block_sums[j];
  pre = block_sum(pre);
  const uint32_t c0 = min(n, blockIdx.x * chunk), c1 = min(n, c0 + chunk);
  for (uint32_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) out[i] += pre;
  if (blockIdx.x == nblocks - 1 && threadIdx.x == 0) {
    unsigned all = 0;
    for (uint32_t j = 0; j < nblocks; ++j) all += block_sums[j];
    out[n] = all;
  }
}

// G^T fill: predecessor u of t goes to itgt[ioff[t] + fill[t]++]
__global__ void trim_transpose_fill_kernel(const uint32_t* off, const uint32_t* tgt, uint32_t n,
                                           const uint32_t* ioff, uint32_t* fill, uint32_t* itgt) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t u = warp; u < n; u += nw) {
    const uint32_t s = off[u], e = off[u + 1];
    for (uint32_t k = s + lane; k < e; k += 32) {
      const uint32_t t = tgt[k];
      itgt[ioff[t] + atomicAdd(&fill[t], 1u)] = u;
    }
  }
}

// offsets: off[0] = 0, non-decreasing, off[n] = m
__global__ void trim_validate_offsets_kernel(const uint32_t* off, uint32_t n, uint64_t m,
                                             uint32_t* bad) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
    if (v == 0 && off[0] != 0u) atomicOr(bad, 2u);
    if (v == n && (uint64_t)off[n] != m) atomicOr(bad, 2u);
    if (v < n && off[v + 1] < off[v]) atomicOr(bad, 2u);
  }
}

// batched graphs: every edge stays inside its graph (vgraph[v] = graph id of v)
__global__ void trim_validate_batch_kernel(const uint32_t* off, const uint32_t* tgt, uint32_t n,
                                           const uint32_t* vgraph, uint32_t* bad) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const uint32_t g = vgraph[u];
    for (uint32_t k = off[u]; k < off[u + 1]; ++k)
      if (vgraph[tgt[k]] != g) atomicOr(bad, 4u);
  }
}
