// trim_internal.cuh -- device state, control block and warp/grid primitives of
// the persistent trimming kernel.
//
// Level semantics (Definition 2 of Guo & Sekerinski, counted from 0): round r
// removes exactly the vertices whose successors were all removed in rounds
// < r. Every variant reads a vertex u as "removed before round r" iff
// level[u] < r; a vertex removed during round r carries level r and still
// counts as present for the rest of that round. This snapshot rule makes every
// variant compute the same levels, so they can be mixed round by round.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/trim.h"

namespace trimk {

constexpr uint32_t LIVE = 0xFFFFFFFFu;
constexpr uint32_t NIL = 0xFFFFFFFFu;
constexpr int NFEAT = 12;
// asynchronous AC-4 tail: in-edges per item of the shared queue (a removed
// vertex's G^T row is cut into pieces of at most this many), and the queue's
// capacity for n vertices and m edges (every removal adds at most
// ceil(in-degree / kAsyncPiece) items)
constexpr uint32_t kAsyncPiece = 256;
__host__ __device__ constexpr uint64_t async_queue_cap(uint64_t n, uint64_t m) {
  return n + m / kAsyncPiece + 1;
}

// flags inside Dev::flags (superset of the public TRIM_FLAG_*)
constexpr uint32_t F_STATS = TRIM_FLAG_STATS;
constexpr uint32_t F_ROUND_LOG = TRIM_FLAG_ROUND_LOG;
constexpr uint32_t F_NEED_FEATURES = 0x100;  // scheduler modes: gather per-frontier degrees
constexpr uint32_t F_AC4_POSSIBLE = 0x200;   // counters initialised, AC-4 work list kept
constexpr uint32_t F_AC6_POSSIBLE = 0x400;
constexpr uint32_t F_AC3_POSSIBLE = 0x800;
constexpr uint32_t F_LIVE_EDGES = 0x1000;    // scheduled run: keep the live-edge count in every flavour
constexpr uint32_t F_CONTINUE = 0x2000;      // continuation launch: resume the run if a segment handed it over

// Per-round accumulators, filled while round r runs (ring slot r & 3). CTA 0
// zeroes slot (k+2) & 3 at the start of round k: that slot was last read at the
// start of round k-1 and is next written in round k+2.
struct RoundStat {
  unsigned long long sum_in;   // sum of in-degrees of F_r
  unsigned long long sum_out;  // sum of out-degrees of F_r
  unsigned int hist[3];        // in-degree < 8, < 256, >= 256
  unsigned int live_count;     // AC-3: survivors written to the output live list in round r
  unsigned int max_din;        // largest in-degree among the work-list entries of F_r
  unsigned int pad;
};

// The schedule state of the current round. Every CTA keeps its own copy in
// shared memory and advances it from the same global inputs after each grid
// barrier, so all copies stay identical without a serial hand-off.
struct Sched {
  uint32_t round;         // r
  uint32_t fb, fe;        // F_{r-1} = log[fb, fe)
  uint32_t variant;       // variant of round r
  uint32_t prev_variant;  // variant of round r-1 (NIL before round 1)
  uint32_t c4w;           // AC-4 work list entries [0, c4w) already pushed
  uint32_t e_c4;          // ... their edges: [0, e_c4)
  uint32_t w_end;         // work list entries / edges of vertices removed before round r
  uint32_t e_end;
  uint32_t ac3_list;      // live list (0/1) holding a superset of the live vertices, NIL = none
  uint32_t live_in_len;   // its length
  uint32_t live_out;      // output list of an AC-3 round
  uint32_t done;
  uint32_t fprev;         // frontier size of round r-1 (timing feature)
  uint32_t mixed;         // 1 once a round ran AC-6 or AC-3 (AC-4 must then re-check levels)
  uint32_t vcount[3];     // rounds run so far by AC-4, AC-6, AC-3
  uint32_t stable;        // rounds in a row the scheduler kept its choice (0 outside schedulers)
  // committed stretch: rounds r < cstop run the committed variant without
  // consulting the scheduler (cstop = 0: none); the scheduler is consulted
  // again after round cstop, whose features it reads
  uint32_t cstop;
  uint32_t cperiod;       // length of the last committed stretch
  uint32_t clast;         // variant of the last commit (NIL: none yet)
  uint32_t bmax;          // largest in-degree among work-list entries AC-4 has not pushed
  unsigned long long m_live;     // out-edges of live vertices
  float feat[12];                // features that chose this round's variant
  // local AC-4 rounds (see trim_kernels.cu): removals counted only through the
  // local barrier are not in Ctrl::log_len; `skew` holds them, so that
  // removals so far = log_len + skew and logged entry i of the count sits at
  // log position i - skew
  uint32_t skew;
  uint32_t supp_valid;           // 1 once an AC-6 or AC-3 round set the support positions
  uint32_t lround;               // local rounds run so far (parity picks the barrier slot)
  unsigned long long lbase[2];   // value of each local-barrier slot after its last round
};

// Global control block. Counters hit by every CTA sit on their own 128-byte lines.
struct Ctrl {
  unsigned int bar;       unsigned int _p0[31];  // monotone grid-barrier arrivals
  unsigned int log_len;   unsigned int _p1[31];  // entries in the dead log
  unsigned long long w4;  unsigned int _p1b[30];  // AC-4 work list: items (low 32) | edges (high 32)
  unsigned int err;       unsigned int err_info; unsigned int _p2[30];
  // published by CTA 0 for the host
  unsigned int rounds;    // alpha
  unsigned int vcount[3];
  unsigned int rlog_len;
  unsigned int _p3[27];
  unsigned long long t_round[4];  // CTA 0's %globaltimer at the start of round r (ring)
  unsigned long long t_work[4];   // ... when CTA 0 finished the work of round r
  unsigned long long t_flush[4];  // ... when CTA 0 finished flushing round r
  unsigned long long stats[4];    // edges inspected, in-edges pushed, candidates, live swept
  RoundStat rs[4];
  // local AC-4 rounds: one 64-bit barrier word per round parity; every CTA adds
  // 2^48 (arrival) + 2^32 (if it sent removals to the global lists) + its local
  // removals, and reads the round's totals as the difference to the slot's
  // value after its previous round
  alignas(128) unsigned long long lbar[2];  unsigned int _p4[28];
  unsigned long long local_edges; // in-edges pushed from the CTAs' local queues (live-edge count)
  unsigned int n_dead;            // removals so far, published by CTA 0
  unsigned int local_rounds;      // local AC-4 rounds so far, published by CTA 0
  // asynchronous AC-4 tail (see async_tail in trim_kernels.cu): work tokens
  // (one per CTA with work; 0: the run is over), pieces written to the global
  // list, the rebalance generation asked for, entries in the two global entry
  // lists, the tail's removals and top level, the round at which it took
  // over, a heartbeat of the CTAs with work (bounds the wait of those
  // without), and the rebalances run
  unsigned int a_tokens;
  unsigned int oq_res;
  unsigned int a_req;
  unsigned int e_n[2];
  unsigned int a_removed;
  unsigned int a_maxlev;
  unsigned int a_round;
  unsigned int a_beat;
  unsigned int a_rebalances;
  unsigned int _p5[18];
  // segmented runs: a kernel that lacks the variant its scheduler picked saves
  // the schedule state here and exits; the kernel that has it resumes from it
  unsigned int resume;            // 1: a segment ended early, state in `saved`
  unsigned int resume_variant;    // the variant the next segment must run
  unsigned int segments;          // kernels that ran part of this run
  unsigned int first_exit_round;  // round at which the first segment handed over (0: never)
  unsigned int consults;          // rounds whose variant the scheduler chose
  unsigned int commit_round0;     // 1: round 1's choice committed the run at once
  Sched saved;
};

struct Dev {
  uint32_t n;
  uint32_t m;
  const uint32_t* __restrict__ off;   // out-CSR (read-only during a run)
  const uint32_t* __restrict__ tgt;
  const uint32_t* __restrict__ ioff;  // in-CSR G^T (nullable)
  const uint32_t* __restrict__ itgt;
  uint32_t* level;
  uint32_t* cnt;      // AC-4 out-degree counters
  uint32_t* supp;     // edge_index of AC-3 / AC-6: position of the current support
  uint32_t* s_head;   // AC-6 supporting sets added during the epoch (intrusive lists)
  uint32_t* s_next;
  uint32_t* s_cnt;    // AC-6 bulk build: member counts per support (zero between builds)
  uint32_t* s_off;    // AC-6 bulk supporting sets: CSR by support vertex (n+1)
  uint32_t* s_list;
  uint32_t* log;      // dead log: F_0 | F_1 | ... (n)
  uint32_t* roff;     // roff[r] = start of F_r in the log (n+2)
  uint32_t* live0;    // AC-3 live lists
  uint32_t* live1;
  // AC-4 work list: one entry per removed vertex with in-edges, in removal order:
  // the start of its G^T row and the exclusive prefix of in-degrees (edge offset).
  uint32_t* w4_row;
  uint32_t* w4_eoff;
  uint32_t* chunk_first;  // [c]: work-list entry that owns edge 32c of the prefix
  // in+out trimming (trim_run_inout): in-degree counters, and per work-list
  // entry the vertex's out-CSR row start and in-degree (its edge range covers
  // its G^T row, then its G row)
  uint32_t* cnt_in;
  uint32_t* w4_orow;
  uint32_t* w4_din;
  // vertex sampling (trim_set_dead_mask): mask[v] != 0 marks a vertex that is
  // DEAD from the start; nullable
  const uint8_t* __restrict__ mask;
  // implicit graph (trim_create_implicit): successors computed on the fly by
  // the implicit flavours; off/tgt are null then
  trim_implicit_graph_t ig;
  uint32_t* bsum;     // per-CTA scratch of the grid-wide scan
  uint32_t sbuf_cap;  // entries of each CTA append buffer (dynamic shared memory)
  uint32_t resume;    // 1: continue the run from Ctrl::saved instead of starting it
  uint32_t commit_after;  // != 0: scheduler flavours commit after this many stable rounds
  uint32_t recheck_rounds;  // length of the first committed stretch (doubles while repeated)
  uint32_t bar_base;  // grid-barrier counter when this kernel starts (0 for a new run)
  uint32_t local_edges_max;  // AC-4: pending in-edges up to which rounds run locally (0: never)
  // asynchronous AC-4 tail: per vertex (top level among its removed successors
  // << 32 | live-successor counter); the global list of G^T row pieces still
  // to push (row start, length, level of the removed vertex) and its
  // capacity; the two global entry lists of rebalances (predecessor, level),
  // ae_cap entries each
  unsigned long long* aw;
  uint32_t* oq_row;
  uint32_t* oq_len;
  uint32_t* oq_lev;
  uint32_t oq_cap;
  uint32_t* ae_id;
  uint32_t* ae_lev;
  uint32_t ae_cap;
  uint32_t async_edges_max;  // pending in-edges up to which the rest of the run is asynchronous (0: never)
  Ctrl* C;
  trim_round_rec_t* rlog;
  uint32_t rlog_cap;
  const float* model; // scheduler MLP blob (nullable)
  const uint8_t* script;
  uint32_t script_len;
  uint32_t mode;      // trim_variant_t requested
  uint32_t flags;
  uint64_t spin_limit_ns;
  float heur_push_ratio;
  float heur_ac6_ratio;
  float commit_confidence;  // LEARNED: commit at once at this softmax probability (0: never)
};

// ---------------------------------------------------------------- primitives

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_relaxed_add64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acqrel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
               : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
// loads of state that other SMs write during the run: served by L2, never a stale L1 line
__device__ __forceinline__ uint32_t ldcg(const uint32_t* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned warp_incl_scan(unsigned x) {
  const unsigned lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  return x;
}

// Warp-collective search: owner lane j of element k, i.e. the largest j with
// excl_j <= k (lanes that own nothing carry excl = total and are never picked).
__device__ __forceinline__ unsigned owner_of(unsigned excl, unsigned k) {
  unsigned lo = 0;
#pragma unroll
  for (unsigned step = 16; step >= 1; step >>= 1) {
    const unsigned cand = lo + step;
    const unsigned ex = __shfl_sync(0xFFFFFFFFu, excl, cand & 31u);
    if (cand < 32u && ex <= k) lo = cand;
  }
  return lo;
}
template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

__device__ __forceinline__ void set_error(const Dev& D, unsigned code, unsigned info) {
  if (atomicCAS(&D.C->err, 0u, code) == 0u) D.C->err_info = info;
}

}  // namespace trimk

// kernels (trim_kernels.cu, one flavour per variant set; trim_aux.cu), launched from trim_api.cu
__global__ void trim_probe_atomic_kernel(const uint32_t* idx, uint64_t n, uint32_t* counters);
__global__ void trim_persistent_kernel_m1(trimk::Dev D);   // AC-4 only
__global__ void trim_persistent_kernel_m2(trimk::Dev D);   // AC-6 only
__global__ void trim_persistent_kernel_m4(trimk::Dev D);   // AC-3 only
__global__ void trim_persistent_kernel_m9(trimk::Dev D);   // AC-4 + schedulers (segments)
__global__ void trim_persistent_kernel_m10(trimk::Dev D);  // AC-6 + schedulers (segments)
__global__ void trim_persistent_kernel_m12(trimk::Dev D);  // AC-3 + schedulers (segments)
__global__ void trim_persistent_kernel_m15(trimk::Dev D);  // all variants + schedulers
__global__ void trim_persistent_kernel_m17(trimk::Dev D);  // in+out trimming (AC-4 pushes on G and G^T)
__global__ void trim_persistent_kernel_m34(trimk::Dev D);  // AC-6 on an implicit graph
__global__ void trim_persistent_kernel_m36(trimk::Dev D);  // AC-3 on an implicit graph
__global__ void trim_implicit_degree_sum_kernel(trimk::Dev D, unsigned long long* m);
__global__ void trim_reset_ctrl_kernel(trimk::Ctrl* C);
__global__ void trim_status_kernel(const uint32_t* level, uint32_t n, uint8_t* status);
// SCC decomposition (trim_scc.cu)
__global__ void scc_init_kernel(const uint32_t* level, uint32_t n, uint32_t* comp, uint32_t* color);
__global__ void scc_trim2_single_kernel(const uint32_t* off, const uint32_t* tgt,
                                        const uint32_t* ioff, const uint32_t* itgt, uint32_t n,
                                        const uint32_t* comp, uint32_t* out1, uint32_t* in1);
__global__ void scc_trim2_pair_kernel(uint32_t n, const uint32_t* out1, const uint32_t* in1,
                                      uint32_t* comp, unsigned long long* pairs);
__global__ void scc_trim1_kernel(const uint32_t* off, const uint32_t* tgt, const uint32_t* ioff,
                                 const uint32_t* itgt, uint32_t n, uint32_t* comp,
                                 unsigned long long* removed);
__global__ void scc_label_start_kernel(uint32_t n, const uint32_t* comp, uint32_t* label,
                                       uint32_t* frontier, uint32_t* count,
                                       unsigned long long* open);
__global__ void scc_label_level_kernel(const uint32_t* off, const uint32_t* tgt,
                                       const uint32_t* comp, uint32_t* label, uint32_t* inq,
                                       uint32_t stamp, const uint32_t* frontier, uint32_t count,
                                       uint32_t* next, uint32_t* next_count);
__global__ void scc_roots_start_kernel(uint32_t n, const uint32_t* comp, const uint32_t* label,
                                       uint32_t* mark, uint32_t stamp, uint32_t* frontier,
                                       uint32_t* count);
__global__ void scc_search_level_kernel(const uint32_t* rowoff, const uint32_t* rowtgt,
                                        const uint32_t* comp, const uint32_t* color,
                                        uint32_t* mark, uint32_t stamp, const uint32_t* frontier,
                                        uint32_t count, uint32_t* next, uint32_t* next_count);
__global__ void scc_close_kernel(uint32_t n, uint32_t* comp, const uint32_t* label,
                                 const uint32_t* mark, uint32_t stamp,
                                 unsigned long long* placed);
__global__ void scc_count_kernel(uint32_t n, const uint32_t* comp, unsigned long long* count);
__global__ void trim_mask_levels_kernel(uint32_t* level, const uint8_t* mask, uint32_t n);
__global__ void trim_indeg_kernel(const uint32_t* tgt, uint64_t m, uint32_t n, uint32_t* cnt,
                                  uint32_t* bad);
__global__ void trim_scan_blocks_kernel(const uint32_t* in, uint32_t n, uint32_t* out,
                                        uint32_t* block_sums, uint32_t chunk);
__global__ void trim_scan_apply_kernel(uint32_t* out, uint32_t n, const uint32_t* block_sums,
                                       uint32_t nblocks, uint32_t chunk);
__global__ void trim_gt_hist_kernel(const uint32_t* off, const uint32_t* tgt, uint32_t n,
                                    uint32_t rows, uint32_t shift, uint32_t nb, uint32_t* counts,
                                    uint32_t* real);
__global__ void trim_gt_scatter_kernel(const uint32_t* off, const uint32_t* tgt, uint32_t n,
                                       uint32_t rows, uint32_t shift, uint32_t nb,
                                       const uint32_t* slots, unsigned long long* pairs);
__global__ void trim_gt_place_kernel(const unsigned long long* pairs, const uint32_t* slots,
                                     const uint32_t* rstart, uint32_t C, uint32_t n, uint32_t m,
                                     uint32_t shift, uint32_t nb, uint32_t* ioff,
                                     uint32_t* itgt);
__global__ void trim_transpose_fill_kernel(const uint32_t* off, const uint32_t* tgt, uint32_t n,
                                           const uint32_t* ioff, uint32_t* fill, uint32_t* itgt);
__global__ void trim_validate_offsets_kernel(const uint32_t* off, uint32_t n, uint64_t m,
                                             uint32_t* bad);
__global__ void trim_validate_batch_kernel(const uint32_t* off, const uint32_t* tgt, uint32_t n,
                                           const uint32_t* vgraph, uint32_t* bad);
