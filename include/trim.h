/*
 * trim.h -- C ABI of the GB300 graph-trimming library.
 *
 * Computes the trimmed graph of Guo & Sekerinski, "Efficient Parallel Graph
 * Trimming by Arc-Consistency" (arXiv 2107.12720): Definition 1 (the maximal
 * subgraph in which every vertex keeps at least one out-edge) together with
 * the peeling step of every removed vertex (Definition 2, counted from 0).
 *
 * Conventions shared by every entry point:
 *  - Every call returns a trim_err_t; nothing aborts. A failed call leaves the
 *    caller's output buffers untouched; trim_last_error() describes it.
 *  - Vertex ids and CSR offsets are uint32: n <= 2^31 vertices (so that no
 *    grid-stride index can wrap) and m <= 2^32 - 64 edges (so that 32-edge
 *    chunk arithmetic cannot wrap); 0xFFFFFFFF is the LIVE sentinel of
 *    trim_level.
 *  - Device pointers passed in are BORROWED: they must stay valid and unchanged
 *    until trim_destroy(); so are host arrays given as TRIM_MEM_HOST_MAPPED.
 *    Other host pointers are copied during the call.
 *  - A context is bound to one CUDA stream and to the device current at
 *    trim_create(); it is not thread-safe. All device work is ordered on that
 *    stream.
 *  - trim_run() is repeatable: it resets all state, and repeated calls give
 *    bit-identical status and level, whatever variant or schedule is used.
 *  - Nothing here calls into any CPU implementation of the method: if the
 *    device or the kernels are unavailable, calls fail with TRIM_ERR_CUDA or
 *    TRIM_ERR_NO_DEVICE.
 */
#ifndef TRIM_H_
#define TRIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRIM_LIVE 0xFFFFFFFFu
#define TRIM_MASKED 0xFFFFFFFEu /* trim_level of a vertex set DEAD by trim_set_dead_mask */

typedef enum {
  TRIM_OK = 0,
  TRIM_ERR_INVALID_ARG = 1, /* null pointer, size mismatch, unknown enum value       */
  TRIM_ERR_BAD_GRAPH = 2,   /* offsets not monotone, target >= n, csr_in not G^T ... */
  TRIM_ERR_TOO_LARGE = 3,   /* n or m beyond the uint32 limits above                  */
  TRIM_ERR_OOM = 4,         /* device allocation failed (or the memory cap was hit)   */
  TRIM_ERR_CUDA = 5,        /* a CUDA runtime call failed                             */
  TRIM_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out (see spin_limit_ns) */
  TRIM_ERR_STATE = 7,       /* call out of order (e.g. trim_status before trim_run)   */
  TRIM_ERR_NO_DEVICE = 8    /* no CUDA device, or not an sm_103 device                */
} trim_err_t;

/* Per-round kernel choice.
 *  TRIM_AC4_PUSH     Section 5, Algorithm 6: out-degree counters decremented through
 *                    the transposed graph G^T (needs csr_in or builds it on device).
 *  TRIM_AC6_SUPPORT  Section 6, Algorithms 7-8 and Definition 3: one support per
 *                    vertex (edge_index) and supporting sets S; no G^T needed.
 *  TRIM_AC3_PULL     Section 4, Algorithm 4 with the edge_index jump of Section 8:
 *                    a sweep over the vertices still live.
 *  TRIM_SCHED_*      choose one of the three per round on the device:
 *    HEURISTIC       a fixed cost rule on frontier and live-set sizes;
 *    LEARNED         the scheduler MLP set by trim_set_model (falls back to the
 *                    heuristic outside the model's training range or without model);
 *    SCRIPTED        the per-round list given to trim_set_schedule.
 * Every choice yields the same status and level. */
typedef enum {
  TRIM_AC4_PUSH = 0,
  TRIM_AC6_SUPPORT = 1,
  TRIM_AC3_PULL = 2,
  TRIM_SCHED_HEURISTIC = 3,
  TRIM_SCHED_LEARNED = 4,
  TRIM_SCHED_SCRIPTED = 5
} trim_variant_t;

/* A graph in CSR form (Section 2.1 "Graph Storage"): the successors of v are
 * targets[offsets[v] .. offsets[v+1]). offsets has n+1 entries with offsets[0]=0
 * and offsets[n]=m; every target is < n. Successor order is free; duplicate
 * edges and self-loops are allowed (a self-loop keeps its vertex LIVE). */
typedef struct {
  uint32_t n;
  uint64_t m;
  const uint32_t* offsets;
  const uint32_t* targets;
  int on_device; /* where the arrays live: one of TRIM_MEM_* below                */
} trim_csr_t;

/* trim_csr_t.on_device */
#define TRIM_MEM_HOST 0        /* host memory; trim_create copies it to the device          */
#define TRIM_MEM_DEVICE 1      /* device memory of the context's GPU; borrowed, not copied  */
#define TRIM_MEM_HOST_MAPPED 2 /* host memory the kernels read in place (borrowed, never
                                  copied): page-locked memory (cudaHostAlloc,
                                  cudaHostRegister), or any host memory on a system whose
                                  GPU reads pageable memory through the host page tables
                                  (coherent CPU-GPU links such as NVLink-C2C). The kernels
                                  then fetch only the CSR entries they use, over the link;
                                  trim_create fails with TRIM_ERR_INVALID_ARG if the GPU
                                  cannot read the memory. The arrays must stay valid and
                                  unchanged until trim_destroy. */

/* flags of trim_create */
#define TRIM_FLAG_VALIDATE 0x1u  /* check the CSR (and that csr_in is its transpose) on device */
#define TRIM_FLAG_STATS 0x2u     /* count edges inspected, atomics, candidates per run          */
#define TRIM_FLAG_ROUND_LOG 0x4u /* record per-round features and device timestamps            */

/* Tunables (filled by the autotuner; defaults are sensible). */
typedef struct {
  uint32_t block_threads;     /* threads per CTA of the persistent kernel (128..512, x32)  */
  uint32_t ctas_per_sm;       /* persistent CTAs per SM (0 = as many as fit)               */
  uint32_t sched_commit_rounds; /* HEURISTIC / LEARNED: after this many rounds in a row
                                 with the same choice, the run commits to that variant:
                                 the following rounds run it without consulting the
                                 scheduler or gathering its features (0 = never commit) */
  uint32_t sched_recheck_rounds; /* ... a committed stretch lasts this many rounds, then the
                                 scheduler is consulted again (keeping the variant
                                 re-commits at once); each stretch that ends in the same
                                 commit doubles the next one                             */
  uint64_t spin_limit_ns;     /* bound of every device-side wait; past it the run stops
                                 with TRIM_ERR_TIMEOUT                                       */
  float heur_push_ratio;      /* heuristic: push while sum(indeg F) < ratio * n_live        */
  float heur_ac6_ratio;       /* heuristic (no G^T): AC-6 while |F| < ratio * n_live        */
  uint32_t local_round_edges; /* AC-4-only kernel: once the in-edges still to push fit a
                                 small round (at most this many, one work-list entry per
                                 warp), rounds run CTA-locally: each CTA queues the vertices
                                 it removes in shared memory and pushes them itself in the
                                 next round, and a round ends at one barrier that carries
                                 its totals; a round whose removals overflow the queues
                                 returns to ordinary rounds (0 = never local)            */
  float sched_commit_confidence; /* LEARNED: a choice whose softmax probability (among the
                                 variants the run can use) is at least this commits the
                                 run at once, as sched_commit_rounds unchanged choices do
                                 (0 = commit only after sched_commit_rounds)              */
  uint32_t sched_handover;    /* which kernels a scheduled run (trim_run, trim_run_async,
                                 trim_batch_run) uses, and who passes the run between
                                 them when the scheduler picks a variant the running
                                 kernel lacks: TRIM_HANDOVER_*                           */
  uint32_t async_round_edges; /* AC-4 (alone or as a committed scheduled variant), from
                                 round 128 on: once the in-edges still to push are at most
                                 this many, the rest of the run is asynchronous: no
                                 rounds, each CTA pushes the rows of the vertices it
                                 removes at its own pace, and a removed vertex takes one
                                 more than the top level among its successors (Definition
                                 2), carried by the pushes. Same levels and alpha; needs
                                 G^T, off in TRIM_FLAG_ROUND_LOG runs (0 = never)        */
} trim_params_t;

/* trim_params_t.sched_handover */
#define TRIM_HANDOVER_DEVICE 0u /* the run starts on the kernel holding the schedulers and
                                   the variant the mode's last run on this context chose
                                   for round 1 (AC-4 with G^T, else AC-3, the first time);
                                   the kernel holding all three variants is enqueued
                                   behind it and finishes the run if the first kernel
                                   handed it over, or returns at once: no host step      */
#define TRIM_HANDOVER_HOST 1u   /* every segment runs a kernel holding one variant plus the
                                   schedulers; the host reads the control block after each
                                   and launches the next (trim_run_async: as _NONE)      */
#define TRIM_HANDOVER_NONE 2u   /* one launch of the kernel holding all three variants and
                                   the schedulers                                        */

/* Statistics of the last run (sizes in vertices/edges, times in ms). */
typedef struct {
  uint32_t rounds;          /* alpha: number of peeling steps that removed something      */
  uint32_t n_dead;          /* vertices removed                                          */
  float device_ms;          /* trim time between events around the device work          */
  uint64_t edges_inspected; /* TRIM_FLAG_STATS: out-edge targets read by AC-6/AC-3 scans.
                               Scans read targets in groups (4 per thread step, up to 32
                               per warp step) and a scan that resumes after its support
                               reads again the targets its last group loaded past it, so
                               the count can exceed m for AC-6, whose logical inspections
                               are at most m (Section 8)                                */
  uint64_t in_edges_pushed; /* TRIM_FLAG_STATS: in-edges walked by AC-4 (atomics issued)   */
  uint64_t candidates;      /* TRIM_FLAG_STATS: AC-6 supporting-set members re-scanned     */
  uint64_t live_swept;      /* TRIM_FLAG_STATS: AC-3 live-list entries visited             */
  uint32_t rounds_by_variant[3]; /* rounds run by AC-4, AC-6, AC-3                         */
  uint32_t segments;        /* persistent-kernel launches of the run (1 unless a scheduled
                               trim_run switched between variant kernels)               */
  uint32_t local_rounds;    /* AC-4 rounds that ran CTA-locally (see local_round_edges)   */
  uint32_t launches;        /* kernel launches of the run: the control-block reset, every
                               segment, a continuation launch, a dead-mask pass          */
  uint32_t async_round;     /* round from which the run was asynchronous (0: never; see
                               async_round_edges)                                        */
  uint32_t async_removed;   /* vertices the asynchronous part removed                   */
  uint32_t async_rebalances; /* times the asynchronous part spread its pending work evenly
                               over the CTAs again                                       */
} trim_run_stats_t;

/* One record per round of a TRIM_FLAG_ROUND_LOG run. features[] are the
 * scheduler inputs computed before the round r, from round r-1 (F = F_{r-1}):
 *   0 log2(1+|F|)            1 log2(1+sum of in-degrees of F)
 *   2 log2(1+in-edges of removed vertices that AC-4 has not pushed yet)
 *   3 log2(1+live vertices)  4 log2(1+live edges)   5 |F| / live vertices
 *   6 sum of in-degrees of F / live edges
 *   7..9 fractions of F with in-degree < 8, < 256, >= 256
 *   10 log2(1 + ns per frontier vertex of round r-2)  11 variant of round r-1 (-1: none)
 * Live edges: edges between live vertices when G^T is present, out-edges of
 * live vertices without it; the in-degree features are 0 without G^T.
 * Features are computed only for TRIM_SCHED_LEARNED runs and for scheduled
 * runs with TRIM_FLAG_ROUND_LOG; otherwise they are 0. */
typedef struct {
  uint32_t round;        /* r: the round that removes the vertices of level r          */
  uint32_t variant;      /* trim_variant_t actually run (0..2)                        */
  uint32_t frontier;     /* |F_{r-1}|                                                 */
  uint32_t removed;      /* |F_r|                                                     */
  uint64_t t_start_ns;   /* device %globaltimer at the start of the round              */
  uint64_t t_end_ns;     /* ... at its end (after the grid-wide barrier)               */
  uint64_t t_work_ns;    /* ... when CTA 0 finished its share of the work              */
  uint64_t t_flush_ns;   /* ... when CTA 0 finished moving its buffers out             */
  float features[12];
} trim_round_rec_t;

typedef struct trim_ctx trim_ctx;

/* Creates a context for G (csr_out) and optionally G^T (csr_in, may be NULL).
 * csr_in, when given, must be the transpose of csr_out (same n and m; checked
 * when TRIM_FLAG_VALIDATE is set); without it the AC-4 variant builds G^T on the
 * device on first use (a counting sort; its time is not part of trim_run).
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * On success *out receives the context. Allocates device memory ~ (40 n + 4 m) B,
 * plus ~ (20 n + m / 64) B + 128 B per resident GPU thread for the asynchronous
 * AC-4 tail once G^T exists (given here, or built on first use). */
trim_err_t trim_create(const trim_csr_t* csr_out, const trim_csr_t* csr_in, void* cuda_stream,
                       uint32_t flags, trim_ctx** out);

/* Runs the whole trimming (all rounds) with the given variant or scheduler.
 * Returns once status/level are final on the device. stats may be NULL.
 * A fixed variant runs as one persistent launch of a kernel that holds only that
 * variant. A scheduled run (HEURISTIC, LEARNED, SCRIPTED) runs on kernels that
 * hold the schedulers: when the scheduler picks a variant the running kernel
 * lacks, the kernel saves the schedule state and exits, and the next launch
 * resumes at the same round; params.sched_handover says which kernels and who
 * starts the next one (by default no host step at all). Once the scheduler
 * commits (sched_commit_rounds, sched_commit_confidence) the committed rounds
 * skip it inside the same kernel. When the scheduler's only decision of a run
 * (the one before round 1) committed it to one variant for all its rounds, the
 * mode's next run on this context runs that variant's single-variant kernel
 * directly (with TRIM_HANDOVER_DEVICE or _HOST): that decision depends only on
 * the graph, dead mask, model and parameters, and changing any of them clears
 * it. Every schedule and handover yields the same status and level. */
trim_err_t trim_run(trim_ctx* ctx, trim_variant_t variant, trim_run_stats_t* stats);

/* ---- Implicit graphs (Section 2.1, "On-the-fly Property") ----
 * A graph given as G = (v0, POST): no CSR in memory, the successors of a vertex
 * are computed when a kernel needs them. AC-6 and AC-3 only ever read
 * successors, so they run on such a graph (AC-4 needs G^T and cannot; the
 * paper's Table 1). The library's built-in family is a seeded planted graph:
 * vertices C = [0, nC) (core), R = [nC, nC+nR) (reaching set) and
 * T = [nC+nR, n) (trimmable, rank = v - nC - nR), n = nC + nR + nT. With
 *   mix(z):    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
 *              z *= 0x94D049BB133111EB; z ^= z >> 31     (SplitMix64)
 *   key(v)   = mix(seed ^ mix(salt + v + 0x9E3779B97F4A7C15))
 *   word(v,i)= mix(key(v) + (i + 1) * 0x9E3779B97F4A7C15)
 *   below(w,k)= floor(w * k / 2^64)                         (Lemire)
 *   draw(lo,hi) = lo + below(word(v, 0), hi - lo + 1)
 * vertex v has degree k(v) and successors s_j(v), j < k(v), with w = word(v, 1+j):
 *   v in C: k = draw(c_kmin, c_kmax),   s_j = below(w, nC)
 *   v in R: k = draw(r_kmin, r_kmax),   s_0 = below(w, nC), s_j = below(w, nC + nR)
 *   v in T, n_chains = 0: k = 0 if rank < t_sinks else draw(t_kmin, t_kmax);
 *                         s_j = nC + nR + below(w, rank)
 *   v in T, n_chains > 0 (chains, pos = rank / n_chains): k = 0 at pos 0, else
 *                         1 + draw(t_kmin, t_kmax); s_0 = v - n_chains (the chain
 *                         predecessor), s_j = nC + nR + below(w, pos * n_chains).
 * Rows may repeat a successor; that changes no result. nR > 0 needs nC > 0. */
typedef struct {
  uint64_t seed;
  uint64_t salt;
  uint32_t nC, nR, nT;
  uint32_t c_kmin, c_kmax;
  uint32_t r_kmin, r_kmax;
  uint32_t t_sinks, t_kmin, t_kmax;
  uint32_t n_chains;
} trim_implicit_graph_t;

/* Creates a context over an implicit graph (no CSR is copied or stored: memory
 * is O(n)). Only TRIM_AC6_SUPPORT and TRIM_AC3_PULL can run on it (trim_run,
 * trim_run_async); every other call that needs edges in memory (other variants
 * and schedules, trim_run_inout, trim_batch_run, a dead mask) fails with
 * TRIM_ERR_INVALID_ARG. The edge count m (the sum of the degrees) is computed
 * on the device here. flags: TRIM_FLAG_STATS, TRIM_FLAG_ROUND_LOG. */
trim_err_t trim_create_implicit(const trim_implicit_graph_t* g, void* cuda_stream, uint32_t flags,
                                trim_ctx** out);

/* ---- SCC decomposition (Section 1: the use trimming is made for) ----
 * trim_run_scc labels every vertex with its strongly connected component:
 * comp[v] = the smallest vertex id of v's component (the same labels whatever
 * the order of the work). Steps, all on the device, driven from the host:
 *  1. in+out trimming (trim_run_inout): every removed vertex is a size-1
 *     component (it has no in-edge or no out-edge among the others);
 *  2. size-2 trimming: two open vertices that are each other's only open
 *     successor (or each other's only open predecessor) form a component;
 *  3. forward-backward steps (Section 1's FW-BW, from every vertex at once):
 *     forward, every open vertex learns the smallest open vertex that reaches
 *     it (label propagation along G); a vertex r that keeps its own label is
 *     reached by no smaller vertex, and the backward search from r through
 *     G^T among the vertices labelled r collects exactly r's component, whose
 *     smallest member r is. Every step closes at least the component of the
 *     smallest open vertex; independent parts of the graph (the graphs of a
 *     batch) advance together. Before every step, trimming passes remove the
 *     open vertices without an open successor or predecessor (size-1
 *     components that became trimmable, as Figure 1's v6 and v7 do once the
 *     large components are gone).
 * comp: n uint32, on the device if out_on_device else on the host. Needs G^T
 * (csr_in, or built on the device). Overwrites the context's level array (with
 * the in+out trimming of step 1). stats may be NULL. Device memory ~ 24 n
 * bytes is allocated on first use. Not for implicit graphs or with a dead mask
 * (TRIM_ERR_INVALID_ARG). */
typedef struct {
  uint32_t components;       /* number of strongly connected components              */
  uint32_t trimmed_size1;    /* size-1 components removed by step 1                  */
  uint32_t trimmed_size2;    /* size-2 components found by step 2                     */
  uint32_t trimmed_in_steps; /* size-1 components removed by the passes of step 3     */
  uint32_t fwbw_steps;       /* forward-backward steps of step 3                       */
  uint32_t search_levels;    /* frontier levels of the label propagations and backward
                                searches, all steps                                     */
  float ms;                  /* elapsed time on the stream, steps 1-3                 */
} trim_scc_stats_t;
trim_err_t trim_run_scc(trim_ctx* ctx, uint32_t* comp, int out_on_device, trim_scc_stats_t* stats);

/* Vertex sampling (Section 9's scalability experiment samples vertices by setting
 * the unsampled ones DEAD before trimming). mask: n bytes, mask[v] != 0 makes v
 * DEAD from the start (status 0, level TRIM_MASKED); on the device if on_device
 * (device memory of the context's GPU), else on the host; copied, so the caller
 * may free it at once. NULL clears the mask. The mask applies to every later
 * trim_run, trim_run_async and trim_batch_run (any variant or schedule) until it
 * is changed; the result equals trimming the subgraph induced by the unmasked
 * vertices. rounds and n_dead of the run statistics count only vertices removed
 * by trimming. trim_run_inout refuses to run while a mask is set
 * (TRIM_ERR_INVALID_ARG). */
trim_err_t trim_set_dead_mask(trim_ctx* ctx, const uint8_t* mask, int on_device);

/* In+out trimming: removes every vertex that has no live successor OR no live
 * predecessor, repeatedly (Section 4's remark on checking the in-degree when
 * the transposed graph is in memory; Section 1: the size-1 SCC trimming that
 * FW-BW and ISPAN run before and after large-SCC detection). Step 0 removes
 * the vertices without out-edges or without in-edges; step r removes every
 * vertex still present that has no successor or no predecessor among the
 * vertices present after step r-1, and trim_level reports that step (the
 * smaller of the vertex's Definition-2 levels in G and in G^T). Survivors are
 * exactly the vertices that reach a directed cycle and are reached from one.
 * Needs G^T (csr_in, or built on the device on first use, outside the timing).
 * Runs as one persistent launch that pushes, for every removed vertex, both
 * its G^T row (out-degree counters of its predecessors) and its G row
 * (in-degree counters of its successors). Results are read with trim_status /
 * trim_level like those of trim_run; stats may be NULL (in_edges_pushed counts
 * the G^T pushes, edges_inspected the G pushes). Graphs with 2m > 2^32 - 64 are
 * refused with TRIM_ERR_TOO_LARGE (the work list counts both rows of a vertex in
 * uint32 edge offsets). */
trim_err_t trim_run_inout(trim_ctx* ctx, trim_run_stats_t* stats);

/* Enqueues the same work as trim_run without waiting (no host synchronisation,
 * so it may be captured into a CUDA graph): a fixed variant is one persistent
 * launch; a scheduled run is the launches of TRIM_HANDOVER_DEVICE (a first
 * segment and the continuation behind it), or with TRIM_HANDOVER_HOST or _NONE
 * one launch of the kernel holding all three variants. Errors raised on the
 * device surface at the next trim_sync(). */
trim_err_t trim_run_async(trim_ctx* ctx, trim_variant_t variant);
/* Waits for the enqueued work and reports its device-side status; stats may be NULL. */
trim_err_t trim_sync(trim_ctx* ctx, trim_run_stats_t* stats);

/* Output of the last run: out[v] = 1 if v is LIVE (Definition 1), 0 if removed.
 * out has n bytes, on the device if out_on_device else on the host. */
trim_err_t trim_status(const trim_ctx* ctx, uint8_t* out, int out_on_device);

/* Output of the last run: out[v] = the peeling step that removed v (0 for a vertex
 * without out-edges; else 1 + the largest level among its successors, i.e. the
 * length of its longest path to a sink), TRIM_LIVE, or TRIM_MASKED for a vertex
 * the dead mask set DEAD. n uint32 values. */
trim_err_t trim_level(const trim_ctx* ctx, uint32_t* out, int out_on_device);

/* Device pointer to the context's level array (n uint32, valid until the next
 * run or trim_destroy): lets callers read results without a copy. */
trim_err_t trim_level_device_ptr(const trim_ctx* ctx, const uint32_t** out);

/* The context's transposed graph G^T (Section 2's in-edges, as CSR): in_offsets
 * n+1 values, in_targets m values, the predecessors of v in
 * in_targets[in_offsets[v] .. in_offsets[v+1]) (their order within a row is
 * unspecified). If the context was created without csr_in, G^T is built on
 * the device first (and kept for AC-4 runs). Both outputs on the device if
 * out_on_device, else on the host. Fails with TRIM_ERR_INVALID_ARG on an
 * implicit graph. */
trim_err_t trim_in_csr(trim_ctx* ctx, uint32_t* in_offsets, uint32_t* in_targets,
                       int out_on_device);

/* Batched trimming of G independent graphs packed into the context's CSR:
 * graph g owns vertices [graph_off[g], graph_off[g+1]) and no edge may cross two
 * graphs (checked with TRIM_FLAG_VALIDATE). graph_off: G+1 host uint32 values,
 * graph_off[0]=0, graph_off[G]=n. The packed CSR is the disjoint union of the
 * graphs, so all of them are trimmed together: every round serves every graph
 * still peeling. A fixed variant is one persistent launch, captured into a
 * CUDA graph on the second call with the same variant and replayed from then
 * on; a scheduled variant runs as trim_run runs it. Results equal
 * trimming each graph alone: read them with trim_status / trim_level. */
trim_err_t trim_batch_run(trim_ctx* ctx, const uint32_t* graph_off, uint32_t G,
                          trim_variant_t variant, trim_run_stats_t* stats);

trim_err_t trim_set_params(trim_ctx* ctx, const trim_params_t* params);
trim_err_t trim_get_params(const trim_ctx* ctx, trim_params_t* params);
/* Default tunables for the current device (no context needed). */
trim_err_t trim_default_params(trim_params_t* params);

/* Scheduler MLP (12 -> 32 -> 32 -> 3, ReLU), TRIM_MLP_NPARAMS fp32 values laid
 * out as W1[32][12] b1[32] W2[32][32] b2[32] W3[3][32] b3[3], followed by the
 * input normalisation mean[12], inv_std[12] and the training range lo[12],
 * hi[12] (TRIM_MLP_NBLOB floats in all). Host pointer, copied. */
#define TRIM_MLP_NIN 12
#define TRIM_MLP_NH 32
#define TRIM_MLP_NOUT 3
#define TRIM_MLP_NPARAMS 1571
#define TRIM_MLP_NBLOB (TRIM_MLP_NPARAMS + 4 * TRIM_MLP_NIN)
trim_err_t trim_set_model(trim_ctx* ctx, const float* blob, size_t n_floats);

/* Per-round variant list for TRIM_SCHED_SCRIPTED (host pointer, copied): round r
 * (1-based) runs variants[(r-1) % len]; each entry 0..2. */
trim_err_t trim_set_schedule(trim_ctx* ctx, const uint8_t* variants, uint32_t len);

/* Copies up to cap records of the last TRIM_FLAG_ROUND_LOG run to out (host). */
trim_err_t trim_get_round_log(const trim_ctx* ctx, trim_round_rec_t* out, size_t cap,
                              size_t* n_out);

void trim_destroy(trim_ctx* ctx);

/* Process-wide cap on the device bytes one context may allocate (0 = no cap).
 * Allocations past it fail with TRIM_ERR_OOM, which lets callers (and tests)
 * exercise out-of-memory paths without exhausting the device. */
trim_err_t trim_set_alloc_limit(uint64_t bytes);

/* Message of the last failed call on ctx (with ctx NULL: of the last failed
 * call that takes no context, such as trim_create). Never NULL. */
const char* trim_last_error(const trim_ctx* ctx);

/* ---- scheduler MLP training kernels (plain fp32, no tensor cores) ----
 * All pointers are DEVICE pointers; work is enqueued on cuda_stream.
 * X: [N][12] fp32 features, y: [N] uint8 labels in 0..2,
 * params: TRIM_MLP_NPARAMS fp32 (layout above, without the normalisation tail;
 * inputs are used as given).
 *
 * trim_mlp_forward: logits[N][3].
 * trim_mlp_loss_grad: mean softmax cross-entropy over the N rows into *loss
 *   (device float) and its gradient w.r.t. params into grad (TRIM_MLP_NPARAMS).
 *   scratch: device buffer of at least trim_mlp_scratch_bytes(N) bytes.
 * trim_mlp_adam_step: one Adam update (Kingma & Ba, 2015) of params from grad;
 *   m, v: TRIM_MLP_NPARAMS fp32 moment buffers; t: the 1-based step number. */
size_t trim_mlp_scratch_bytes(uint32_t N);
trim_err_t trim_mlp_forward(const float* params, const float* X, uint32_t N, float* logits,
                            void* cuda_stream);
trim_err_t trim_mlp_loss_grad(const float* params, const float* X, const uint8_t* y, uint32_t N,
                              float* loss, float* grad, void* scratch, void* cuda_stream);
trim_err_t trim_mlp_adam_step(float* params, const float* grad, float* m, float* v, uint32_t t,
                              float lr, float beta1, float beta2, float eps, void* cuda_stream);

/* ---- Diagnostic: the device's L2 atomic ceiling (no counterpart in the paper) ----
 * AC-4 issues one returning atomicSub per in-edge it pushes; on large frontiers
 * its time is bound by how many such atomics the L2 completes per second, not
 * by DRAM bandwidth. trim_probe_atomic_rate measures that ceiling for a given
 * stream of counter indices: it sets counters[0..n_counters) to 0xFFFFFFFF and
 * runs one fully parallel kernel that applies atomicSub(&counters[idx[i]], 1)
 * for i in [0, n_idx) and keeps the returned values (as AC-4 does), timed with
 * CUDA events on cuda_stream; the kernel runs `reps` times and *ms_out receives
 * the fastest. idx (n_idx values, each < n_counters) and counters are DEVICE
 * pointers owned by the caller; counters is overwritten. Waits for the stream.
 * Errors: TRIM_ERR_INVALID_ARG for null pointers, n_idx = 0, n_counters = 0 or
 * reps = 0; TRIM_ERR_CUDA if a launch fails. */
trim_err_t trim_probe_atomic_rate(const uint32_t* idx, uint64_t n_idx, uint32_t* counters,
                                  uint32_t n_counters, uint32_t reps, void* cuda_stream,
                                  float* ms_out);

/* ---- Trimming without any device allocation (no counterpart in the paper) ----
 * For callers that cannot call cudaMalloc when they need a result: processes
 * under an allocator discipline that forbids new device allocations, plugins
 * that must not touch the host application's allocator, or paths that must
 * not synchronise the device the way cudaMalloc/cudaFree can.
 *
 * trim_run_ac4_noalloc runs the same AC-4 kernel as trim_run(TRIM_AC4_PUSH) and
 * writes the same levels, but takes all its scratch (counters, dead log, AC-4
 * work list, control block) from one fixed __device__ array compiled into the
 * library: TRIM_NOALLOC_SCRATCH_BYTES per GPU, held by every GPU that loads the
 * library until the process exits. Nothing is allocated per call.
 *
 * All pointers are DEVICE pointers supplied by the caller: the graph in CSR
 * (offsets n+1, targets m), its transpose G^T (in_offsets n+1, in_targets m;
 * the caller builds it, e.g. once with trim_create + a trim_run of AC-4 on a
 * context, or on its own), and level_out (n uint32: levels as trim_level,
 * TRIM_LIVE for survivors). rounds_out (host, nullable) receives alpha.
 * Sizes above TRIM_NOALLOC_MAX_N vertices or TRIM_NOALLOC_MAX_M edges are
 * rejected with TRIM_ERR_TOO_LARGE before any device work. The arrays
 * themselves are not checked (as with trim_create without TRIM_FLAG_VALIDATE):
 * offsets must be monotone with offsets[n] = m, every target < n, and
 * (in_offsets, in_targets) exactly the transpose of (offsets, targets);
 * otherwise the kernel may write outside level_out or the scratch array.
 * cuda_stream must belong to the current device (NULL: its legacy default
 * stream); a stream of another device is refused with TRIM_ERR_INVALID_ARG.
 *
 * The first call on each device (with that device current) looks up the
 * array's device address and the launch shape; make that first call before
 * any stream capture. Every call on a device uses the same array, which keeps
 * the previous call's contents (the call clears what must start at zero):
 * calls whose GPU work overlaps (several streams, several host threads) race
 * on it and must be serialised by the caller. The call waits for its work on
 * cuda_stream before it returns, to report device-side errors. */
#define TRIM_NOALLOC_MAX_N (1u << 18)
#define TRIM_NOALLOC_MAX_M (1u << 22)
#define TRIM_NOALLOC_SCRATCH_BYTES 5769472u
trim_err_t trim_run_ac4_noalloc(const uint32_t* offsets, const uint32_t* targets,
                                const uint32_t* in_offsets, const uint32_t* in_targets,
                                uint32_t n, uint32_t m, uint32_t* level_out,
                                uint32_t* rounds_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TRIM_H_ */
