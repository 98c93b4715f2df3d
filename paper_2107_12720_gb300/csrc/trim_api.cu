// trim_api.cu -- the C ABI (include/trim.h): contexts, device memory, launches.
//
// Host code only marshals: every step of the trimming runs in the kernels of
// trim_kernels.cu. There is no CPU implementation of the method behind this ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "trim_internal.cuh"

using trimk::Ctrl;
using trimk::Dev;

namespace {

thread_local std::string g_create_error = "no error";
uint64_t g_alloc_limit = 0;  // process-wide cap on bytes one context may allocate (0 = none)

}  // namespace

struct trim_ctx {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  uint32_t flags = 0;
  uint32_t n = 0;
  uint64_t m = 0;
  const uint32_t* off = nullptr;
  const uint32_t* tgt = nullptr;
  const uint32_t* ioff = nullptr;
  const uint32_t* itgt = nullptr;
  std::vector<void*> owned;  // every device allocation of this context (library pool)
  uint64_t allocated = 0;
  uint32_t *level = nullptr, *cnt = nullptr, *supp = nullptr, *s_head = nullptr,
           *s_next = nullptr, *s_cnt = nullptr, *s_off = nullptr, *s_list = nullptr,
           *log = nullptr, *roff = nullptr, *live0 = nullptr, *live1 = nullptr, *bsum = nullptr;
  uint32_t *w4_row = nullptr, *w4_eoff = nullptr, *chunk_first = nullptr;
  // asynchronous AC-4 tail: per-vertex words, the global list of G^T row
  // pieces and the two rebalance entry lists (allocated once G^T exists)
  unsigned long long* aw = nullptr;
  uint32_t *oq_row = nullptr, *oq_len = nullptr, *oq_lev = nullptr;
  uint32_t oq_cap = 0;
  uint32_t *ae_id = nullptr, *ae_lev = nullptr;
  uint32_t ae_cap = 0;
  // in+out runs: in-degree counters, the work list's G rows and in-degrees, and
  // the chunk-owner index of its edge space (both rows: up to 2m edges)
  uint32_t *cnt_in = nullptr, *w4_orow = nullptr, *w4_din = nullptr, *chunk_io = nullptr;
  uint8_t* mask = nullptr;  // trim_set_dead_mask: device copy of the dead mask
  bool has_mask = false;
  bool implicit = false;      // trim_create_implicit: successors computed, no CSR
  trim_implicit_graph_t ig{};
  // trim_run_scc: component labels, propagated labels, label-frontier stamps,
  // backward-search marks, two frontiers, counters (allocated on first use)
  uint32_t *scc_comp = nullptr, *scc_color = nullptr, *scc_fw = nullptr, *scc_bw = nullptr,
           *scc_fa = nullptr, *scc_fb = nullptr;
  unsigned long long* scc_cnt = nullptr;
  uint32_t scc_stamp = 0;  // last search stamp: marks of earlier runs stay below it
  cudaEvent_t scc_ev0 = nullptr, scc_ev1 = nullptr;
  Ctrl* ctrl = nullptr;
  Ctrl* h_ctrl = nullptr;  // host mirror of the control block for read-back
  bool h_ctrl_pinned = false;
  trim_round_rec_t* rlog = nullptr;
  uint32_t rlog_cap = 0;
  float* model = nullptr;
  bool has_model = false;
  uint8_t* script = nullptr;
  uint32_t script_len = 0;
  uint8_t* status_tmp = nullptr;
  trim_params_t params{};
  int grids[10] = {};  // cooperative grid size of each kernel flavour
  trimk::Dev last_dev{};        // arguments of the last launch (segments reuse them)
  int seg_first[3] = {-1, -1, -1};  // per scheduled mode: flavour of its last first round
  uint64_t last_segments = 0;       // segments of the last trim_run
  uint64_t last_launches = 0;       // kernel launches of the last trim_run
  int cont_mode = -1;               // the pending run has a continuation launch: its mode
  int sched_mode = -1;              // the pending run is scheduled: its mode
  // per scheduled mode: the variant of its last run on this context if that
  // run's only scheduler decision (before round 1) committed it for good
  int seg_whole[3] = {-1, -1, -1};
  std::vector<uint8_t> h_script;    // host copy of the scripted schedule
  cudaGraphExec_t batch_exec = nullptr;  // captured batched launch (trim_batch_run)
  cudaStream_t cap_stream = nullptr;      // private stream used only for that capture
  bool capturing = false;
  int batch_variant = -1;
  int batch_last_variant = -1;
  bool ran = false;
  bool pending = false;
  bool s_cnt_dirty = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err = "no error";
  trim_run_stats_t last{};
};

namespace {

trim_err_t fail(trim_ctx* c, trim_err_t code, const std::string& msg) {
  if (c) c->err = msg; else g_create_error = msg;
  return code;
}

// The graph, its dead mask, the model or the parameters changed: a scheduled
// run's round-1 choice may differ from the one its last run made.
void forget_first_flavours(trim_ctx* c) {
  c->seg_first[0] = c->seg_first[1] = c->seg_first[2] = -1;
  c->seg_whole[0] = c->seg_whole[1] = c->seg_whole[2] = -1;
}

trim_err_t cuda_fail(trim_ctx* c, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, TRIM_ERR_OOM, msg);
  return fail(c, TRIM_ERR_CUDA, msg);
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);        \
  } while (0)

// Device memory comes from a stream-ordered pool owned by the library (one per
// device): freeing a context returns its memory to the pool instead of
// unmapping it, so creating and destroying contexts stays cheap. Up to
// kPoolKeepBytes stay reserved between contexts; the rest goes back to the
// system at the next synchronisation.
constexpr uint64_t kPoolKeepBytes = 4ull << 30;
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};

cudaError_t device_pool(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = kPoolKeepBytes;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return e;
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

template <class T>
trim_err_t dalloc(trim_ctx* c, T** p, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (g_alloc_limit && c->allocated + bytes > g_alloc_limit)
    return fail(c, TRIM_ERR_OOM, "device memory cap reached");
  void* q = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = device_pool(c->device, &pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&q, bytes, pool, c->stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_fail(c, e, "cudaMallocFromPoolAsync");
  }
  c->owned.push_back(q);
  c->allocated += bytes;
  *p = static_cast<T*>(q);
  return TRIM_OK;
}

// Returns a temporary allocation of dalloc to the pool (stream-ordered).
template <class T>
void dfree(trim_ctx* c, T* p, size_t count) {
  if (!p) return;
  auto it = std::find(c->owned.begin(), c->owned.end(), static_cast<void*>(p));
  if (it == c->owned.end()) return;
  c->owned.erase(it);
  c->allocated -= std::max<size_t>(count, 1) * sizeof(T);
  cudaFreeAsync(p, c->stream);
}

// Carves 256-byte aligned pieces out of one device allocation (an "arena"),
// so a context costs one cudaMalloc and one cudaFree instead of one per array.
struct ArenaPlan {
  size_t bytes = 0;
  template <class T>
  size_t add(size_t count) {
    const size_t at = bytes;
    bytes += (std::max<size_t>(count, 1) * sizeof(T) + 255) & ~size_t(255);
    return at;
  }
};

#define TRY(x)                       \
  do {                               \
    trim_err_t t_ = (x);             \
    if (t_ != TRIM_OK) return t_;    \
  } while (0)

// Page-locked host slots for the control-block mirrors: a read-back into
// page-locked memory is a short DMA, into pageable memory a staged copy. The
// slots come from one block allocated on first use and shared by all contexts
// of the process (page-locking per context would cost more than it saves).
constexpr int kCtrlSlots = 64;
std::mutex g_slot_mutex;
char* g_slot_block = nullptr;
bool g_slot_used[kCtrlSlots] = {};
constexpr size_t kSlotBytes = (sizeof(Ctrl) + 255) / 256 * 256;

Ctrl* take_ctrl_slot() {
  std::lock_guard<std::mutex> lock(g_slot_mutex);
  if (!g_slot_block) {
    void* p = nullptr;
    if (cudaHostAlloc(&p, kSlotBytes * kCtrlSlots, cudaHostAllocPortable) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    g_slot_block = static_cast<char*>(p);
  }
  for (int i = 0; i < kCtrlSlots; ++i)
    if (!g_slot_used[i]) {
      g_slot_used[i] = true;
      return new (g_slot_block + i * kSlotBytes) Ctrl();
    }
  return nullptr;
}

void give_ctrl_slot(Ctrl* h) {
  std::lock_guard<std::mutex> lock(g_slot_mutex);
  const int i = (int)((reinterpret_cast<char*>(h) - g_slot_block) / (ptrdiff_t)kSlotBytes);
  if (i >= 0 && i < kCtrlSlots) g_slot_used[i] = false;
}

void release(trim_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (void* p : c->owned) cudaFreeAsync(p, c->stream);
  c->owned.clear();
  if (c->h_ctrl_pinned) give_ctrl_slot(c->h_ctrl);
  else delete c->h_ctrl;
  c->h_ctrl = nullptr;
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->scc_ev0) cudaEventDestroy(c->scc_ev0);
  if (c->scc_ev1) cudaEventDestroy(c->scc_ev1);
}

trim_err_t check_device(trim_ctx* c, int* dev, int* sms) {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    (void)cudaGetLastError();
    return fail(c, TRIM_ERR_NO_DEVICE, "no CUDA device available");
  }
  CK(cudaGetDevice(dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, *dev));
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(c, TRIM_ERR_NO_DEVICE,
                "this library is built for sm_103a (GB300); device is sm_" +
                    std::to_string(prop.major) + std::to_string(prop.minor));
  *sms = prop.multiProcessorCount;
  return TRIM_OK;
}

void default_params(trim_params_t* p) {
  p->block_threads = 512;
  p->ctas_per_sm = 0;
  p->sched_commit_rounds = 8;
  p->sched_recheck_rounds = 128;
  p->spin_limit_ns = 5ull * 1000 * 1000 * 1000;  // 5 s
  p->heur_push_ratio = 1.0f;
  p->heur_ac6_ratio = 1.0f;
  p->local_round_edges = 1u << 18;
  p->sched_commit_confidence = 0.9f;
  p->sched_handover = TRIM_HANDOVER_DEVICE;
  p->async_round_edges = 1u << 18;
}

// per-warp append slices in dynamic shared memory: 4 buffers (dead log, AC-4
// work-list rows and edge offsets, AC-3 live list) of kSliceEntries words per
// warp of the block (64 KB for 512 threads)
constexpr uint32_t kSliceEntries = 256;
constexpr uint32_t kSbufCap = kSliceEntries;
size_t dyn_smem_bytes(uint32_t block_threads) {
  return (block_threads / 32) * 4 * (size_t)kSliceEntries * sizeof(uint32_t);
}

// kernel flavours: index 0..3 = AC-4 only, AC-6 only, AC-3 only, everything;
// 4..6 = AC-4, AC-6, AC-3 each with the per-round schedulers (segments);
// 7 = in+out trimming; 8, 9 = AC-6, AC-3 on an implicit graph
typedef void (*persistent_fn)(trimk::Dev);
constexpr int kNumFlavours = 10;
constexpr int kFlavourAll = 3;
constexpr int kFlavourSeg = 4;  // + variant
constexpr int kFlavourInout = 7;
constexpr int kFlavourImplicitAC6 = 8, kFlavourImplicitAC3 = 9;
const persistent_fn kFlavours[kNumFlavours] = {
    trim_persistent_kernel_m1,  trim_persistent_kernel_m2,  trim_persistent_kernel_m4,
    trim_persistent_kernel_m15, trim_persistent_kernel_m9,  trim_persistent_kernel_m10,
    trim_persistent_kernel_m12, trim_persistent_kernel_m17, trim_persistent_kernel_m34,
    trim_persistent_kernel_m36};

// launch shapes are a property of the device and the block size: computed once
// per (device, block_threads, ctas_per_sm) for the whole process
struct GridCache {
  int device = -1;
  uint32_t block = 0, cps = 0;
  int grids[kNumFlavours] = {};
};
std::mutex g_grid_mutex;
GridCache g_grid_cache[8];

trim_err_t compute_grid(trim_ctx* c) {
  std::lock_guard<std::mutex> lock(g_grid_mutex);
  for (const GridCache& e : g_grid_cache)
    if (e.device == c->device && e.block == c->params.block_threads &&
        e.cps == c->params.ctas_per_sm) {
      for (int k = 0; k < kNumFlavours; ++k) c->grids[k] = e.grids[k];
      return TRIM_OK;
    }
  for (int k = 0; k < kNumFlavours; ++k) {
    int per_sm = 0;
    CK(cudaFuncSetAttribute(kFlavours[k], cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)dyn_smem_bytes(512)));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kFlavours[k],
                                                     (int)c->params.block_threads,
                                                     dyn_smem_bytes(c->params.block_threads)));
    if (per_sm <= 0) return fail(c, TRIM_ERR_INVALID_ARG, "block_threads does not fit on an SM");
    if (c->params.ctas_per_sm) per_sm = std::min<int>(per_sm, (int)c->params.ctas_per_sm);
    c->grids[k] = per_sm * c->sm_count;
  }
  for (GridCache& e : g_grid_cache)
    if (e.device < 0) {
      e.device = c->device;
      e.block = c->params.block_threads;
      e.cps = c->params.ctas_per_sm;
      for (int k = 0; k < kNumFlavours; ++k) e.grids[k] = c->grids[k];
      break;
    }
  return TRIM_OK;
}

trim_err_t sync_check(trim_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  return TRIM_OK;
}

// Waits for the stream and copies the control block to the host mirror.
trim_err_t read_ctrl(trim_ctx* c) {
  CK(cudaMemcpyAsync(c->h_ctrl, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
  return sync_check(c);
}

// exclusive scan of in[0..n) into out[0..n], out[n] = total (device, on c->stream)
trim_err_t device_scan(trim_ctx* c, const uint32_t* in, uint32_t n, uint32_t* out) {
  const uint32_t nb = std::max<uint32_t>(1, std::min<uint32_t>(1024, (n + 4095) / 4096));
  const uint32_t chunk = (n + nb - 1) / nb;
  uint32_t* sums = nullptr;
  TRY(dalloc(c, &sums, nb));
  trim_scan_blocks_kernel<<<nb, 512, 0, c->stream>>>(in, n, out, sums, chunk);
  CK(cudaGetLastError());
  trim_scan_apply_kernel<<<nb, 512, 0, c->stream>>>(out, n, sums, nb, chunk);
  CK(cudaGetLastError());
  return TRIM_OK;
}

// The asynchronous AC-4 tail's per-vertex words, its global list of G^T row
// pieces and its two rebalance entry lists, allocated once G^T exists
// (kernels without them never start the tail). An entry list holds every
// queue of a cooperative grid: 8 entries per resident thread.
trim_err_t alloc_async(trim_ctx* c) {
  if (c->aw != nullptr) return TRIM_OK;
  const uint64_t cap = trimk::async_queue_cap(c->n, c->m);  // < 2^32: n <= 2^31, m < 2^32
  int per_sm = 0;
  CK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, c->device));
  const uint64_t ecap = (uint64_t)c->sm_count * (uint64_t)per_sm * 8u;
  TRY(dalloc(c, &c->aw, c->n));
  TRY(dalloc(c, &c->oq_row, cap));
  TRY(dalloc(c, &c->oq_len, cap));
  TRY(dalloc(c, &c->oq_lev, cap));
  TRY(dalloc(c, &c->ae_id, 2 * ecap));
  TRY(dalloc(c, &c->ae_lev, 2 * ecap));
  c->oq_cap = (uint32_t)cap;
  c->ae_cap = (uint32_t)ecap;
  return TRIM_OK;
}

// G^T on the device (the transposed graph of Section 2), by a counting sort
// whose counts and placements are shared-memory atomics (trim_gt_*_kernel: no
// same-address global atomics on hub targets); graphs with more than 2^27
// vertices use the direct global counting sort.
trim_err_t build_transpose(trim_ctx* c) {
  const uint32_t n = c->n;
  const uint32_t m = (uint32_t)c->m;  // offsets are uint32: m < 2^32
  uint32_t *ioff = nullptr, *itgt = nullptr;
  TRY(dalloc(c, &ioff, (size_t)n + 1));
  TRY(dalloc(c, &itgt, m));
  uint32_t lg = 0;
  while (lg < 32 && (1ull << lg) < n) ++lg;
  if (m == 0) {
    CK(cudaMemsetAsync(ioff, 0, ((size_t)n + 1) * 4, c->stream));
  } else if (lg <= 27) {
    // buckets of 2^shift targets, at most 32,768 each (128 KB of counters in
    // pass 4): up to 2^26 vertices 2,048 buckets and two CTAs per SM in passes
    // 1 and 3 (96 KB of shared memory each in pass 3), above that 4,096
    // buckets and one CTA per SM; either way the open sectors of all (bucket,
    // CTA) ranges, 32 B each, stay in the L2
    const bool wide = lg > 26;
    const uint32_t keep = wide ? 12u : 11u;
    const uint32_t shift = lg > keep ? lg - keep : 0;
    const uint32_t nb = (uint32_t)(((uint64_t)n + (1u << shift) - 1) >> shift);
    const uint32_t C = (uint32_t)c->sm_count * (wide ? 1u : 2u);
    const uint32_t rows = (n + C - 1) / C;
    // (bucket, CTA) ranges hold whole sectors: up to 3 unused slots each
    const size_t cap = (size_t)m + 3 * (size_t)nb * C;
    uint32_t *counts = nullptr, *slots = nullptr, *real = nullptr, *rstart = nullptr;
    unsigned long long* pairs = nullptr;
    TRY(dalloc(c, &counts, (size_t)nb * C));
    TRY(dalloc(c, &slots, (size_t)nb * C + 1));
    TRY(dalloc(c, &real, nb));
    TRY(dalloc(c, &rstart, (size_t)nb + 1));
    TRY(dalloc(c, &pairs, cap));
    CK(cudaMemsetAsync(real, 0, (size_t)nb * 4, c->stream));
    const size_t hist_bytes = (size_t)nb * 4, scatter_bytes = (size_t)nb * 48;
    const size_t place_bytes = ((size_t)1 << shift) * 4;
    CK(cudaFuncSetAttribute(trim_gt_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)scatter_bytes));
    CK(cudaFuncSetAttribute(trim_gt_place_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)place_bytes));
    trim_gt_hist_kernel<<<C, 1024, hist_bytes, c->stream>>>(c->off, c->tgt, n, rows, shift, nb,
                                                            counts, real);
    CK(cudaGetLastError());
    TRY(device_scan(c, counts, nb * C, slots));
    TRY(device_scan(c, real, nb, rstart));
    trim_gt_scatter_kernel<<<C, 1024, scatter_bytes, c->stream>>>(c->off, c->tgt, n, rows, shift,
                                                                  nb, slots, pairs);
    CK(cudaGetLastError());
    trim_gt_place_kernel<<<std::min<uint32_t>(nb, (uint32_t)c->sm_count * 4), 512, place_bytes,
                           c->stream>>>(pairs, slots, rstart, C, n, m, shift, nb, ioff, itgt);
    CK(cudaGetLastError());
    dfree(c, pairs, cap);
    dfree(c, rstart, (size_t)nb + 1);
    dfree(c, real, nb);
    dfree(c, slots, (size_t)nb * C + 1);
    dfree(c, counts, (size_t)nb * C);
  } else {
    uint32_t *fill = nullptr, *bad = nullptr;
    TRY(dalloc(c, &fill, (size_t)n + 1));
    TRY(dalloc(c, &bad, 1));
    CK(cudaMemsetAsync(fill, 0, ((size_t)n + 1) * 4, c->stream));
    CK(cudaMemsetAsync(bad, 0, 4, c->stream));
    const int blocks = c->sm_count * 8;
    trim_indeg_kernel<<<blocks, 512, 0, c->stream>>>(c->tgt, m, n, fill, bad);
    CK(cudaGetLastError());
    TRY(device_scan(c, fill, n, ioff));
    CK(cudaMemsetAsync(fill, 0, ((size_t)n + 1) * 4, c->stream));
    trim_transpose_fill_kernel<<<blocks, 512, 0, c->stream>>>(c->off, c->tgt, n, ioff, fill, itgt);
    CK(cudaGetLastError());
    dfree(c, bad, 1);
    dfree(c, fill, (size_t)n + 1);
  }
  TRY(sync_check(c));
  c->ioff = ioff;
  c->itgt = itgt;
  TRY(alloc_async(c));
  forget_first_flavours(c);
  return TRIM_OK;
}

trim_err_t validate(trim_ctx* c, const uint32_t* ioff_given) {
  uint32_t *bad = nullptr, *indeg = nullptr;
  TRY(dalloc(c, &bad, 1));
  TRY(dalloc(c, &indeg, (size_t)c->n + 1));
  CK(cudaMemsetAsync(bad, 0, 4, c->stream));
  CK(cudaMemsetAsync(indeg, 0, ((size_t)c->n + 1) * 4, c->stream));
  const int blocks = c->sm_count * 8;
  trim_validate_offsets_kernel<<<blocks, 512, 0, c->stream>>>(c->off, c->n, c->m, bad);
  CK(cudaGetLastError());
  uint32_t hbad = 0;
  CK(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_check(c));
  if (hbad) return fail(c, TRIM_ERR_BAD_GRAPH, "csr_out: offsets not monotone or off[n] != m");
  if (c->m) {
    trim_indeg_kernel<<<blocks, 512, 0, c->stream>>>(c->tgt, c->m, c->n, indeg, bad);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_check(c));
  if (hbad) return fail(c, TRIM_ERR_BAD_GRAPH, "csr_out: a target is >= n");
  if (ioff_given) {
    trim_validate_offsets_kernel<<<blocks, 512, 0, c->stream>>>(ioff_given, c->n, c->m, bad);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, c->stream));
    TRY(sync_check(c));
    if (hbad) return fail(c, TRIM_ERR_BAD_GRAPH, "csr_in: offsets not monotone or off[n] != m");
    // G^T must list every edge once: its degrees equal the in-degree histogram of
    // csr_out, and the multiset of (source, target) pairs matches (checked by
    // building G^T here and comparing row by row after sorting).
    const uint32_t* keep_ioff = c->ioff;
    const uint32_t* keep_itgt = c->itgt;
    TRY(build_transpose(c));
    std::vector<uint32_t> a((size_t)c->n + 1), b((size_t)c->n + 1);
    CK(cudaMemcpy(a.data(), c->ioff, a.size() * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(b.data(), keep_ioff, b.size() * 4, cudaMemcpyDeviceToHost));
    if (a != b) return fail(c, TRIM_ERR_BAD_GRAPH, "csr_in is not the transpose (degrees differ)");
    std::vector<uint32_t> ta(c->m), tb(c->m);
    if (c->m) {
      CK(cudaMemcpy(ta.data(), c->itgt, c->m * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(tb.data(), keep_itgt, c->m * 4, cudaMemcpyDeviceToHost));
    }
    for (uint32_t v = 0; v < c->n; ++v) {
      std::sort(ta.begin() + a[v], ta.begin() + a[v + 1]);
      std::sort(tb.begin() + a[v], tb.begin() + a[v + 1]);
    }
    if (ta != tb) return fail(c, TRIM_ERR_BAD_GRAPH, "csr_in is not the transpose (edges differ)");
    c->ioff = keep_ioff;
    c->itgt = keep_itgt;
  }
  return TRIM_OK;
}

// Device-side address of host memory the kernels read in place
// (TRIM_MEM_HOST_MAPPED): page-locked memory maps through its device pointer;
// other host memory only where the GPU walks the host page tables.
trim_err_t map_host(trim_ctx* c, const uint32_t* p, const uint32_t** out) {
  *out = nullptr;
  if (p == nullptr) return TRIM_OK;
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) (void)cudaGetLastError();
  if (e == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer != nullptr) {
    *out = static_cast<const uint32_t*>(at.devicePointer);
    return TRIM_OK;
  }
  if (e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged))
    return fail(c, TRIM_ERR_INVALID_ARG, "TRIM_MEM_HOST_MAPPED given device memory");
  int pageable = 0;
  CK(cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccessUsesHostPageTables,
                            c->device));
  if (!pageable)
    return fail(c, TRIM_ERR_INVALID_ARG,
                "host memory is not readable by this GPU: page-lock it or use TRIM_MEM_HOST");
  *out = p;
  return TRIM_OK;
}

trim_err_t create_impl(const trim_csr_t* g, const trim_csr_t* gi, void* stream, uint32_t flags,
                       trim_ctx* c) {
  if (g->on_device < TRIM_MEM_HOST || g->on_device > TRIM_MEM_HOST_MAPPED ||
      (gi && (gi->on_device < TRIM_MEM_HOST || gi->on_device > TRIM_MEM_HOST_MAPPED)))
    return fail(c, TRIM_ERR_INVALID_ARG, "on_device must be one of TRIM_MEM_*");
  if (g->n > (1u << 31) || g->m > (1ull << 32) - 64)
    return fail(c, TRIM_ERR_TOO_LARGE, "n must be <= 2^31 and m <= 2^32 - 64");
  if (g->offsets == nullptr || (g->m && g->targets == nullptr))
    return fail(c, TRIM_ERR_INVALID_ARG, "csr_out: null array");
  if (gi) {
    if (gi->n != g->n || gi->m != g->m)
      return fail(c, TRIM_ERR_INVALID_ARG, "csr_in: n and m must equal those of csr_out");
    if (gi->offsets == nullptr || (gi->m && gi->targets == nullptr))
      return fail(c, TRIM_ERR_INVALID_ARG, "csr_in: null array");
  }
  if (g->on_device == TRIM_MEM_HOST && g->n) {
    // cheap host checks before any device work
    if (g->offsets[0] != 0 || (uint64_t)g->offsets[g->n] != g->m)
      return fail(c, TRIM_ERR_BAD_GRAPH, "csr_out: offsets[0] != 0 or offsets[n] != m");
  }
  TRY(check_device(c, &c->device, &c->sm_count));
  if (g->on_device == TRIM_MEM_HOST_MAPPED && g->n) {
    // the same checks once the memory is known to be host memory
    const uint32_t* probe = nullptr;
    TRY(map_host(c, g->offsets, &probe));
    if (g->offsets[0] != 0 || (uint64_t)g->offsets[g->n] != g->m)
      return fail(c, TRIM_ERR_BAD_GRAPH, "csr_out: offsets[0] != 0 or offsets[n] != m");
  }
  c->stream = static_cast<cudaStream_t>(stream);
  c->flags = flags;
  c->n = g->n;
  c->m = g->m;
  default_params(&c->params);
  CK(cudaEventCreate(&c->ev0));
  CK(cudaEventCreate(&c->ev1));
  // one arena: copies of host inputs, then all per-run state
  const size_t n = c->n;
  if (flags & TRIM_FLAG_ROUND_LOG) c->rlog_cap = (uint32_t)std::min<uint64_t>(n + 1, 1u << 20);
  ArenaPlan A;
  const bool out_host = g->on_device == TRIM_MEM_HOST;
  const size_t a_off = out_host ? A.add<uint32_t>(n + 1) : 0;
  const size_t a_tgt = out_host ? A.add<uint32_t>(c->m) : 0;
  const bool in_host = gi && gi->on_device == TRIM_MEM_HOST;
  const size_t a_ioff = in_host ? A.add<uint32_t>(n + 1) : 0;
  const size_t a_itgt = in_host ? A.add<uint32_t>(c->m) : 0;
  const size_t a_level = A.add<uint32_t>(n), a_cnt = A.add<uint32_t>(n), a_supp = A.add<uint32_t>(n);
  const size_t a_shead = A.add<uint32_t>(n), a_snext = A.add<uint32_t>(n);
  const size_t a_scnt = A.add<uint32_t>(n), a_soff = A.add<uint32_t>(n + 1);
  const size_t a_slist = A.add<uint32_t>(n), a_log = A.add<uint32_t>(n);
  const size_t a_roff = A.add<uint32_t>(n + 2), a_live0 = A.add<uint32_t>(n);
  const size_t a_live1 = A.add<uint32_t>(n), a_bsum = A.add<uint32_t>(8192);
  const size_t a_ctrl = A.add<Ctrl>(1);
  const size_t a_w4r = A.add<uint32_t>(n), a_w4e = A.add<uint32_t>(n);
  const size_t a_chunk = A.add<uint32_t>((c->m >> 5) + 2);
  const size_t a_rlog = c->rlog_cap ? A.add<trim_round_rec_t>(c->rlog_cap) : 0;
  char* base = nullptr;
  TRY(dalloc(c, &base, A.bytes));
  auto at = [&](size_t o) { return reinterpret_cast<uint32_t*>(base + o); };
  if (out_host) {
    CK(cudaMemcpyAsync(at(a_off), g->offsets, (n + 1) * 4, cudaMemcpyHostToDevice, c->stream));
    if (c->m)
      CK(cudaMemcpyAsync(at(a_tgt), g->targets, c->m * 4, cudaMemcpyHostToDevice, c->stream));
    c->off = at(a_off);
    c->tgt = at(a_tgt);
  } else if (g->on_device == TRIM_MEM_HOST_MAPPED) {
    TRY(map_host(c, g->offsets, &c->off));
    TRY(map_host(c, c->m ? g->targets : nullptr, &c->tgt));
  } else {
    c->off = g->offsets;
    c->tgt = g->targets;
  }
  if (gi) {
    if (in_host) {
      CK(cudaMemcpyAsync(at(a_ioff), gi->offsets, (n + 1) * 4, cudaMemcpyHostToDevice, c->stream));
      if (c->m)
        CK(cudaMemcpyAsync(at(a_itgt), gi->targets, c->m * 4, cudaMemcpyHostToDevice, c->stream));
      c->ioff = at(a_ioff);
      c->itgt = at(a_itgt);
    } else if (gi->on_device == TRIM_MEM_HOST_MAPPED) {
      TRY(map_host(c, gi->offsets, &c->ioff));
      TRY(map_host(c, c->m ? gi->targets : nullptr, &c->itgt));
    } else {
      c->ioff = gi->offsets;
      c->itgt = gi->targets;
    }
  }
  c->level = at(a_level); c->cnt = at(a_cnt); c->supp = at(a_supp);
  c->s_head = at(a_shead); c->s_next = at(a_snext); c->s_cnt = at(a_scnt);
  c->s_off = at(a_soff); c->s_list = at(a_slist); c->log = at(a_log); c->roff = at(a_roff);
  c->live0 = at(a_live0); c->live1 = at(a_live1); c->bsum = at(a_bsum);
  c->ctrl = reinterpret_cast<Ctrl*>(base + a_ctrl);
  c->w4_row = at(a_w4r); c->w4_eoff = at(a_w4e); c->chunk_first = at(a_chunk);
  if (c->rlog_cap) c->rlog = reinterpret_cast<trim_round_rec_t*>(base + a_rlog);
  if (flags & TRIM_FLAG_VALIDATE) TRY(validate(c, gi ? c->ioff : nullptr));
  if (c->ioff != nullptr) TRY(alloc_async(c));
  CK(cudaMemsetAsync(c->s_cnt, 0, n * 4, c->stream));
  c->h_ctrl = take_ctrl_slot();
  c->h_ctrl_pinned = c->h_ctrl != nullptr;
  if (!c->h_ctrl) c->h_ctrl = new (std::nothrow) Ctrl();
  if (!c->h_ctrl) return fail(c, TRIM_ERR_OOM, "host allocation failed");
  TRY(compute_grid(c));
  TRY(sync_check(c));
  return TRIM_OK;
}

// A context over an implicit graph: O(n) state only; m is the degree sum,
// computed on the device.
trim_err_t create_implicit_impl(const trim_implicit_graph_t* g, void* stream, uint32_t flags,
                                trim_ctx* c) {
  const uint64_t n64 = (uint64_t)g->nC + g->nR + g->nT;
  if (n64 > (1u << 31)) return fail(c, TRIM_ERR_TOO_LARGE, "n must be <= 2^31");
  if (g->nR && !g->nC) return fail(c, TRIM_ERR_INVALID_ARG, "a reaching set needs a core");
  if (g->c_kmin > g->c_kmax || g->r_kmin > g->r_kmax || g->t_kmin > g->t_kmax)
    return fail(c, TRIM_ERR_INVALID_ARG, "degree bounds: kmin > kmax");
  if ((g->nC && g->c_kmax > (1u << 20)) || (g->nR && g->r_kmax > (1u << 20)) ||
      g->t_kmax > (1u << 20))
    return fail(c, TRIM_ERR_TOO_LARGE, "degrees above 2^20");
  TRY(check_device(c, &c->device, &c->sm_count));
  c->stream = static_cast<cudaStream_t>(stream);
  c->flags = flags;
  c->n = (uint32_t)n64;
  c->implicit = true;
  c->ig = *g;
  default_params(&c->params);
  CK(cudaEventCreate(&c->ev0));
  CK(cudaEventCreate(&c->ev1));
  const size_t n = c->n;
  if (flags & TRIM_FLAG_ROUND_LOG) c->rlog_cap = (uint32_t)std::min<uint64_t>(n + 1, 1u << 20);
  ArenaPlan A;
  const size_t a_level = A.add<uint32_t>(n), a_supp = A.add<uint32_t>(n);
  const size_t a_shead = A.add<uint32_t>(n), a_snext = A.add<uint32_t>(n);
  const size_t a_scnt = A.add<uint32_t>(n), a_soff = A.add<uint32_t>(n + 1);
  const size_t a_slist = A.add<uint32_t>(n), a_log = A.add<uint32_t>(n);
  const size_t a_roff = A.add<uint32_t>(n + 2), a_live0 = A.add<uint32_t>(n);
  const size_t a_live1 = A.add<uint32_t>(n), a_bsum = A.add<uint32_t>(8192);
  const size_t a_ctrl = A.add<Ctrl>(1), a_m = A.add<unsigned long long>(1);
  const size_t a_rlog = c->rlog_cap ? A.add<trim_round_rec_t>(c->rlog_cap) : 0;
  char* base = nullptr;
  TRY(dalloc(c, &base, A.bytes));
  auto at = [&](size_t o) { return reinterpret_cast<uint32_t*>(base + o); };
  c->level = at(a_level); c->supp = at(a_supp); c->cnt = nullptr;
  c->s_head = at(a_shead); c->s_next = at(a_snext); c->s_cnt = at(a_scnt);
  c->s_off = at(a_soff); c->s_list = at(a_slist); c->log = at(a_log); c->roff = at(a_roff);
  c->live0 = at(a_live0); c->live1 = at(a_live1); c->bsum = at(a_bsum);
  c->ctrl = reinterpret_cast<Ctrl*>(base + a_ctrl);
  if (c->rlog_cap) c->rlog = reinterpret_cast<trim_round_rec_t*>(base + a_rlog);
  CK(cudaMemsetAsync(c->s_cnt, 0, n * 4, c->stream));
  // m = the sum of the degrees
  unsigned long long* dm = reinterpret_cast<unsigned long long*>(base + a_m);
  CK(cudaMemsetAsync(dm, 0, 8, c->stream));
  Dev D{};
  D.n = c->n;
  D.ig = c->ig;
  trim_implicit_degree_sum_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(D, dm);
  CK(cudaGetLastError());
  unsigned long long hm = 0;
  CK(cudaMemcpyAsync(&hm, dm, 8, cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_check(c));
  if (hm > (1ull << 32) - 64) return fail(c, TRIM_ERR_TOO_LARGE, "m must be <= 2^32 - 64");
  c->m = hm;
  c->h_ctrl = take_ctrl_slot();
  c->h_ctrl_pinned = c->h_ctrl != nullptr;
  if (!c->h_ctrl) c->h_ctrl = new (std::nothrow) Ctrl();
  if (!c->h_ctrl) return fail(c, TRIM_ERR_OOM, "host allocation failed");
  TRY(compute_grid(c));
  return TRIM_OK;
}

// AC-4 work list (one entry per removed vertex with in-edges) and the owner
// index of every 32-edge chunk of its in-edge prefix; allocated on first use.
trim_err_t ensure_work_list(trim_ctx* c) {
  if (c->w4_row) return TRIM_OK;  // carved from the arena at create time
  TRY(dalloc(c, &c->w4_row, c->n));
  TRY(dalloc(c, &c->w4_eoff, c->n));
  TRY(dalloc(c, &c->chunk_first, (c->m >> 5) + 2));
  return TRIM_OK;
}

// In+out trimming's arrays: in-degree counters and the work list's out-CSR
// row starts and in-degrees; allocated on first use.
trim_err_t ensure_inout(trim_ctx* c) {
  if (c->cnt_in) return TRIM_OK;
  // the work list's edge offsets are uint32 and cover both rows of every vertex
  if (2 * c->m > (1ull << 32) - 64)
    return fail(c, TRIM_ERR_TOO_LARGE, "in+out trimming needs 2m <= 2^32 - 64");
  TRY(dalloc(c, &c->cnt_in, c->n));
  TRY(dalloc(c, &c->w4_orow, c->n));
  TRY(dalloc(c, &c->w4_din, c->n));
  TRY(dalloc(c, &c->chunk_io, ((2 * c->m) >> 5) + 2));
  return TRIM_OK;
}

// Enqueues one run. A scheduled variant runs on the all-variant kernel, or with
// seg_flavour >= 0 on that flavour as the first segment: followed, with cont,
// by a continuation launch of the all-variant kernel (which finishes the run
// if the first segment handed it over), else by host-side segments
// (run_segmented). With inout, the run is in+out trimming (variant must be
// TRIM_AC4_PUSH).
trim_err_t enqueue_run(trim_ctx* c, trim_variant_t variant, int seg_flavour = -1,
                       uint32_t commit_after = 0, bool inout = false, bool cont = false) {
  if ((int)variant < 0 || variant > TRIM_SCHED_SCRIPTED)
    return fail(c, TRIM_ERR_INVALID_ARG, "unknown variant");
  if (c->implicit) {
    if ((variant != TRIM_AC6_SUPPORT && variant != TRIM_AC3_PULL) || inout || seg_flavour >= 0)
      return fail(c, TRIM_ERR_INVALID_ARG,
                  "an implicit graph runs TRIM_AC6_SUPPORT or TRIM_AC3_PULL only");
    if (c->has_mask) return fail(c, TRIM_ERR_INVALID_ARG, "an implicit graph takes no dead mask");
  }
  if (inout) {
    if (c->has_mask) return fail(c, TRIM_ERR_INVALID_ARG, "trim_run_inout does not take a dead mask");
    if (c->ioff == nullptr) TRY(build_transpose(c));
    TRY(ensure_inout(c));
  }
  if (variant == TRIM_SCHED_SCRIPTED && c->script_len == 0)
    return fail(c, TRIM_ERR_STATE, "TRIM_SCHED_SCRIPTED needs trim_set_schedule first");
  if (variant == TRIM_AC4_PUSH && c->ioff == nullptr) TRY(build_transpose(c));
  uint32_t f = c->flags & (TRIM_FLAG_STATS | TRIM_FLAG_ROUND_LOG);
  bool ac4 = false, ac6 = false, ac3 = false;
  switch (variant) {
    case TRIM_AC4_PUSH: ac4 = true; break;
    case TRIM_AC6_SUPPORT: ac6 = true; break;
    case TRIM_AC3_PULL: ac3 = true; break;
    default:
      ac4 = c->ioff != nullptr;
      ac6 = ac3 = true;
      if (variant == TRIM_SCHED_LEARNED) f |= trimk::F_NEED_FEATURES;
  }
  // scheduler features: for the learned scheduler, and in round logs of scheduled runs
  if ((c->flags & TRIM_FLAG_ROUND_LOG) && variant >= TRIM_SCHED_HEURISTIC)
    f |= trimk::F_NEED_FEATURES;
  if (variant == TRIM_SCHED_SCRIPTED) {
    ac4 = ac6 = ac3 = false;
    for (uint8_t x : c->h_script) {
      if (x == TRIM_AC4_PUSH) ac4 = true;
      else if (x == TRIM_AC6_SUPPORT) ac6 = true;
      else ac3 = true;
    }
    if (ac4 && c->ioff == nullptr) TRY(build_transpose(c));
  }
  if (ac4) { f |= trimk::F_AC4_POSSIBLE; TRY(ensure_work_list(c)); }
  if (ac6) f |= trimk::F_AC6_POSSIBLE;
  if (ac3) f |= trimk::F_AC3_POSSIBLE;
  c->cont_mode = -1;
  c->sched_mode = (variant >= TRIM_SCHED_HEURISTIC) ? (int)variant : -1;
  c->last_launches = 0;
  if (c->n == 0) {
    c->ran = true;
    c->pending = false;
    std::memset(c->h_ctrl, 0, sizeof(Ctrl));
    CK(cudaEventRecord(c->ev0, c->stream));
    CK(cudaEventRecord(c->ev1, c->stream));
    return TRIM_OK;
  }
  if (ac6 && c->s_cnt_dirty) {
    CK(cudaMemsetAsync(c->s_cnt, 0, (size_t)c->n * 4, c->stream));
    c->s_cnt_dirty = false;
  }
  Dev D{};
  D.n = c->n;
  D.m = (uint32_t)c->m;
  D.off = c->off; D.tgt = c->tgt; D.ioff = c->ioff; D.itgt = c->itgt;
  D.level = c->level; D.cnt = c->cnt; D.supp = c->supp;
  D.s_head = c->s_head; D.s_next = c->s_next; D.s_cnt = c->s_cnt; D.s_off = c->s_off;
  D.s_list = c->s_list; D.log = c->log; D.roff = c->roff; D.live0 = c->live0;
  D.live1 = c->live1; D.w4_row = c->w4_row; D.w4_eoff = c->w4_eoff;
  D.chunk_first = c->chunk_first; D.bsum = c->bsum; D.C = c->ctrl;
  D.cnt_in = c->cnt_in; D.w4_orow = c->w4_orow; D.w4_din = c->w4_din;
  D.mask = c->has_mask ? c->mask : nullptr;
  D.ig = c->ig;
  if (inout) D.chunk_first = c->chunk_io;
  D.sbuf_cap = kSbufCap;
  D.rlog = c->rlog; D.rlog_cap = c->rlog_cap;
  D.model = c->has_model ? c->model : nullptr;
  D.script = c->script; D.script_len = c->script_len;
  D.mode = variant; D.flags = f;
  D.spin_limit_ns = c->params.spin_limit_ns;
  D.heur_push_ratio = c->params.heur_push_ratio;
  D.heur_ac6_ratio = c->params.heur_ac6_ratio;
  D.commit_after = commit_after;
  D.commit_confidence = c->params.sched_commit_confidence;
  D.recheck_rounds = c->params.sched_recheck_rounds;
  D.local_edges_max = c->params.local_round_edges;
  D.aw = c->aw;
  D.oq_row = c->oq_row; D.oq_len = c->oq_len; D.oq_lev = c->oq_lev; D.oq_cap = c->oq_cap;
  D.ae_id = c->ae_id; D.ae_lev = c->ae_lev; D.ae_cap = c->ae_cap;
  D.async_edges_max = (c->aw != nullptr && c->ioff != nullptr) ? c->params.async_round_edges : 0u;
  // scheduled runs keep the live-edge count (a feature); with G^T and AC-4 the
  // scheduler kernels derive it from running totals instead
  if (variant >= TRIM_SCHED_HEURISTIC && !(ac4 && c->ioff)) D.flags |= trimk::F_LIVE_EDGES;
  // a fixed variant runs on its lean single-variant flavour
  int flavour = kFlavourAll;
  if (c->implicit) flavour = variant == TRIM_AC6_SUPPORT ? kFlavourImplicitAC6 : kFlavourImplicitAC3;
  else if (inout) flavour = kFlavourInout;
  else if (variant <= TRIM_AC3_PULL) flavour = (int)variant;
  else if (seg_flavour >= 0) flavour = seg_flavour;
  c->last_dev = D;
  const int grid = c->grids[flavour];
  if ((uint32_t)grid > 8192) return fail(c, TRIM_ERR_INVALID_ARG, "grid too large");
  c->last_launches = 2;  // control-block reset + persistent kernel
  trim_reset_ctrl_kernel<<<1, 32, 0, c->stream>>>(c->ctrl);
  CK(cudaGetLastError());
  // device_ms covers the persistent kernel alone; inside a stream capture the
  // records must be "external" to become event-record nodes of the graph
  const unsigned rec = c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  CK(cudaEventRecordWithFlags(c->ev0, c->stream, rec));
  void* args[] = {&D};
  CK(cudaLaunchCooperativeKernel((const void*)kFlavours[flavour], dim3(grid),
                                 dim3(c->params.block_threads), args,
                                 dyn_smem_bytes(c->params.block_threads),
                                 c->stream));
  if (cont) {
    // the all-variant kernel finishes the run if the first segment handed it
    // over (its scheduler chose a variant that kernel lacks); else it returns
    // at once
    Dev Dc = D;
    Dc.flags |= trimk::F_CONTINUE;
    void* cargs[] = {&Dc};
    CK(cudaLaunchCooperativeKernel((const void*)kFlavours[kFlavourAll],
                                   dim3(c->grids[kFlavourAll]), dim3(c->params.block_threads),
                                   cargs, dyn_smem_bytes(c->params.block_threads), c->stream));
    c->cont_mode = (int)variant;
    c->last_launches = 3;
  }
  CK(cudaEventRecordWithFlags(c->ev1, c->stream, rec));
  c->pending = true;
  c->ran = false;
  return TRIM_OK;
}

trim_err_t finish_run(trim_ctx* c, trim_run_stats_t* stats, bool ctrl_read = false);

// ---- SCC decomposition (trim_run_scc) ----

trim_err_t ensure_scc(trim_ctx* c) {
  if (c->scc_comp) return TRIM_OK;
  const size_t n = c->n;
  TRY(dalloc(c, &c->scc_comp, n));
  TRY(dalloc(c, &c->scc_color, n));
  TRY(dalloc(c, &c->scc_fw, n));
  TRY(dalloc(c, &c->scc_bw, n));
  TRY(dalloc(c, &c->scc_fa, n));
  TRY(dalloc(c, &c->scc_fb, n));
  TRY(dalloc(c, &c->scc_cnt, 4));
  CK(cudaMemsetAsync(c->scc_fw, 0, n * 4, c->stream));  // marks hold search stamps (>= 1)
  CK(cudaMemsetAsync(c->scc_bw, 0, n * 4, c->stream));
  if (!c->scc_ev0) CK(cudaEventCreate(&c->scc_ev0));
  if (!c->scc_ev1) CK(cudaEventCreate(&c->scc_ev1));
  return TRIM_OK;
}

// reads counter i of the SCC counters (waits for the stream)
trim_err_t scc_read(trim_ctx* c, int i, unsigned long long* v) {
  CK(cudaMemcpyAsync(v, c->scc_cnt + i, 8, cudaMemcpyDeviceToHost, c->stream));
  return sync_check(c);
}

// Runs frontier levels until the frontier is empty: the first frontier (k
// vertices) is in c->scc_fa; `level` enqueues one level from fa (k vertices)
// into fb, counting into the given device counter. Returns the levels run.
template <class Level>
trim_err_t scc_levels(trim_ctx* c, uint32_t k, Level level, uint32_t* levels) {
  uint32_t* cnt32 = reinterpret_cast<uint32_t*>(c->scc_cnt + 3);
  const int blocks = c->sm_count * 8;
  uint32_t *fa = c->scc_fa, *fb = c->scc_fb;
  while (k > 0) {
    CK(cudaMemsetAsync(cnt32 + 1, 0, 4, c->stream));
    const uint32_t warps_needed = std::min<uint32_t>(k, (uint32_t)blocks * 8u);
    level(std::max<uint32_t>(1u, (warps_needed + 7u) / 8u), fa, k, fb, cnt32 + 1);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&k, cnt32 + 1, 4, cudaMemcpyDeviceToHost, c->stream));
    TRY(sync_check(c));
    std::swap(fa, fb);
    ++*levels;
  }
  c->scc_fa = fa;  // the two frontier buffers may have traded places
  c->scc_fb = fb;
  return TRIM_OK;
}

// the next search stamp (marks of earlier searches stay below it; the mark
// arrays are cleared before the counter could wrap)
trim_err_t scc_next_stamp(trim_ctx* c, uint32_t* stamp) {
  if (c->scc_stamp >= 0xFFFFFFF0u) {
    CK(cudaMemsetAsync(c->scc_fw, 0, (size_t)c->n * 4, c->stream));
    CK(cudaMemsetAsync(c->scc_bw, 0, (size_t)c->n * 4, c->stream));
    c->scc_stamp = 0;
  }
  *stamp = ++c->scc_stamp;
  return TRIM_OK;
}

trim_err_t run_scc(trim_ctx* c, uint32_t* out, int out_on_device, trim_scc_stats_t* stats) {
  if (c->implicit) return fail(c, TRIM_ERR_INVALID_ARG, "SCC decomposition needs a CSR");
  if (c->has_mask) return fail(c, TRIM_ERR_INVALID_ARG, "SCC decomposition takes no dead mask");
  trim_scc_stats_t st{};
  if (c->n == 0) {
    if (stats) *stats = st;
    return TRIM_OK;
  }
  TRY(ensure_scc(c));
  CK(cudaEventRecord(c->scc_ev0, c->stream));
  // 1. size-1 components: in+out trimming
  TRY(enqueue_run(c, TRIM_AC4_PUSH, -1, 0, true));
  TRY(finish_run(c, nullptr));
  st.trimmed_size1 = c->last.n_dead;
  const uint32_t n = c->n;
  const int blocks = c->sm_count * 8;
  scc_init_kernel<<<blocks, 256, 0, c->stream>>>(c->level, n, c->scc_comp, c->scc_color);
  CK(cudaGetLastError());
  // 2. size-2 components
  CK(cudaMemsetAsync(c->scc_cnt, 0, 24, c->stream));
  scc_trim2_single_kernel<<<blocks, 256, 0, c->stream>>>(c->off, c->tgt, c->ioff, c->itgt, n,
                                                         c->scc_comp, c->scc_fa, c->scc_fb);
  CK(cudaGetLastError());
  scc_trim2_pair_kernel<<<blocks, 256, 0, c->stream>>>(n, c->scc_fa, c->scc_fb, c->scc_comp,
                                                       c->scc_cnt);
  CK(cudaGetLastError());
  unsigned long long v = 0;
  TRY(scc_read(c, 0, &v));
  st.trimmed_size2 = (uint32_t)v;
  // 3. steps: trimming passes, then label propagation along G (every open
  // vertex learns the smallest open vertex that reaches it) and backward
  // searches through G^T from the vertices that kept their own label
  const uint32_t* off = c->off;
  const uint32_t* tgt = c->tgt;
  const uint32_t* ioff = c->ioff;
  const uint32_t* itgt = c->itgt;
  uint32_t* comp = c->scc_comp;
  uint32_t* label = c->scc_color;
  uint32_t* cnt32 = reinterpret_cast<uint32_t*>(c->scc_cnt + 3);
  for (uint32_t step = 0; step <= n; ++step) {
    for (int pass = 0; pass < 1024; ++pass) {  // trimming passes
      CK(cudaMemsetAsync(c->scc_cnt + 1, 0, 8, c->stream));
      scc_trim1_kernel<<<blocks, 256, 0, c->stream>>>(off, tgt, ioff, itgt, n, comp,
                                                      c->scc_cnt + 1);
      CK(cudaGetLastError());
      TRY(scc_read(c, 1, &v));
      st.trimmed_in_steps += (uint32_t)v;
      if (v == 0) break;
    }
    // labels
    CK(cudaMemsetAsync(c->scc_cnt + 2, 0, 16, c->stream));  // open count, two frontier counters
    scc_label_start_kernel<<<blocks, 256, 0, c->stream>>>(n, comp, label, c->scc_fa, cnt32,
                                                          c->scc_cnt + 2);
    CK(cudaGetLastError());
    TRY(scc_read(c, 2, &v));
    if (v == 0) break;  // every vertex has its component
    uint32_t k = 0;
    CK(cudaMemcpyAsync(&k, cnt32, 4, cudaMemcpyDeviceToHost, c->stream));
    TRY(sync_check(c));
    while (k > 0) {  // one stamp per level: a vertex joins a level's frontier once
      uint32_t stamp = 0;
      TRY(scc_next_stamp(c, &stamp));
      uint32_t lv = 0;
      uint32_t* fa = c->scc_fa;
      uint32_t* fb = c->scc_fb;
      CK(cudaMemsetAsync(cnt32 + 1, 0, 4, c->stream));
      const uint32_t warps_needed = std::min<uint32_t>(k, (uint32_t)blocks * 8u);
      scc_label_level_kernel<<<std::max<uint32_t>(1u, (warps_needed + 7u) / 8u), 256, 0,
                               c->stream>>>(off, tgt, comp, label, c->scc_fw, stamp, fa, k, fb,
                                            cnt32 + 1);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(&k, cnt32 + 1, 4, cudaMemcpyDeviceToHost, c->stream));
      TRY(sync_check(c));
      std::swap(c->scc_fa, c->scc_fb);
      (void)lv;
      ++st.search_levels;
    }
    // backward searches from the roots
    uint32_t stamp = 0;
    TRY(scc_next_stamp(c, &stamp));
    CK(cudaMemsetAsync(cnt32, 0, 4, c->stream));
    scc_roots_start_kernel<<<blocks, 256, 0, c->stream>>>(n, comp, label, c->scc_bw, stamp,
                                                          c->scc_fa, cnt32);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&k, cnt32, 4, cudaMemcpyDeviceToHost, c->stream));
    TRY(sync_check(c));
    TRY(scc_levels(c, k,
                   [&](uint32_t b, uint32_t* fa, uint32_t kk, uint32_t* fb, uint32_t* nc) {
                     scc_search_level_kernel<<<b, 256, 0, c->stream>>>(
                         ioff, itgt, comp, label, c->scc_bw, stamp, fa, kk, fb, nc);
                   },
                   &st.search_levels));
    scc_close_kernel<<<blocks, 256, 0, c->stream>>>(n, comp, label, c->scc_bw, stamp, c->scc_cnt);
    CK(cudaGetLastError());
    ++st.fwbw_steps;
  }
  CK(cudaMemsetAsync(c->scc_cnt, 0, 8, c->stream));
  scc_count_kernel<<<blocks, 256, 0, c->stream>>>(n, c->scc_comp, c->scc_cnt);
  CK(cudaGetLastError());
  CK(cudaEventRecord(c->scc_ev1, c->stream));
  TRY(scc_read(c, 0, &v));
  st.components = (uint32_t)v;
  CK(cudaEventElapsedTime(&st.ms, c->scc_ev0, c->scc_ev1));
  CK(cudaMemcpyAsync(out, c->scc_comp, (size_t)n * 4,
                     out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_check(c));
  if (stats) *stats = st;
  return TRIM_OK;
}

// Launches the next segment of a host-segmented run: `flavour` resumes the run
// from the schedule state the last segment saved.
trim_err_t launch_segment(trim_ctx* c, int flavour, uint32_t bar_base) {
  trimk::Dev D = c->last_dev;
  D.resume = 1;
  D.bar_base = bar_base;
  void* args[] = {&D};
  CK(cudaLaunchCooperativeKernel((const void*)kFlavours[flavour], dim3(c->grids[flavour]),
                                 dim3(c->params.block_threads), args,
                                 dyn_smem_bytes(c->params.block_threads),
                                 c->stream));
  CK(cudaEventRecord(c->ev1, c->stream));
  return TRIM_OK;
}

// The first segment's commit length of a scheduled mode (a scripted run never
// commits: its script decides every round).
uint32_t commit_rounds(const trim_ctx* c, trim_variant_t variant) {
  return variant == TRIM_SCHED_SCRIPTED ? 0u : c->params.sched_commit_rounds;
}

// The kernel flavour a scheduled mode's run starts on: the one with the
// schedulers and the variant its last run chose for round 1 (a scripted run:
// its first entry; else AC-4 with G^T, AC-3 without).
int first_flavour(const trim_ctx* c, trim_variant_t variant) {
  const int mi = (int)variant - (int)TRIM_SCHED_HEURISTIC;
  if (c->seg_first[mi] >= 0) return c->seg_first[mi];
  if (variant == TRIM_SCHED_SCRIPTED && !c->h_script.empty())
    return kFlavourSeg + std::min<int>(c->h_script[0], TRIM_AC3_PULL);
  return kFlavourSeg + (c->ioff ? TRIM_AC4_PUSH : TRIM_AC3_PULL);
}

// A scheduled run (heuristic, learned, scripted) with host-side handover: each
// segment is one launch of a kernel that holds one variant plus the
// schedulers; when the scheduler picks a variant the running kernel lacks,
// the kernel saves the schedule state and exits, and the host launches the
// kernel of that variant, which resumes at the same round. Commits stay
// inside a kernel (a committed stretch skips the scheduler).
trim_err_t run_segmented(trim_ctx* c, trim_variant_t variant, trim_run_stats_t* stats) {
  const int mi = (int)variant - (int)TRIM_SCHED_HEURISTIC;
  TRY(enqueue_run(c, variant, first_flavour(c, variant), commit_rounds(c, variant)));
  if (!c->pending) return finish_run(c, stats);
  uint64_t segments = 1;
  while (true) {
    TRY(read_ctrl(c));
    const Ctrl& h = *c->h_ctrl;
    if (h.err || !h.resume) break;
    if (h.resume_variant > TRIM_AC3_PULL || ++segments > (uint64_t)c->n + 3) {
      c->pending = false;
      c->s_cnt_dirty = true;
      return fail(c, TRIM_ERR_STATE, "invalid segment handover");
    }
    const uint32_t v = h.resume_variant;
    if (segments == 2 && h.saved.round == 1) c->seg_first[mi] = kFlavourSeg + (int)v;
    TRY(launch_segment(c, kFlavourSeg + (int)v, h.bar));
  }
  c->last_segments = segments;
  c->last_launches = 1 + segments;
  return finish_run(c, stats, true);
}

// A scheduled run, with the kernels and handover params.sched_handover names;
// waits for it.
trim_err_t run_scheduled(trim_ctx* c, trim_variant_t variant, trim_run_stats_t* stats) {
  const int whole = c->seg_whole[(int)variant - (int)TRIM_SCHED_HEURISTIC];
  if (whole >= 0 && c->params.sched_handover != TRIM_HANDOVER_NONE) {
    TRY(enqueue_run(c, (trim_variant_t)whole));  // the schedule is known: one variant
    return finish_run(c, stats);
  }
  switch (c->params.sched_handover) {
    case TRIM_HANDOVER_HOST:
      return run_segmented(c, variant, stats);
    case TRIM_HANDOVER_NONE:
      TRY(enqueue_run(c, variant, -1, commit_rounds(c, variant)));
      return finish_run(c, stats);
    default:
      TRY(enqueue_run(c, variant, first_flavour(c, variant), commit_rounds(c, variant), false,
                      true));
      return finish_run(c, stats);
  }
}

// Waits for the enqueued run and publishes its statistics (ctrl_read: the
// control block is already in h_ctrl).
trim_err_t finish_run(trim_ctx* c, trim_run_stats_t* stats, bool ctrl_read) {
  if (c->pending) {
    if (!ctrl_read) TRY(read_ctrl(c));
    c->pending = false;
    const Ctrl& h = *c->h_ctrl;
    if (h.err) {
      c->s_cnt_dirty = true;
      if (h.err == TRIM_ERR_TIMEOUT)
        return fail(c, TRIM_ERR_TIMEOUT, "a device-side wait exceeded spin_limit_ns");
      return fail(c, (trim_err_t)h.err,
                  "device reported error " + std::to_string(h.err) + " (info " +
                      std::to_string(h.err_info) + ")");
    }
    if (c->has_mask && c->n) {  // masked vertices report TRIM_MASKED (level 0 inside the run)
      trim_mask_levels_kernel<<<c->sm_count * 4, 512, 0, c->stream>>>(c->level, c->mask, c->n);
      CK(cudaGetLastError());
      TRY(sync_check(c));
    }
    uint64_t launches = c->last_launches;
    if (c->cont_mode >= 0) {  // first segment + continuation: what ran, as counted
      c->last_segments = h.segments;
      // the next run of this mode starts on the kernel of round 1's variant
      if (h.first_exit_round == 1 && h.resume_variant <= TRIM_AC3_PULL)
        c->seg_first[c->cont_mode - (int)TRIM_SCHED_HEURISTIC] =
            kFlavourSeg + (int)h.resume_variant;
      c->cont_mode = -1;
    }
    if (c->sched_mode >= 0) {
      // a run whose only scheduler decision, before round 1, committed it to
      // one variant for all its rounds: that decision depends only on the
      // graph, mask, model and parameters, so the mode's next run on this
      // context is the same single-variant run
      int v = -1, used = 0;
      for (int i = 0; i < 3; ++i)
        if (h.vcount[i]) v = i, ++used;
      c->seg_whole[c->sched_mode - (int)TRIM_SCHED_HEURISTIC] =
          (h.consults == 1 && h.commit_round0 && h.first_exit_round == 0 && used == 1) ? v : -1;
      c->sched_mode = -1;
    }
    if (c->has_mask && c->n) launches += 1;
    trim_run_stats_t s{};
    s.rounds = h.rounds;
    s.n_dead = h.n_dead;
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    s.device_ms = ms;
    s.edges_inspected = h.stats[0];
    s.in_edges_pushed = h.stats[1];
    s.candidates = h.stats[2];
    s.live_swept = h.stats[3];
    for (int i = 0; i < 3; ++i) s.rounds_by_variant[i] = h.vcount[i];
    s.segments = (uint32_t)c->last_segments;
    s.local_rounds = h.local_rounds;
    s.launches = (uint32_t)std::min<uint64_t>(launches, 0xFFFFFFFFu);
    s.async_round = h.a_round;
    s.async_removed = h.a_removed;
    s.async_rebalances = h.a_rebalances;
    c->last = s;
    c->ran = true;
  }
  if (!c->ran) return fail(c, TRIM_ERR_STATE, "no run was enqueued");
  if (stats) *stats = c->last;
  return TRIM_OK;
}

// no edge of the packed CSR may join two graphs
trim_err_t validate_batch(trim_ctx* c, const uint32_t* graph_off, uint32_t G) {
  std::vector<uint32_t> vg(c->n);
  for (uint32_t g = 0; g < G; ++g)
    for (uint32_t v = graph_off[g]; v < graph_off[g + 1]; ++v) vg[v] = g;
  uint32_t *dvg = nullptr, *bad = nullptr;
  TRY(dalloc(c, &dvg, c->n));
  TRY(dalloc(c, &bad, 1));
  CK(cudaMemcpyAsync(dvg, vg.data(), (size_t)c->n * 4, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(bad, 0, 4, c->stream));
  trim_validate_batch_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(c->off, c->tgt, c->n, dvg,
                                                                     bad);
  CK(cudaGetLastError());
  uint32_t h = 0;
  CK(cudaMemcpyAsync(&h, bad, 4, cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_check(c));
  if (h) return fail(c, TRIM_ERR_BAD_GRAPH, "an edge joins two graphs of the batch");
  return TRIM_OK;
}

// The packed CSR of independent graphs is itself one graph (their disjoint
// union), whose levels equal those of each graph trimmed alone. All graphs run
// in one persistent launch, so every round's fixed cost (barrier, bookkeeping)
// is shared by all graphs still peeling. The launch (control-block reset plus
// persistent kernel) is captured once into a CUDA graph and replayed.
trim_err_t enqueue_batch(trim_ctx* c, const uint32_t* graph_off, uint32_t G,
                         trim_variant_t variant) {
  (void)graph_off;
  (void)G;
  if (c->n == 0) return enqueue_run(c, variant);  // nothing to launch, nothing to capture
  if (c->batch_exec == nullptr || c->batch_variant != (int)variant) {
    // the first call with a variant runs directly (a one-shot caller pays no
    // capture; it also builds G^T if needed and makes every allocation the run
    // needs); the second captures the launch, then launches and replays it.
    if (c->batch_last_variant != (int)variant) {
      c->batch_last_variant = (int)variant;
      return enqueue_run(c, variant);
    }
    if (c->batch_exec) {
      cudaGraphExecDestroy(c->batch_exec);
      c->batch_exec = nullptr;
    }
    // capture on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is then launched on c->stream
    if (c->cap_stream == nullptr)
      CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaStream_t user_stream = c->stream;
    c->stream = c->cap_stream;
    c->capturing = true;
    cudaError_t be = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    trim_err_t e = be == cudaSuccess ? enqueue_run(c, variant) : TRIM_ERR_CUDA;
    cudaError_t ce = be == cudaSuccess ? cudaStreamEndCapture(c->cap_stream, &graph) : be;
    c->capturing = false;
    c->stream = user_stream;
    if (e != TRIM_OK || ce != cudaSuccess) {  // not capturable here: launch directly
      if (graph) cudaGraphDestroy(graph);
      (void)cudaGetLastError();
      c->pending = false;
      return enqueue_run(c, variant);
    }
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      (void)cudaGetLastError();
      c->pending = false;
      return enqueue_run(c, variant);
    }
    c->batch_exec = exec;
    c->batch_variant = (int)variant;
  }
  CK(cudaGraphLaunch(c->batch_exec, c->stream));
  c->cont_mode = -1;
  c->last_launches = 2;  // the replayed reset + persistent kernel
  c->pending = true;
  c->ran = false;
  return TRIM_OK;
}

}  // namespace

extern "C" {

trim_err_t trim_create(const trim_csr_t* csr_out, const trim_csr_t* csr_in, void* cuda_stream,
                       uint32_t flags, trim_ctx** out) {
  if (!csr_out || !out) return fail(nullptr, TRIM_ERR_INVALID_ARG, "null csr_out or out");
  if (flags & ~(TRIM_FLAG_VALIDATE | TRIM_FLAG_STATS | TRIM_FLAG_ROUND_LOG))
    return fail(nullptr, TRIM_ERR_INVALID_ARG, "unknown flag bits");
  trim_ctx* c = new (std::nothrow) trim_ctx();
  if (!c) return fail(nullptr, TRIM_ERR_OOM, "host allocation failed");
  trim_err_t e = create_impl(csr_out, csr_in, cuda_stream, flags, c);
  if (e != TRIM_OK) {
    g_create_error = c->err;
    release(c);
    delete c;
    return e;
  }
  *out = c;
  return TRIM_OK;
}

trim_err_t trim_create_implicit(const trim_implicit_graph_t* g, void* cuda_stream, uint32_t flags,
                                trim_ctx** out) {
  if (!g || !out) return fail(nullptr, TRIM_ERR_INVALID_ARG, "null graph or out");
  if (flags & ~(TRIM_FLAG_STATS | TRIM_FLAG_ROUND_LOG))
    return fail(nullptr, TRIM_ERR_INVALID_ARG, "flags: TRIM_FLAG_STATS, TRIM_FLAG_ROUND_LOG only");
  trim_ctx* c = new (std::nothrow) trim_ctx();
  if (!c) return fail(nullptr, TRIM_ERR_OOM, "host allocation failed");
  trim_err_t e = create_implicit_impl(g, cuda_stream, flags, c);
  if (e != TRIM_OK) {
    g_create_error = c->err;
    release(c);
    delete c;
    return e;
  }
  *out = c;
  return TRIM_OK;
}

trim_err_t trim_run(trim_ctx* c, trim_variant_t variant, trim_run_stats_t* stats) {
  if (!c) return fail(nullptr, TRIM_ERR_INVALID_ARG, "null context");
  c->last_segments = 1;
  if (c->implicit && variant != TRIM_AC6_SUPPORT && variant != TRIM_AC3_PULL)
    return fail(c, TRIM_ERR_INVALID_ARG, "an implicit graph runs TRIM_AC6_SUPPORT or TRIM_AC3_PULL only");
  if (variant >= TRIM_SCHED_HEURISTIC && variant <= TRIM_SCHED_SCRIPTED)
    return run_scheduled(c, variant, stats);
  TRY(enqueue_run(c, variant));
  return finish_run(c, stats);
}

trim_err_t trim_run_inout(trim_ctx* c, trim_run_stats_t* stats) {
  if (!c) return fail(nullptr, TRIM_ERR_INVALID_ARG, "null context");
  c->last_segments = 1;
  TRY(enqueue_run(c, TRIM_AC4_PUSH, -1, 0, true));
  return finish_run(c, stats);
}

trim_err_t trim_run_scc(trim_ctx* c, uint32_t* comp, int out_on_device, trim_scc_stats_t* stats) {
  if (!c) return fail(nullptr, TRIM_ERR_INVALID_ARG, "null context");
  if (!comp && c->n) return fail(c, TRIM_ERR_INVALID_ARG, "null comp");
  return run_scc(c, comp, out_on_device, stats);
}

trim_err_t trim_run_async(trim_ctx* c, trim_variant_t variant) {
  if (!c) return fail(nullptr, TRIM_ERR_INVALID_ARG, "null context");
  c->last_segments = 1;
  if (variant >= TRIM_SCHED_HEURISTIC && variant <= TRIM_SCHED_SCRIPTED && !c->implicit) {
    const int whole = c->seg_whole[(int)variant - (int)TRIM_SCHED_HEURISTIC];
    if (whole >= 0 && c->params.sched_handover == TRIM_HANDOVER_DEVICE)
      return enqueue_run(c, (trim_variant_t)whole);  // the schedule is known: one variant
    if (c->params.sched_handover == TRIM_HANDOVER_DEVICE)
      return enqueue_run(c, variant, first_flavour(c, variant), commit_rounds(c, variant), false,
                         true);
    return enqueue_run(c, variant, -1, commit_rounds(c, variant));
  }
  return enqueue_run(c, variant);
}

trim_err_t trim_sync(trim_ctx* c, trim_run_stats_t* stats) {
  if (!c) return fail(nullptr, TRIM_ERR_INVALID_ARG, "null context");
  return finish_run(c, stats);
}

trim_err_t trim_batch_run(trim_ctx* c, const uint32_t* graph_off, uint32_t G,
                          trim_variant_t variant, trim_run_stats_t* stats) {
  if (!c || !graph_off || G == 0) return fail(c, TRIM_ERR_INVALID_ARG, "null argument or G = 0");
  if (c->implicit) return fail(c, TRIM_ERR_INVALID_ARG, "batched runs need a CSR");
  if (graph_off[0] != 0 || graph_off[G] != c->n)
    return fail(c, TRIM_ERR_INVALID_ARG, "graph_off must start at 0 and end at n");
  for (uint32_t g = 0; g < G; ++g)
    if (graph_off[g + 1] < graph_off[g])
      return fail(c, TRIM_ERR_INVALID_ARG, "graph_off must be non-decreasing");
  if (c->flags & TRIM_FLAG_VALIDATE) TRY(validate_batch(c, graph_off, G));
  c->last_segments = 1;
  // a scheduled variant runs as trim_run runs it (its first kernel depends on
  // the mode's last run: nothing is captured)
  if (variant >= TRIM_SCHED_HEURISTIC && variant <= TRIM_SCHED_SCRIPTED)
    return run_scheduled(c, variant, stats);
  TRY(enqueue_batch(c, graph_off, G, variant));
  return finish_run(c, stats);
}

trim_err_t trim_status(const trim_ctx* cc, uint8_t* out, int out_on_device) {
  trim_ctx* c = const_cast<trim_ctx*>(cc);
  if (!c || (!out && c->n)) return fail(c, TRIM_ERR_INVALID_ARG, "null argument");
  if (c->pending) TRY(finish_run(c, nullptr));
  if (!c->ran) return fail(c, TRIM_ERR_STATE, "trim_status before a successful trim_run");
  if (c->n == 0) return TRIM_OK;
  uint8_t* dst = out;
  if (!out_on_device) {
    if (!c->status_tmp) TRY(dalloc(c, &c->status_tmp, c->n));
    dst = c->status_tmp;
  }
  trim_status_kernel<<<c->sm_count * 4, 512, 0, c->stream>>>(c->level, c->n, dst);
  CK(cudaGetLastError());
  if (!out_on_device)
    CK(cudaMemcpyAsync(out, dst, c->n, cudaMemcpyDeviceToHost, c->stream));
  return sync_check(c);
}

trim_err_t trim_level(const trim_ctx* cc, uint32_t* out, int out_on_device) {
  trim_ctx* c = const_cast<trim_ctx*>(cc);
  if (!c || (!out && c->n)) return fail(c, TRIM_ERR_INVALID_ARG, "null argument");
  if (c->pending) TRY(finish_run(c, nullptr));
  if (!c->ran) return fail(c, TRIM_ERR_STATE, "trim_level before a successful trim_run");
  if (c->n == 0) return TRIM_OK;
  CK(cudaMemcpyAsync(out, c->level, (size_t)c->n * 4,
                     out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->stream));
  return sync_check(c);
}

trim_err_t trim_in_csr(trim_ctx* c, uint32_t* in_offsets, uint32_t* in_targets,
                       int out_on_device) {
  if (!c || !in_offsets || (!in_targets && c->m))
    return fail(c, TRIM_ERR_INVALID_ARG, "null argument");
  if (c->implicit) return fail(c, TRIM_ERR_INVALID_ARG, "an implicit graph has no CSR");
  if (c->pending) TRY(finish_run(c, nullptr));
  if (c->ioff == nullptr) TRY(build_transpose(c));
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(in_offsets, c->ioff, ((size_t)c->n + 1) * 4, kind, c->stream));
  if (c->m) CK(cudaMemcpyAsync(in_targets, c->itgt, (size_t)c->m * 4, kind, c->stream));
  return sync_check(c);
}

trim_err_t trim_level_device_ptr(const trim_ctx* c, const uint32_t** out) {
  if (!c || !out) return fail(const_cast<trim_ctx*>(c), TRIM_ERR_INVALID_ARG, "null argument");
  *out = c->level;
  return TRIM_OK;
}

trim_err_t trim_default_params(trim_params_t* p) {
  if (!p) return fail(nullptr, TRIM_ERR_INVALID_ARG, "null params");
  default_params(p);
  return TRIM_OK;
}

// a captured batched launch embeds the kernel arguments: drop it when they change
static void drop_batch_graph(trim_ctx* c) {
  if (c && c->batch_exec) {
    cudaStreamSynchronize(c->stream);
    cudaGraphExecDestroy(c->batch_exec);
    c->batch_exec = nullptr;
    c->batch_variant = -1;
  }
}

trim_err_t trim_set_params(trim_ctx* c, const trim_params_t* p) {
  if (!c || !p) return fail(c, TRIM_ERR_INVALID_ARG, "null argument");
  if (p->block_threads < 128 || p->block_threads > 512 || p->block_threads % 32)
    return fail(c, TRIM_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in [128,512]");
  if (p->spin_limit_ns == 0) return fail(c, TRIM_ERR_INVALID_ARG, "spin_limit_ns must be > 0");
  if (!(p->heur_push_ratio > 0.0f) || !(p->heur_ac6_ratio > 0.0f))
    return fail(c, TRIM_ERR_INVALID_ARG, "heuristic ratios must be > 0");
  if (p->sched_commit_rounds && !p->sched_recheck_rounds)
    return fail(c, TRIM_ERR_INVALID_ARG, "sched_recheck_rounds must be > 0 when committing");
  if (!(p->sched_commit_confidence >= 0.0f && p->sched_commit_confidence <= 1.0f))
    return fail(c, TRIM_ERR_INVALID_ARG, "sched_commit_confidence must be in [0, 1]");
  if (p->sched_handover > TRIM_HANDOVER_NONE)
    return fail(c, TRIM_ERR_INVALID_ARG, "unknown sched_handover");
  drop_batch_graph(c);
  forget_first_flavours(c);
  const trim_params_t old = c->params;
  c->params = *p;
  trim_err_t e = compute_grid(c);
  if (e != TRIM_OK) {
    c->params = old;
    compute_grid(c);
    return e;
  }
  return TRIM_OK;
}

trim_err_t trim_get_params(const trim_ctx* c, trim_params_t* p) {
  if (!c || !p) return fail(const_cast<trim_ctx*>(c), TRIM_ERR_INVALID_ARG, "null argument");
  *p = c->params;
  return TRIM_OK;
}

trim_err_t trim_set_model(trim_ctx* c, const float* blob, size_t n_floats) {
  if (!c) return fail(nullptr, TRIM_ERR_INVALID_ARG, "null context");
  forget_first_flavours(c);
  if (blob == nullptr) {
    drop_batch_graph(c);
    c->has_model = false;
    return TRIM_OK;
  }
  if (n_floats != TRIM_MLP_NBLOB)
    return fail(c, TRIM_ERR_INVALID_ARG, "model blob must hold TRIM_MLP_NBLOB floats");
  drop_batch_graph(c);
  if (!c->model) TRY(dalloc(c, &c->model, TRIM_MLP_NBLOB));
  CK(cudaMemcpyAsync(c->model, blob, TRIM_MLP_NBLOB * 4, cudaMemcpyHostToDevice, c->stream));
  TRY(sync_check(c));
  c->has_model = true;
  return TRIM_OK;
}

trim_err_t trim_set_dead_mask(trim_ctx* c, const uint8_t* mask, int on_device) {
  if (!c) return fail(nullptr, TRIM_ERR_INVALID_ARG, "null context");
  if (c->pending) TRY(finish_run(c, nullptr));
  drop_batch_graph(c);
  forget_first_flavours(c);
  if (mask == nullptr) {
    c->has_mask = false;
    return TRIM_OK;
  }
  if (c->n && !c->mask) TRY(dalloc(c, &c->mask, c->n));
  if (c->n)
    CK(cudaMemcpyAsync(c->mask, mask, c->n,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  TRY(sync_check(c));
  c->has_mask = true;
  return TRIM_OK;
}

trim_err_t trim_set_schedule(trim_ctx* c, const uint8_t* v, uint32_t len) {
  if (!c || (!v && len)) return fail(c, TRIM_ERR_INVALID_ARG, "null argument");
  for (uint32_t i = 0; i < len; ++i)
    if (v[i] > 2) return fail(c, TRIM_ERR_INVALID_ARG, "schedule entries must be 0..2");
  drop_batch_graph(c);
  if (len > c->script_len || !c->script) {
    uint8_t* s = nullptr;
    TRY(dalloc(c, &s, len));
    c->script = s;
  }
  if (len) CK(cudaMemcpyAsync(c->script, v, len, cudaMemcpyHostToDevice, c->stream));
  TRY(sync_check(c));
  c->script_len = len;
  c->h_script.assign(v, v + len);
  forget_first_flavours(c);
  return TRIM_OK;
}

trim_err_t trim_get_round_log(const trim_ctx* cc, trim_round_rec_t* out, size_t cap,
                              size_t* n_out) {
  trim_ctx* c = const_cast<trim_ctx*>(cc);
  if (!c || !n_out || (!out && cap)) return fail(c, TRIM_ERR_INVALID_ARG, "null argument");
  if (!(c->flags & TRIM_FLAG_ROUND_LOG))
    return fail(c, TRIM_ERR_STATE, "context was created without TRIM_FLAG_ROUND_LOG");
  if (c->pending) TRY(finish_run(c, nullptr));
  if (!c->ran) return fail(c, TRIM_ERR_STATE, "no completed run");
  const size_t have = std::min<size_t>(c->h_ctrl->rlog_len, c->rlog_cap);
  const size_t k = std::min(have, cap);
  if (k) CK(cudaMemcpy(out, c->rlog, k * sizeof(trim_round_rec_t), cudaMemcpyDeviceToHost));
  *n_out = k;
  return TRIM_OK;
}

void trim_destroy(trim_ctx* c) {
  if (!c) return;
  release(c);
  delete c;
}

const char* trim_last_error(const trim_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

trim_err_t trim_set_alloc_limit(uint64_t bytes) {
  g_alloc_limit = bytes;
  return TRIM_OK;
}

trim_err_t trim_probe_atomic_rate(const uint32_t* idx, uint64_t n_idx, uint32_t* counters,
                                  uint32_t n_counters, uint32_t reps, void* cuda_stream,
                                  float* ms_out) {
  trim_ctx* c = nullptr;  // errors go to the context-free message
  if (!idx || !counters || !ms_out || n_idx == 0 || n_counters == 0 || reps == 0)
    return fail(c, TRIM_ERR_INVALID_ARG, "null pointer or zero size");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 3.0e38f;
  cudaError_t e = cudaSuccess;
  for (uint32_t r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaMemsetAsync(counters, 0xFF, (size_t)n_counters * 4, st);
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) {
      trim_probe_atomic_kernel<<<sms * 32, 256, 0, st>>>(idx, n_idx, counters);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(c, e, "trim_probe_atomic_rate");
  *ms_out = best;
  return TRIM_OK;
}

}  // extern "C"
