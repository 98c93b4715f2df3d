// trim_aux.cu -- small helper kernels of the trimming library: control-block
// reset, status extraction, and the device-side CSR utilities (G^T by counting
// sort, grid scans, validation).
#include "trim_internal.cuh"

using namespace trimk;

namespace {

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

}  // namespace

// Control block reset before every run (one thread).
__global__ void trim_reset_ctrl_kernel(Ctrl* C) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned* w = reinterpret_cast<unsigned*>(C);
    for (size_t i = 0; i < sizeof(Ctrl) / 4; ++i) w[i] = 0u;
  }
}

__global__ void trim_status_kernel(const uint32_t* level, uint32_t n, uint8_t* status) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    status[v] = level[v] == LIVE ? 1 : 0;
}

// After a run with a dead mask: masked vertices carry level 0 inside the run
// (removed before round 1, so every variant's "level[u] < r" test skips them);
// their reported level is TRIM_MASKED.
__global__ void trim_mask_levels_kernel(uint32_t* level, const uint8_t* mask, uint32_t n) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (mask[v]) level[v] = TRIM_MASKED;
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

// Diagnostic: returning atomicSub over an index stream, fully parallel. The
// returned values are folded into `acc` so the atomics keep their return path
// (the form AC-4 uses); the guarded store never fires for counters that start
// at 0xFFFFFFFF and are decremented at most 2^32 - 2 times.
__global__ void trim_probe_atomic_kernel(const uint32_t* idx, uint64_t n, uint32_t* counters) {
  uint32_t acc = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    acc |= (atomicSub(&counters[idx[i]], 1u) == 0u) ? 1u : 0u;
  if (acc) counters[0] = 0u;
}
