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

// ---- G^T by a two-level counting sort (bucket of the target, then target) ----
// Same-address atomics on the in-degree counters of hub targets serialise at
// the L2, so the global counting sort above is slow on skewed graphs. Here
// every count and every placement is a shared-memory atomic:
//   1. each CTA counts, for its rows, the edges per target bucket b = t >> shift
//      (counts[b * C + c], bucket-major, rounded up to whole 32-byte sectors of
//      8-byte pairs; the exact totals per bucket go to real[b]);
//   2. exclusive scans give every (bucket, CTA) its sector-aligned slot range
//      and every bucket its start in itgt;
//   3. the same traversal writes each edge's (t, u) into its range: pairs wait
//      in shared memory in groups of four per bucket and leave as one full
//      32-byte sector (a partial sector written to DRAM costs a read first);
//      pairs that find their bucket's group taken go out one by one from the
//      range's other end; slots left over get the fill value ~0;
//   4. one CTA per bucket counts the bucket's targets in shared memory, scans
//      them into ioff, and places every u at its target's next slot in itgt.
// Targets >= n are skipped (only TRIM_FLAG_VALIDATE reports them).

// Rows with more out-edges than kHeavyRow are walked by the whole CTA (one
// warp would take a skewed graph's longest rows alone, one dependent load per
// 32 edges); up to kHeavyCap of them per CTA, any further ones by their warp.
constexpr uint32_t kHeavyRow = 256;
constexpr uint32_t kHeavyCap = 1024;

// All threads of the CTA: f(u, t) for every out-edge of rows [r0, r1).
// Light rows: each warp takes 32 rows at a time and walks their edges laid end
// to end, 32 per step, four steps' loads in flight. Heavy rows: afterwards,
// one at a time, the whole CTA strides over the row. `heavy` and `nheavy` are
// shared scratch (*nheavy = 0 on entry).
template <class F>
__device__ __forceinline__ void cta_row_edges(const uint32_t* off, const uint32_t* tgt,
                                              uint32_t r0, uint32_t r1, uint32_t* heavy,
                                              uint32_t* nheavy, F f) {
  const unsigned lane = lane_id();
  const uint32_t nw = blockDim.x >> 5;
  for (uint32_t r = r0 + (threadIdx.x >> 5) * 32u; r < r1; r += nw * 32u) {  // warp-uniform
    const uint32_t v = r + lane;
    const bool has = v < r1;
    const uint32_t s = has ? off[v] : 0u;
    uint32_t d = has ? off[v + 1] - s : 0u;
    if (d > kHeavyRow) {
      const uint32_t at = atomicAdd(nheavy, 1u);
      if (at < kHeavyCap) {
        heavy[at] = v;
        d = 0u;
      }
    }
    const uint32_t incl = warp_incl_scan(d);
    const uint32_t excl = incl - d;
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    for (uint32_t k0 = 0; k0 < total; k0 += 128u) {  // warp-uniform
      uint32_t u[4], t[4];
      bool ok[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t k = k0 + (uint32_t)q * 32u + lane;
        const unsigned o = owner_of(excl, k);
        const uint32_t so = __shfl_sync(0xFFFFFFFFu, s, o);
        const uint32_t xo = __shfl_sync(0xFFFFFFFFu, excl, o);
        ok[q] = k < total;
        u[q] = r + o;
        t[q] = ok[q] ? __ldg(&tgt[so + (k - xo)]) : 0u;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (ok[q]) f(u[q], t[q]);
    }
  }
  __syncthreads();
  const uint32_t nh = min(*nheavy, kHeavyCap);
  for (uint32_t h = 0; h < nh; ++h) {  // block-uniform
    const uint32_t v = heavy[h];
    const uint32_t s = off[v], e = off[v + 1];
    for (uint32_t k0 = s; k0 < e; k0 += 4u * blockDim.x) {
      uint32_t t[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t k = k0 + (uint32_t)q * blockDim.x + threadIdx.x;
        t[q] = k < e ? __ldg(&tgt[k]) : 0u;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (k0 + (uint32_t)q * blockDim.x + threadIdx.x < e) f(v, t[q]);
    }
  }
}

// Pass 1: per-CTA histogram of target buckets over rows [c * rows, (c+1) * rows).
__global__ void trim_gt_hist_kernel(const uint32_t* off, const uint32_t* tgt, uint32_t n,
                                    uint32_t rows, uint32_t shift, uint32_t nb,
                                    uint32_t* counts, uint32_t* real) {
  extern __shared__ uint32_t hist[];
  __shared__ uint32_t heavy[kHeavyCap];
  __shared__ uint32_t nheavy;
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0u;
  if (threadIdx.x == 0) nheavy = 0u;
  __syncthreads();
  const uint32_t r0 = min(n, blockIdx.x * rows), r1 = min(n, r0 + rows);
  cta_row_edges(off, tgt, r0, r1, heavy, &nheavy, [&](uint32_t, uint32_t t) {
    if (t < n) atomicAdd(&hist[t >> shift], 1u);
  });
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
    counts[(size_t)i * gridDim.x + blockIdx.x] = (hist[i] + 3u) & ~3u;
    if (hist[i]) atomicAdd(&real[i], hist[i]);
  }
}

// Pass 3: the edges of the same rows go to their (bucket, CTA) slot ranges.
// Shared memory per bucket: a group of four pairs, its slot requests and
// completed writes, and the range's two cursors (groups from the start,
// single pairs from the end).
__global__ void trim_gt_scatter_kernel(const uint32_t* off, const uint32_t* tgt, uint32_t n,
                                       uint32_t rows, uint32_t shift, uint32_t nb,
                                       const uint32_t* slots, unsigned long long* pairs) {
  extern __shared__ unsigned long long gbuf[];  // nb x 4 pairs, then the counters
  uint32_t* req = reinterpret_cast<uint32_t*>(gbuf + (size_t)nb * 4u);
  uint32_t* done = req + nb;
  uint32_t* lo = done + nb;
  uint32_t* hi = lo + nb;
  __shared__ uint32_t heavy[kHeavyCap];
  __shared__ uint32_t nheavy;
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
    const size_t at = (size_t)i * gridDim.x + blockIdx.x;
    req[i] = 0u;
    done[i] = 0u;
    lo[i] = slots[at];
    hi[i] = slots[at + 1];
  }
  if (threadIdx.x == 0) nheavy = 0u;
  __syncthreads();
  volatile unsigned long long* vbuf = gbuf;
  const uint32_t r0 = min(n, blockIdx.x * rows), r1 = min(n, r0 + rows);
  cta_row_edges(off, tgt, r0, r1, heavy, &nheavy, [&](uint32_t u, uint32_t t) {
    if (t >= n) return;
    const uint32_t b = t >> shift;
    const unsigned long long pr = ((unsigned long long)t << 32) | u;
    const uint32_t slot = atomicAdd(&req[b], 1u);
    if (slot >= 4u) {  // the group is taken: this pair goes out alone
      pairs[atomicSub(&hi[b], 1u) - 1u] = pr;
      return;
    }
    vbuf[b * 4u + slot] = pr;
    __threadfence_block();
    if (atomicAdd(&done[b], 1u) != 3u) return;
    // the fourth write of the group: send it as one sector and open the next
    __threadfence_block();
    const uint32_t at = atomicAdd(&lo[b], 4u);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(pairs + at);
    dst[0] = make_ulonglong2(vbuf[b * 4u], vbuf[b * 4u + 1u]);
    dst[1] = make_ulonglong2(vbuf[b * 4u + 2u], vbuf[b * 4u + 3u]);
    __threadfence_block();
    atomicExch(&done[b], 0u);
    __threadfence_block();
    atomicExch(&req[b], 0u);
  });
  __syncthreads();
  // groups that never filled: their pairs go out one by one; the range's
  // unused slots (at most 3) get the fill value
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
    for (uint32_t k = 0; k < done[i]; ++k) pairs[--hi[i]] = vbuf[i * 4u + k];
    for (uint32_t k = lo[i]; k < hi[i]; ++k) pairs[k] = ~0ull;
  }
}

// Warp-collective: lanes whose target equals lane 0's form `same` when at
// least 8 of them do (a hub's in-edges dominate this warp's pairs); they take
// one combined atomic, every other lane its own.
__device__ __forceinline__ unsigned hub_lanes(uint32_t t) {
  const uint32_t t0 = __shfl_sync(0xFFFFFFFFu, t, 0);
  const unsigned same = __ballot_sync(0xFFFFFFFFu, t == t0 && t != 0xFFFFFFFFu);
  return __popc(same) >= 8 ? same : 0u;
}

// Pass 4: CTA per bucket (grid-stride).
__global__ void trim_gt_place_kernel(const unsigned long long* pairs, const uint32_t* slots,
                                     const uint32_t* rstart, uint32_t C, uint32_t n, uint32_t m,
                                     uint32_t shift, uint32_t nb, uint32_t* ioff,
                                     uint32_t* itgt) {
  extern __shared__ uint32_t cnt[];
  const unsigned lane = lane_id();
  const uint32_t nw = blockDim.x >> 5;
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const uint32_t base = b << shift;
    const uint32_t nt = min(1u << shift, n - base);
    const uint32_t p0 = slots[(size_t)b * C];
    const uint32_t p1 = slots[(size_t)(b + 1u) * C];  // slots[nb * C] = all slots
    for (uint32_t i = threadIdx.x; i < nt; i += blockDim.x) cnt[i] = 0u;
    __syncthreads();
    // four loads in flight per lane, then the combined atomics
    for (uint32_t q = p0 + (threadIdx.x >> 5) * 32u; q < p1; q += 4u * nw * 32u) {  // warp-uniform
      uint32_t t[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t p = q + (uint32_t)k * nw * 32u + lane;
        const unsigned long long pr = p < p1 ? pairs[p] : ~0ull;  // ~0: an unused slot
        t[k] = pr != ~0ull ? (uint32_t)(pr >> 32) - base : 0xFFFFFFFFu;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const unsigned same = hub_lanes(t[k]);
        if (same >> lane & 1u) {
          if (lane == 0) atomicAdd(&cnt[t[k]], (uint32_t)__popc(same));
        } else if (t[k] != 0xFFFFFFFFu) {
          atomicAdd(&cnt[t[k]], 1u);
        }
      }
    }
    __syncthreads();
    uint32_t carry = rstart[b];  // edges of the buckets before b
    for (uint32_t j0 = 0; j0 < nt; j0 += blockDim.x) {  // block-uniform
      const uint32_t j = j0 + threadIdx.x;
      const uint32_t x = j < nt ? cnt[j] : 0u;
      unsigned tot;
      const uint32_t ex = block_excl_scan(x, &tot);
      if (j < nt) {
        cnt[j] = carry + ex;
        ioff[base + j] = carry + ex;
      }
      carry += tot;
    }
    __syncthreads();
    for (uint32_t q = p0 + (threadIdx.x >> 5) * 32u; q < p1; q += 4u * nw * 32u) {
      unsigned long long pr[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t p = q + (uint32_t)k * nw * 32u + lane;
        pr[k] = p < p1 ? pairs[p] : ~0ull;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool valid = pr[k] != ~0ull;
        const uint32_t t = valid ? (uint32_t)(pr[k] >> 32) - base : 0xFFFFFFFFu;
        const unsigned same = hub_lanes(t);
        uint32_t at = 0;
        if (lane == 0 && same) at = atomicAdd(&cnt[t], (uint32_t)__popc(same));
        at = __shfl_sync(0xFFFFFFFFu, at, 0) + __popc(same & ((1u << lane) - 1u));
        if (valid && !(same >> lane & 1u)) at = atomicAdd(&cnt[t], 1u);
        if (valid) itgt[at] = (uint32_t)pr[k];
      }
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ioff[n] = m;
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
