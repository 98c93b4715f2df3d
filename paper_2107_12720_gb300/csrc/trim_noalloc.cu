// trim_noalloc.cu -- AC-4 trimming for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a result: code
// running inside a memory-pool discipline that forbids new device allocations
// (allocator hooks, fixed-budget serving processes), plugins that must not
// touch the host application's allocator, or code paths that must not
// synchronise the device the way cudaMalloc/cudaFree can. trim_run_ac4_noalloc
// serves them: it runs the same AC-4 persistent kernel as trim_run, but every
// byte of scratch it needs (counters, dead log, AC-4 work list, control block)
// lives in one file-scope __device__ array of fixed size. The caller passes the
// graph, its transpose and the output array; nothing is allocated per call.
//
// The array exists in every GPU context that loads this library and stays
// there until the process exits (about TRIM_NOALLOC_SCRATCH_BYTES per device).
#include <cuda_runtime.h>

#include <mutex>

#include "trim_internal.cuh"

namespace {

constexpr uint32_t kMaxN = TRIM_NOALLOC_MAX_N;
constexpr uint32_t kMaxM = TRIM_NOALLOC_MAX_M;
constexpr size_t kAlignWords = 64;  // 256-byte alignment of every region
constexpr size_t round_up(size_t x) { return (x + kAlignWords - 1) / kAlignWords * kAlignWords; }

// region layout inside the scratch array, in 32-bit words
constexpr size_t kCtrlWords = round_up((sizeof(trimk::Ctrl) + 3) / 4);
constexpr size_t kOffCnt = kCtrlWords;
constexpr size_t kOffLog = kOffCnt + round_up(kMaxN);
constexpr size_t kOffRoff = kOffLog + round_up(kMaxN);
constexpr size_t kOffRow = kOffRoff + round_up(kMaxN + 2);
constexpr size_t kOffEoff = kOffRow + round_up(kMaxN);
constexpr size_t kOffChunk = kOffEoff + round_up(kMaxN);
constexpr size_t kOffSpare = kOffChunk + round_up((kMaxM >> 5) + 2);
constexpr size_t kWords = kOffSpare + kAlignWords;
static_assert(kWords * 4 == TRIM_NOALLOC_SCRATCH_BYTES,
              "TRIM_NOALLOC_SCRATCH_BYTES in trim.h must match the scratch layout");

// The scratch shared by every call on a device (host code only ever uses the
// address obtained with cudaGetSymbolAddress below, never this name).
static __device__ __align__(256) uint32_t g_noalloc_scratch[kWords];

constexpr uint32_t kSliceEntries = 256;  // per-warp append slices of the AC-4 kernel
constexpr uint32_t kBlock = 512;
size_t dyn_smem() { return 16 * 4 * (size_t)kSliceEntries * sizeof(uint32_t); }

struct DeviceSetup {
  bool ready = false;
  uint32_t* scratch = nullptr;
  int grid = 0;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: the device address of the scratch
// array and the cooperative grid size of the AC-4 kernel.
trim_err_t setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return TRIM_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(trim_persistent_kernel_m1,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn_smem()) != cudaSuccess) {
      (void)cudaGetLastError();
      return TRIM_ERR_CUDA;
    }
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trim_persistent_kernel_m1,
                                                      (int)kBlock, dyn_smem()) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        per_sm <= 0) {
      (void)cudaGetLastError();
      return TRIM_ERR_CUDA;
    }
    s.scratch = static_cast<uint32_t*>(p);
    s.grid = per_sm * sms;
    s.ready = true;
  }
  *out = &s;
  return TRIM_OK;
}

}  // namespace

extern "C" trim_err_t trim_run_ac4_noalloc(const uint32_t* offsets, const uint32_t* targets,
                                           const uint32_t* in_offsets, const uint32_t* in_targets,
                                           uint32_t n, uint32_t m, uint32_t* level_out,
                                           uint32_t* rounds_out, void* cuda_stream) {
  if (n > kMaxN || m > kMaxM) return TRIM_ERR_TOO_LARGE;
  if (offsets == nullptr || in_offsets == nullptr || level_out == nullptr ||
      (m && (targets == nullptr || in_targets == nullptr)))
    return TRIM_ERR_INVALID_ARG;
  if (rounds_out) *rounds_out = 0;
  if (n == 0) return TRIM_OK;
  int dev = 0, count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    (void)cudaGetLastError();
    return TRIM_ERR_NO_DEVICE;
  }
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TRIM_ERR_CUDA;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (!(major == 10 && minor == 3)) return TRIM_ERR_NO_DEVICE;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  // the scratch address and the launch shape belong to the current device: a
  // stream of another device would receive pointers of the wrong context
  int stream_dev = -1;
  if (cudaStreamGetDevice(stream, &stream_dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return TRIM_ERR_INVALID_ARG;
  }
  if (stream_dev != dev) return TRIM_ERR_INVALID_ARG;
  DeviceSetup* s = nullptr;
  trim_err_t e = setup_device(dev, &s);
  if (e != TRIM_OK) return e;
  uint32_t* base = s->scratch;

  trimk::Dev D{};
  D.n = n;
  D.m = m;
  D.off = offsets;
  D.tgt = targets;
  D.ioff = in_offsets;
  D.itgt = in_targets;
  D.level = level_out;
  D.cnt = base + kOffCnt;
  D.log = base + kOffLog;
  D.roff = base + kOffRoff;
  D.w4_row = base + kOffRow;
  D.w4_eoff = base + kOffEoff;
  D.chunk_first = base + kOffChunk;
  D.live0 = D.live1 = base + kOffSpare;  // never written by the AC-4 kernel
  D.bsum = base + kOffSpare;
  D.C = reinterpret_cast<trimk::Ctrl*>(base);
  D.mode = TRIM_AC4_PUSH;
  D.flags = trimk::F_AC4_POSSIBLE;
  D.sbuf_cap = kSliceEntries;
  D.spin_limit_ns = 5ull * 1000 * 1000 * 1000;
  D.heur_push_ratio = 1.0f;
  D.heur_ac6_ratio = 1.0f;
  D.local_edges_max = 1u << 18;  // as trim_run's default

  // The control block must start at zero; every other region is written
  // before it is read within a call, so stale contents of earlier calls are harmless.
  trim_reset_ctrl_kernel<<<1, 32, 0, stream>>>(D.C);
  if (cudaGetLastError() != cudaSuccess) return TRIM_ERR_CUDA;
  void* args[] = {&D};
  if (cudaLaunchCooperativeKernel((const void*)trim_persistent_kernel_m1, dim3(s->grid),
                                  dim3(kBlock), args, dyn_smem(), stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return TRIM_ERR_CUDA;
  }
  unsigned int status[2] = {0, 0};  // err, err_info
  uint32_t rounds = 0;
  const trimk::Ctrl* C = D.C;
  if (cudaMemcpyAsync(status, &C->err, sizeof(status), cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(&rounds, &C->rounds, sizeof(rounds), cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return TRIM_ERR_CUDA;
  }
  if (status[0] != 0) return (trim_err_t)status[0];
  if (rounds_out) *rounds_out = rounds;
  return TRIM_OK;
}
