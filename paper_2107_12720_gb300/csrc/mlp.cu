// mlp.cu -- training and inference kernels of the per-round scheduler MLP.
//
// 12 -> 32 -> 32 -> 3 with ReLU, softmax cross-entropy, Adam. Plain fp32 FMA:
// the network is ~1.6k multiply-adds per sample, far too small for tensor cores.
// One warp handles one sample at a time with lane j owning hidden unit j of both
// layers; gradients are accumulated per warp in registers, reduced per block in
// shared memory and written to per-block slots of the scratch buffer, which a
// second kernel sums in a fixed order (deterministic, no float atomics).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/trim.h"

namespace {

constexpr int NIN = TRIM_MLP_NIN, NH = TRIM_MLP_NH, NOUT = TRIM_MLP_NOUT;
constexpr int P = TRIM_MLP_NPARAMS;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH,
              OW3 = OB2 + NH, OB3 = OW3 + NOUT * NH;
static_assert(OB3 + NOUT == P, "parameter layout");
constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ float wsum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

struct Fwd {
  float a1, h1, a2, h2, z[NOUT];
};

// forward of one sample; W = parameters in shared memory; x in registers (all lanes)
__device__ __forceinline__ Fwd forward(const float* W, const float* x, unsigned lane) {
  Fwd f;
  float a = W[OB1 + lane];
#pragma unroll
  for (int i = 0; i < NIN; ++i) a = fmaf(W[OW1 + lane * NIN + i], x[i], a);
  f.a1 = a;
  f.h1 = fmaxf(a, 0.0f);
  float b = W[OB2 + lane];
#pragma unroll
  for (int k = 0; k < NH; ++k) b = fmaf(W[OW2 + lane * NH + k], __shfl_sync(FULL, f.h1, k), b);
  f.a2 = b;
  f.h2 = fmaxf(b, 0.0f);
#pragma unroll
  for (int o = 0; o < NOUT; ++o) f.z[o] = wsum(W[OW3 + o * NH + lane] * f.h2) + W[OB3 + o];
  return f;
}

__global__ void __launch_bounds__(THREADS) mlp_forward_kernel(const float* __restrict__ params,
                                                              const float* __restrict__ X,
                                                              uint32_t N, float* logits) {
  __shared__ float W[P];
  for (int i = threadIdx.x; i < P; i += THREADS) W[i] = params[i];
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t warp = blockIdx.x * WARPS + (threadIdx.x >> 5);
  const uint32_t nw = gridDim.x * WARPS;
  for (uint32_t row = warp; row < N; row += nw) {
    float x[NIN];
#pragma unroll
    for (int i = 0; i < NIN; ++i) x[i] = __ldg(&X[(size_t)row * NIN + i]);
    const Fwd f = forward(W, x, lane);
    if (lane < NOUT) logits[(size_t)row * NOUT + lane] = f.z[lane];
  }
}

// per-block partial gradients (and loss) of sum_rows CE / N
__global__ void __launch_bounds__(THREADS) mlp_grad_kernel(const float* __restrict__ params,
                                                           const float* __restrict__ X,
                                                           const uint8_t* __restrict__ y,
                                                           uint32_t N, float* partial) {
  __shared__ float W[P];
  __shared__ float G[P + 1];
  for (int i = threadIdx.x; i < P; i += THREADS) W[i] = params[i];
  for (int i = threadIdx.x; i < P + 1; i += THREADS) G[i] = 0.0f;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t warp = blockIdx.x * WARPS + (threadIdx.x >> 5);
  const uint32_t nw = gridDim.x * WARPS;
  const float invN = 1.0f / (float)N;
  float gW1[NIN], gW2[NH], gb1 = 0.0f, gb2 = 0.0f, gW3[NOUT], gb3 = 0.0f, loss = 0.0f;
#pragma unroll
  for (int i = 0; i < NIN; ++i) gW1[i] = 0.0f;
#pragma unroll
  for (int k = 0; k < NH; ++k) gW2[k] = 0.0f;
#pragma unroll
  for (int o = 0; o < NOUT; ++o) gW3[o] = 0.0f;
  for (uint32_t row = warp; row < N; row += nw) {
    float x[NIN];
#pragma unroll
    for (int i = 0; i < NIN; ++i) x[i] = __ldg(&X[(size_t)row * NIN + i]);
    const int label = (int)__ldg(&y[row]);
    const Fwd f = forward(W, x, lane);
    float mx = f.z[0];
#pragma unroll
    for (int o = 1; o < NOUT; ++o) mx = fmaxf(mx, f.z[o]);
    float e[NOUT], se = 0.0f;
#pragma unroll
    for (int o = 0; o < NOUT; ++o) { e[o] = expf(f.z[o] - mx); se += e[o]; }
    float dz[NOUT];
#pragma unroll
    for (int o = 0; o < NOUT; ++o) dz[o] = (e[o] / se - (o == label ? 1.0f : 0.0f)) * invN;
    if (lane == 0) loss += (mx + logf(se) - f.z[label]) * invN;
    // layer 3
    float dh2 = 0.0f;
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
      gW3[o] = fmaf(dz[o], f.h2, gW3[o]);
      dh2 = fmaf(W[OW3 + o * NH + lane], dz[o], dh2);
    }
    if (lane < NOUT) gb3 += dz[lane];
    const float da2 = f.a2 > 0.0f ? dh2 : 0.0f;
    // layer 2: lane j owns row j of W2; dh1 for lane k needs column k
    float dh1 = 0.0f;
#pragma unroll
    for (int k = 0; k < NH; ++k) {
      gW2[k] = fmaf(da2, __shfl_sync(FULL, f.h1, k), gW2[k]);
      dh1 = fmaf(W[OW2 + k * NH + lane], __shfl_sync(FULL, da2, k), dh1);
    }
    gb2 += da2;
    const float da1 = f.a1 > 0.0f ? dh1 : 0.0f;
#pragma unroll
    for (int i = 0; i < NIN; ++i) gW1[i] = fmaf(da1, x[i], gW1[i]);
    gb1 += da1;
  }
  // block reduction in shared memory (per warp in turn: deterministic order)
  for (int w = 0; w < WARPS; ++w) {
    if ((int)(threadIdx.x >> 5) == w) {
#pragma unroll
      for (int i = 0; i < NIN; ++i) G[OW1 + lane * NIN + i] += gW1[i];
      G[OB1 + lane] += gb1;
#pragma unroll
      for (int k = 0; k < NH; ++k) G[OW2 + lane * NH + k] += gW2[k];
      G[OB2 + lane] += gb2;
#pragma unroll
      for (int o = 0; o < NOUT; ++o) G[OW3 + o * NH + lane] += gW3[o];
      if (lane < NOUT) G[OB3 + lane] += gb3;
      if (lane == 0) G[P] += loss;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < P + 1; i += THREADS) partial[(size_t)blockIdx.x * (P + 1) + i] = G[i];
}

__global__ void mlp_reduce_kernel(const float* partial, uint32_t nblocks, float* grad,
                                  float* loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > P) return;
  float s = 0.0f;
  for (uint32_t b = 0; b < nblocks; ++b) s += partial[(size_t)b * (P + 1) + i];
  if (i < P) grad[i] = s;
  else *loss = s;
}

__global__ void mlp_adam_kernel(float* params, const float* grad, float* m, float* v, float lr,
                                float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

uint32_t grad_blocks(uint32_t N) {
  uint32_t b = (N + WARPS * 16 - 1) / (WARPS * 16);
  if (b < 1) b = 1;
  if (b > 296) b = 296;
  return b;
}

trim_err_t ck(cudaError_t e) { return e == cudaSuccess ? TRIM_OK : TRIM_ERR_CUDA; }

}  // namespace

extern "C" {

size_t trim_mlp_scratch_bytes(uint32_t N) {
  return (size_t)grad_blocks(N) * (P + 1) * sizeof(float);
}

trim_err_t trim_mlp_forward(const float* params, const float* X, uint32_t N, float* logits,
                            void* stream) {
  if (!params || (!X && N) || (!logits && N)) return TRIM_ERR_INVALID_ARG;
  if (N == 0) return TRIM_OK;
  const uint32_t blocks = (N + WARPS - 1) / WARPS < 1184 ? (N + WARPS - 1) / WARPS : 1184;
  mlp_forward_kernel<<<blocks, THREADS, 0, (cudaStream_t)stream>>>(params, X, N, logits);
  return ck(cudaGetLastError());
}

trim_err_t trim_mlp_loss_grad(const float* params, const float* X, const uint8_t* y, uint32_t N,
                              float* loss, float* grad, void* scratch, void* stream) {
  if (!params || !X || !y || !loss || !grad || !scratch || N == 0) return TRIM_ERR_INVALID_ARG;
  const uint32_t nb = grad_blocks(N);
  float* partial = static_cast<float*>(scratch);
  mlp_grad_kernel<<<nb, THREADS, 0, (cudaStream_t)stream>>>(params, X, y, N, partial);
  if (cudaGetLastError() != cudaSuccess) return TRIM_ERR_CUDA;
  mlp_reduce_kernel<<<(P + 1 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(partial, nb, grad, loss);
  return ck(cudaGetLastError());
}

trim_err_t trim_mlp_adam_step(float* params, const float* grad, float* m, float* v, uint32_t t,
                              float lr, float beta1, float beta2, float eps, void* stream) {
  if (!params || !grad || !m || !v || t == 0) return TRIM_ERR_INVALID_ARG;
  const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
  mlp_adam_kernel<<<(P + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, lr, beta1,
                                                                     beta2, eps, c1, c2);
  return ck(cudaGetLastError());
}

}  // extern "C"
