// Learned selectivity surrogate (not in the paper; evaluated against exact ESC):
// an MLP 64 -> 128 -> ReLU -> 128 -> ReLU -> 1 predicting log10 selectivity
// from encoded predicate features.  Weights are used in bfloat16, biases
// and every accumulation are float32, the optimiser keeps float32 master
// weights (Adam).
//
// Flat parameter layout (ESC_MLP_PARAMS = 24961 floats): W1 [128][64], b1
// [128], W2 [128][128], b2 [128], w3 [128], b3.  The bfloat16 copy has the
// same layout (its bias entries are unused).
//
// Kernel shape: one thread per hidden unit (128), 8 samples per pass; the
// weight matrices sit in shared memory as float32 with a padded row stride
// (65 / 129) so that threads reading one column, and threads reading their
// own rows, hit distinct banks.  The gradient kernel keeps the block's
// weight-gradient sums in shared memory (each thread owns rows) and adds
// them to the global gradient once, at the end.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "esc_internal.h"

namespace esc {

constexpr int kIn = 64, kH = 128, kS = 8;  // inputs, hidden width, samples per pass
constexpr int kW1 = 0, kB1 = kW1 + kH * kIn, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH, kB3 = kW3 + kH;
constexpr int kParams = kB3 + 1;  // 24961
constexpr int kS1 = kIn + 1, kS2 = kH + 1;  // padded row strides

__device__ __forceinline__ float bf(const uint16_t v) {
  return __uint_as_float((uint32_t)v << 16);
}

struct MlpSmem {
  float W1[kH * kS1];
  float W2[kH * kS2];
  float w3[kH], b1[kH], b2[kH];
  float x[kS][kIn];
  float z1[kS][kH];   // relu(a1)
  float a1[kS][kH];
  float d2[kS][kH];   // d loss / d a2
  float red[kS][4];   // per-warp partial sums of y
  float b3;
};

struct GradSmem {
  float gW1[kH * kS1];
  float gW2[kH * kS2];
};

__device__ void load_weights(MlpSmem &S, const uint16_t *wbf, const float *pf) {
  for (int i = threadIdx.x; i < kH * kIn; i += blockDim.x) S.W1[(i / kIn) * kS1 + i % kIn] = bf(wbf[kW1 + i]);
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) S.W2[(i / kH) * kS2 + i % kH] = bf(wbf[kW2 + i]);
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    S.w3[i] = bf(wbf[kW3 + i]);
    S.b1[i] = pf[kB1 + i];
    S.b2[i] = pf[kB2 + i];
  }
  if (threadIdx.x == 0) S.b3 = pf[kB3];
}

// Forward of samples s0 .. s0+kS-1 (those < B): leaves z1, a1 in shared
// memory, returns this thread's (unit j) a2 per sample, and the outputs y in
// S.red[s][0] (valid after the final barrier).
__device__ void forward_pass(MlpSmem &S, const uint16_t *x, uint64_t B, uint64_t s0, float (&a2)[kS]) {
  const int j = threadIdx.x;
  for (int i = j; i < kS * kIn; i += blockDim.x) {
    const uint64_t s = s0 + i / kIn;
    S.x[i / kIn][i % kIn] = s < B ? bf(x[s * kIn + i % kIn]) : 0.0f;
  }
  __syncthreads();
  float acc[kS];
#pragma unroll
  for (int s = 0; s < kS; ++s) acc[s] = S.b1[j];
  for (int k = 0; k < kIn; ++k) {
    const float w = S.W1[j * kS1 + k];
#pragma unroll
    for (int s = 0; s < kS; ++s) acc[s] = fmaf(w, S.x[s][k], acc[s]);
  }
#pragma unroll
  for (int s = 0; s < kS; ++s) {
    S.a1[s][j] = acc[s];
    S.z1[s][j] = fmaxf(acc[s], 0.0f);
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < kS; ++s) acc[s] = S.b2[j];
  for (int k = 0; k < kH; ++k) {
    const float w = S.W2[j * kS2 + k];
#pragma unroll
    for (int s = 0; s < kS; ++s) acc[s] = fmaf(w, S.z1[s][k], acc[s]);
  }
  const float w3 = S.w3[j];
#pragma unroll
  for (int s = 0; s < kS; ++s) {
    a2[s] = acc[s];
    float v = w3 * fmaxf(acc[s], 0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((j & 31) == 0) S.red[s][j >> 5] = v;
  }
  __syncthreads();
  if (j < kS) S.red[j][0] = S.red[j][0] + S.red[j][1] + S.red[j][2] + S.red[j][3] + S.b3;
  __syncthreads();
}

__global__ void __launch_bounds__(kH) mlp_forward_kernel(const uint16_t *x, uint64_t B, const uint16_t *wbf,
                                                          const float *pf, float *y) {
  extern __shared__ __align__(16) uint8_t smem[];
  MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem);
  load_weights(S, wbf, pf);
  __syncthreads();
  for (uint64_t s0 = (uint64_t)blockIdx.x * kS; s0 < B; s0 += (uint64_t)gridDim.x * kS) {
    float a2[kS];
    forward_pass(S, x, B, s0, a2);
    if (threadIdx.x < kS && s0 + threadIdx.x < B) y[s0 + threadIdx.x] = S.red[threadIdx.x][0];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kH) mlp_grad_kernel(const uint16_t *x, const float *t, uint64_t B,
                                                       const uint16_t *wbf, const float *pf, float *grad,
                                                       float *loss_sum) {
  extern __shared__ __align__(16) uint8_t smem[];
  MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem);
  GradSmem &G = *reinterpret_cast<GradSmem *>(smem + ((sizeof(MlpSmem) + 15) & ~(size_t)15));
  const int j = threadIdx.x;
  load_weights(S, wbf, pf);
  for (int i = j; i < kH * kS1; i += blockDim.x) G.gW1[i] = 0.0f;
  for (int i = j; i < kH * kS2; i += blockDim.x) G.gW2[i] = 0.0f;
  __syncthreads();
  float gb1 = 0.0f, gb2 = 0.0f, gw3 = 0.0f, gb3 = 0.0f, lsum = 0.0f;
  const float inv_b = 2.0f / (float)B;
  for (uint64_t s0 = (uint64_t)blockIdx.x * kS; s0 < B; s0 += (uint64_t)gridDim.x * kS) {
    float a2[kS];
    forward_pass(S, x, B, s0, a2);
    // output layer and second hidden layer: thread j owns unit j (row j of W2)
    float dy[kS];
    const float w3 = S.w3[j];
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      const bool ok = s0 + s < B;
      const float e = ok ? S.red[s][0] - t[s0 + s] : 0.0f;
      dy[s] = e * inv_b;
      if (j == 0) {
        lsum += e * e;
        gb3 += dy[s];
      }
      const float z2 = fmaxf(a2[s], 0.0f);
      gw3 = fmaf(dy[s], z2, gw3);
      const float d2 = a2[s] > 0.0f ? dy[s] * w3 : 0.0f;
      S.d2[s][j] = d2;
      gb2 += d2;
    }
    for (int k = 0; k < kH; ++k) {
      float g = G.gW2[j * kS2 + k];
#pragma unroll
      for (int s = 0; s < kS; ++s) g = fmaf(S.d2[s][j], S.z1[s][k], g);
      G.gW2[j * kS2 + k] = g;
    }
    __syncthreads();
    // first hidden layer: thread k owns unit k (row k of W1), reads column k of W2
    const int k = j;
    float d1[kS];
#pragma unroll
    for (int s = 0; s < kS; ++s) d1[s] = 0.0f;
    for (int i = 0; i < kH; ++i) {
      const float w = S.W2[i * kS2 + k];
#pragma unroll
      for (int s = 0; s < kS; ++s) d1[s] = fmaf(w, S.d2[s][i], d1[s]);
    }
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      d1[s] = S.a1[s][k] > 0.0f ? d1[s] : 0.0f;
      gb1 += d1[s];
    }
    for (int m = 0; m < kIn; ++m) {
      float g = G.gW1[k * kS1 + m];
#pragma unroll
      for (int s = 0; s < kS; ++s) g = fmaf(d1[s], S.x[s][m], g);
      G.gW1[k * kS1 + m] = g;
    }
    __syncthreads();
  }
  // add this block's sums to the global gradient
  for (int i = j; i < kH * kIn; i += blockDim.x) atomicAdd(&grad[kW1 + i], G.gW1[(i / kIn) * kS1 + i % kIn]);
  for (int i = j; i < kH * kH; i += blockDim.x) atomicAdd(&grad[kW2 + i], G.gW2[(i / kH) * kS2 + i % kH]);
  atomicAdd(&grad[kB1 + j], gb1);
  atomicAdd(&grad[kB2 + j], gb2);
  atomicAdd(&grad[kW3 + j], gw3);
  if (j == 0) {
    atomicAdd(&grad[kB3], gb3);
    atomicAdd(loss_sum, lsum);
  }
}

__global__ void adam_kernel(float *p, uint16_t *wbf, const float *g, float *m, float *v, uint64_t n, float lr,
                            float beta1, float beta2, float eps, float bc1, float bc2) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
    const __nv_bfloat16 h = __float2bfloat16_rn(pi);
    wbf[i] = *reinterpret_cast<const uint16_t *>(&h);
  }
}

size_t fwd_smem() { return sizeof(MlpSmem); }
size_t grad_smem() { return ((sizeof(MlpSmem) + 15) & ~(size_t)15) + sizeof(GradSmem); }

}  // namespace esc

using namespace esc;

#define ESC_MLP_CK(call)                                                                      \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(ESC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {
int grid_for(uint64_t B) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t chunks = (B + kS - 1) / kS;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(chunks, (uint64_t)sms));
}
}  // namespace

extern "C" {

esc_status esc_mlp_forward(const uint16_t *x_bf16, uint64_t batch, const uint16_t *w_bf16, const float *params,
                           float *y, void *stream) {
  ESC_RANGE("esc_mlp_forward");
  if (batch == 0) return ESC_OK;
  if (!x_bf16 || !w_bf16 || !params || !y) return fail(ESC_EINVAL, "esc_mlp_forward: NULL argument");
  ESC_MLP_CK(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem()));
  mlp_forward_kernel<<<grid_for(batch) * 2, kH, fwd_smem(), static_cast<cudaStream_t>(stream)>>>(x_bf16, batch, w_bf16,
                                                                                              params, y);
  ESC_MLP_CK(cudaGetLastError());
  clear_error();
  return ESC_OK;
}

esc_status esc_mlp_grad(const uint16_t *x_bf16, const float *target, uint64_t batch, const uint16_t *w_bf16,
                        const float *params, float *grad, float *loss_sum, void *stream) {
  ESC_RANGE("esc_mlp_grad");
  if (batch == 0) return ESC_OK;
  if (!x_bf16 || !target || !w_bf16 || !params || !grad || !loss_sum)
    return fail(ESC_EINVAL, "esc_mlp_grad: NULL argument");
  ESC_MLP_CK(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()));
  mlp_grad_kernel<<<grid_for(batch), kH, grad_smem(), static_cast<cudaStream_t>(stream)>>>(
      x_bf16, target, batch, w_bf16, params, grad, loss_sum);
  ESC_MLP_CK(cudaGetLastError());
  clear_error();
  return ESC_OK;
}

esc_status esc_mlp_adam(float *params, uint16_t *w_bf16, const float *grad, float *m, float *v, uint64_t n, float lr,
                        float beta1, float beta2, float eps, int32_t step, void *stream) {
  ESC_RANGE("esc_mlp_adam");
  if (!params || !w_bf16 || !grad || !m || !v || step < 1) return fail(ESC_EINVAL, "esc_mlp_adam: bad argument");
  const float bc1 = 1.0f - powf(beta1, (float)step);
  const float bc2 = 1.0f - powf(beta2, (float)step);
  adam_kernel<<<(int)std::min<uint64_t>((n + 255) / 256, 1024), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      params, w_bf16, grad, m, v, n, lr, beta1, beta2, eps, bc1, bc2);
  ESC_MLP_CK(cudaGetLastError());
  clear_error();
  return ESC_OK;
}

}  // extern "C"
