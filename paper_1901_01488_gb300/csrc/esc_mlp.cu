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
// Kernel shape: kSets sets of 128 threads per block; in each set, one thread
// per hidden unit, 8 samples per pass (a block: kSets x 8 samples per pass,
// one set of weights).  The weight matrices sit in shared memory as bfloat16
// with padded row strides (66 / 130 elements) so that threads reading their
// own rows, and threads reading one column, hit distinct banks.  The gradient
// kernel keeps the block's weight-gradient sums in shared memory (float32);
// each thread adds the samples of every set into its share of a row (a
// quarter of the columns), so no two threads update the same sum, and the
// sums go to the global gradient once, at the end.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "esc_internal.h"

namespace esc {

constexpr int kIn = 64, kH = 128, kS = 8;  // inputs, hidden width, samples per pass and set
constexpr int kSets = 4;                     // sample sets per block
constexpr int kMlpThreads = kSets * kH;      // 512
constexpr int kW1 = 0, kB1 = kW1 + kH * kIn, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH, kB3 = kW3 + kH;
constexpr int kParams = kB3 + 1;  // 24961
constexpr int kT1 = kIn + 4, kT2 = kH + 4;  // padded bf16 row strides (34 and 66 words: 8-byte loads
                                            // of 16 threads, their rows, hit distinct banks)
constexpr int kG1 = kIn + 1, kG2 = kH + 1;  // padded float32 row strides of the gradient sums
static_assert(kH % kSets == 0 && kIn % kSets == 0, "columns split evenly over the sets");
static_assert(kParams == ESC_MLP_PARAMS, "flat parameter layout");

__device__ __forceinline__ float bf(const uint16_t v) {
  return __uint_as_float((uint32_t)v << 16);
}

struct MlpWeights {
  uint16_t W1[kH * kT1];  // bfloat16
  uint16_t W2[kH * kT2];
  float w3[kH], b1[kH], b2[kH];
  float b3;
};

// One set's samples of a pass (16-byte aligned rows: 4 values a load).
struct alignas(16) MlpSet {
  float x[kS][kIn];
  float z1[kS][kH];   // relu(a1)
  float a1[kS][kH];   // pre-activation; the gradient kernel overwrites it with d loss / d a1
  float d2[kS][kH];   // d loss / d a2
  float red[kS][4];   // per-warp partial sums of y
};

struct MlpSmem {
  MlpWeights W;
  MlpSet set[kSets];
};

struct GradSmem {
  float gW1[kH * kG1];
  float gW2[kH * kG2];
};

__device__ void load_weights(MlpWeights &W, const uint16_t *wbf, const float *pf) {
  for (int i = threadIdx.x; i < kH * kIn; i += blockDim.x) W.W1[(i / kIn) * kT1 + i % kIn] = wbf[kW1 + i];
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) W.W2[(i / kH) * kT2 + i % kH] = wbf[kW2 + i];
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    W.w3[i] = bf(wbf[kW3 + i]);
    W.b1[i] = pf[kB1 + i];
    W.b2[i] = pf[kB2 + i];
  }
  if (threadIdx.x == 0) W.b3 = pf[kB3];
}

// Forward of this thread's set (samples s0 .. s0+kS-1, those < B; thread j =
// hidden unit j of the set): leaves z1, a1 in the set's buffers, returns a2
// per sample, and the outputs y in S.red[s][0] (valid after the final
// barrier).  Every thread of the block calls it together (block barriers).
__device__ void forward_pass(const MlpWeights &W, MlpSet &S, const uint16_t *x, uint64_t B, uint64_t s0,
                             float (&a2)[kS]) {
  const int j = threadIdx.x % kH;
  for (int i = j; i < kS * kIn; i += kH) {
    const uint64_t s = s0 + i / kIn;
    S.x[i / kIn][i % kIn] = s < B ? bf(x[s * kIn + i % kIn]) : 0.0f;
  }
  __syncthreads();
  float acc[kS];
#pragma unroll
  for (int s = 0; s < kS; ++s) acc[s] = W.b1[j];
  // 4 inputs a step: 4 weights in one 8-byte load, 4 values of each sample in one 16-byte load
  for (int k = 0; k < kIn; k += 4) {
    const uint2 w2 = *reinterpret_cast<const uint2 *>(&W.W1[j * kT1 + k]);
    const float w0 = __uint_as_float(w2.x << 16), w1 = __uint_as_float(w2.x & 0xffff0000u);
    const float w2f = __uint_as_float(w2.y << 16), w3f = __uint_as_float(w2.y & 0xffff0000u);
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      const float4 v = *reinterpret_cast<const float4 *>(&S.x[s][k]);
      acc[s] = fmaf(w0, v.x, acc[s]);
      acc[s] = fmaf(w1, v.y, acc[s]);
      acc[s] = fmaf(w2f, v.z, acc[s]);
      acc[s] = fmaf(w3f, v.w, acc[s]);
    }
  }
#pragma unroll
  for (int s = 0; s < kS; ++s) {
    S.a1[s][j] = acc[s];
    S.z1[s][j] = fmaxf(acc[s], 0.0f);
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < kS; ++s) acc[s] = W.b2[j];
  for (int k = 0; k < kH; k += 4) {
    const uint2 w2 = *reinterpret_cast<const uint2 *>(&W.W2[j * kT2 + k]);
    const float w0 = __uint_as_float(w2.x << 16), w1 = __uint_as_float(w2.x & 0xffff0000u);
    const float w2f = __uint_as_float(w2.y << 16), w3f = __uint_as_float(w2.y & 0xffff0000u);
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      const float4 v = *reinterpret_cast<const float4 *>(&S.z1[s][k]);
      acc[s] = fmaf(w0, v.x, acc[s]);
      acc[s] = fmaf(w1, v.y, acc[s]);
      acc[s] = fmaf(w2f, v.z, acc[s]);
      acc[s] = fmaf(w3f, v.w, acc[s]);
    }
  }
  const float w3 = W.w3[j];
#pragma unroll
  for (int s = 0; s < kS; ++s) {
    a2[s] = acc[s];
    float v = w3 * fmaxf(acc[s], 0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((j & 31) == 0) S.red[s][j >> 5] = v;
  }
  __syncthreads();
  if (j < kS) S.red[j][0] = S.red[j][0] + S.red[j][1] + S.red[j][2] + S.red[j][3] + W.b3;
  __syncthreads();
}

__global__ void __launch_bounds__(kMlpThreads, 2) mlp_forward_kernel(const uint16_t *x, uint64_t B, const uint16_t *wbf,
                                                                  const float *pf, float *y) {
  extern __shared__ __align__(16) uint8_t smem[];
  MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem);
  const int q = threadIdx.x / kH, j = threadIdx.x % kH;
  load_weights(S.W, wbf, pf);
  __syncthreads();
  // block-uniform trip count: every set of the block passes together
  for (uint64_t c0 = (uint64_t)blockIdx.x * (kSets * kS); c0 < B; c0 += (uint64_t)gridDim.x * (kSets * kS)) {
    const uint64_t s0 = c0 + (uint64_t)q * kS;
    float a2[kS];
    forward_pass(S.W, S.set[q], x, B, s0, a2);
    if (j < kS && s0 + j < B) y[s0 + j] = S.set[q].red[j][0];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kMlpThreads) mlp_grad_kernel(const uint16_t *x, const float *t, uint64_t B,
                                                               const uint16_t *wbf, const float *pf, float *grad,
                                                               float *loss_sum) {
  extern __shared__ __align__(16) uint8_t smem[];
  MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem);
  GradSmem &G = *reinterpret_cast<GradSmem *>(smem + ((sizeof(MlpSmem) + 15) & ~(size_t)15));
  const int q = threadIdx.x / kH, j = threadIdx.x % kH;
  MlpSet &me = S.set[q];
  load_weights(S.W, wbf, pf);
  for (int i = threadIdx.x; i < kH * kG1; i += blockDim.x) G.gW1[i] = 0.0f;
  for (int i = threadIdx.x; i < kH * kG2; i += blockDim.x) G.gW2[i] = 0.0f;
  __syncthreads();
  float gb1 = 0.0f, gb2 = 0.0f, gw3 = 0.0f, gb3 = 0.0f, lsum = 0.0f;
  const float inv_b = 2.0f / (float)B;
  constexpr int kC2 = kH / kSets, kC1 = kIn / kSets;  // this thread's columns of a gradient row
  for (uint64_t c0 = (uint64_t)blockIdx.x * (kSets * kS); c0 < B; c0 += (uint64_t)gridDim.x * (kSets * kS)) {
    const uint64_t s0 = c0 + (uint64_t)q * kS;
    float a2[kS];
    forward_pass(S.W, me, x, B, s0, a2);
    // output layer and second hidden layer: thread j owns unit j of its set's samples
    const float w3 = S.W.w3[j];
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      const bool ok = s0 + s < B;
      const float e = ok ? me.red[s][0] - t[s0 + s] : 0.0f;
      const float dy = e * inv_b;
      if (j == 0) {
        lsum += e * e;
        gb3 += dy;
      }
      const float z2 = fmaxf(a2[s], 0.0f);
      gw3 = fmaf(dy, z2, gw3);
      const float d2 = a2[s] > 0.0f ? dy * w3 : 0.0f;
      me.d2[s][j] = d2;
      gb2 += d2;
    }
    __syncthreads();
    // row j of W2's gradient, columns q*kC2 .. q*kC2+kC2-1, over every set's samples
    for (int kk = 0; kk < kC2; ++kk) {
      const int k = q * kC2 + kk;
      float g = G.gW2[j * kG2 + k];
#pragma unroll
      for (int p = 0; p < kSets; ++p)
#pragma unroll
        for (int s = 0; s < kS; ++s) g = fmaf(S.set[p].d2[s][j], S.set[p].z1[s][k], g);
      G.gW2[j * kG2 + k] = g;
    }
    // first hidden layer: thread k owns unit k of its set's samples (column k of W2)
    const int k = j;
    float d1[kS];
#pragma unroll
    for (int s = 0; s < kS; ++s) d1[s] = 0.0f;
    for (int i = 0; i < kH; ++i) {
      const float w = bf(S.W.W2[i * kT2 + k]);
#pragma unroll
      for (int s = 0; s < kS; ++s) d1[s] = fmaf(w, me.d2[s][i], d1[s]);
    }
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      d1[s] = me.a1[s][k] > 0.0f ? d1[s] : 0.0f;
      gb1 += d1[s];
    }
    __syncthreads();  // every thread has read its a1 before any overwrites it
#pragma unroll
    for (int s = 0; s < kS; ++s) me.a1[s][k] = d1[s];  // a1 now holds d loss / d a1
    __syncthreads();
    // row k of W1's gradient, columns q*kC1 .. q*kC1+kC1-1, over every set's samples
    for (int mm = 0; mm < kC1; ++mm) {
      const int m = q * kC1 + mm;
      float g = G.gW1[k * kG1 + m];
#pragma unroll
      for (int p = 0; p < kSets; ++p)
#pragma unroll
        for (int s = 0; s < kS; ++s) g = fmaf(S.set[p].a1[s][k], S.set[p].x[s][m], g);
      G.gW1[k * kG1 + m] = g;
    }
    __syncthreads();
  }
  // add this block's sums to the global gradient
  for (int i = threadIdx.x; i < kH * kIn; i += blockDim.x) atomicAdd(&grad[kW1 + i], G.gW1[(i / kIn) * kG1 + i % kIn]);
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) atomicAdd(&grad[kW2 + i], G.gW2[(i / kH) * kG2 + i % kH]);
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
// Blocks for a batch: one per kSets x kS samples, at most `per_sm` per SM.
int grid_for(uint64_t B, int per_sm) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t chunks = (B + kSets * kS - 1) / (kSets * kS);
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(chunks, (uint64_t)sms * per_sm));
}
}  // namespace

extern "C" {

esc_status esc_mlp_forward(const uint16_t *x_bf16, uint64_t batch, const uint16_t *w_bf16, const float *params,
                           float *y, void *stream) {
  ESC_RANGE("esc_mlp_forward");
  if (batch == 0) return ESC_OK;
  if (!x_bf16 || !w_bf16 || !params || !y) return fail(ESC_EINVAL, "esc_mlp_forward: NULL argument");
  ESC_MLP_CK(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem()));
  // two blocks per SM: the weights (bfloat16) and the sets' buffers take 110 KB
  mlp_forward_kernel<<<grid_for(batch, 2), kMlpThreads, fwd_smem(), static_cast<cudaStream_t>(stream)>>>(
      x_bf16, batch, w_bf16, params, y);
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
  mlp_grad_kernel<<<grid_for(batch, 1), kMlpThreads, grad_smem(), static_cast<cudaStream_t>(stream)>>>(
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
