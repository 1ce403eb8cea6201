// Training and inference kernels of the birth network (the learned proposal
// p_k(.|Z_k) of Eq. 6): forward, loss gradient and Adam, behind the
// stateless phd_mlp_* entry points.
//
// k_mlp_forward: one thread per input, the parameters staged in shared
//   memory (bfloat16 values), the first hidden layer in registers.
// k_mlp_grad: 64 inputs per CTA, one thread each for the forward and the
//   backward pass (pre-activations and bfloat16 activations kept in shared
//   memory rows), then the CTA's weight-gradient sums over its 64 inputs as
//   small products in shared memory (thread t owns hidden unit t), written
//   as one FP32 partial vector per CTA.
// k_mlp_reduce: the partials summed per parameter in CTA order (fixed order:
//   deterministic), divided by n.
// k_mlp_adam: one thread per parameter (Kingma & Ba, Algorithm 1; the bias
//   corrections are passed in).
//
// Loss per input with target (t, vx, vy), v~ = v / s_b, outputs
// y = (m_x, m_y, l_x, l_y, logit):
//   L = softplus(logit) - t logit + t sum_d [ l_d + (v~_d - m_d)^2 e^{-2 l_d} / 2 ]
// (cross-entropy of "the filter extracted an estimate for this measurement"
// and the Gaussian negative log-likelihood of the extracted velocity).
// The backward pass uses the bfloat16 weights and activations of the forward
// pass with FP32 deltas.
#include <cmath>

#include <cuda_bf16.h>

#include "mlp_device.cuh"
#include "phd.h"
#include "phd_internal.cuh"

namespace phd {

constexpr int kGradRows = 64;              // inputs per CTA of k_mlp_grad
constexpr int kRowPad = kNH + 1;           // padded shared rows (bank-conflict free)

__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X,
                                                     int n, float* __restrict__ Y) {
  __shared__ float W[kNParams];
  stage_params(W, P);
  __syncthreads();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    float y[kNOut];
    mlp_forward_one(W, X[3 * s], X[3 * s + 1], X[3 * s + 2], y);
#pragma unroll
    for (int o = 0; o < kNOut; ++o) Y[5 * s + o] = y[o];
  }
}

__device__ __forceinline__ float softplus_f(float a) { return fmaxf(a, 0.0f) + log1pf(expf(-fabsf(a))); }

__global__ void __launch_bounds__(kGradRows) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                       const float* __restrict__ T, int n, float inv_vs,
                                                       float* __restrict__ part) {
  extern __shared__ __align__(16) float sm[];
  float* W = sm;                                  // [kNParams]
  float* A1 = W + kNParams;                       // [64][65] pre-activations, then deltas of layer 1
  float* A2 = A1 + kGradRows * kRowPad;           // [64][65] same for layer 2
  float* H1 = A2 + kGradRows * kRowPad;           // [64][65] bfloat16 activations of layer 1
  float* H2 = H1 + kGradRows * kRowPad;           // [64][65] same for layer 2
  float* U = H2 + kGradRows * kRowPad;            // [64][3] bfloat16 inputs
  float* DY = U + kGradRows * kNIn;               // [64][5] output deltas
  float* LS = DY + kGradRows * kNOut;             // [64] per-input loss
  stage_params(W, P);
  __syncthreads();
  const int s = threadIdx.x;
  const int gs = blockIdx.x * kGradRows + s;
  const bool live = gs < n;
  float* a1 = A1 + s * kRowPad;
  float* a2 = A2 + s * kRowPad;
  float* h1 = H1 + s * kRowPad;
  float* h2 = H2 + s * kRowPad;
  // forward
  const float u0 = bf16r(live ? X[3 * gs] : 0.0f), u1 = bf16r(live ? X[3 * gs + 1] : 0.0f),
              u2 = bf16r(live ? X[3 * gs + 2] : 0.0f);
  U[3 * s] = u0;
  U[3 * s + 1] = u1;
  U[3 * s + 2] = u2;
  for (int j = 0; j < kNH; ++j) {
    float a = W[kOffB1 + j];
    a = fmaf(W[kOffW1 + j * kNIn + 0], u0, a);
    a = fmaf(W[kOffW1 + j * kNIn + 1], u1, a);
    a = fmaf(W[kOffW1 + j * kNIn + 2], u2, a);
    a1[j] = a;
    h1[j] = bf16r(gelu_f(a));
  }
  float y[kNOut];
#pragma unroll
  for (int o = 0; o < kNOut; ++o) y[o] = W[kOffB3 + o];
  for (int j = 0; j < kNH; ++j) {
    float a = W[kOffB2 + j];
#pragma unroll 16
    for (int k = 0; k < kNH; ++k) a = fmaf(W[kOffW2 + j * kNH + k], h1[k], a);
    a2[j] = a;
    const float hv = bf16r(gelu_f(a));
    h2[j] = hv;
#pragma unroll
    for (int o = 0; o < kNOut; ++o) y[o] = fmaf(W[kOffW3 + o * kNH + j], hv, y[o]);
  }
  // loss and output deltas (zero for the padding rows of the last CTA)
  float dy[kNOut] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  float L = 0.0f;
  if (live) {
    const float t = T[3 * gs];
    L = softplus_f(y[4]) - t * y[4];
    dy[4] = 1.0f / (1.0f + expf(-y[4])) - t;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const float r = T[3 * gs + 1 + d] * inv_vs - y[d];
      const float e = expf(-2.0f * y[2 + d]);
      L += t * (y[2 + d] + 0.5f * r * r * e);
      dy[d] = -t * r * e;
      dy[2 + d] = t * (1.0f - r * r * e);
    }
  }
  LS[s] = L;
#pragma unroll
  for (int o = 0; o < kNOut; ++o) DY[kNOut * s + o] = dy[o];
  // backward: deltas of layer 2, then layer 1 (overwriting the pre-activations)
  for (int j = 0; j < kNH; ++j) {
    float g = 0.0f;
#pragma unroll
    for (int o = 0; o < kNOut; ++o) g = fmaf(W[kOffW3 + o * kNH + j], dy[o], g);
    a2[j] = g * gelu_grad_f(a2[j]);
  }
  for (int k = 0; k < kNH; ++k) {
    float g = 0.0f;
#pragma unroll 16
    for (int j = 0; j < kNH; ++j) g = fmaf(W[kOffW2 + j * kNH + k], a2[j], g);
    a1[k] = g * gelu_grad_f(a1[k]);
  }
  __syncthreads();
  // weight gradients summed over the CTA's inputs; thread t owns unit t
  const int t = threadIdx.x;
  float* out = part + (size_t)blockIdx.x * (kNParams + 1);
  {
    float acc[kNH];
#pragma unroll
    for (int k = 0; k < kNH; ++k) acc[k] = 0.0f;
    float db = 0.0f;
    for (int r = 0; r < kGradRows; ++r) {
      const float d = A2[r * kRowPad + t];
      db += d;
#pragma unroll
      for (int k = 0; k < kNH; ++k) acc[k] = fmaf(d, H1[r * kRowPad + k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < kNH; ++k) out[kOffW2 + t * kNH + k] = acc[k];
    out[kOffB2 + t] = db;
  }
  {
    float w0 = 0.0f, w1 = 0.0f, w2 = 0.0f, db = 0.0f;
    for (int r = 0; r < kGradRows; ++r) {
      const float d = A1[r * kRowPad + t];
      db += d;
      w0 = fmaf(d, U[3 * r], w0);
      w1 = fmaf(d, U[3 * r + 1], w1);
      w2 = fmaf(d, U[3 * r + 2], w2);
    }
    out[kOffW1 + t * kNIn + 0] = w0;
    out[kOffW1 + t * kNIn + 1] = w1;
    out[kOffW1 + t * kNIn + 2] = w2;
    out[kOffB1 + t] = db;
  }
  {
    float acc[kNOut] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    for (int r = 0; r < kGradRows; ++r) {
      const float h = H2[r * kRowPad + t];
#pragma unroll
      for (int o = 0; o < kNOut; ++o) acc[o] = fmaf(DY[kNOut * r + o], h, acc[o]);
    }
#pragma unroll
    for (int o = 0; o < kNOut; ++o) out[kOffW3 + o * kNH + t] = acc[o];
  }
  if (t < kNOut) {
    float db = 0.0f;
    for (int r = 0; r < kGradRows; ++r) db += DY[kNOut * r + t];
    out[kOffB3 + t] = db;
  }
  if (t == kNOut) {
    float l = 0.0f;
    for (int r = 0; r < kGradRows; ++r) l += LS[r];
    out[kNParams] = l;
  }
}

size_t mlp_grad_smem() {
  return sizeof(float) * ((size_t)kNParams + 4 * kGradRows * kRowPad + kGradRows * (kNIn + kNOut + 1));
}

__global__ void k_mlp_reduce(const float* __restrict__ part, int blocks, float inv_n, float* __restrict__ G,
                             float* __restrict__ loss) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= kNParams; i += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < blocks; ++b) s += part[(size_t)b * (kNParams + 1) + i];
    if (i < kNParams) G[i] = s * inv_n;
    else if (loss) *loss = s * inv_n;
  }
}

__global__ void k_mlp_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m1,
                           float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float a = b1 * m1[i] + (1.0f - b1) * g;
    const float v = b2 * m2[i] + (1.0f - b2) * g * g;
    m1[i] = a;
    m2[i] = v;
    P[i] -= lr * (a * c1) / (sqrtf(v * c2) + eps);
  }
}

}  // namespace phd

using namespace phd;

extern "C" {

int32_t phd_mlp_nparams(void) { return kNParams; }

phd_status phd_mlp_forward(const float* d_params, const float* d_X, int32_t n, float* d_Y, void* stream) {
  if (n < 0 || !d_params || (n > 0 && (!d_X || !d_Y))) return PHD_ERR_INVALID_ARG;
  if (n == 0) return PHD_OK;
  int blocks = (n + 127) / 128;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_mlp_forward<<<blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(d_params, d_X, n, d_Y);
  return cudaGetLastError() == cudaSuccess ? PHD_OK : PHD_ERR_CUDA;
}

phd_status phd_mlp_grad_scratch_size(int32_t n, size_t* bytes) {
  if (n < 0 || !bytes) return PHD_ERR_INVALID_ARG;
  const size_t blocks = ((size_t)n + kGradRows - 1) / kGradRows;
  *bytes = blocks * (kNParams + 1) * sizeof(float);
  return PHD_OK;
}

phd_status phd_mlp_grad(const float* d_params, const float* d_X, const float* d_T, int32_t n, float vel_scale,
                        float* d_grad, float* d_loss, void* d_scratch, size_t scratch_bytes, void* stream) {
  if (n < 1 || !d_params || !d_X || !d_T || !d_grad || !d_scratch || !(vel_scale > 0.0f))
    return PHD_ERR_INVALID_ARG;
  size_t need = 0;
  phd_mlp_grad_scratch_size(n, &need);
  if (scratch_bytes < need) return PHD_ERR_CAPACITY;
  // per device (host-side call, also legal while the stream is captured)
  if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_grad_smem()) !=
      cudaSuccess)
    return PHD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = (n + kGradRows - 1) / kGradRows;
  float* part = static_cast<float*>(d_scratch);
  k_mlp_grad<<<blocks, kGradRows, mlp_grad_smem(), s>>>(d_params, d_X, d_T, n, 1.0f / vel_scale, part);
  k_mlp_reduce<<<(kNParams + 256) / 256, 256, 0, s>>>(part, blocks, 1.0f / (float)n, d_grad, d_loss);
  return cudaGetLastError() == cudaSuccess ? PHD_OK : PHD_ERR_CUDA;
}

phd_status phd_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int32_t t, float lr,
                        float beta1, float beta2, float eps, void* stream) {
  if (!d_params || !d_grad || !d_m || !d_v || t < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return PHD_ERR_INVALID_ARG;
  const double c1 = 1.0 / (1.0 - std::pow((double)beta1, (double)t));
  const double c2 = 1.0 / (1.0 - std::pow((double)beta2, (double)t));
  k_mlp_adam<<<(kNParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      d_params, d_grad, d_m, d_v, lr, beta1, beta2, eps, (float)c1, (float)c2);
  return cudaGetLastError() == cudaSuccess ? PHD_OK : PHD_ERR_CUDA;
}

}  // extern "C"
