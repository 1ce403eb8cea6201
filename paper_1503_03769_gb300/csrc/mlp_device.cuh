// The birth network on the device: a 3-64-64-5 perceptron with exact-erf
// GELU after the two hidden layers, bfloat16 operands and FP32 accumulation.
//
// Parameter vector (kNParams floats, or bfloat16 in a filter's workspace):
// W1[64][3], b1[64], W2[64][64], b2[64], W3[5][64], b3[5], W[j][k] the weight
// from input k into unit j.  Every matrix-product operand (weights, biases,
// the network input and the two hidden activations) is rounded to bfloat16
// (round to nearest even); products and sums are FP32.  Thread-per-input
// form (mlp_forward_one): every layer sum runs over k in increasing order.
// Warp-per-input form (mlp_forward_warp): lane l owns hidden units l and
// l + 32; the hidden-layer sums run over k in increasing order, the output
// sum is the lanes' pairs (l, l + 32) combined by a butterfly over the warp.
#pragma once

#include <cuda_bf16.h>

namespace phd {

constexpr int kNH = 64, kNIn = 3, kNOut = 5;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kNH * kNIn;
constexpr int kOffW2 = kOffB1 + kNH;
constexpr int kOffB2 = kOffW2 + kNH * kNH;
constexpr int kOffW3 = kOffB2 + kNH;
constexpr int kOffB3 = kOffW3 + kNOut * kNH;
constexpr int kNParams = kOffB3 + kNOut;   // 4741

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// GELU(a) = a Phi(a) = a (1 + erf(a / sqrt 2)) / 2
__device__ __forceinline__ float gelu_f(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }
// d GELU / da = Phi(a) + a phi(a)
__device__ __forceinline__ float gelu_grad_f(float a) {
  return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * expf(-0.5f * a * a);
}

// Stage the parameters into shared memory as (bfloat16-valued) floats.
__device__ __forceinline__ void stage_params(float* __restrict__ W, const float* __restrict__ P) {
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) W[i] = bf16r(P[i]);
}
__device__ __forceinline__ void stage_params(float* __restrict__ W, const __nv_bfloat16* __restrict__ P) {
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) W[i] = __bfloat162float(P[i]);
}

// Forward pass of one input with the staged weights W; y gets the 5 outputs.
__device__ __forceinline__ void mlp_forward_one(const float* __restrict__ W, float u0, float u1, float u2,
                                                float* y) {
  u0 = bf16r(u0);
  u1 = bf16r(u1);
  u2 = bf16r(u2);
  float h1[kNH];
#pragma unroll
  for (int j = 0; j < kNH; ++j) {
    float a = W[kOffB1 + j];
    a = fmaf(W[kOffW1 + j * kNIn + 0], u0, a);
    a = fmaf(W[kOffW1 + j * kNIn + 1], u1, a);
    a = fmaf(W[kOffW1 + j * kNIn + 2], u2, a);
    h1[j] = bf16r(gelu_f(a));
  }
#pragma unroll
  for (int o = 0; o < kNOut; ++o) y[o] = W[kOffB3 + o];
  for (int j = 0; j < kNH; ++j) {
    float a = W[kOffB2 + j];
#pragma unroll
    for (int k = 0; k < kNH; ++k) a = fmaf(W[kOffW2 + j * kNH + k], h1[k], a);
    const float h2 = bf16r(gelu_f(a));
#pragma unroll
    for (int o = 0; o < kNOut; ++o) y[o] = fmaf(W[kOffW3 + o * kNH + j], h2, y[o]);
  }
}

// Shared-memory image for the warp form: W2 rows padded to kW2Pad floats so
// that the 32 lanes reading 32 different rows at the same column hit 32
// different banks.
constexpr int kW2Pad = kNH + 1;
constexpr int kWarpImage = kNParams - kNH * kNH + kNH * kW2Pad;   // floats
__device__ __forceinline__ int warp_image_index(int i) {
  if (i < kOffW2 || i >= kOffB2) return i < kOffW2 ? i : i - kNH * kNH + kNH * kW2Pad;
  const int r = (i - kOffW2) / kNH, c = (i - kOffW2) - r * kNH;
  return kOffW2 + r * kW2Pad + c;
}
__device__ __forceinline__ void stage_params_warp(float* __restrict__ W, const __nv_bfloat16* __restrict__ P) {
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) W[warp_image_index(i)] = __bfloat162float(P[i]);
}

// Forward pass of one input by a whole warp (all 32 lanes, converged), with
// the padded shared image W; every lane returns the 5 outputs.
__device__ __forceinline__ void mlp_forward_warp(const float* __restrict__ W, float u0, float u1, float u2,
                                                 float* y) {
  const int l = threadIdx.x & 31;
  const float* W2 = W + kOffW2;
  const float* B2 = W + kOffW2 + kNH * kW2Pad;
  const float* W3 = B2 + kNH;
  const float* B3 = W3 + kNOut * kNH;
  u0 = bf16r(u0);
  u1 = bf16r(u1);
  u2 = bf16r(u2);
  float ha, hb;
  {
    float a = W[kOffB1 + l];
    a = fmaf(W[kOffW1 + l * kNIn + 0], u0, a);
    a = fmaf(W[kOffW1 + l * kNIn + 1], u1, a);
    a = fmaf(W[kOffW1 + l * kNIn + 2], u2, a);
    ha = bf16r(gelu_f(a));
    float b = W[kOffB1 + l + 32];
    b = fmaf(W[kOffW1 + (l + 32) * kNIn + 0], u0, b);
    b = fmaf(W[kOffW1 + (l + 32) * kNIn + 1], u1, b);
    b = fmaf(W[kOffW1 + (l + 32) * kNIn + 2], u2, b);
    hb = bf16r(gelu_f(b));
  }
  float a2 = B2[l], b2 = B2[l + 32];
#pragma unroll 8
  for (int k = 0; k < 32; ++k) {
    const float hk = __shfl_sync(0xffffffffu, ha, k);
    a2 = fmaf(W2[l * kW2Pad + k], hk, a2);
    b2 = fmaf(W2[(l + 32) * kW2Pad + k], hk, b2);
  }
#pragma unroll 8
  for (int k = 0; k < 32; ++k) {
    const float hk = __shfl_sync(0xffffffffu, hb, k);
    a2 = fmaf(W2[l * kW2Pad + 32 + k], hk, a2);
    b2 = fmaf(W2[(l + 32) * kW2Pad + 32 + k], hk, b2);
  }
  const float ga = bf16r(gelu_f(a2)), gb = bf16r(gelu_f(b2));
#pragma unroll
  for (int o = 0; o < kNOut; ++o) {
    float s = fmaf(W3[o * kNH + l + 32], gb, W3[o * kNH + l] * ga);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    y[o] = B3[o] + s;
  }
}

}  // namespace phd
