// Measured issue rate of the MUFU ex2 instruction: the denominator of the
// pair passes' roofline (every particle x measurement pair of Eq. 7 and Eq. 8
// costs one ex2 of its exponent).  The kernel runs kChains independent
// dependency chains v <- 2^-v per thread (the pair kernels' own exp2_neg, one
// MUFU instruction each) over a full-occupancy grid, so the MUFU pipes, not
// latency, bound it.
#include <cstdint>

#include "phd.h"
#include "phd_internal.cuh"

namespace phd {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;

// written only if a chain leaves (0, 1), which 2^-v started in (0, 1) cannot:
// keeps the chains live without a caller buffer
static __device__ float g_ex2_sink[1];

__global__ void __launch_bounds__(kPeakThreads) k_ex2_rate(int iters) {
  float v[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) v[c] = 0.125f * (float)(c + 1) + 1e-6f * (float)threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) v[c] = exp2_neg(v[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += v[c];
  if (!(s > 0.f && s < (float)kPeakChains)) g_ex2_sink[0] = s;
}

}  // namespace phd

extern "C" phd_status phd_measure_ex2_rate(int32_t reps, double* h_per_s, double* h_best_ms, void* stream) {
  if (reps < 1 || reps > 10000 || !h_per_s) return PHD_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PHD_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PHD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = sms * (2048 / phd::kPeakThreads);
  const int iters = 4096;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PHD_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PHD_ERR_CUDA;
  }
  float best = 0.f;
  cudaError_t err = cudaSuccess;
  phd::k_ex2_rate<<<blocks, phd::kPeakThreads, 0, s>>>(iters);   // warm-up
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    cudaEventRecord(e0, s);
    phd::k_ex2_rate<<<blocks, phd::kPeakThreads, 0, s>>>(iters);
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && (r == 0 || ms < best)) best = ms;
  }
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || best <= 0.f) return PHD_ERR_CUDA;
  const double ex2 = (double)blocks * phd::kPeakThreads * phd::kPeakChains * (double)iters;
  *h_per_s = ex2 / (best * 1e-3);
  if (h_best_ms) *h_best_ms = best;
  return PHD_OK;
}
