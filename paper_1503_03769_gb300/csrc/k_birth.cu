// Measurement-driven birth: Eq. 6 with the birth proposal p_k(.|Z_k) a
// mixture over the current measurements whose velocity Gaussian and mixture
// logit come from the birth network, and the importance weights that keep
// the PHD unbiased under it.  FP32 handles of one filter (all PEs share Z).
//
// k_birth_head: one warp per measurement: the network input (position in
//   the plane scaled to the birth region, log1p of the number of other
//   measurements inside +-3 sigma per coordinate, bearing wrapped), then the
//   network (bfloat16 operands, FP32 sums) -> head (m_x, m_y, l_x, l_y, logit).
// Mixture table (the last CTA of k_birth_head, or k_birth_table when the
//   caller supplies the head): pi = softmax(logit), its inclusive CDF, and per
//   component the constants of the ratio of its density to the plain birth
//   density: s_v = s_b exp(clamp(l, log 0.05, log 5)), mu = s_b m,
//   L_p = log2 pi_p + log2(area s_b^2 / (2 pi s_z0 s_z1)) - log2(s_vx s_vy).
// k_birth_draw: eight lanes per birth slot (after k_predict has written the
//   plain births there): u_c < alpha keeps the plain draw (same random
//   numbers as the plain birth), otherwise the component is the smallest p
//   with CDF_p > (u_c - alpha) / (1 - alpha), the position is the
//   measurement plus its noise (linear sensor), or range |z_r + s_r n1| and
//   bearing z_th + s_th n2 around the sensor (range-bearing sensor), the
//   velocity mu_p + s_v (n1, n2).  Weight (Eq. 6, defensive mixture):
//     w = (nu_b / J_j) / (alpha + (1 - alpha) R(x)),
//     R(x) = sum_p pi_p q_p(x) / (U(pos) N(v; 0, s_b^2 I)),
//   0 outside the region; R is summed over all M components in exp2 form
//   (range-bearing: folded range density and the 1/r Jacobian).
//
// Random numbers: the plain rows (n1, n2, u1, u2) of k_predict's slot, and
// (u_c, nz1, nz2) from the caller's extra rows [K][jmax] after the K x pe_cap
// plain rows, or from Philox-4x32-10 with the birth tag.
#include <cstdint>
#include <cuda_bf16.h>

#include "mlp_device.cuh"
#include "phd.h"
#include "phd_internal.cuh"

namespace phd {

__device__ __forceinline__ float wrap_pm_pi(float a) {
  const float two_pi = 6.283185307179586f;
  return a - two_pi * rintf(a * (1.0f / two_pi));
}

// Network input of measurement p: position in the plane scaled to the
// region, log1p of the number of other measurements in the +-3 sigma window.
// `lanes` consecutive lanes (a power of two, converged) split the count.
__device__ __forceinline__ float3 birth_feature(const Model& m, const V2<float>* __restrict__ Z, int M, int p,
                                                int lane = 0, int lanes = 1) {
  const V2<float> z = Z[p];
  float px = z.a, py = z.b;
  if (m.meas_model) {
    float sn, cs;
    sincosf(z.b, &sn, &cs);
    px = m.f_sx + z.a * cs;
    py = m.f_sy + z.a * sn;
  }
  int count = 0;
  for (int q = lane; q < M; q += lanes) {
    const V2<float> o = Z[q];
    const float d0 = o.a - z.a;
    float d1 = o.b - z.b;
    if (m.meas_model) d1 = wrap_pm_pi(d1);
    count += (q != p && fabsf(d0) <= m.f_win0 && fabsf(d1) <= m.f_win1) ? 1 : 0;
  }
  if (lanes == 32) count = __reduce_add_sync(0xffffffffu, count);
  return make_float3((px - m.f_cx) * m.f_ihx, (py - m.f_cy) * m.f_ihy, log1pf((float)count));
}

// One warp per measurement: features (lanes split the neighbour count) and
// the network (lanes own hidden units).
__device__ void birth_table_block(const Dev& d, const Model& m);

__global__ void __launch_bounds__(256) k_birth_head(Dev d, Model m) {
  pdl_enter();
  __shared__ float W[kWarpImage];
  stage_params_warp(W, static_cast<const __nv_bfloat16*>(d.mlp_w));
  __syncthreads();
  const int M = *d.M;
  const V2<float>* __restrict__ Z = static_cast<const V2<float>*>(d.Z);
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < M; p += nw) {
    const float3 u = birth_feature(m, Z, M, p, lane, 32);
    float y[kNOut];
    mlp_forward_warp(W, u.x, u.y, u.z, y);
#pragma unroll
    for (int o = 0; o < kNOut; ++o)
      if (lane == o) d.bhead[5 * p + o] = y[o];
  }
  // the last CTA to finish builds the mixture table from every CTA's head
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(d.bdone, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  birth_table_block(d, m);
  if (threadIdx.x == 0) *d.bdone = 0u;
}

__global__ void k_birth_features(Model m, const V2<float>* __restrict__ Z, int M, float* __restrict__ X) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < M; p += gridDim.x * blockDim.x) {
    const float3 u = birth_feature(m, Z, M, p);
    X[3 * p] = u.x;
    X[3 * p + 1] = u.y;
    X[3 * p + 2] = u.z;
  }
}

// The mixture table, built by one CTA of kTableThreads threads: pi =
// softmax(logit) (max-shifted), its inclusive CDF, and per component the
// constants of k_birth_draw's ratio terms.
constexpr int kTableThreads = 256;

__device__ void birth_table_block(const Dev& d, const Model& m) {
  __shared__ float sh[kTableThreads / 32];
  __shared__ float wsum[kTableThreads / 32];
  const int M = *d.M;
  if (M == 0) return;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  // heads written by other CTAs of this launch: read through L2 (__ldcg)
  float mx = -INFINITY;
  for (int p = t; p < M; p += kTableThreads) mx = fmaxf(mx, __ldcg(d.bhead + 5 * p + 4));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) sh[wid] = mx;
  __syncthreads();
  mx = sh[0];
  for (int k = 1; k < kTableThreads / 32; ++k) mx = fmaxf(mx, sh[k]);
  // unnormalised inclusive CDF in rounds of kTableThreads consecutive measurements
  float carry = 0.0f;
  for (int r0 = 0; r0 < M; r0 += kTableThreads) {
    const int p = r0 + t;
    const float e = p < M ? expf(__ldcg(d.bhead + 5 * p + 4) - mx) : 0.0f;
    float incl = e;
    for (int o = 1; o < 32; o <<= 1) {
      const float u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    __syncthreads();   // wsum of the previous round has been read
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    float base = carry, rtot = 0.0f;
    for (int k = 0; k < kTableThreads / 32; ++k) {
      if (k < wid) base += wsum[k];
      rtot += wsum[k];
    }
    if (p < M) d.bcdf[p] = base + incl;
    carry += rtot;
  }
  const float inv = 1.0f / carry;
  const float lo = -4.3219281f, hi = 2.3219281f;   // log2(0.05), log2(5)
  const float sb = m.f_bv;
  for (int p = t; p < M; p += kTableThreads) {
    float hd[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) hd[o] = __ldcg(d.bhead + 5 * p + o);
    d.bcdf[p] *= inv;
    const float pi = expf(hd[4] - mx) * inv;
    const float l2x = fminf(fmaxf(hd[2] * 1.4426950408889634f, lo), hi);   // log2 of s_v / s_b
    const float l2y = fminf(fmaxf(hd[3] * 1.4426950408889634f, lo), hi);
    const V2<float> z = static_cast<const V2<float>*>(d.Z)[p];
    float4* out = reinterpret_cast<float4*>(d.bcomp + 8 * p);
    out[0] = make_float4(z.a, z.b, sb * hd[0], sb * hd[1]);
    out[1] = make_float4(exp2f(-l2x) / sb, exp2f(-l2y) / sb,                   // 1 / s_v
                         log2f(pi) + m.f_blog - l2x - l2y - 2.0f * log2f(sb), 0.0f);
  }
}

// Table only (the network head was supplied by the caller).
__global__ void __launch_bounds__(kTableThreads) k_birth_table(Dev d, Model m) {
  pdl_enter(); birth_table_block(d, m); }

static size_t birth_draw_smem(const Model& m) { return (size_t)m.m_max * (2 * sizeof(float4) + sizeof(float)); }

// kDrawLanes consecutive lanes per birth slot: each draws the same random
// numbers and particle (the draw is cheap), then they split the M-term sum
// of R (p = lane, lane + kDrawLanes, ...) and combine it by shuffles.
constexpr int kDrawLanes = 8;

__global__ void __launch_bounds__(256) k_birth_draw(Dev d, Model m, const float* __restrict__ noise) {
  pdl_enter();
  const int K = m.K;
  const int M = *d.M;
  const float alpha = M > 0 ? m.f_alpha : 1.0f;
  const unsigned long long step = *d.step;
  const Cst<float> cst = consts<float>(m);
  const float c = 0.72134752044448170f;             // log2(e) / 2
  const float b0 = c / (float)(m.sz0 * m.sz0), b1 = c / (float)(m.sz1 * m.sz1);
  const float bv = c / (m.f_bv * m.f_bv);
  St4<float>* __restrict__ xp = static_cast<St4<float>*>(d.x_alt);
  float* __restrict__ wp = static_cast<float*>(d.w_alt);
  // the mixture table in shared memory: the component search and the M-term
  // sums read it for every birth
  extern __shared__ __align__(16) float4 smem_tab[];
  float4* comp = smem_tab;                                   // [M][2]
  float* cdf = reinterpret_cast<float*>(smem_tab + 2 * m.m_max);   // [M]
  for (int i = threadIdx.x; i < 2 * M; i += blockDim.x) comp[i] = reinterpret_cast<const float4*>(d.bcomp)[i];
  for (int i = threadIdx.x; i < M; i += blockDim.x) cdf[i] = d.bcdf[i];
  __syncthreads();
  const int sub = threadIdx.x & (kDrawLanes - 1);
  const unsigned gmask = ((1u << kDrawLanes) - 1u) << (threadIdx.x & 31 & ~(kDrawLanes - 1));
  const long total = (long)K * m.jmax;
  const long stride = ((long)gridDim.x * blockDim.x) / kDrawLanes;
  for (long it = ((long)blockIdx.x * blockDim.x + threadIdx.x) / kDrawLanes; it < total; it += stride) {
    const int j = (int)(it / m.jmax), b = (int)(it - (long)j * m.jmax);
    if (b >= d.Jb[j]) continue;
    const long g = (long)j * m.pe_cap + d.n_cur[j] + b;
    float n1, n2, u1, u2;
    draw_noise<float>(m, noise, g, step, n1, n2, u1, u2);
    float uc, nz1, nz2;
    if (noise) {
      const float4 ex = reinterpret_cast<const float4*>(noise)[(long)K * m.pe_cap + it];
      uc = ex.x;
      nz1 = ex.y;
      nz2 = ex.z;
    } else {
      const U4 r = philox4x32_10(U4{(uint32_t)g, (uint32_t)step, kTagBirth, (uint32_t)(step >> 32)},
                                 (uint32_t)m.seed, (uint32_t)(m.seed >> 32));
      uc = unit_open<float>(r.a);
      const float rad = sqrtf(-2.0f * logf(unit_open<float>(r.b)));
      float sn, cs;
      sincospif(2.0f * unit_open<float>(r.c), &sn, &cs);
      nz1 = rad * cs;
      nz2 = rad * sn;
    }
    St4<float> o;
    if (uc < alpha) {
      o.x = cst.rx0 + u1 * cst.rw;
      o.vx = cst.bv * n1;
      o.y = cst.ry0 + u2 * cst.rh;
      o.vy = cst.bv * n2;
    } else {
      const float uu = (uc - alpha) / (1.0f - alpha);
      int lo = 0, hi = M - 1;                        // smallest p with CDF_p > uu (else M - 1)
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cdf[mid] > uu) hi = mid; else lo = mid + 1;
      }
      const float4 c0 = comp[2 * lo], c1 = comp[2 * lo + 1];
      if (m.meas_model) {
        const float r = fabsf(c0.x + (float)m.sz0 * nz1);
        float sn, cs;
        sincosf(c0.y + (float)m.sz1 * nz2, &sn, &cs);
        o.x = cst.sx + r * cs;
        o.y = cst.sy + r * sn;
      } else {
        o.x = c0.x + (float)m.sz0 * nz1;
        o.y = c0.y + (float)m.sz1 * nz2;
      }
      o.vx = c0.z + n1 / c1.x;
      o.vy = c0.w + n2 / c1.y;
    }
    const bool inside = o.x >= cst.rx0 && o.x <= cst.rx0 + cst.rw && o.y >= cst.ry0 && o.y <= cst.ry0 + cst.rh;
    float w = 0.0f;
    const float bw = d.bwf[j];
    if (inside && alpha >= 1.0f) {
      w = bw;
    } else if (inside) {
      const float vplain = bv * (o.vx * o.vx + o.vy * o.vy);
      float R = 0.0f;
      if (m.meas_model) {
        const float px = o.x - cst.sx, py = o.y - cst.sy;
        const float r = sqrtf(px * px + py * py);
        const float th = atan2f(py, px);
        const float ir = 1.0f / r;
        for (int p = sub; p < M; p += kDrawLanes) {
          const float4 c0 = comp[2 * p], c1 = comp[2 * p + 1];
          const float e1 = r - c0.x, e2 = r + c0.x, dt = wrap_pm_pi(th - c0.y);
          const float ex = (o.vx - c0.z) * c1.x, ey = (o.vy - c0.w) * c1.y;
          const float base = c1.z + vplain - b1 * dt * dt - c * (ex * ex + ey * ey);
          R += (exp2f(base - b0 * e1 * e1) + exp2f(base - b0 * e2 * e2)) * ir;
        }
      } else {
        for (int p = sub; p < M; p += kDrawLanes) {
          const float4 c0 = comp[2 * p], c1 = comp[2 * p + 1];
          const float dx = o.x - c0.x, dy = o.y - c0.y;
          const float ex = (o.vx - c0.z) * c1.x, ey = (o.vy - c0.w) * c1.y;
          R += exp2f(c1.z + vplain - b0 * dx * dx - b1 * dy * dy - c * (ex * ex + ey * ey));
        }
      }
#pragma unroll
      for (int off = kDrawLanes / 2; off > 0; off >>= 1) R += __shfl_xor_sync(gmask, R, off);
      w = bw / (alpha + (1.0f - alpha) * R);
    }
    if (sub == 0) {
      xp[g] = o;
      wp[g] = w;
    }
  }
}

__global__ void k_params_bf16(__nv_bfloat16* __restrict__ dst, const float* __restrict__ src) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

cudaError_t launch_birth_head(const Dev& d, const Model& m, cudaStream_t s) {
  int blocks = (m.m_max + 7) / 8;   // a warp per measurement slot
  if (blocks > 152 * 2) blocks = 152 * 2;
  launch_k(k_birth_head, dim3(blocks), dim3(256), 0, s, d, m);
  return cudaGetLastError();
}

cudaError_t launch_birth_table(const Dev& d, const Model& m, cudaStream_t s) {
  launch_k(k_birth_table, dim3(1), dim3(kTableThreads), 0, s, d, m);
  return cudaGetLastError();
}

cudaError_t launch_birth_draw(const Dev& d, const Model& m, const float* noise, cudaStream_t s) {
  const long items = (long)m.K * m.jmax * kDrawLanes;
  int blocks = (int)((items + 255) / 256);
  if (blocks > 152 * 4) blocks = 152 * 4;
  if (blocks < 1) blocks = 1;
  launch_k(k_birth_draw, dim3(blocks), dim3(256), birth_draw_smem(m), s, d, m, noise);
  return cudaGetLastError();
}

cudaError_t prepare_birth(const Model& m) {
  return cudaFuncSetAttribute(k_birth_draw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)birth_draw_smem(m));
}

cudaError_t launch_params_bf16(void* dst, const float* src, cudaStream_t s) {
  k_params_bf16<<<(kNParams + 255) / 256, 256, 0, s>>>(static_cast<__nv_bfloat16*>(dst), src);
  return cudaGetLastError();
}

}  // namespace phd

extern "C" phd_status phd_birth_features(const phd_config* cfg, const float* d_Z, int32_t M, float* d_X,
                                         void* stream) {
  if (!cfg || M < 0 || (M > 0 && (!d_Z || !d_X))) return PHD_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_Z) % 8 != 0) return PHD_ERR_INVALID_ARG;   // rows read as float pairs
  if (phd::config_problem(*cfg)) return PHD_ERR_INVALID_ARG;
  if (M == 0) return PHD_OK;
  const phd::Model m = phd::model_from_config(*cfg);
  int blocks = (M + 127) / 128;
  if (blocks > 152 * 8) blocks = 152 * 8;
  phd::k_birth_features<<<blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(
      m, reinterpret_cast<const phd::V2<float>*>(d_Z), M, d_X);
  return cudaGetLastError() == cudaSuccess ? PHD_OK : PHD_ERR_CUDA;
}
