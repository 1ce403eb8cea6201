// Prediction (Eq. 5-6) and measurement staging.
//
// k_predict: one thread per particle slot of every PE.  Survivor slots
// (i < n_cur[j]) move by the constant-velocity model of Sec. 4,
//   x' = x + T vx + T^2/2 a_x,  vx' = vx + T a_x  (same for y),
// with a = sigma_a (n1, n2), and take weight p_S w (proposal = transition, so
// Eq. 5's phi/q is the survival probability).  Birth slots
// (n_cur[j] <= i < n_cur[j] + J_j) draw position U(region) and velocity
// N(0, s_b^2 I) and take weight nu_b / J_j (Eq. 6 with gamma = nu_b p_k);
// with a birth network loaded the birth slots are left to k_birth_draw.
// Survivors keep their slot index, births follow them; the predicted set is
// written to the alternate buffers (x_alt, w_alt), the current set is read.
// Random numbers come from the caller (noise rows n1, n2, u1, u2) or from
// Philox-4x32-10 keyed by the seed with counter (slot, step, tag).
//
// Memory traffic per particle: 16 B (float) state read + 16 B written, 4 B
// weight read + written, plus 16 B of injected noise when given.
#include "phd_internal.cuh"

namespace phd {


template <class R>
__global__ void __launch_bounds__(256) k_predict(Dev d, Model m, const R* __restrict__ noise) {
  pdl_enter();
  __shared__ int pref[kMaxPE + 1];
  const int K = m.K;
  // work items: tiles of 256 over each slice's survivors + births
  // with a birth network loaded k_birth_draw fills the birth slots
  const bool births = !m.learned;
  slice_prefix(K, pref, [&](int j) { return (d.n_cur[j] + (births ? d.Jb[j] : 0) + 255) / 256; });
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < K; j += blockDim.x) d.n_pred[j] = d.n_cur[j] + d.Jb[j];
  const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x);
  const R* __restrict__ w = static_cast<const R*>(d.w);
  St4<R>* __restrict__ xp = static_cast<St4<R>*>(d.x_alt);
  R* __restrict__ wp = static_cast<R*>(d.w_alt);
  const unsigned long long step = *d.step;
  const Cst<R> c = consts<R>(m);
  for (int item = blockIdx.x; item < pref[K]; item += gridDim.x) {
    const int j = item_pe(pref, K, item);
    const int i = (item - pref[j]) * 256 + threadIdx.x;
    const int L = d.n_cur[j];
    if (i >= L + (births ? d.Jb[j] : 0)) continue;
    const long g = (long)j * m.pe_cap + i;
    R n1, n2, u1, u2;
    draw_noise<R>(m, noise, g, step, n1, n2, u1, u2);
    const bool surv = i < L;
    St4<R> o;
    R wo;
    predict_slot<R>(c, surv, surv ? x[g] : St4<R>{0, 0, 0, 0}, surv ? w[g] : (R)0, slice_bw<R>(d, j), n1, n2,
                    u1, u2, o, wo);
    xp[g] = o;
    wp[g] = wo;
  }
}

// Copy Z_k into the workspace (in place when it is already there), publish M,
// and flag non-finite measurements.
template <class R>
__global__ void k_stage_z(Dev d, Model, const R* Z, int M) {
  pdl_enter();
  V2<R>* zs = static_cast<V2<R>*>(d.Z);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < M; p += gridDim.x * blockDim.x) {
    V2<R> z = reinterpret_cast<const V2<R>*>(Z)[p];
    if (!isfinite(z.a) || !isfinite(z.b)) atomicOr(d.err, kErrNonFinite);
    zs[p] = z;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *d.M = M;
}

template <class R>
cudaError_t launch_predict(const Dev& d, const Model& m, const R* noise, cudaStream_t s) {
  long items = (long)m.K * ((m.pe_cap + 255) / 256);
  int blocks = (int)(items < 152 * 16 ? (items > 0 ? items : 1) : 152 * 16);
  launch_k(k_predict<R>, dim3(blocks), dim3(256), 0, s, d, m, noise);
  return cudaGetLastError();
}

// Batch staging: the scans of all runs back to back; run j owns rows
// off[j] .. off[j+1]-1 (each at most m_max, all within the workspace).
template <class R>
__global__ void k_stage_zb(Dev d, Model m, const R* Z, const int* __restrict__ off) {
  pdl_enter();
  const int K = m.K;
  const int rows = off[K];
  const bool ok_total = rows >= 0 && rows <= K * m.m_max;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < K; j += gridDim.x * blockDim.x) {
    int Mj = off[j + 1] - off[j];
    if (!ok_total || off[j] < 0 || Mj < 0 || Mj > m.m_max) {
      atomicOr(d.err, kErrCapacity);
      Mj = 0;
    }
    d.zoff[j] = ok_total && off[j] >= 0 ? off[j] : 0;
    d.Mj[j] = Mj;
  }
  if (!ok_total) return;
  V2<R>* zs = static_cast<V2<R>*>(d.Z);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < rows; p += gridDim.x * blockDim.x) {
    V2<R> z = reinterpret_cast<const V2<R>*>(Z)[p];
    if (!isfinite(z.a) || !isfinite(z.b)) atomicOr(d.err, kErrNonFinite);
    zs[p] = z;
  }
}

template <class R>
cudaError_t launch_stage_zb(const Dev& d, const Model& m, const R* Z, const int* off, cudaStream_t s) {
  long rows = (long)m.K * m.m_max;
  int blocks = (int)((rows + 255) / 256);
  if (blocks > 152 * 4) blocks = 152 * 4;
  if (blocks < 1) blocks = 1;
  launch_k(k_stage_zb<R>, dim3(blocks), dim3(256), 0, s, d, m, Z, off);
  return cudaGetLastError();
}

template cudaError_t launch_stage_zb<float>(const Dev&, const Model&, const float*, const int*, cudaStream_t);
template cudaError_t launch_stage_zb<double>(const Dev&, const Model&, const double*, const int*, cudaStream_t);

template <class R>
cudaError_t launch_stage_z(const Dev& d, const Model& m, const R* Z, int M, cudaStream_t s) {
  int blocks = (M + 255) / 256;
  if (blocks < 1) blocks = 1;
  launch_k(k_stage_z<R>, dim3(blocks), dim3(256), 0, s, d, m, Z, M);
  return cudaGetLastError();
}

template cudaError_t launch_predict<float>(const Dev&, const Model&, const float*, cudaStream_t);
template cudaError_t launch_predict<double>(const Dev&, const Model&, const double*, cudaStream_t);
template cudaError_t launch_stage_z<float>(const Dev&, const Model&, const float*, int, cudaStream_t);
template cudaError_t launch_stage_z<double>(const Dev&, const Model&, const double*, int, cudaStream_t);

}  // namespace phd
