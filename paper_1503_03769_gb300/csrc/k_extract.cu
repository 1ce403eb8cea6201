// Measurement-labelled state extraction (Eq. 10-18, Step 3) and CU fusion
// (Step 4).
//
// k_select (one CTA per PE): LT_j = round(N^j) with the updated mass N^j,
//   dW^{j,p} = C^j_p / (kappa + C_p) (Eq. 16 in closed
//   form), and the LT_j largest dW by rank counting: rank_p = #{q : dW_q > dW_p
//   or (dW_q = dW_p and q < p)}; label p is taken when dW_p > 0 and
//   rank_p < LT_j.  O(M^2) comparisons per PE on M <= 4096 values in shared
//   memory, made on the FP64 values' bit patterns as unsigned integers (same
//   order, integer instructions).
// k_selsum (pass 3, selected labels only): per label the sums of
//   e w, e w (x - r_x), e w vx, e w (y - r_y), e w vy over the PE's particles,
//   with e = 2^-q the unnormalised likelihood and r the measurement's
//   Cartesian point; the offsets keep the FP32 sums small.  Eq. 18's
//   zeta_p = sum_i dw^{i,p} x_i / dW^p does not depend on the per-label
//   factor p_D cnorm / (kappa + C_p), which cancels.
// k_est_local: per (PE, rank) FP64 reduction of the pass-3 partials to zeta.
// k_fuse (one CTA): for every label the PEs that took it vote; a label is
//   valid with more than K/2 votes, and its state is the FP64 mean of the
//   voters' local states in PE order.  Output in ascending label order.
#include "phd_internal.cuh"

namespace phd {

template <class R>
__global__ void __launch_bounds__(1024) k_select(Dev d, Model m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem_raw);
  __shared__ int npos_s;
  const int j = blockIdx.x;
  const int M = *d.M;
  if (threadIdx.x == 0) npos_s = 0;
  for (int p = threadIdx.x; p < M; p += blockDim.x) {
    const double den = m.kappa + d.Cused[j * m.m_max + p];
    key[p] = order_key(den > 0.0 ? d.C[j * m.m_max + p] / den : 0.0);
  }
  __syncthreads();
  const double mass = d.mass[j];
  int npos_t = 0;
  for (int p = threadIdx.x; p < M; p += blockDim.x) npos_t += key[p] > 0ull ? 1 : 0;
  npos_t = __reduce_add_sync(0xffffffffu, npos_t);
  if ((threadIdx.x & 31) == 0) atomicAdd(&npos_s, npos_t);
  __syncthreads();
  long long LT = llround(mass);
  if (LT > npos_s) LT = npos_s;
  if (LT < 0) LT = 0;
  for (int p = threadIdx.x; p < M; p += blockDim.x) {
    const unsigned long long v = key[p];
    int rank = 0;
    for (int q = 0; q < M; ++q) {
      const unsigned long long u = key[q];
      rank += (u > v || (u == v && q < p)) ? 1 : 0;
    }
    const bool take = v > 0ull && rank < LT;
    d.selrank[j * m.m_max + p] = take ? rank : -1;
    if (take) d.sel[j * m.m_max + rank] = p;
  }
  if (threadIdx.x == 0) d.nsel[j] = (int)LT;
}

// Cartesian point of a measurement, the offset origin of the labelled sums.
template <class R>
__device__ __forceinline__ void meas_point(const Model& m, V2<R> z, R& rx, R& ry) {
  if (m.meas_model == 0) {
    rx = z.a;
    ry = z.b;
  } else {
    R sn, cs;
    sincos(z.b, &sn, &cs);
    rx = (R)m.sx + z.a * cs;
    ry = (R)m.sy + z.a * sn;
  }
}

template <class R>
__global__ void __launch_bounds__(kThreads) k_selsum(Dev d, Model m) {
  __shared__ int pref[kMaxPE + 1];
  __shared__ R sh0[kTile], sh1[kTile], shl[kTile], sw[kTile];
  __shared__ St4<R> sx[kTile];
  __shared__ double red[kThreads];
  const int K = m.K;
  item_prefix(d.n_pred, K, pref);
  const int total = pref[K];
  const V2<R>* __restrict__ Z = static_cast<const V2<R>*>(d.Z);
  const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x_alt);
  const R* __restrict__ w = static_cast<const R*>(d.w_alt);
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);
  const Lik<R> L = make_lik<R>(m);

  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = item_pe(pref, K, item);
    const int ns = d.nsel[j];
    if (ns <= 0) continue;   // uniform over the block
    const int tile = item - pref[j];
    const long base = (long)j * m.pe_cap + (long)tile * kTile;
    const int cnt = min(kTile, d.n_pred[j] - tile * kTile);
    const int mper = ns < kThreads ? ns : kThreads;
    const int nsplit = kThreads / mper;
    const int rl = threadIdx.x % mper;
    const int split = threadIdx.x / mper;
    const bool active = split < nsplit;
    __syncthreads();
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
      H3<R> h = {0, 0, 0};
      R wi = 0;
      St4<R> s = {0, 0, 0, 0};
      if (i < cnt) {
        s = x[base + i];
        h = meas_h<R>(m, s, tab);
        wi = w[base + i];
      }
      sh0[i] = h.h0;
      sh1[i] = h.h1;
      shl[i] = h.h1lo;
      sw[i] = wi;
      sx[i] = s;
    }
    __syncthreads();
    for (int r0 = 0; r0 < ns; r0 += mper) {
      const int r = r0 + rl;
      R a[5] = {0, 0, 0, 0, 0};
      if (active && r < ns) {
        const int p = d.sel[j * m.m_max + r];
        const V2<R> z = Z[p];
        R px, py;
        meas_point<R>(m, z, px, py);
        for (int i = split; i < cnt; i += nsplit) {
          const R q = qform<R>(L, z.a, z.b, sh0[i], sh1[i], shl[i]);
          const R ew = exp2_neg(q) * sw[i];
          const St4<R> s = sx[i];
          a[0] += ew;
          a[1] = fma(ew, s.x - px, a[1]);
          a[2] = fma(ew, s.vx, a[2]);
          a[3] = fma(ew, s.y - py, a[3]);
          a[4] = fma(ew, s.vy, a[4]);
        }
      }
      for (int c = 0; c < 5; ++c) {
        red[threadIdx.x] = (double)a[c];
        __syncthreads();
        if (split == 0 && r < ns) {
          double t = red[threadIdx.x];
          for (int k = 1; k < nsplit; ++k) t += red[threadIdx.x + k * mper];
          d.spart[((long)item * m.m_max + r) * 5 + c] = t;
        }
        __syncthreads();
      }
    }
  }
}

template <class R>
__global__ void k_est_local(Dev d, Model m) {
  __shared__ int pref[kMaxPE + 1];
  const int K = m.K;
  item_prefix(d.n_pred, K, pref);
  St4<R>* est = static_cast<St4<R>*>(d.est_local);
  const V2<R>* Zr = static_cast<const V2<R>*>(d.Z);
  const long total = (long)K * m.m_max;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
    const int j = (int)(g / m.m_max);
    const int r = (int)(g - (long)j * m.m_max);
    if (r >= d.nsel[j]) continue;
    double a[5] = {0, 0, 0, 0, 0};
    for (int it = pref[j]; it < pref[j + 1]; ++it)
      for (int c = 0; c < 5; ++c) a[c] += d.spart[((long)it * m.m_max + r) * 5 + c];
    const int p = d.sel[j * m.m_max + r];
    R px, py;
    meas_point<R>(m, Zr[p], px, py);
    St4<R> o;
    if (a[0] > 0.0) {
      o.x = (R)((double)px + a[1] / a[0]);
      o.vx = (R)(a[2] / a[0]);
      o.y = (R)((double)py + a[3] / a[0]);
      o.vy = (R)(a[4] / a[0]);
    } else {
      o = St4<R>{px, (R)0, py, (R)0};
    }
    est[g] = o;
  }
}

template <class R>
__global__ void __launch_bounds__(1024) k_fuse(Dev d, Model m, R* out_states, int* out_labels, int cap,
                                               int* d_count) {
  __shared__ int wsum[32];
  __shared__ int carry_s;
  const int K = m.K;
  const int M = *d.M;
  const St4<R>* est = static_cast<const St4<R>*>(d.est_local);
  St4<R>* out = reinterpret_cast<St4<R>*>(out_states);
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int p0 = 0; p0 < M; p0 += blockDim.x) {
    const int p = p0 + threadIdx.x;
    int votes = 0;
    if (p < M)
      for (int j = 0; j < K; ++j) votes += d.selrank[j * m.m_max + p] >= 0 ? 1 : 0;
    const int valid = (p < M && 2 * votes > K) ? 1 : 0;
    // block exclusive scan of the valid flags
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = valid;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      wsum[lane] = v;   // inclusive warp totals
    }
    __syncthreads();
    const int carry = carry_s;
    const int idx = carry + (wid > 0 ? wsum[wid - 1] : 0) + incl - valid;
    if (valid && idx < cap) {
      double a[4] = {0, 0, 0, 0};
      for (int j = 0; j < K; ++j) {
        const int r = d.selrank[j * m.m_max + p];
        if (r >= 0) {
          const St4<R> e = est[j * m.m_max + r];
          a[0] += (double)e.x;
          a[1] += (double)e.vx;
          a[2] += (double)e.y;
          a[3] += (double)e.vy;
        }
      }
      out[idx] = St4<R>{(R)(a[0] / votes), (R)(a[1] / votes), (R)(a[2] / votes), (R)(a[3] / votes)};
      out_labels[idx] = p;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + wsum[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *d.out_count = carry_s;
    if (d_count) *d_count = carry_s;
  }
}

template <class R>
cudaError_t launch_extract(const Dev& d, const Model& m, R* out_states, int* out_labels, int cap,
                           int* d_count, cudaStream_t s) {
  k_select<R><<<m.K, 1024, sizeof(unsigned long long) * (size_t)m.m_max, s>>>(d, m);
  k_selsum<R><<<grid_items(m), kThreads, 0, s>>>(d, m);
  long tot = (long)m.K * m.m_max;
  int b = (int)((tot + 255) / 256);
  if (b > 152 * 8) b = 152 * 8;
  k_est_local<R><<<b, 256, 0, s>>>(d, m);
  k_fuse<R><<<1, 1024, 0, s>>>(d, m, out_states, out_labels, cap, d_count);
  return cudaGetLastError();
}

template cudaError_t launch_extract<float>(const Dev&, const Model&, float*, int*, int, int*, cudaStream_t);
template cudaError_t launch_extract<double>(const Dev&, const Model&, double*, int*, int, int*, cudaStream_t);

}  // namespace phd
