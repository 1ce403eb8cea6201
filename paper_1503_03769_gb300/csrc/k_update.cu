// Update, Eq. 7-8, as two passes over the particle x measurement pairs.
//
// The likelihood is kept in exp2 form:
//   g(z|x) = cnorm * 2^-q,  q = b0 (z0 - h0(x))^2 + b1 (z1 - h1(x))^2,
//   b = log2(e) / (2 sigma^2),
// so one MUFU ex2 per pair evaluates it; the bearing difference is wrapped
// to [0, pi].  The N x M likelihood matrix is never stored.
//
// Pass 1 (k_colsum): C^j_p = p_D cnorm sum_i 2^-q_ip w_i.  A work item is a
//   tile of kTile particles of one PE, staged in shared memory as
//   (h0, h1, h1lo, w);
//   threads own measurements (and, when M < 256, a split of the tile) and
//   accumulate in FP32 over at most one tile; the per-item partials go to
//   memory in FP64 and are summed in a fixed order by k_finalize, so the
//   normaliser is accumulated in FP64 and is deterministic.
// Finalize: C^j, the normaliser each PE applies (its own, or the PE mean),
//   and ginv_p = cnorm p_D / (kappa + C_p) (0 when kappa + C_p = 0).
// Pass 2 (k_rowsum): w_i <- [(1 - p_D) + sum_p 2^-q_ip ginv_p] w_i with one
//   thread per particle and Z_k, ginv staged in shared memory; per-item FP64
//   partial sums of the updated weights feed N^j.  The updated weights go to
//   their own buffer: the extraction (Eq. 13, 18) still needs the predicted
//   ones.
//
// Algorithmic work per pair and pass: one ex2 and ~5 FP32 operations; bytes
// per particle and pass: 16 B state + 4 B weight (+ 4 B weight written in
// pass 2); per measurement: 8 B (+ 8 B of FP64 partial per work item).
#include "phd_internal.cuh"

namespace phd {

template <class R>
__global__ void __launch_bounds__(kThreads) k_colsum(Dev d, Model m) {
  __shared__ int pref[kMaxPE + 1];
  __shared__ R sh0[kTile], sh1[kTile], shl[kTile], sw[kTile];
  __shared__ double red[kThreads];
  const int K = m.K;
  item_prefix(d.n_pred, K, pref);
  const int total = pref[K];
  const int M = *d.M;
  if (M <= 0) return;
  const V2<R>* __restrict__ Z = static_cast<const V2<R>*>(d.Z);
  const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x_alt);
  const R* __restrict__ w = static_cast<const R*>(d.w_alt);
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);
  const Lik<R> L = make_lik<R>(m);
  const int mper = M < kThreads ? M : kThreads;
  const int nsplit = kThreads / mper;
  const int pl = threadIdx.x % mper;
  const int split = threadIdx.x / mper;
  const bool active = split < nsplit;

  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = item_pe(pref, K, item);
    const int tile = item - pref[j];
    const long base = (long)j * m.pe_cap + (long)tile * kTile;
    const int cnt = min(kTile, d.n_pred[j] - tile * kTile);
    __syncthreads();
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
      H3<R> h = {0, 0, 0};
      R wi = 0;
      if (i < cnt) {
        h = meas_h<R>(m, x[base + i], tab);
        wi = w[base + i];
      }
      sh0[i] = h.h0;
      sh1[i] = h.h1;
      shl[i] = h.h1lo;
      sw[i] = wi;
    }
    __syncthreads();
    for (int p0 = 0; p0 < M; p0 += mper) {
      const int p = p0 + pl;
      R acc = 0;
      if (active && p < M) {
        const V2<R> z = Z[p];
        R part = 0;
        int i = split, k = 0;
        for (; i < cnt; i += nsplit) {
          const R q = qform<R>(L, z.a, z.b, sh0[i], sh1[i], shl[i]);
          part = fma(exp2_neg(q), sw[i], part);
          if (++k == 32) { acc += part; part = 0; k = 0; }
        }
        acc += part;
      }
      red[threadIdx.x] = (double)acc;
      __syncthreads();
      if (split == 0 && p < M) {
        double s = red[threadIdx.x];
        for (int k = 1; k < nsplit; ++k) s += red[threadIdx.x + k * mper];
        d.colpart[(long)item * m.m_max + p] = s;
      }
      __syncthreads();
    }
  }
}

template <class R>
__global__ void k_finalize(Dev d, Model m) {
  __shared__ int pref[kMaxPE + 1];
  const int K = m.K;
  item_prefix(d.n_pred, K, pref);
  const int M = *d.M;
  const double cs = m.p_d * m.cnorm;
  R* ginv = static_cast<R*>(d.ginv);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < M; p += gridDim.x * blockDim.x) {
    double mean = 0.0;
    for (int j = 0; j < K; ++j) {
      double c = 0.0;
      for (int it = pref[j]; it < pref[j + 1]; ++it) c += d.colpart[(long)it * m.m_max + p];
      c *= cs;
      d.C[j * m.m_max + p] = c;
      mean += c;
    }
    mean /= (double)K;
    for (int j = 0; j < K; ++j) {
      const double cu = m.ck_global ? mean : d.C[j * m.m_max + p];
      d.Cused[j * m.m_max + p] = cu;
      const double den = m.kappa + cu;
      ginv[j * m.m_max + p] = den > 0.0 ? (R)(cs / den) : (R)0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long n = 0;
    for (int j = 0; j < K; ++j) n += (unsigned long long)d.n_pred[j];
    d.stats[0] += n * (unsigned long long)M;
    d.stats[1] += n;
    d.stats[2] += (unsigned long long)M;
    d.stats[3] += 1ull;
  }
}

template <class R>
__global__ void __launch_bounds__(kThreads) k_rowsum(Dev d, Model m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int pref[kMaxPE + 1];
  __shared__ double red[kThreads / 32];
  V2<R>* zs = reinterpret_cast<V2<R>*>(smem_raw);
  R* gs = reinterpret_cast<R*>(smem_raw + sizeof(V2<R>) * m.m_max);
  const int K = m.K;
  item_prefix(d.n_pred, K, pref);
  const int total = pref[K];
  const int M = *d.M;
  const V2<R>* __restrict__ Z = static_cast<const V2<R>*>(d.Z);
  const R* __restrict__ ginv = static_cast<const R*>(d.ginv);
  const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x_alt);
  const R* __restrict__ w = static_cast<const R*>(d.w_alt);
  R* __restrict__ wu = static_cast<R*>(d.wu);
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);
  const Lik<R> L = make_lik<R>(m);
  const R miss = (R)(1.0 - m.p_d);

  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = item_pe(pref, K, item);
    const int tile = item - pref[j];
    __syncthreads();
    for (int p = threadIdx.x; p < M; p += kThreads) {
      zs[p] = Z[p];
      gs[p] = ginv[j * m.m_max + p];
    }
    __syncthreads();
    const int i = tile * kTile + threadIdx.x;
    double wn = 0.0;
    if (i < d.n_pred[j]) {
      const long g = (long)j * m.pe_cap + i;
      const H3<R> h = meas_h<R>(m, x[g], tab);
      R acc = 0, part = 0;
      int k = 0;
      for (int p = 0; p < M; ++p) {
        const V2<R> z = zs[p];
        const R q = qform<R>(L, z.a, z.b, h.h0, h.h1, h.h1lo);
        part = fma(exp2_neg(q), gs[p], part);
        if (++k == 64) { acc += part; part = 0; k = 0; }
      }
      acc += part;
      const R wv = (miss + acc) * w[g];
      wu[g] = wv;
      wn = (double)wv;
    }
    // fixed-order block reduction of the updated weights (FP64)
    for (int o = 16; o > 0; o >>= 1) wn += __shfl_down_sync(0xffffffffu, wn, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = wn;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int k2 = 0; k2 < kThreads / 32; ++k2) s += red[k2];
      d.rowpart[item] = s;
    }
  }
}

// N^j = sum of PE j's pass-2 partials, in item order (deterministic).
__global__ void __launch_bounds__(256) k_mass(Dev d, Model m) {
  __shared__ int pref[kMaxPE + 1];
  __shared__ double red[8];
  const int j = blockIdx.x;
  item_prefix(d.n_pred, m.K, pref);
  double s = 0.0;
  for (int it = pref[j] + threadIdx.x; it < pref[j + 1]; it += blockDim.x) s += d.rowpart[it];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k];
    d.mass[j] = t;
  }
}

int grid_items(const Model& m) {
  long items = (long)m.K * ((m.pe_cap + kTile - 1) / kTile);
  long g = 152L * 4;
  return (int)(items < g ? (items > 0 ? items : 1) : g);
}

template <class R>
cudaError_t prepare_kernels(const Model& m) {
  size_t sm = (sizeof(V2<R>) + sizeof(R)) * (size_t)m.m_max;
  return cudaFuncSetAttribute(k_rowsum<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <class R>
cudaError_t launch_update(const Dev& d, const Model& m, cudaStream_t s) {
  const int g = grid_items(m);
  k_colsum<R><<<g, kThreads, 0, s>>>(d, m);
  k_finalize<R><<<(m.m_max + 255) / 256, 256, 0, s>>>(d, m);
  size_t sm = (sizeof(V2<R>) + sizeof(R)) * (size_t)m.m_max;
  k_rowsum<R><<<g, kThreads, sm, s>>>(d, m);
  k_mass<<<m.K, 256, 0, s>>>(d, m);
  return cudaGetLastError();
}

template cudaError_t launch_update<float>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_update<double>(const Dev&, const Model&, cudaStream_t);
template cudaError_t prepare_kernels<float>(const Model&);
template cudaError_t prepare_kernels<double>(const Model&);

}  // namespace phd
