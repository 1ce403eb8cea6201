// Update, Eq. 7-8, as two passes over the particle x measurement pairs.
//
// The likelihood is kept in exp2 form:
//   g(z|x) = cnorm * 2^-q,  q = b0 (z0 - h0(x))^2 + b1 (z1 - h1(x))^2,
//   b = log2(e) / (2 sigma^2),
// so one MUFU ex2 per pair evaluates it; the bearing difference is wrapped
// to [0, pi].  The N x M likelihood matrix is never stored.
//
// Pass 1 (k_colsum): C^j_p = p_D cnorm sum_i 2^-q_ip w_i.  A work item is a
//   tile of kTile particles of one PE (staged in shared memory as packed
//   (h0, h1, h1lo, w)) times a chunk of kMChunk measurements; threads own
//   measurements (and, when the chunk is short, a split of the tile) and
//   accumulate in FP32 over at most one tile; the per-tile partials go to
//   memory in FP64 and are summed in a fixed order by k_finalize, so the
//   normaliser is accumulated in FP64 and is deterministic.
// Finalize: C^j, the normaliser each PE applies (its own, or the PE mean),
//   and ginv_p = cnorm p_D / (kappa + C_p) (0 when kappa + C_p = 0).
// Pass 2 (k_rowsum): w_i <- [(1 - p_D) + sum_p 2^-q_ip ginv_p] w_i with four
//   lanes per particle and Z_k, ginv staged in shared memory; per-tile FP64
//   sums and maxima of the updated weights feed N^j and the resampling plan
//   (k_mass).  The updated weights go to their own buffer: the extraction
//   (Eq. 13, 18) still needs the predicted ones.
//
// Algorithmic work per pair and pass: one ex2 and ~5 FP32 operations; bytes
// per particle and pass: 16 B state + 4 B weight (+ 4 B weight written in
// pass 2); per measurement: 8 B (+ 8 B of FP64 partial per work item).
#include "phd_internal.cuh"

namespace phd {

template <class R>
__global__ void __launch_bounds__(kThreads) k_colsum(Dev d, Model m) {
  __shared__ int tpref[kMaxPE + 1];   // tiles per slice (pass-1 partial rows)
  __shared__ int ipref[kMaxPE + 1];   // work items per slice (tiles x measurement chunks)
  __shared__ P4<R> sp[kTile];
  __shared__ R red[kThreads];
  const int K = m.K;
  item_prefix(d.n_pred, K, tpref);
  slice_prefix(K, ipref, [&](int j) {
    return ((d.n_pred[j] + kTile - 1) / kTile) * ((slice_M(d, j) + kMChunk - 1) / kMChunk);
  });
  const int total = ipref[K];
  const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x_alt);
  const R* __restrict__ w = static_cast<const R*>(d.w_alt);
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);
  const Lik<R> L = make_lik<R>(m);
  int staged = -1;
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = item_pe(ipref, K, item);
    const int M = slice_M(d, j);
    const V2<R>* __restrict__ Z = slice_Z<R>(d, j);
    const int chunks = (M + kMChunk - 1) / kMChunk;
    const int local = item - ipref[j];
    const int tile = local / chunks, chunk = local - tile * chunks;
    const int titem = tpref[j] + tile;
    const long base = (long)j * m.pe_cap + (long)tile * kTile;
    const int cnt = min(kTile, d.n_pred[j] - tile * kTile);
    if (titem != staged) {   // consecutive items of a CTA often share the tile
      __syncthreads();
      for (int i = threadIdx.x; i < kTile; i += kThreads) {
        P4<R> q = {0, 0, 0, 0};
        if (i < cnt) {
          const H3<R> h = meas_h<R>(m, x[base + i], tab);
          q = P4<R>{h.h0, h.h1, h.h1lo, w[base + i]};
        }
        sp[i] = q;
      }
      __syncthreads();
      staged = titem;
    }
    const int pbeg = chunk * kMChunk;
    const int Mc = min(kMChunk, M - pbeg);
    const int nsplit = kThreads / Mc;
    const int pl = threadIdx.x % Mc;
    const int split = threadIdx.x / Mc;
    const int p = pbeg + pl;
    R acc = 0;
    if (split < nsplit) {
      // four independent partial sums (ILP), each over at most 64 pairs
      const V2<R> z = Z[p];
      R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      int i = split;
      for (; i + 3 * nsplit < cnt; i += 4 * nsplit) {
        const P4<R> q0 = sp[i], q1 = sp[i + nsplit], q2 = sp[i + 2 * nsplit], q3 = sp[i + 3 * nsplit];
        a0 = fma(exp2_neg(qform<R>(L, z.a, z.b, q0.h0, q0.h1, q0.h1lo)), q0.w, a0);
        a1 = fma(exp2_neg(qform<R>(L, z.a, z.b, q1.h0, q1.h1, q1.h1lo)), q1.w, a1);
        a2 = fma(exp2_neg(qform<R>(L, z.a, z.b, q2.h0, q2.h1, q2.h1lo)), q2.w, a2);
        a3 = fma(exp2_neg(qform<R>(L, z.a, z.b, q3.h0, q3.h1, q3.h1lo)), q3.w, a3);
      }
      for (; i < cnt; i += nsplit) {
        const P4<R> q0 = sp[i];
        a0 = fma(exp2_neg(qform<R>(L, z.a, z.b, q0.h0, q0.h1, q0.h1lo)), q0.w, a0);
      }
      acc = (a0 + a1) + (a2 + a3);
    }
    // the tile's partial for measurement p: splits combined in the kernel's
    // precision (a tile is at most 256 particles), one conversion to FP64
    red[threadIdx.x] = acc;
    __syncthreads();
    if (split == 0) {
      R s = red[threadIdx.x];
      for (int k = 1; k < nsplit; ++k) s += red[threadIdx.x + k * Mc];
      d.colpart[(long)titem * m.m_max + p] = (double)s;
    }
    __syncthreads();
  }
}

// One warp per (slice, measurement): C^j_p = p_D cnorm * (FP64 tree over
// slice j's tile partials, fixed order), the normaliser the slice applies
// (its own, or for one filter's PEs in "global" mode the PE mean), ginv and
// the dW order keys.
template <class R>
__global__ void __launch_bounds__(256) k_finalize(Dev d, Model m) {
  __shared__ int pref[kMaxPE + 1];
  __shared__ int mpref[kMaxPE + 1];
  const int K = m.K;
  item_prefix(d.n_pred, K, pref);
  slice_prefix(K, mpref, [&](int j) { return slice_M(d, j); });
  const double cs = m.p_d * m.cnorm;
  R* ginv = static_cast<R*>(d.ginv);
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int wid0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (m.ck_global && d.zshared) {
    // one filter's PEs share Z: a warp per measurement handles every PE
    const int M = *d.M;
    for (int p = wid0; p < M; p += nwarps) {
      double mean = 0.0;
      for (int j = 0; j < K; ++j) {
        double c = 0.0;
        for (int it = pref[j] + lane; it < pref[j + 1]; it += 32) c += d.colpart[(long)it * m.m_max + p];
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        c = __shfl_sync(0xffffffffu, c, 0) * cs;
        if (lane == 0) d.C[j * m.m_max + p] = c;
        mean += c;
      }
      mean /= (double)K;
      for (int j = lane; j < K; j += 32) {
        const double cj = d.C[j * m.m_max + p];
        d.Cused[j * m.m_max + p] = mean;
        const double den = d.kap[j] + mean;
        ginv[j * m.m_max + p] = den > 0.0 ? (R)(cs / den) : (R)0;
        d.dwkey[j * m.m_max + p] = order_key(den > 0.0 ? cj / den : 0.0);
      }
    }
  } else {
    for (int gw = wid0; gw < mpref[K]; gw += nwarps) {
      const int j = item_pe(mpref, K, gw);
      const int p = gw - mpref[j];
      double c = 0.0;
      for (int it = pref[j] + lane; it < pref[j + 1]; it += 32) c += d.colpart[(long)it * m.m_max + p];
      for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
      if (lane == 0) {
        c *= cs;
        d.C[j * m.m_max + p] = c;
        d.Cused[j * m.m_max + p] = c;
        const double den = d.kap[j] + c;
        ginv[j * m.m_max + p] = den > 0.0 ? (R)(cs / den) : (R)0;
        d.dwkey[j * m.m_max + p] = order_key(den > 0.0 ? c / den : 0.0);
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long n = 0, pairs = 0, meas = 0;
    for (int j = 0; j < K; ++j) {
      const unsigned long long Mj = (unsigned long long)slice_M(d, j);
      n += (unsigned long long)d.n_pred[j];
      pairs += (unsigned long long)d.n_pred[j] * Mj;
      meas += Mj;
    }
    d.stats[0] += pairs;
    d.stats[1] += n;
    d.stats[2] += d.zshared ? (unsigned long long)*d.M : meas;
    d.stats[3] += 1ull;
  }
}

// Pass 2: tiles of kRowTile particles; four consecutive lanes share a particle
// and split the measurements (p = g, g+4, ...), combined by shuffles.
template <class R>
__global__ void __launch_bounds__(kThreads) k_rowsum(Dev d, Model m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int pref[kMaxPE + 1];
  __shared__ double rs[kThreads / 32];
  __shared__ double rm[kThreads / 32];
  Z4<R>* zs = reinterpret_cast<Z4<R>*>(smem_raw);
  const int K = m.K;
  item_prefix(d.n_pred, K, pref, kRowTile);
  const int total = pref[K];
  const R* __restrict__ ginv = static_cast<const R*>(d.ginv);
  const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x_alt);
  const R* __restrict__ w = static_cast<const R*>(d.w_alt);
  R* __restrict__ wu = static_cast<R*>(d.wu);
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);
  const Lik<R> L = make_lik<R>(m);
  const R miss = consts<R>(m).miss;
  const int il = threadIdx.x >> 2, g = threadIdx.x & 3;
  int staged = -1;
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = item_pe(pref, K, item);
    const int tile = item - pref[j];
    const int M = slice_M(d, j);
    const V2<R>* __restrict__ Z = slice_Z<R>(d, j);
    if (j != staged) {
      __syncthreads();
      for (int p = threadIdx.x; p < M; p += kThreads) {
        const V2<R> z = Z[p];
        zs[p] = Z4<R>{z.a, z.b, ginv[j * m.m_max + p], (R)0};
      }
      __syncthreads();
      staged = j;
    }
    const int i = tile * kRowTile + il;
    const bool live = i < d.n_pred[j];
    const long gi = (long)j * m.pe_cap + i;
    R acc = 0;
    if (live) {
      // four independent partial sums (ILP) over measurements g, g+4, ...,
      // folded into acc every 32 rounds
      const H3<R> h = meas_h<R>(m, x[gi], tab);
      R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      int p = g, k = 0;
      for (; p + 12 < M; p += 16) {
        const Z4<R> z0 = zs[p], z1 = zs[p + 4], z2 = zs[p + 8], z3 = zs[p + 12];
        a0 = fma(exp2_neg(qform<R>(L, z0.z0, z0.z1, h.h0, h.h1, h.h1lo)), z0.g, a0);
        a1 = fma(exp2_neg(qform<R>(L, z1.z0, z1.z1, h.h0, h.h1, h.h1lo)), z1.g, a1);
        a2 = fma(exp2_neg(qform<R>(L, z2.z0, z2.z1, h.h0, h.h1, h.h1lo)), z2.g, a2);
        a3 = fma(exp2_neg(qform<R>(L, z3.z0, z3.z1, h.h0, h.h1, h.h1lo)), z3.g, a3);
        if (++k == 32) {
          acc += (a0 + a1) + (a2 + a3);
          a0 = a1 = a2 = a3 = 0;
          k = 0;
        }
      }
      for (; p < M; p += 4) {
        const Z4<R> z0 = zs[p];
        a0 = fma(exp2_neg(qform<R>(L, z0.z0, z0.z1, h.h0, h.h1, h.h1lo)), z0.g, a0);
      }
      acc += (a0 + a1) + (a2 + a3);
    }
    acc += __shfl_down_sync(0xffffffffu, acc, 2, 4);
    acc += __shfl_down_sync(0xffffffffu, acc, 1, 4);
    R wv = 0;
    if (live && g == 0) {
      wv = (miss + acc) * w[gi];
      wu[gi] = wv;
    }
    // tile sum and max: the warp's 8 particles in the kernel's precision, the
    // 8 warp totals in FP64 by one thread (FP64 is ~1/60 of the FP32 rate)
    R sv = wv, mv = wv;
    for (int o = 16; o > 0; o >>= 1) {
      sv += __shfl_down_sync(0xffffffffu, sv, o);
      const R u = __shfl_down_sync(0xffffffffu, mv, o);
      mv = u > mv ? u : mv;
    }
    if ((threadIdx.x & 31) == 0) {
      rs[threadIdx.x >> 5] = (double)sv;
      rm[threadIdx.x >> 5] = (double)mv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0, mx = 0.0;
      for (int k = 0; k < kThreads / 32; ++k) {
        s += rs[k];
        mx = fmax(mx, rm[k]);
      }
      d.rowpart[item] = s;
      d.rowmax[item] = mx;
    }
    __syncthreads();
  }
}

// Per PE: N^j = sum of the pass-2 tile sums (fixed order), the largest
// updated weight, and the resampling plan (L_j and the CDF scale).
__global__ void __launch_bounds__(256) k_mass(Dev d, Model m) {
  __shared__ int pref[kMaxPE + 1];
  __shared__ double red[8], redm[8];
  const int j = blockIdx.x;
  item_prefix(d.n_pred, m.K, pref, kRowTile);
  double s = 0.0, mx = 0.0;
  for (int it = pref[j] + threadIdx.x; it < pref[j + 1]; it += blockDim.x) {
    s += d.rowpart[it];
    mx = fmax(mx, d.rowmax[it]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = s;
    redm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, tm = 0.0;
    for (int k = 0; k < 8; ++k) {
      t += red[k];
      tm = fmax(tm, redm[k]);
    }
    d.mass[j] = t;
    int L, sc;
    resample_plan(d.rho[j], d.lmax[j], d.n_pred[j], t, tm, L, sc);
    d.rs_mass[j] = t;
    d.rs_s[j] = sc;
    d.rs_L[j] = L;
  }
}

int grid_items(const Model& m) {
  long items = (long)m.K * ((m.pe_cap + kTile - 1) / kTile);
  long g = 152L * 4;
  return (int)(items < g ? (items > 0 ? items : 1) : g);
}

static int grid_cap(long items, long cap) { return (int)(items < cap ? (items > 0 ? items : 1) : cap); }

template <class R>
cudaError_t prepare_kernels(const Model& m) {
  size_t sm = sizeof(Z4<R>) * (size_t)m.m_max;
  return cudaFuncSetAttribute(k_rowsum<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <class R>
cudaError_t launch_update(const Dev& d, const Model& m, cudaStream_t s) {
  const long tiles = (long)m.K * ((m.pe_cap + kTile - 1) / kTile);
  const long chunks = (m.m_max + kMChunk - 1) / kMChunk;
  k_colsum<R><<<grid_cap(tiles * chunks, 152L * 8), kThreads, 0, s>>>(d, m);
  k_finalize<R><<<grid_cap(((long)m.K * m.m_max + 7) / 8, 152L * 8), 256, 0, s>>>(d, m);
  const long rtiles = (long)m.K * ((m.pe_cap + kRowTile - 1) / kRowTile);
  k_rowsum<R><<<grid_cap(rtiles, 152L * 8), kThreads, sizeof(Z4<R>) * (size_t)m.m_max, s>>>(d, m);
  k_mass<<<m.K, 256, 0, s>>>(d, m);
  return cudaGetLastError();
}

template cudaError_t launch_update<float>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_update<double>(const Dev&, const Model&, cudaStream_t);
template cudaError_t prepare_kernels<float>(const Model&);
template cudaError_t prepare_kernels<double>(const Model&);

}  // namespace phd
