// Measurement-labelled state extraction (Eq. 10-18, Step 3) and CU fusion
// (Step 4).
//
// k_select (one CTA per PE and chunk of measurements; the last kernel of the
//   update stage): N^j from the pass-2 tile sums (and, in the first CTA of
//   the slice, the resampling plan), LT_j = round(N^j),
//   dW^{j,p} = C^j_p / (kappa + C_p) (Eq. 16 in closed
//   form), and the LT_j largest dW by rank counting: rank_p = #{q : dW_q > dW_p
//   or (dW_q = dW_p and q < p)}; label p is taken when dW_p > 0 and
//   rank_p < LT_j.  O(M^2) comparisons per PE on M <= 4096 values in shared
//   memory, made on the FP64 values' bit patterns as unsigned integers (same
//   order, integer instructions).
// k_selsum (pass 3, selected labels only; pass-1 tiles): per label the sums of
//   e w, e w (x - r_x), e w vx, e w (y - r_y), e w vy over the PE's particles,
//   with e = 2^-q the unnormalised likelihood and r the measurement's
//   Cartesian point; the offsets keep the FP32 sums small.  Eq. 18's
//   zeta_p = sum_i dw^{i,p} x_i / dW^p does not depend on the per-label
//   factor p_D cnorm / (kappa + C_p), which cancels.
// k_est_local: per (PE, rank) FP64 reduction of the pass-3 partials to zeta
//   (one filter on one PE: also the output, in ascending label order).
// k_fuse (one CTA, K > 1): for every label the PEs that took it vote; a label is
//   valid with more than K/2 votes, and its state is the mean of the voters'
//   local states in PE order (FP32 kernels: positions as offsets from the
//   label's measurement point, summed and scaled in FP32; FP64 kernels: FP64
//   sums).  Output in
//   ascending label order.
#include "phd_internal.cuh"

namespace phd {

template <class R>
__global__ void __launch_bounds__(256) k_select(Dev d, Model m) {
  pdl_enter();
  extern __shared__ __align__(32) unsigned char smem_raw[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem_raw);
  __shared__ int npos_s;
  __shared__ int pref[kMaxPE + 1];
  __shared__ double red[8], redm[8], mass_s;
  const int j = blockIdx.x;
  const int M = slice_M(d, j);
  item_prefix(d.n_pred, m.K, pref, row_tile(m.tune));
  const double N = slice_mass(d, m, j, pref, blockIdx.y == 0, red, redm, &mass_s);
  if (threadIdx.x == 0) npos_s = 0;
  for (int p = threadIdx.x; p < M; p += blockDim.x) key[p] = d.dwkey[j * m.m_max + p];
  __syncthreads();
  int npos_t = 0;
  for (int p = threadIdx.x; p < M; p += blockDim.x) npos_t += key[p] > 0ull ? 1 : 0;
  npos_t = __reduce_add_sync(0xffffffffu, npos_t);
  if ((threadIdx.x & 31) == 0) atomicAdd(&npos_s, npos_t);
  __syncthreads();
  long long LT = llround(N);
  if (LT > npos_s) LT = npos_s;
  if (LT < 0) LT = 0;
  // one warp per measurement, lanes split the comparisons
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int p = blockIdx.y * wpb + (threadIdx.x >> 5); p < M; p += gridDim.y * wpb) {
    const unsigned long long v = key[p];
    int cnt = 0;
    for (int q = lane; q < M; q += 32) {
      const unsigned long long u = key[q];
      cnt += (u > v || (u == v && q < p)) ? 1 : 0;
    }
    const int rank = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) {
      const bool take = v > 0ull && rank < LT;
      d.selrank[j * m.m_max + p] = take ? rank : -1;
      if (take) d.sel[j * m.m_max + rank] = p;
    }
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) d.nsel[j] = (int)LT;
}


// Pass 3: a work item is a tile of c_tile particles of one slice (the pass-1
// tile), staged as packed geometry + weight and state; groups of nsplit
// consecutive lanes own kSelLB selected labels each (one pair of shared loads
// feeds kSelLB pairs) and split the tile; FP32 sums of offsets from each
// label's point, reduced by shuffles within the group, one FP64 partial per
// (tile, label).
constexpr int kSelLB = 2;

template <class R, int RB>
__global__ void __launch_bounds__(kThreads) k_selsum(Dev d, Model m) {
  pdl_enter();
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ int pref[kMaxPE + 1];
  const int TP = m.tune.c_tile;
  P4<R>* sp = reinterpret_cast<P4<R>*>(smem_raw);   // [TP]
  St4<R>* sx = reinterpret_cast<St4<R>*>(sp + TP);  // [TP]
  int* lr = reinterpret_cast<int*>(sx + TP);        // [m_max] selected ranks past no gate
  __shared__ R bsh[4 * (kThreads / 32)];
  __shared__ int wcnt[kThreads / 32];
  const int K = m.K;
  item_prefix(d.n_pred, K, pref, TP);
  const int total = pref[K];
  const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x_alt);
  const R* __restrict__ w = static_cast<const R*>(d.w_alt);
  const P4<R>* __restrict__ geo = static_cast<const P4<R>*>(d.geo);
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);
  const PairQ<R, RB> Q(m);
  const Lik<R> LB = make_lik<R>(m);
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = item_pe(pref, K, item);
    const int ns = d.nsel[j];
    if (ns <= 0) continue;   // uniform over the block
    const V2<R>* __restrict__ Z = slice_Z<R>(d, j);
    const int tile = item - pref[j];
    const long base = (long)j * m.pe_cap + (long)tile * TP;
    const int cnt = min(TP, d.n_pred[j] - tile * TP);
    __syncthreads();
    const R inf = (R)INFINITY;
    R lo0 = inf, hi0 = -inf, lo1 = inf, hi1 = -inf;
    for (int i = threadIdx.x; i < TP; i += kThreads) {
      P4<R> q = {0, 0, 0, 0};
      St4<R> st = {0, 0, 0, 0};
      if (i < cnt) {
        // the pass-1 tiles: the spatial order (and its geometry records) when
        // the update built it
        if (m.tune.order) {
          q = geo[base + i];
          st = x[(long)j * m.pe_cap + d.perm[base + i]];
        } else {
          st = x[base + i];
          const H3<R> h = meas_h<R>(m, st, tab);
          q = P4<R>{h.h0, h.h1, h.h1lo, w[base + i]};
        }
        lo0 = fmin(lo0, q.h0);
        hi0 = fmax(hi0, q.h0);
        lo1 = fmin(lo1, q.h1);
        hi1 = fmax(hi1, q.h1);
      }
      sp[i] = q;
      sx[i] = st;
    }
    const Box<R> box = block_box<R>(lo0, hi0, lo1, hi1, bsh);
    // every selected label's partial is written: zeros first, then the
    // labels that can reach the tile (the gate's survivors, in rank order)
    for (int t = threadIdx.x; t < ns * 5; t += kThreads) d.spart[(long)item * m.m_max * 5 + t] = 0.0;
    int nl = 0;
    {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      for (int r0 = 0; r0 < ns; r0 += kThreads) {
        const int r = r0 + (int)threadIdx.x;
        bool keep = false;
        if (r < ns) {
          const V2<R> z = Z[d.sel[j * m.m_max + r]];
          keep = !m.tune.gate || box_qmin<R, RB>(box, LB.b0, LB.b1, z.a, z.b) < gate_limit<R>(m);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wcnt[wid] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int k = 0; k < kThreads / 32; ++k) {
          before += k < wid ? wcnt[k] : 0;
          all += wcnt[k];
        }
        if (keep) lr[nl + before + __popc(bal & ((1u << lane) - 1u))] = r;
        nl += all;
        __syncthreads();
      }
    }
    const int ng = (nl + kSelLB - 1) / kSelLB;   // label groups
    int nsplit = 1;
    while (nsplit * 2 <= 32 && nsplit * 2 * ng <= kThreads) nsplit *= 2;
    const int gpr = kThreads / nsplit;           // label groups per round
    const int rl = threadIdx.x / nsplit, split = threadIdx.x % nsplit;
    for (int g0 = 0; g0 < ng; g0 += gpr) {
      const int g = g0 + rl;
      R s[kSelLB][5];
      R z0[kSelLB], z1[kSelLB], px[kSelLB], py[kSelLB];
#pragma unroll
      for (int k = 0; k < kSelLB; ++k) {
#pragma unroll
        for (int c = 0; c < 5; ++c) s[k][c] = 0;
        const int q = g * kSelLB + k;
        V2<R> z = {0, 0};
        if (g < ng && q < nl) z = Z[d.sel[j * m.m_max + lr[q]]];
        z0[k] = z.a;
        z1[k] = z.b;
        meas_point<R>(m, z, px[k], py[k]);
      }
      if (g < ng) {
        for (int i = split; i < cnt; i += nsplit) {
          const P4<R> q = sp[i];
          const St4<R> st = sx[i];
#pragma unroll
          for (int k = 0; k < kSelLB; ++k) {
            const R ew = exp2_neg(Q(z0[k], z1[k], q.h0, q.h1, q.h1lo)) * q.w;
            s[k][0] += ew;
            s[k][1] = fma(ew, st.x - px[k], s[k][1]);
            s[k][2] = fma(ew, st.vx, s[k][2]);
            s[k][3] = fma(ew, st.y - py[k], s[k][3]);
            s[k][4] = fma(ew, st.vy, s[k][4]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kSelLB; ++k)
#pragma unroll
        for (int c = 0; c < 5; ++c)
          for (int o = nsplit >> 1; o > 0; o >>= 1) s[k][c] += __shfl_down_sync(0xffffffffu, s[k][c], o, nsplit);
      if (split == 0 && g < ng) {
#pragma unroll
        for (int k = 0; k < kSelLB; ++k) {
          const int q = g * kSelLB + k;
          if (q < nl) {
            double* o = d.spart + ((long)item * m.m_max + lr[q]) * 5;
#pragma unroll
            for (int c = 0; c < 5; ++c) o[c] = (double)s[k][c];
          }
        }
      }
    }
  }
}

// One warp per (PE, rank): lanes take the PE's pass-3 tile partials in a
// strided order, an FP64 shuffle tree combines them (fixed order), then
// zeta = r + S / C (Eq. 18).  With one filter on one PE (`direct`) the fusion
// rule has a single voter, so the output is the local estimates themselves in
// ascending label order: each warp places its label after the selected labels
// below it, and the count is the selection's size.
template <class R>
__global__ void __launch_bounds__(256) k_est_local(Dev d, Model m, bool direct, R* out_states, int* out_labels,
                                                   int cap, int* d_count) {
  pdl_enter();
  __shared__ int pref[kMaxPE + 1];
  const int K = m.K;
  item_prefix(d.n_pred, K, pref, m.tune.c_tile);
  St4<R>* est = static_cast<St4<R>*>(d.est_local);
  const int lane = threadIdx.x & 31;
  const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
  const long total = (long)K * m.m_max;
  for (long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < total; gw += nwarps) {
    const int j = (int)(gw / m.m_max);
    const int r = (int)(gw - (long)j * m.m_max);
    const int nsel = d.nsel[j];
    if (direct && r == 0 && lane == 0) {
      *d.out_count = nsel;
      if (d_count) *d_count = nsel;
    }
    if (r >= nsel) continue;   // uniform over the warp
    // the label's measurement, fetched ahead of the partials
    const int p = d.sel[j * m.m_max + r];
    int below = 0;
    if (direct) {
      for (int t = lane; t < nsel; t += 32) below += d.sel[j * m.m_max + t] < p ? 1 : 0;
      below = __reduce_add_sync(0xffffffffu, below);
    }
    const V2<R> z = slice_Z<R>(d, j)[p];
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
#pragma unroll 4
    for (int it = pref[j] + lane; it < pref[j + 1]; it += 32) {
      const double* q = d.spart + ((long)it * m.m_max + r) * 5;
      a0 += q[0];
      a1 += q[1];
      a2 += q[2];
      a3 += q[3];
      a4 += q[4];
    }
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_down_sync(0xffffffffu, a0, o);
      a1 += __shfl_down_sync(0xffffffffu, a1, o);
      a2 += __shfl_down_sync(0xffffffffu, a2, o);
      a3 += __shfl_down_sync(0xffffffffu, a3, o);
      a4 += __shfl_down_sync(0xffffffffu, a4, o);
    }
    if (lane == 0) {
      R px, py;
      meas_point<R>(m, z, px, py);
      St4<R> o;
      if (a0 > 0.0) {
        if constexpr (sizeof(R) == 4) {
          // the offsets from the label's point are small: FP32 suffices
          const float inv = 1.0f / (float)a0;
          o.x = px + (float)a1 * inv;
          o.vx = (float)a2 * inv;
          o.y = py + (float)a3 * inv;
          o.vy = (float)a4 * inv;
        } else {
          o.x = (R)((double)px + a1 / a0);
          o.vx = (R)(a2 / a0);
          o.y = (R)((double)py + a3 / a0);
          o.vy = (R)(a4 / a0);
        }
      } else {
        o = St4<R>{px, (R)0, py, (R)0};
      }
      est[gw] = o;
      if (direct && below < cap) {
        reinterpret_cast<St4<R>*>(out_states)[below] = o;
        out_labels[below] = p;
      }
    }
  }
}

template <class R>
__global__ void __launch_bounds__(1024) k_fuse(Dev d, Model m, R* out_states, int* out_labels, int cap,
                                               int* d_count) {
  pdl_enter();
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
      if constexpr (sizeof(R) == 4) {
        // positions as offsets from the label's measurement point, FP32 sums
        // and scale (as the fused CU)
        R px, py;
        meas_point<R>(m, slice_Z<R>(d, 0)[p], px, py);
        float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int j = 0; j < K; ++j) {
          const int r = d.selrank[j * m.m_max + p];
          if (r >= 0) {
            const St4<R> e = est[j * m.m_max + r];
            a0 += e.x - px;
            a1 += e.vx;
            a2 += e.y - py;
            a3 += e.vy;
          }
        }
        const float iv = 1.0f / (float)votes;
        out[idx] = St4<R>{px + a0 * iv, a1 * iv, py + a2 * iv, a3 * iv};
      } else {
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
      }
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

// Independent runs (a batch): run j's estimates are its local estimates, in
// ascending label order (the fusion rule with one voter).  One CTA per run.
template <class R>
__global__ void __launch_bounds__(1024) k_batch_out(Dev d, Model m, R* out_states, int* out_labels, int* counts,
                                                    int cap) {
  pdl_enter();
  __shared__ int wsum[32];
  __shared__ int carry_s;
  const int j = blockIdx.x;
  const int M = slice_M(d, j);
  const St4<R>* est = static_cast<const St4<R>*>(d.est_local);
  St4<R>* out = reinterpret_cast<St4<R>*>(out_states) + (long)j * cap;
  int* lab = out_labels + (long)j * cap;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int p0 = 0; p0 < M; p0 += blockDim.x) {
    const int p = p0 + threadIdx.x;
    const int r = p < M ? d.selrank[j * m.m_max + p] : -1;
    const int valid = r >= 0 ? 1 : 0;
    int incl = valid;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int v = lane < nw ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (lane < nw) wsum[lane] = v;
    }
    __syncthreads();
    const int carry = carry_s;
    const int idx = carry + (wid > 0 ? wsum[wid - 1] : 0) + incl - valid;
    if (valid && idx < cap) {
      out[idx] = est[j * m.m_max + r];
      lab[idx] = p;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + wsum[nw - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[j] = carry_s;
}

template <class R>
cudaError_t launch_batch_out(const Dev& d, const Model& m, R* out_states, int* out_labels, int* counts, int cap,
                             cudaStream_t s) {
  launch_k(k_batch_out<R>, dim3(m.K), dim3(1024), 0, s, d, m, out_states, out_labels, counts, cap);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_extract(const Dev& d, const Model& m, R* out_states, int* out_labels, int cap,
                           int* d_count, cudaStream_t s) {
  {
    const long items = (long)m.K * ((m.pe_cap + m.tune.c_tile - 1) / m.tune.c_tile);
    const int g = (int)(items < 152L * 8 ? (items > 0 ? items : 1) : 152L * 8);
    const size_t smem = (sizeof(P4<R>) + sizeof(St4<R>)) * (size_t)m.tune.c_tile + sizeof(int) * (size_t)m.m_max;
    switch (model_flag(m)) {
      case 1: launch_k(k_selsum<R, 1>, dim3(g), dim3(kThreads), smem, s, d, m); break;
      case 2: launch_k(k_selsum<R, 2>, dim3(g), dim3(kThreads), smem, s, d, m); break;
      case 3: launch_k(k_selsum<R, 3>, dim3(g), dim3(kThreads), smem, s, d, m); break;
      default: launch_k(k_selsum<R, 0>, dim3(g), dim3(kThreads), smem, s, d, m); break;
    }
  }
  long warps = (long)m.K * m.m_max;
  int b = (int)((warps + 7) / 8);
  if (b > 152 * 8) b = 152 * 8;
  const bool direct = d.zshared && m.K == 1;
  launch_k(k_est_local<R>, dim3(b), dim3(256), 0, s, d, m, direct, out_states, out_labels, cap, d_count);
  if (d.zshared && !direct)
    launch_k(k_fuse<R>, dim3(1), dim3(1024), 0, s, d, m, out_states, out_labels, cap, d_count);
  return cudaGetLastError();
}

template cudaError_t launch_batch_out<float>(const Dev&, const Model&, float*, int*, int*, int, cudaStream_t);
template cudaError_t launch_batch_out<double>(const Dev&, const Model&, double*, int*, int*, int, cudaStream_t);
template <class R>
cudaError_t launch_select(const Dev& d, const Model& m, cudaStream_t s) {
  launch_k(k_select<R>, dim3(m.K, (m.m_max + 63) / 64), dim3(256), sizeof(unsigned long long) * (size_t)m.m_max, s,
           d, m);
  return cudaGetLastError();
}
template cudaError_t launch_select<float>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_select<double>(const Dev&, const Model&, cudaStream_t);

template <class R>
cudaError_t launch_fuse(const Dev& d, const Model& m, R* out_states, int* out_labels, int cap, int* d_count,
                        cudaStream_t s) {
  launch_k(k_fuse<R>, dim3(1), dim3(1024), 0, s, d, m, out_states, out_labels, cap, d_count);
  return cudaGetLastError();
}
template cudaError_t launch_fuse<float>(const Dev&, const Model&, float*, int*, int, int*, cudaStream_t);
template cudaError_t launch_fuse<double>(const Dev&, const Model&, double*, int*, int, int*, cudaStream_t);

template cudaError_t launch_extract<float>(const Dev&, const Model&, float*, int*, int, int*, cudaStream_t);
template cudaError_t launch_extract<double>(const Dev&, const Model&, double*, int*, int, int*, cudaStream_t);

}  // namespace phd

namespace phd {
template <class R>
cudaError_t prepare_extract() {
  const int sm = (int)((sizeof(P4<R>) + sizeof(St4<R>)) * 1024 + sizeof(int) * kMaxM);
  cudaError_t e = cudaFuncSetAttribute(k_selsum<R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_selsum<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_selsum<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_selsum<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}
template cudaError_t prepare_extract<float>();
template cudaError_t prepare_extract<double>();
}  // namespace phd
