// Resampling (Sec. 2.2 step 3; Algorithm 1 "Resample", Step 5) and the ring
// exchange (Step 6).
//
// Systematic resampling on an exact integer-valued CDF, per PE j:
//   plan (k_select, the update's last kernel): N^j = sum_i w_i (FP64, fixed order),
//               e with max w < 2^e, c = ceil(log2 n), s = 52 - c - e,
//               L_j = min(pe_cap - J_j, round((rho / K) max(1, N^j))).
//   k_rs_q / k_rs_off: q_i = floor(w_i 2^s) (exact, from the float's bits),
//               chunk totals and their exclusive scan.  Every Q_i < 2^52 is
//               an exact FP64 integer, so the prefix is accumulated in 64-bit
//               integers, which gives the same values as FP64 and cannot
//               depend on the summation order.
//   k_rs_count: Q_i = chunk offset + in-chunk prefix; c_i = #{t : T_t < Q_i}
//               with T_t = floor((t 2^32 + U) Q_n / (L 2^32)), in closed form
//               with 128-bit integers: V = floor((Q_i L 2^32 - 1) / Q_n) (one
//               multiply by the reciprocal of Q_n that k_rs_off prepares),
//               c_i = min(L, V < U ? 0 : ((V - U) >> 32) + 1).  Child t's
//               parent is then the least i with c_i > t, i.e. the least i
//               with Q_i > T_t.
//   k_rs_gather: one thread per child: binary search of c, copy the parent's
//               predicted state into the current set, weight N^j / L_j.
// Ring exchange (K > 1): L_x = floor(frac min_j L_j); PE j takes the first L_x
// entries of a Fisher-Yates shuffle of its L_j slots (r = t + floor(u_t
// (L_j - t) / 2^32)); the particles in PE j's slots move, through an outbox,
// into the slots PE j+1 chose, so slice sizes and the union of particles are
// unchanged.
#include "phd_internal.cuh"

namespace phd {

// Exact CDF in three passes over chunks of kChunk particles (any PE size):
// chunk totals of q_i = floor(w_i 2^s), an exclusive scan of the totals per
// PE, then every chunk rescans its own q_i and turns Q_i into offspring ends.
template <class R>
__global__ void __launch_bounds__(kChunk) k_rs_q(Dev d, Model m) {
  pdl_enter();
  __shared__ int pref[kMaxPE + 1];
  __shared__ unsigned long long wt[32];
  item_prefix(d.n_pred, m.K, pref, kChunk);
  const R* wu = static_cast<const R*>(d.wu);
  for (int c = blockIdx.x; c < pref[m.K]; c += gridDim.x) {
    const int j = item_pe(pref, m.K, c);
    const int i = (c - pref[j]) * kChunk + threadIdx.x;
    const unsigned long long q = i < d.n_pred[j] ? scaled_floor(wu[(long)j * m.pe_cap + i], d.rs_s[j]) : 0ull;
    unsigned long long tot = 0;
    block_scan_u64<R>(q, wt, &tot);
    if (threadIdx.x == 0) d.csum[c] = tot;
  }
}

__global__ void __launch_bounds__(1024) k_rs_off(Dev d, Model m) {
  pdl_enter();
  __shared__ int pref[kMaxPE + 1];
  __shared__ unsigned long long wt[32];
  const int j = blockIdx.x;
  item_prefix(d.n_pred, m.K, pref, kChunk);
  unsigned long long carry = 0ull;
  for (int c0 = pref[j]; c0 < pref[j + 1]; c0 += blockDim.x) {
    const int c = c0 + threadIdx.x;
    const unsigned long long v = c < pref[j + 1] ? d.csum[c] : 0ull;
    unsigned long long tot = 0;
    const unsigned long long incl = block_scan_u64<float>(v, wt, &tot);
    if (c < pref[j + 1]) d.coff[c] = carry + incl - v;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    d.rs_Qn[j] = carry;
    const Recip r = make_recip(carry);
    d.rs_rcp[2 * j] = r.d;
    d.rs_rcp[2 * j + 1] = r.v;
  }
}

template <class R>
__global__ void __launch_bounds__(kChunk) k_rs_count(Dev d, Model m, const uint32_t* __restrict__ u) {
  pdl_enter();
  __shared__ int pref[kMaxPE + 1];
  __shared__ unsigned long long wt[32];
  item_prefix(d.n_pred, m.K, pref, kChunk);
  const R* wu = static_cast<const R*>(d.wu);
  const unsigned long long st = *d.step;
  for (int c = blockIdx.x; c < pref[m.K]; c += gridDim.x) {
    const int j = item_pe(pref, m.K, c);
    const int i = (c - pref[j]) * kChunk + threadIdx.x;
    const long g = (long)j * m.pe_cap + i;
    const bool live = i < d.n_pred[j];
    const unsigned long long q = live ? scaled_floor(wu[g], d.rs_s[j]) : 0ull;
    const unsigned long long Qi = d.coff[c] + block_scan_u64<R>(q, wt, nullptr);
    if (live) {
      const uint32_t U = u ? u[j] : philox_u32(m, (uint32_t)j, st, kTagResample);
      const unsigned long long Qn = d.rs_Qn[j];
      const Recip rq{d.rs_rcp[2 * j], d.rs_rcp[2 * j + 1], Qn ? __clzll((long long)Qn) : 0};
      d.child_end[g] = offspring_end(Qi, Qn, (unsigned long long)d.rs_L[j], U, rq);
    }
  }
}

// Scatter by parent, a warp per 32 consecutive parents: parent i of PE j has
// children child_end[i-1] .. child_end[i]-1 (parents in order, children in
// order); the warp writes its parents' children as one contiguous range,
// lane by lane (coalesced), each child finding its parent among the warp's
// 32 by a shuffle search and taking its predicted state (shuffled from the
// parent's lane) and the weight N^j / L_j.  Work items: 256-particle tiles
// of each slice.
template <class R>
__global__ void __launch_bounds__(256) k_rs_gather(Dev d, Model m, bool last) {
  pdl_enter();
  __shared__ int pref[kMaxPE + 1];
  const int K = m.K;
  item_prefix(d.n_pred, K, pref);
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < K; j += blockDim.x) d.n_cur[j] = d.rs_L[j];
  // the step's last kernel advances the step counter (every reader of this
  // step's counter has completed: each kernel waits for its predecessor)
  if (last && blockIdx.x == 0 && threadIdx.x == 0) *d.step += 1ull;
  const St4<R>* xp = static_cast<const St4<R>*>(d.x_alt);
  St4<R>* x = static_cast<St4<R>*>(d.x);
  R* w = static_cast<R*>(d.w);
  const int lane = threadIdx.x & 31;
  for (int item = blockIdx.x; item < pref[K]; item += gridDim.x) {
    const int j = item_pe(pref, K, item);
    const int n = d.n_pred[j];
    const int L = d.rs_L[j];
    if (L == 0) continue;   // uniform over the block
    const int wb = (item - pref[j]) * kTile + (threadIdx.x & ~31);   // the warp's first parent
    if (wb >= n) continue;   // uniform over the warp
    const long base = (long)j * m.pe_cap;
    const int i = wb + lane;
    const bool live = i < n;
    const int ce = d.child_end[base + (live ? i : n - 1)];
    const int c0 = __shfl_sync(0xffffffffu, wb > 0 ? d.child_end[base + wb - 1] : 0, 0);
    const int c1 = __shfl_sync(0xffffffffu, ce, 31);
    const St4<R> s = live ? xp[base + i] : St4<R>{0, 0, 0, 0};
    const R wn = (R)d.rs_wn[j];
    for (int t0 = c0; t0 < c1; t0 += 32) {
      const int t = t0 + lane;
      // smallest lane k with child_end > t (lanes past the slice repeat the last end)
      int lo = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int e = __shfl_sync(0xffffffffu, ce, lo + step - 1);
        if (e <= t) lo += step;
      }
      const R sx = __shfl_sync(0xffffffffu, s.x, lo), svx = __shfl_sync(0xffffffffu, s.vx, lo);
      const R sy = __shfl_sync(0xffffffffu, s.y, lo), svy = __shfl_sync(0xffffffffu, s.vy, lo);
      if (t < c1) {
        x[base + t] = St4<R>{sx, svx, sy, svy};
        w[base + t] = wn;
        d.parent[base + t] = wb + lo;
      }
    }
  }
}

// Ring exchange plan: L_x = floor(frac min_j L_j); PE j's slots are the first
// L_x entries of a partial Fisher-Yates shuffle of 0..L_j-1.
__global__ void k_xplan(Dev d, Model m, const uint32_t* __restrict__ xu) {
  pdl_enter();
  extern __shared__ int perm[];
  __shared__ double msm[kMaxPE];
  __shared__ int lx_s;
  const int j = blockIdx.x;
  const int n = d.rs_L[j];
  if (threadIdx.x < 32) {
    const int c = exchange_count_warp(d, m, msm);
    if (threadIdx.x == 0) lx_s = c;
  }
  __syncthreads();
  const int lx = lx_s;
  if (j == 0 && threadIdx.x == 0) *d.lx = lx;
  if (lx <= 0) return;
  // perm in the first n ints, the (independent) draws after it; swaps serial
  unsigned int* ud = reinterpret_cast<unsigned int*>(perm + n);
  const unsigned long long st = *d.step;
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = i;
  for (int t = threadIdx.x; t < lx; t += blockDim.x)
    ud[t] = xu ? xu[(long)j * m.pe_cap + t] : philox_u32(m, (uint32_t)((long)j * m.pe_cap + t), st, kTagExchange);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 0; t < lx; ++t) {
      const uint32_t u = ud[t];
      const int r = t + (int)(((unsigned long long)u * (unsigned long long)(n - t)) >> 32);
      const int tmp = perm[t];
      perm[t] = perm[r];
      perm[r] = tmp;
      d.xslots[(long)j * m.pe_cap + t] = perm[t];
    }
  }
}

// Outgoing particle-weight couples of each PE into the outbox.
template <class R>
__global__ void k_xout(Dev d, Model m) {
  pdl_enter();
  const St4<R>* x = static_cast<const St4<R>*>(d.x);
  const R* w = static_cast<const R*>(d.w);
  St4<R>* xo = static_cast<St4<R>*>(d.x_out);
  R* wo = static_cast<R*>(d.w_out);
  const int lx = *d.lx;
  const long total = (long)m.K * lx;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
    const int j = (int)(g / lx);
    const int t = (int)(g - (long)j * lx);
    const long src = (long)j * m.pe_cap + d.xslots[(long)j * m.pe_cap + t];
    xo[(long)j * m.pe_cap + t] = x[src];
    wo[(long)j * m.pe_cap + t] = w[src];
  }
}

// PE j's chosen slots receive the outboxes of its sources (exchange_source).
template <class R>
__global__ void k_xin(Dev d, Model m) {
  pdl_enter();
  if (blockIdx.x == 0 && threadIdx.x == 0) *d.step += 1ull;   // the step's last kernel
  St4<R>* x = static_cast<St4<R>*>(d.x);
  R* w = static_cast<R*>(d.w);
  const St4<R>* xo = static_cast<const St4<R>*>(d.x_out);
  const R* wo = static_cast<const R*>(d.w_out);
  const int lx = *d.lx;
  const long total = (long)m.K * lx;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
    const int j = (int)(g / lx);
    const int t = (int)(g - (long)j * lx);
    const int from = exchange_source(m, j, t);
    const long dst = (long)j * m.pe_cap + d.xslots[(long)j * m.pe_cap + t];
    x[dst] = xo[(long)from * m.pe_cap + t];
    w[dst] = wo[(long)from * m.pe_cap + t];
  }
}

template <class R>
cudaError_t launch_resample(const Dev& d, const Model& m, const uint32_t* u, const uint32_t* xu,
                            cudaStream_t s) {
  const long total = (long)m.K * m.pe_cap;
  int b = (int)((total + 255) / 256);
  if (b > 152 * 16) b = 152 * 16;
  const long chunks = (long)m.K * ((m.pe_cap + kChunk - 1) / kChunk);
  const int gc = (int)(chunks < 152L * 2 ? (chunks > 0 ? chunks : 1) : 152L * 2);
  launch_k(k_rs_q<R>, dim3(gc), dim3(kChunk), 0, s, d, m);
  launch_k(k_rs_off, dim3(m.K), dim3(1024), 0, s, d, m);
  launch_k(k_rs_count<R>, dim3(gc), dim3(kChunk), 0, s, d, m, u);
  const long gitems = (long)m.K * ((m.pe_cap + kTile - 1) / kTile);
  const bool xchg = m.K > 1 && m.exchange_frac > 0.0;
  launch_k(k_rs_gather<R>, dim3((int)(gitems < 152 * 16 ? (gitems > 0 ? gitems : 1) : 152 * 16)), dim3(256), 0, s, d, m,
           !xchg);
  if (xchg) return launch_exchange<R>(d, m, xu, s);
  return cudaGetLastError();
}

// Step 6 on the resampled slices: plan, outboxes, receivers; the last kernel
// advances the step counter.
template <class R>
cudaError_t launch_exchange(const Dev& d, const Model& m, const uint32_t* xu, cudaStream_t s) {
  int bx = (int)(((long)m.K * (long)(m.exchange_frac * m.pe_cap) + 255) / 256);
  if (bx < 1) bx = 1;
  if (bx > 152 * 8) bx = 152 * 8;
  launch_k(k_xplan, dim3(m.K), dim3(256), sizeof(int) * 2 * (size_t)m.pe_cap, s, d, m, xu);
  launch_k(k_xout<R>, dim3(bx), dim3(256), 0, s, d, m);
  launch_k(k_xin<R>, dim3(bx), dim3(256), 0, s, d, m);
  return cudaGetLastError();
}
template cudaError_t launch_exchange<float>(const Dev&, const Model&, const uint32_t*, cudaStream_t);
template cudaError_t launch_exchange<double>(const Dev&, const Model&, const uint32_t*, cudaStream_t);

cudaError_t prepare_exchange(const Model& m) {
  return cudaFuncSetAttribute(k_xplan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(int) * 2 * (size_t)m.pe_cap));
}

template cudaError_t launch_resample<float>(const Dev&, const Model&, const uint32_t*, const uint32_t*, cudaStream_t);
template cudaError_t launch_resample<double>(const Dev&, const Model&, const uint32_t*, const uint32_t*, cudaStream_t);

}  // namespace phd
