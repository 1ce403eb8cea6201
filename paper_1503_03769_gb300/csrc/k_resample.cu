// Resampling (Sec. 2.2 step 3; Algorithm 1 "Resample", Step 5) and the ring
// exchange (Step 6).
//
// Systematic resampling on an exact integer-valued CDF, per PE j:
//   k_rs_mass : N^j = sum_i w_i (FP64, fixed order), e with max w < 2^e,
//               c = ceil(log2 n), s = 52 - c - e,
//               L_j = min(pe_cap - J_j, round((rho / K) max(1, N^j))).
//   k_rs_scan : q_i = floor(w_i 2^s) (an FP64 power-of-two scaling then
//               floor: exact), Q_i = q_0 + ... + q_i.  Every Q_i < 2^52 is an
//               exact FP64 integer, so the prefix is accumulated in 64-bit
//               integers, which gives the same values as FP64 and cannot
//               depend on the summation order.
//   k_rs_count: c_i = #{t : T_t < Q_i} with T_t = floor((t 2^32 + U) Q_n /
//               (L 2^32)), in closed form with 128-bit integers:
//               V = floor((Q_i L 2^32 - 1) / Q_n), c_i = min(L, V < U ? 0 :
//               ((V - U) >> 32) + 1).  Child t's parent is then the least i
//               with c_i > t, i.e. the least i with Q_i > T_t.
//   k_rs_gather: one thread per child: binary search of c, copy the parent's
//               predicted state into the current set, weight N^j / L_j.
// Ring exchange (K > 1): L_x = floor(frac min_j L_j); PE j takes the first L_x
// entries of a Fisher-Yates shuffle of its L_j slots (r = t + floor(u_t
// (L_j - t) / 2^32)); the particles in PE j's slots move, through an outbox,
// into the slots PE j+1 chose, so slice sizes and the union of particles are
// unchanged.
#include "phd_internal.cuh"

namespace phd {

template <class R>
__global__ void __launch_bounds__(256) k_rs_mass(Dev d, Model m) {
  __shared__ double rs[8], rm[8];
  const int j = blockIdx.x;
  const int n = d.n_pred[j];
  const R* w = static_cast<const R*>(d.wu) + (long)j * m.pe_cap;
  // FP32 runs of 64 weights per thread, FP64 across runs and threads
  double s = 0.0;
  R run = 0, mxr = 0;
  int k = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const R v = w[i];
    run += v;
    mxr = v > mxr ? v : mxr;
    if (++k == 64) {
      s += (double)run;
      run = 0;
      k = 0;
    }
  }
  s += (double)run;
  double mx = (double)mxr;
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    rs[threadIdx.x >> 5] = s;
    rm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double N = 0.0, wmax = 0.0;
    for (int k = 0; k < 8; ++k) {
      N += rs[k];
      wmax = fmax(wmax, rm[k]);
    }
    int L, sc;
    resample_plan(m, j, n, N, wmax, L, sc);
    d.rs_mass[j] = N;
    d.rs_s[j] = sc;
    d.rs_L[j] = L;
  }
}

template <class R>
__global__ void __launch_bounds__(1024) k_rs_scan(Dev d, Model m) {
  constexpr int IT = 4;
  __shared__ unsigned long long wtot[32];
  __shared__ unsigned long long carry_s;
  const int j = blockIdx.x;
  const int n = d.n_pred[j];
  const int s = d.rs_s[j];
  const R* w = static_cast<const R*>(d.wu) + (long)j * m.pe_cap;
  unsigned long long* Q = d.Q + (long)j * m.pe_cap;
  if (threadIdx.x == 0) carry_s = 0ull;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c0 = 0; c0 < n; c0 += 1024 * IT) {
    unsigned long long q[IT];
    unsigned long long run = 0ull;
#pragma unroll
    for (int k = 0; k < IT; ++k) {
      const int i = c0 + threadIdx.x * IT + k;
      q[k] = i < n ? scaled_floor(w[i], s) : 0ull;
      run += q[k];
      q[k] = run;
    }
    unsigned long long incl = run;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      unsigned long long v = wtot[lane];
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      wtot[lane] = v;
    }
    __syncthreads();
    const unsigned long long off = carry_s + (wid > 0 ? wtot[wid - 1] : 0ull) + (incl - run);
#pragma unroll
    for (int k = 0; k < IT; ++k) {
      const int i = c0 + threadIdx.x * IT + k;
      if (i < n) Q[i] = off + q[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_s += wtot[31];
    __syncthreads();
  }
}

__global__ void k_rs_count(Dev d, Model m, const uint32_t* __restrict__ u) {
  const long total = (long)m.K * m.pe_cap;
  const unsigned long long st = *d.step;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
    const int j = (int)(g / m.pe_cap);
    const int i = (int)(g - (long)j * m.pe_cap);
    const int n = d.n_pred[j];
    if (i >= n) continue;
    const uint32_t U = u ? u[j] : philox_u32(m, (uint32_t)j, st, kTagResample);
    d.child_end[g] = offspring_end(d.Q[g], d.Q[(long)j * m.pe_cap + n - 1], (unsigned long long)d.rs_L[j], U);
  }
}

// Children t < L_j of PE j: parent = least i with child_end[i] > t; the
// predicted state is gathered into the current set with weight N^j / L_j.
template <class R>
__global__ void k_rs_gather(Dev d, Model m) {
  const St4<R>* xp = static_cast<const St4<R>*>(d.x_alt);
  St4<R>* x = static_cast<St4<R>*>(d.x);
  R* w = static_cast<R*>(d.w);
  const long total = (long)m.K * m.pe_cap;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
    const int j = (int)(g / m.pe_cap);
    const int t = (int)(g - (long)j * m.pe_cap);
    const int L = d.rs_L[j];
    if (t == 0) d.n_cur[j] = L;
    if (t >= L) continue;
    const long base = (long)j * m.pe_cap;
    int lo = 0, hi = d.n_pred[j] - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (d.child_end[base + mid] > t) hi = mid; else lo = mid + 1;
    }
    x[g] = xp[base + lo];
    w[g] = (R)(d.rs_mass[j] / (double)L);
    d.parent[g] = lo;
  }
}

// Ring exchange plan: L_x = floor(frac min_j L_j); PE j's slots are the first
// L_x entries of a partial Fisher-Yates shuffle of 0..L_j-1.
__global__ void k_xplan(Dev d, Model m, const uint32_t* __restrict__ xu) {
  extern __shared__ int perm[];
  const int j = blockIdx.x;
  const int K = m.K;
  const int n = d.rs_L[j];
  int nmin = d.rs_L[0];
  for (int k = 1; k < K; ++k) nmin = min(nmin, d.rs_L[k]);
  const int lx = (int)floor(m.exchange_frac * (double)nmin);
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

// PE j's chosen slots receive PE j-1's outbox (ring).
template <class R>
__global__ void k_xin(Dev d, Model m) {
  St4<R>* x = static_cast<St4<R>*>(d.x);
  R* w = static_cast<R*>(d.w);
  const St4<R>* xo = static_cast<const St4<R>*>(d.x_out);
  const R* wo = static_cast<const R*>(d.w_out);
  const int lx = *d.lx;
  const long total = (long)m.K * lx;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
    const int j = (int)(g / lx);
    const int t = (int)(g - (long)j * lx);
    const int from = (j + m.K - 1) % m.K;
    const long dst = (long)j * m.pe_cap + d.xslots[(long)j * m.pe_cap + t];
    x[dst] = xo[(long)from * m.pe_cap + t];
    w[dst] = wo[(long)from * m.pe_cap + t];
  }
}

__global__ void k_advance(Dev d) { *d.step += 1ull; }

template <class R>
cudaError_t launch_resample(const Dev& d, const Model& m, const uint32_t* u, const uint32_t* xu,
                            cudaStream_t s) {
  const long total = (long)m.K * m.pe_cap;
  int b = (int)((total + 255) / 256);
  if (b > 152 * 16) b = 152 * 16;
  k_rs_mass<R><<<m.K, 256, 0, s>>>(d, m);
  k_rs_scan<R><<<m.K, 1024, 0, s>>>(d, m);
  k_rs_count<<<b, 256, 0, s>>>(d, m, u);
  k_rs_gather<R><<<b, 256, 0, s>>>(d, m);
  if (m.K > 1 && m.exchange_frac > 0.0) {
    int bx = (int)(((long)m.K * (long)(m.exchange_frac * m.pe_cap) + 255) / 256);
    if (bx < 1) bx = 1;
    if (bx > 152 * 8) bx = 152 * 8;
    k_xplan<<<m.K, 256, sizeof(int) * 2 * (size_t)m.pe_cap, s>>>(d, m, xu);
    k_xout<R><<<bx, 256, 0, s>>>(d, m);
    k_xin<R><<<bx, 256, 0, s>>>(d, m);
  }
  return cudaGetLastError();
}

cudaError_t launch_advance_step(const Dev& d, cudaStream_t s) {
  k_advance<<<1, 1, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t prepare_exchange(const Model& m) {
  return cudaFuncSetAttribute(k_xplan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(int) * 2 * (size_t)m.pe_cap));
}

template cudaError_t launch_resample<float>(const Dev&, const Model&, const uint32_t*, const uint32_t*, cudaStream_t);
template cudaError_t launch_resample<double>(const Dev&, const Model&, const uint32_t*, const uint32_t*, cudaStream_t);

}  // namespace phd
