// Fused filter step: one cooperative launch runs S whole steps (Algorithm 1)
// with one CTA per processing element.
//
// Each PE (CTA j, 1024 threads) keeps its predicted slice in shared memory
// for the step: states, the sensor-space geometry h(x) and the weights.  The
// stages are the staged path's, in order, separated by __syncthreads:
//   predict (Eq. 5-6)       current set (global) -> predicted slice (smem + x_alt)
//   pass 1 (Eq. 7)          C^j_p: threads own (measurement, particle split)
//   [GLOBAL mode]           grid barrier, C_p = mean over PEs
//   pass 2 (Eq. 8)          updated weights, mass N^j and max weight
//   selection (Step 3)      LT_j = round(N^j), rank counting over dW^{j,p}
//   pass 3 (Eq. 18)         labelled sums for the selected labels -> zeta
//   resampling (Step 5)     exact integer CDF scan, offspring counts, gather
//   grid barrier            all L_j, masses and local estimates visible
//   exchange plan (Step 6)  L_x (or 0 when the adaptive trigger holds off),
//                           Fisher-Yates slots by one lane while the other
//                           warps fuse their share of the labels (Step 4),
//                           outgoing couples to the outbox
//   grid barrier
//   exchange in             PE j's slots take their sources' outboxes (ring:
//                           PE j-1; all-to-all: a rotation per slot)
// The only cross-PE waits are the two (three) grid barriers the scheme needs:
// the exchange count and the CU fusion depend on every PE.  Barriers poll
// with an iteration limit; on expiry the kernel records kErrTimeout and every
// CTA returns.  All arithmetic matches the staged kernels (same helpers), but
// reductions run in a different fixed order.
#include "phd_internal.cuh"

namespace phd {

constexpr int kFusedThreads = 1024;

struct FusedArgs {
  const void* Z;            // packed measurements of S steps
  const int* zoff;          // [S+1] row offsets into Z, or NULL for one step of M1 rows
  int M1;
  const void* noise;        // injected predict draws (S == 1) or NULL
  const uint32_t* u;        // injected resampling uniforms (S == 1) or NULL
  const uint32_t* xu;       // injected exchange draws (S == 1) or NULL
  void* out_states;         // [S][cap][4] fused estimates
  int* out_labels;          // [S][cap]
  int* out_count;           // [S]
  int cap;
  int S;
};

// Shared-memory layout of the fused kernel (bytes), for pe_cap P and m_max Mm.
struct FusedSmem {
  size_t sx, sh0, sh1, shl, sw, swu, zs, ginv, Cd, Cu, dW, sel, selrank, red, total;
};

template <class R>
__host__ __device__ inline FusedSmem fused_smem(int P, int Mm) {
  FusedSmem L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = (o + 31) & ~(size_t)31;
    o = at + bytes;
    return at;
  };
  L.sx = take(sizeof(St4<R>) * P);
  // sh0..sw are reused for the resampling CDF (8 B), offspring ends (4 B) and
  // the Fisher-Yates permutation (4 B) once the pair passes are done
  const size_t per = (4 * sizeof(R) > 16 ? 4 * sizeof(R) : 16);
  const size_t blk = take(per * P);
  L.sh0 = blk;
  L.sh1 = blk + sizeof(R) * P;
  L.shl = blk + 2 * sizeof(R) * P;
  L.sw = blk + 3 * sizeof(R) * P;
  L.swu = take(sizeof(R) * P);
  L.zs = take(sizeof(V2<R>) * Mm);
  L.ginv = take(sizeof(R) * Mm);
  L.Cd = take(sizeof(double) * Mm);
  L.Cu = take(sizeof(double) * Mm);
  L.dW = take(sizeof(unsigned long long) * Mm);
  L.sel = take(sizeof(int) * Mm);
  L.selrank = take(sizeof(int) * Mm);
  L.red = take(sizeof(double) * kFusedThreads);
  L.total = (o + 31) & ~(size_t)31;
  return L;
}

__device__ __forceinline__ int pow2_floor(int v) {
  int p = 1;
  while (p * 2 <= v) p *= 2;
  return p;
}

// The three block reductions after pass 2 with two barriers: the mass N^j
// (within each warp in R, the 32 warp totals in FP64 by warp 0 in a fixed
// order; in FP32 mode the FP64 work is 5 shuffle-adds in one warp), the
// largest weight, and the count of measurements with dW > 0.  wred: 64 reals,
// ired: 32 ints (distinct shared scratch); every thread gets all three.
template <class R>
__device__ __forceinline__ void block_mass_stats(R sum, R mx, int cnt, R* wred, int* ired, double* bN, double& N,
                                                 R& wmax, int& npos) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_down_sync(0xffffffffu, sum, o);
    const R u = __shfl_down_sync(0xffffffffu, mx, o);
    mx = u > mx ? u : mx;
  }
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) {
    wred[wid] = sum;
    wred[32 + wid] = mx;
    ired[wid] = cnt;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < nw ? (double)wred[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) *bN = t;
  }
  R m = 0;
  int c = 0;
  for (int k = 0; k < nw; ++k) {
    m = wred[32 + k] > m ? wred[32 + k] : m;
    c += ired[k];
  }
  __syncthreads();
  N = *bN;
  wmax = m;
  npos = c;
}

// Cartesian point of a measurement (offset origin of the labelled sums).
template <class R>
__device__ __forceinline__ void meas_point_f(const Cst<R>& c, int rb, V2<R> z, R& rx, R& ry) {
  if (rb == 0) {
    rx = z.a;
    ry = z.b;
  } else {
    R sn, cs;
    sincos(z.b, &sn, &cs);
    rx = c.sx + z.a * cs;
    ry = c.sy + z.a * sn;
  }
}

// CU fusion of one step by one CTA (Step 4): labels taken by more than K/2
// PEs, FP64 mean of their local states, ascending label order.
// Mean of the voters' local states, in PE order.  FP32: positions as offsets
// from the label's measurement point (close values subtract exactly; the
// point's own rounding cancels), summed and scaled in FP32, with loads that
// do not wait on one another; FP64: plain sums and divides.
template <class R>
__device__ __forceinline__ St4<R> fuse_mean(const St4<R>* __restrict__ est, const int* srank, int Pc, int q, int K,
                                            int m_max, int votes, R px, R py) {
  if constexpr (sizeof(R) == 4) {
    R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    constexpr int U = 8;   // PEs' states in flight per thread
    for (int k0 = 0; k0 < K; k0 += U) {
      St4<R> e[U];
      bool v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = k0 + u < K ? srank[(k0 + u) * Pc + q] : -1;
        v[u] = r >= 0;
        e[u] = v[u] ? est[(k0 + u) * m_max + r] : St4<R>{0, 0, 0, 0};
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (v[u]) {
          a0 += e[u].x - px;
          a1 += e[u].vx;
          a2 += e[u].y - py;
          a3 += e[u].vy;
        }
      }
    }
    const R iv = (R)1 / (R)votes;
    return St4<R>{px + a0 * iv, a1 * iv, py + a2 * iv, a3 * iv};
  } else {
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int k = 0; k < K; ++k) {
      const int r = srank[k * Pc + q];
      if (r >= 0) {
        const St4<R> e = est[k * m_max + r];
        a0 += (double)e.x;
        a1 += (double)e.vx;
        a2 += (double)e.y;
        a3 += (double)e.vy;
      }
    }
    return St4<R>{(R)(a0 / votes), (R)(a1 / votes), (R)(a2 / votes), (R)(a3 / votes)};
  }
}

template <class R>
__device__ void cu_fuse(const Dev& d, const Model& m, int M, St4<R>* out, int* out_lab, int cap, int* count,
                        int* wsum, int* srank, int srank_cap, const V2<R>* zs, const Cst<R>& cc) {
  // Step 4 on CTA 0: the K PEs' ranks of a chunk of measurements are staged
  // in shared memory with independent loads (srank[k][q]); a label's votes
  // are counted from there and the voters' local states read in PE order.
  __shared__ int carry_s;
  const St4<R>* est = static_cast<const St4<R>*>(d.est_local);
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int K = m.K;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int chunk = srank_cap / K;
  if (chunk > (int)blockDim.x) chunk = blockDim.x;
  for (int p0 = 0; p0 < M; p0 += chunk) {
    const int Pc = min(chunk, M - p0);
    for (int idx = threadIdx.x; idx < K * Pc; idx += blockDim.x) {
      const int k = idx / Pc, q = idx - k * Pc;
      srank[idx] = d.selrank[k * m.m_max + p0 + q];
    }
    __syncthreads();
    const int q = threadIdx.x;
    const int p = p0 + q;
    int votes = 0;
    if (q < Pc)
      for (int k = 0; k < K; ++k) votes += srank[k * Pc + q] >= 0 ? 1 : 0;
    const int valid = (q < Pc && 2 * votes > K) ? 1 : 0;
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
      R px, py;
      meas_point_f<R>(cc, m.meas_model, zs[p], px, py);
      out[idx] = fuse_mean<R>(est, srank, Pc, q, K, m.m_max, votes, px, py);
      out_lab[idx] = p;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + wsum[nw - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *count = carry_s;
    *d.out_count = carry_s;
  }
  __syncthreads();
}

// Step 4 shared by the K CTAs after the grid barrier, on the CTA's threads
// tid0 .. blockDim.x - 1 (named barrier 2; warps below tid0 are busy with
// the exchange swaps): every CTA stages all PEs' ranks and counts the votes
// and the output positions of all labels, and forms the states of the valid
// labels p with p mod K == j (CTA 0 writes the count).  The voters' states
// of the CTA's own labels are fetched while the ranks are staged (one load
// per (PE, label) pair, all in flight at once), then summed per label in PE
// order as fuse_mean does.  Same output as cu_fuse on one CTA.
// Labels per chunk of cu_fuse_share in `bytes` of scratch: K ranks per label
// plus at most chunk + K states of the CTA's own labels (0: too small).
template <class R>
__device__ __forceinline__ int share_chunk(int K, size_t bytes, int NT) {
  const long need0 = 16 + (long)sizeof(St4<R>) * K;
  if ((long)bytes <= need0) return 0;
  const long c = ((long)bytes - need0) / ((long)sizeof(int) * K + (long)sizeof(St4<R>));
  return (int)(c < NT ? c : NT);
}

template <class R>
__device__ void cu_fuse_share(const Dev& d, const Model& m, int j, int M, St4<R>* out, int* out_lab, int cap,
                              int* count, int* wsum, unsigned char* scratch, int chunk, const V2<R>* zs,
                              const Cst<R>& cc, int tid0) {
  const int NT = (int)blockDim.x - tid0, lt = (int)threadIdx.x - tid0;
  const int lane = threadIdx.x & 31, lw = lt >> 5, nw = NT >> 5;
  const St4<R>* est = static_cast<const St4<R>*>(d.est_local);
  const int K = m.K;
  int* srank = reinterpret_cast<int*>(scratch);
  St4<R>* sest = reinterpret_cast<St4<R>*>(scratch + ((sizeof(int) * K * chunk + 15) & ~(size_t)15));
  int carry = 0;
  for (int p0 = 0; p0 < M; p0 += chunk) {
    const int Pc = min(chunk, M - p0);
    // own labels of the chunk: p = p0 + q with p mod K == j, i.e. q = q0 + K o
    const int q0 = ((j - p0) % K + K) % K;
    const int no = q0 < Pc ? (Pc - 1 - q0) / K + 1 : 0;
    for (int idx = lt; idx < K * Pc; idx += NT) {
      const int k = idx / Pc, q = idx - k * Pc;
      const int r = __ldcg(d.selrank + k * m.m_max + p0 + q);
      srank[idx] = r;
      if (q >= q0 && (q - q0) % K == 0 && r >= 0) sest[k * no + (q - q0) / K] = est[k * m.m_max + r];
    }
    asm volatile("bar.sync 2, %0;" ::"r"(NT));
    const int q = lt, p = p0 + q;
    int votes = 0;
    if (q < Pc)
      for (int k = 0; k < K; ++k) votes += srank[k * Pc + q] >= 0 ? 1 : 0;
    const int valid = (q < Pc && 2 * votes > K) ? 1 : 0;
    int incl = valid;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[lw] = incl;
    asm volatile("bar.sync 2, %0;" ::"r"(NT));
    if (lw == 0) {
      int v = lane < nw ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (lane < nw) wsum[lane] = v;
    }
    asm volatile("bar.sync 2, %0;" ::"r"(NT));
    const int idx = carry + (lw > 0 ? wsum[lw - 1] : 0) + incl - valid;
    if (valid && idx < cap && p % K == j) {
      R px, py;
      meas_point_f<R>(cc, m.meas_model, zs[p], px, py);
      const int o = (q - q0) / K;
      St4<R> f;
      if constexpr (sizeof(R) == 4) {
        R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int k = 0; k < K; ++k) {
          if (srank[k * Pc + q] >= 0) {
            const St4<R> e = sest[k * no + o];
            a0 += e.x - px;
            a1 += e.vx;
            a2 += e.y - py;
            a3 += e.vy;
          }
        }
        const R iv = (R)1 / (R)votes;
        f = St4<R>{px + a0 * iv, a1 * iv, py + a2 * iv, a3 * iv};
      } else {
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int k = 0; k < K; ++k) {
          if (srank[k * Pc + q] >= 0) {
            const St4<R> e = sest[k * no + o];
            a0 += (double)e.x;
            a1 += (double)e.vx;
            a2 += (double)e.y;
            a3 += (double)e.vy;
          }
        }
        f = St4<R>{(R)(a0 / votes), (R)(a1 / votes), (R)(a2 / votes), (R)(a3 / votes)};
      }
      out[idx] = f;
      out_lab[idx] = p;
    }
    carry += wsum[nw - 1];
    asm volatile("bar.sync 2, %0;" ::"r"(NT));   // srank, sest and wsum are reused
  }
  if (j == 0 && lt == 0) {
    *count = carry;
    *d.out_count = carry;
  }
}

template <class R, int RB>
__global__ void __launch_bounds__(kFusedThreads, 1) k_step_fused(Dev d, Model m, FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const FusedSmem SL = fused_smem<R>(m.pe_cap, m.m_max);
  St4<R>* sx = reinterpret_cast<St4<R>*>(smem + SL.sx);
  P4<R>* sp = reinterpret_cast<P4<R>*>(smem + SL.sh0);
  R* swu = reinterpret_cast<R*>(smem + SL.swu);
  V2<R>* zs = reinterpret_cast<V2<R>*>(smem + SL.zs);
  R* ginv = reinterpret_cast<R*>(smem + SL.ginv);
  double* Cd = reinterpret_cast<double*>(smem + SL.Cd);
  double* Cu = reinterpret_cast<double*>(smem + SL.Cu);
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem + SL.dW);
  int* sel = reinterpret_cast<int*>(smem + SL.sel);
  int* selrank = reinterpret_cast<int*>(smem + SL.selrank);
  R* wred = reinterpret_cast<R*>(smem + SL.red);
  int* ired = reinterpret_cast<int*>(smem + SL.red + 256);
  // resampling arrays alias the pair-pass block (sh0 .. sw)
  unsigned long long* Q = reinterpret_cast<unsigned long long*>(smem + SL.sh0);
  int* cend = reinterpret_cast<int*>(smem + SL.sh0 + sizeof(unsigned long long) * m.pe_cap);
  int* perm = cend + m.pe_cap;
  // CU fusion's rank scratch: the predicted states' block, free after the gather
  int* srank = reinterpret_cast<int*>(smem + SL.sx);
  const int srank_cap = (int)(sizeof(St4<R>) * m.pe_cap / sizeof(int));
  __shared__ double bN;
  __shared__ int bL, bS;
  __shared__ R bW;

  const int j = blockIdx.x;
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31;
  const long base = (long)j * m.pe_cap;
  const int Jj = births_of(m.J, m.K, j);
  const unsigned long long step0 = *d.step;
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);
  const PairQ<R, RB> PQ(m);   // pair exponent, sensor model and truncation fixed at compile time
  const Cst<R> cc = consts<R>(m);
  const R bw = birth_weight<R>(cc, m, j);
  const double cs = m.p_d * m.cnorm;
  const R csr = (R)cs;
  const R kapr = (R)m.kappa;
  St4<R>* gx = static_cast<St4<R>*>(d.x);
  R* gw = static_cast<R*>(d.w);
  St4<R>* gxp = static_cast<St4<R>*>(d.x_alt);
  R* gwp = static_cast<R*>(d.w_alt);
  R* gwu = static_cast<R*>(d.wu);
  St4<R>* gest = static_cast<St4<R>*>(d.est_local);
  const bool xchg = m.K > 1 && m.exchange_frac > 0.0;
  int n = d.n_cur[j];
  // host-injected failure: PE 0 leaves at its first grid barrier
  const bool lost = j == 0 && tid == 0 && reinterpret_cast<volatile unsigned int*>(d.bar)[2] != 0u;

  for (int s = 0; s < a.S; ++s) {
    const unsigned long long step = step0 + (unsigned long long)s;
    const int z0 = a.zoff ? a.zoff[s] : 0;
    int M = a.zoff ? a.zoff[s + 1] - z0 : a.M1;
    if (M < 0 || M > m.m_max) {
      if (tid == 0) atomicOr(d.err, kErrCapacity);
      M = 0;
    }
    const V2<R>* Zg = static_cast<const V2<R>*>(a.Z) + z0;
    for (int p = tid; p < M; p += T) {
      const V2<R> z = Zg[p];
      if (!isfinite(z.a) || !isfinite(z.b)) atomicOr(d.err, kErrNonFinite);
      zs[p] = z;
    }
    if (j == 0 && tid == 0) *d.M = M;
    // ---- predict (Eq. 5-6)
    const int np = n + Jj;
    for (int i = tid; i < np; i += T) {
      R n1, n2, u1, u2;
      draw_noise<R>(m, static_cast<const R*>(a.noise), base + i, step, n1, n2, u1, u2);
      const bool surv = i < n;
      St4<R> o;
      R wo;
      predict_slot<R>(cc, surv, surv ? gx[base + i] : St4<R>{0, 0, 0, 0}, surv ? gw[base + i] : (R)0, bw, n1, n2,
                      u1, u2, o, wo);
      gxp[base + i] = o;
      gwp[base + i] = wo;
      sx[i] = o;
      const H3<R> h = meas_h<R>(m, o, tab);
      sp[i] = P4<R>{h.h0, h.h1, h.h1lo, wo};
    }
    if (tid == 0) {
      d.n_pred[j] = np;
      atomicAdd(&d.stats[0], (unsigned long long)np * (unsigned long long)M);
      atomicAdd(&d.stats[4], (unsigned long long)np * (unsigned long long)M);
      atomicAdd(&d.stats[1], (unsigned long long)np);
      if (j == 0) {
        atomicAdd(&d.stats[2], (unsigned long long)M);
        atomicAdd(&d.stats[3], 1ull);
      }
    }
    __syncthreads();
    // ---- pass 1: C^j_p (Eq. 7).  Groups of nsplit consecutive lanes share a
    // measurement and split the particles.  Accumulation: FP32 runs of at
    // most 256 pairs per thread, the runs summed in FP64, and the nsplit
    // lanes' FP64 sums added in lane order by one thread per measurement.
    if (M > 0) {
      const int nsplit = pow2_floor(min(32, max(1, T / M)));
      const int mper = T / nsplit;
      const int pl = tid / nsplit, split = tid % nsplit;
      double* dred = reinterpret_cast<double*>(smem + SL.red);
      for (int p0 = 0; p0 < M; p0 += mper) {
        const int p = p0 + pl;
        double acc = 0.0;
        if (p < M) {
          // four independent partial sums (ILP), a run of 4 x 64 pairs each
          // time they are folded into the FP64 sum (the FP64 pipe runs ~2
          // lanes/clk/SM: one add per run)
          const V2<R> z = zs[p];
          R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
          int i = split, k = 0;
          for (; i + 3 * nsplit < np; i += 4 * nsplit) {
            const P4<R> q0 = sp[i], q1 = sp[i + nsplit], q2 = sp[i + 2 * nsplit], q3 = sp[i + 3 * nsplit];
            a0 = fma(exp2_neg(PQ(z.a, z.b, q0.h0, q0.h1, q0.h1lo)), q0.w, a0);
            a1 = fma(exp2_neg(PQ(z.a, z.b, q1.h0, q1.h1, q1.h1lo)), q1.w, a1);
            a2 = fma(exp2_neg(PQ(z.a, z.b, q2.h0, q2.h1, q2.h1lo)), q2.w, a2);
            a3 = fma(exp2_neg(PQ(z.a, z.b, q3.h0, q3.h1, q3.h1lo)), q3.w, a3);
            if (++k == 64) {
              acc += (double)((a0 + a1) + (a2 + a3));
              a0 = a1 = a2 = a3 = 0;
              k = 0;
            }
          }
          for (; i < np; i += nsplit) {
            const P4<R> q0 = sp[i];
            a0 = fma(exp2_neg(PQ(z.a, z.b, q0.h0, q0.h1, q0.h1lo)), q0.w, a0);
          }
          acc += (double)((a0 + a1) + (a2 + a3));
        }
        dred[tid] = acc;
        __syncthreads();
        if (split == 0 && p < M) {
          double c = dred[tid];
          for (int o = 1; o < nsplit; ++o) c += dred[tid + o];
          c *= cs;
          Cd[p] = c;
          d.C[j * m.m_max + p] = c;
        }
        __syncthreads();
      }
    }
    if (m.ck_global && m.K > 1) {
      if (!grid_sync(d, m.spin_limit, lost)) return;
      for (int p = tid; p < M; p += T) {
        double mean = 0.0;
        for (int k = 0; k < m.K; ++k) mean += d.C[k * m.m_max + p];
        Cu[p] = mean / (double)m.K;
      }
    } else {
      __syncthreads();
      for (int p = tid; p < M; p += T) Cu[p] = Cd[p];
    }
    __syncthreads();
    // ginv in the kernel's precision; dW order keys in FP64 (one divide per
    // measurement, by M threads)
    for (int p = tid; p < M; p += T) {
      const double den = m.kappa + Cu[p];
      ginv[p] = den > 0.0 ? csr / (R)den : (R)0;
      key[p] = order_key(den > 0.0 ? (double)quot<R>(Cd[p], den) : 0.0);
      d.Cused[j * m.m_max + p] = Cu[p];
    }
    __syncthreads();
    // ---- pass 2: updated weights (Eq. 8), mass and largest weight
    R msum = 0, mmax = 0;
    for (int i = tid; i < np; i += T) {
      const P4<R> q = sp[i];
      R acc = 0, a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      int p = 0, k = 0;
      for (; p + 3 < M; p += 4) {
        const V2<R> z0 = zs[p], z1 = zs[p + 1], z2 = zs[p + 2], z3 = zs[p + 3];
        a0 = fma(exp2_neg(PQ(z0.a, z0.b, q.h0, q.h1, q.h1lo)), ginv[p], a0);
        a1 = fma(exp2_neg(PQ(z1.a, z1.b, q.h0, q.h1, q.h1lo)), ginv[p + 1], a1);
        a2 = fma(exp2_neg(PQ(z2.a, z2.b, q.h0, q.h1, q.h1lo)), ginv[p + 2], a2);
        a3 = fma(exp2_neg(PQ(z3.a, z3.b, q.h0, q.h1, q.h1lo)), ginv[p + 3], a3);
        if (++k == 32) {
          acc += (a0 + a1) + (a2 + a3);
          a0 = a1 = a2 = a3 = 0;
          k = 0;
        }
      }
      for (; p < M; ++p) {
        const V2<R> z0 = zs[p];
        a0 = fma(exp2_neg(PQ(z0.a, z0.b, q.h0, q.h1, q.h1lo)), ginv[p], a0);
      }
      acc += (a0 + a1) + (a2 + a3);
      const R wv = (cc.miss + acc) * q.w;
      swu[i] = wv;
      gwu[base + i] = wv;
      msum += wv;
      mmax = wv > mmax ? wv : mmax;
    }
    // mass, largest weight and the count of labels with dW > 0 in one pass
    int npos_t = 0;
    for (int p = tid; p < M; p += T) npos_t += key[p] > 0ull ? 1 : 0;
    double N;
    R wmaxr;
    int npos;
    block_mass_stats<R>(msum, mmax, npos_t, wred, reinterpret_cast<int*>(smem + SL.red + 64 * sizeof(double)), &bN,
                        N, wmaxr, npos);
    if (tid == 0) d.mass[j] = N;
    // resampling plan (Step 5) by the last warp's lane 0, beside the selection
    // (the last warp ranks the fewest labels); read after pass 3's barrier
    if (tid == T - 32) {
      int Lp, sp_;
      resample_plan(m.rho_pe, m.pe_cap - Jj, np, N, (double)wmaxr, Lp, sp_);
      bL = Lp;
      bS = sp_;
      bW = Lp > 0 ? (R)(N / (double)Lp) : (R)0;
    }
    // ---- selection (Step 3): rank of dW by integer compares of the keys
    long long LTl = llround(N);
    if (LTl > npos) LTl = npos;
    if (LTl < 0) LTl = 0;
    const int LT = (int)LTl;
    // a warp per measurement, lanes split the comparisons
    for (int p = tid >> 5; p < M; p += T >> 5) {
      const unsigned long long v = key[p];
      int cnt = 0;
      for (int q = lane; q < M; q += 32) {
        const unsigned long long u = key[q];
        cnt += (u > v || (u == v && q < p)) ? 1 : 0;
      }
      const int rank = __reduce_add_sync(0xffffffffu, cnt);
      if (lane == 0) {
        const bool take = v > 0ull && rank < LT;
        selrank[p] = take ? rank : -1;
        d.selrank[j * m.m_max + p] = take ? rank : -1;
        if (take) {
          sel[rank] = p;
          d.sel[j * m.m_max + rank] = p;
        }
      }
    }
    if (tid == 0) d.nsel[j] = LT;
    __syncthreads();
    // ---- pass 3: labelled sums for the selected labels (Eq. 18), FP32 sums
    // of offsets from the label's point, zeta formed by one thread per label.
    // Up to one label per warp: wpl = (warps / LT) warps per label split the
    // particles, warp totals by shuffles, the wpl totals summed in warp order
    // through shared memory; more labels: groups of nsplit lanes per label.
    if (LT > 0) {
      const int nw = T >> 5, wid = tid >> 5;
      auto zeta_out = [&](int r, R s0, R s1, R s2, R s3, R s4, R px, R py) {
        St4<R> o;
        if (s0 > (R)0) {
          if constexpr (sizeof(R) == 4) {
            const R inv = (R)1 / s0;
            o.x = px + s1 * inv;
            o.vx = s2 * inv;
            o.y = py + s3 * inv;
            o.vy = s4 * inv;
          } else {
            o.x = px + s1 / s0;
            o.vx = s2 / s0;
            o.y = py + s3 / s0;
            o.vy = s4 / s0;
          }
        } else {
          o = St4<R>{px, (R)0, py, (R)0};
        }
        gest[j * m.m_max + r] = o;
      };
      if (LT <= nw) {
        const int wpl = nw / LT;
        const int r = wid / wpl, part = wid - r * wpl;
        R* pbuf = reinterpret_cast<R*>(smem + SL.red);   // [LT][wpl][5]
        R s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
        if (r < LT) {
          const V2<R> z = zs[sel[r]];
          R px, py;
          meas_point_f<R>(cc, m.meas_model, z, px, py);
          for (int i = part * 32 + lane; i < np; i += wpl * 32) {
            const P4<R> q = sp[i];
            const R ew = exp2_neg(PQ(z.a, z.b, q.h0, q.h1, q.h1lo)) * q.w;
            const St4<R> st = sx[i];
            s0 += ew;
            s1 = fma(ew, st.x - px, s1);
            s2 = fma(ew, st.vx, s2);
            s3 = fma(ew, st.y - py, s3);
            s4 = fma(ew, st.vy, s4);
          }
          for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_down_sync(0xffffffffu, s0, o);
            s1 += __shfl_down_sync(0xffffffffu, s1, o);
            s2 += __shfl_down_sync(0xffffffffu, s2, o);
            s3 += __shfl_down_sync(0xffffffffu, s3, o);
            s4 += __shfl_down_sync(0xffffffffu, s4, o);
          }
          if (lane == 0) {
            R* b = pbuf + (r * wpl + part) * 5;
            b[0] = s0;
            b[1] = s1;
            b[2] = s2;
            b[3] = s3;
            b[4] = s4;
          }
        }
        __syncthreads();
        if (tid < LT) {
          const V2<R> z = zs[sel[tid]];
          R px, py;
          meas_point_f<R>(cc, m.meas_model, z, px, py);
          R t[5] = {0, 0, 0, 0, 0};
          for (int k = 0; k < wpl; ++k)
            for (int c = 0; c < 5; ++c) t[c] += pbuf[(tid * wpl + k) * 5 + c];
          zeta_out(tid, t[0], t[1], t[2], t[3], t[4], px, py);
        }
      } else {
        const int nsplit = pow2_floor(min(32, max(1, T / LT)));
        const int mper = T / nsplit;
        const int rl = tid / nsplit, split = tid % nsplit;
        for (int r0 = 0; r0 < LT; r0 += mper) {
          const int r = r0 + rl;
          R s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
          R px = 0, py = 0;
          if (r < LT) {
            const V2<R> z = zs[sel[r]];
            meas_point_f<R>(cc, m.meas_model, z, px, py);
            for (int i = split; i < np; i += nsplit) {
              const P4<R> q = sp[i];
              const R ew = exp2_neg(PQ(z.a, z.b, q.h0, q.h1, q.h1lo)) * q.w;
              const St4<R> st = sx[i];
              s0 += ew;
              s1 = fma(ew, st.x - px, s1);
              s2 = fma(ew, st.vx, s2);
              s3 = fma(ew, st.y - py, s3);
              s4 = fma(ew, st.vy, s4);
            }
          }
          for (int o = nsplit >> 1; o > 0; o >>= 1) {
            s0 += __shfl_down_sync(0xffffffffu, s0, o, nsplit);
            s1 += __shfl_down_sync(0xffffffffu, s1, o, nsplit);
            s2 += __shfl_down_sync(0xffffffffu, s2, o, nsplit);
            s3 += __shfl_down_sync(0xffffffffu, s3, o, nsplit);
            s4 += __shfl_down_sync(0xffffffffu, s4, o, nsplit);
          }
          if (split == 0 && r < LT) zeta_out(r, s0, s1, s2, s3, s4, px, py);
        }
      }
    }
    // ---- resampling (Step 5): exact integer CDF, offspring counts, gather
    __syncthreads();
    const int Lc = bL, sc = bS;
    {
      constexpr int IT = 4;
      unsigned long long carry = 0ull;
      unsigned long long* wt = reinterpret_cast<unsigned long long*>(smem + SL.red);
      const int wid = tid >> 5, nw = T >> 5;
      for (int c0 = 0; c0 < np; c0 += T * IT) {
        unsigned long long q[IT];
        unsigned long long run = 0ull;
#pragma unroll
        for (int k = 0; k < IT; ++k) {
          const int i = c0 + tid * IT + k;
          q[k] = i < np ? scaled_floor(swu[i], sc) : 0ull;
          run += q[k];
          q[k] = run;
        }
        unsigned long long incl = run;
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        if (lane == 31) wt[wid] = incl;
        __syncthreads();
        if (wid == 0) {
          unsigned long long v = lane < nw ? wt[lane] : 0ull;
          for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
          }
          if (lane < nw) wt[lane] = v;
        }
        __syncthreads();
        const unsigned long long off = carry + (wid > 0 ? wt[wid - 1] : 0ull) + (incl - run);
#pragma unroll
        for (int k = 0; k < IT; ++k) {
          const int i = c0 + tid * IT + k;
          if (i < np) Q[i] = off + q[k];
        }
        carry += wt[nw - 1];
        __syncthreads();
      }
    }
    const uint32_t U = a.u ? a.u[j] : philox_u32(m, (uint32_t)j, step, kTagResample);
    const unsigned long long Qn = np > 0 ? Q[np - 1] : 0ull;
    __shared__ Recip rq_s;
    if (tid == 0) rq_s = make_recip(Qn);
    __syncthreads();
    const Recip rq = rq_s;
    for (int i = tid; i < np; i += T) cend[i] = offspring_end(Q[i], Qn, (unsigned long long)Lc, U, rq);
    __syncthreads();
    const R wnew = bW;
    for (int t = tid; t < Lc; t += T) {
      int lo = 0, hi = np - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cend[mid] > t) hi = mid; else lo = mid + 1;
      }
      gx[base + t] = sx[lo];
      gw[base + t] = wnew;
      d.parent[base + t] = lo;
    }
    if (tid == 0) {
      d.rs_L[j] = Lc;
      d.rs_mass[j] = N;
      d.rs_s[j] = sc;
    }
    n = Lc;
    // ---- CU fusion (Step 4) and ring exchange (Step 6)
    St4<R>* out_s = static_cast<St4<R>*>(a.out_states) + (long)s * a.cap;
    int* out_l = a.out_labels + (long)s * a.cap;
    if (m.K > 1) {
      if (!grid_sync(d, m.spin_limit, lost)) return;
      // warp 0: the exchange count, its draws (independent) and the serial
      // Fisher-Yates swaps; the other warps, at the same time: this CTA's
      // share of the CU fusion (the predicted states' block, free after the
      // gather, is its scratch)
      __shared__ int lx_s;
      unsigned int* ud = reinterpret_cast<unsigned int*>(cend);
      const int fchunk = share_chunk<R>(m.K, sizeof(St4<R>) * (size_t)m.pe_cap, T - 32);
      if (tid < 32) {
        const int c = xchg ? exchange_count_warp(d, m, reinterpret_cast<double*>(smem + SL.red + 1024)) : 0;
        if (c > 0) {
          for (int i = lane; i < Lc; i += 32) perm[i] = i;
          for (int t = lane; t < c; t += 32)
            ud[t] = a.xu ? a.xu[base + t] : philox_u32(m, (uint32_t)(base + t), step, kTagExchange);
          __syncwarp();
          if (lane == 0) {
            for (int t = 0; t < c; ++t) {
              const int r = t + (int)(((unsigned long long)ud[t] * (unsigned long long)(Lc - t)) >> 32);
              const int tmp = perm[t];
              perm[t] = perm[r];
              perm[r] = tmp;
            }
          }
        }
        if (lane == 0) {
          lx_s = c;
          if (j == 0) *d.lx = c;
        }
      } else if (fchunk > 0) {
        cu_fuse_share<R>(d, m, j, M, out_s, out_l, a.cap, a.out_count + s, ired, smem + SL.sx, fchunk, zs, cc, 32);
      }
      __syncthreads();
      const int lx = lx_s;
      // scratch too small for a share (many PEs, tiny slices): CTA 0 fuses alone
      if (fchunk <= 0 && j == 0) cu_fuse<R>(d, m, M, out_s, out_l, a.cap, a.out_count + s, ired, srank, srank_cap, zs, cc);
      if (lx > 0) {
        St4<R>* xo = static_cast<St4<R>*>(d.x_out);
        R* wo = static_cast<R*>(d.w_out);
        for (int t = tid; t < lx; t += T) {
          const int slot = perm[t];
          d.xslots[base + t] = slot;
          xo[base + t] = gx[base + slot];
          wo[base + t] = gw[base + slot];
        }
      }
      if (!grid_sync(d, m.spin_limit, lost)) return;
      if (xchg && lx > 0) {
        const St4<R>* xo = static_cast<const St4<R>*>(d.x_out);
        const R* wo = static_cast<const R*>(d.w_out);
        for (int t = tid; t < lx; t += T) {
          const int from = exchange_source(m, j, t);
          const long dst = base + perm[t];
          gx[dst] = xo[(long)from * m.pe_cap + t];
          gw[dst] = wo[(long)from * m.pe_cap + t];
        }
      }
    } else {
      __syncthreads();
      cu_fuse<R>(d, m, M, out_s, out_l, a.cap, a.out_count + s, ired, srank, srank_cap, zs, cc);
    }
    if (tid == 0) d.n_cur[j] = n;
    __syncthreads();
  }
  if (j == 0 && tid == 0) *d.step = step0 + (unsigned long long)a.S;
}

template <class R>
static const void* fused_fn(const Model& m) {
  switch (model_flag(m)) {
    case 1: return (const void*)k_step_fused<R, 1>;
    case 2: return (const void*)k_step_fused<R, 2>;
    case 3: return (const void*)k_step_fused<R, 3>;
    default: return (const void*)k_step_fused<R, 0>;
  }
}

template <class R>
size_t fused_smem_bytes(const Model& m) {
  return fused_smem<R>(m.pe_cap, m.m_max).total;
}

// Whether the fused kernel can run this configuration: the shared-memory
// layout fits and all K CTAs are co-resident.
template <class R>
bool fused_eligible(const Model& m, int device) {
  const size_t sm = fused_smem_bytes<R>(m);
  int optin = 0, nsm = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return false;
  if (sm + 2048 > (size_t)optin) return false;
  if (cudaFuncSetAttribute(fused_fn<R>(m), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return false;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fused_fn<R>(m), kFusedThreads, sm) != cudaSuccess)
    return false;
  return (long)per * nsm >= m.K;
}

template <class R>
cudaError_t launch_fused(const Dev& d, const Model& m, const void* Z, const int* zoff, int M1, int S, const R* noise,
                         const uint32_t* u, const uint32_t* xu, R* out_states, int* out_labels, int* out_count,
                         int cap, cudaStream_t s) {
  FusedArgs a{Z, zoff, M1, noise, u, xu, out_states, out_labels, out_count, cap, S};
  const size_t sm = fused_smem_bytes<R>(m);
  // the grid barrier resets itself (the last arrival clears the count); it is
  // zeroed with the workspace and again whenever a device error is read
  void* args[] = {(void*)&d, (void*)&m, (void*)&a};
  return cudaLaunchCooperativeKernel(fused_fn<R>(m), dim3(m.K), dim3(kFusedThreads), args, sm, s);
}

template bool fused_eligible<float>(const Model&, int);
template bool fused_eligible<double>(const Model&, int);
template cudaError_t launch_fused<float>(const Dev&, const Model&, const void*, const int*, int, int, const float*,
                                         const uint32_t*, const uint32_t*, float*, int*, int*, int, cudaStream_t);
template cudaError_t launch_fused<double>(const Dev&, const Model&, const void*, const int*, int, int, const double*,
                                          const uint32_t*, const uint32_t*, double*, int*, int*, int, cudaStream_t);

}  // namespace phd
