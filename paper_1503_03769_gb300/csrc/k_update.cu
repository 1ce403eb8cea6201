// Update, Eq. 7-8, as two passes over the particle x measurement pairs.
//
// The likelihood is kept in exp2 form:
//   g(z|x) = cnorm * 2^-q,  q = b0 (z0 - h0(x))^2 + b1 (z1 - h1(x))^2,
//   b = log2(e) / (2 sigma^2),
// so one MUFU ex2 per pair evaluates it; the bearing difference is wrapped
// to [0, pi].  The N x M likelihood matrix is never stored.  The sensor model
// is a template parameter of the pair loops (no per-pair branch).
//
// Pass 1 (k_colsum): C^j_p = p_D cnorm sum_i 2^-q_ip w_i.  A work item is a
//   tile of c_tile particles of one slice (staged in shared memory as packed
//   (h0, h1, h1lo, w)) times a chunk of 64 c_mb measurements.  A thread holds
//   c_mb measurements in registers (one broadcast shared load then feeds c_mb
//   pairs) and runs over a strided split of the tile; the splits of a
//   measurement are combined by a fixed-shape tree in shared memory, and the
//   per-tile partial goes to memory in FP64.  k_finalize sums the partials of
//   a slice in a fixed order, so C is accumulated in FP64 and deterministic.
// Finalize: C^j, the normaliser each slice applies (its own, or the PE mean),
//   and ginv_p = cnorm p_D / (kappa + C_p) (0 when kappa + C_p = 0).
// Pass 2 (k_rowsum): w_i <- [(1 - p_D) + sum_p 2^-q_ip ginv_p] w_i.  A thread
//   holds r_pb particles in registers and r_g lanes share them, splitting the
//   measurements (combined by shuffles); Z_k and ginv are staged in shared
//   memory.  Per-tile FP64 sums and maxima of the updated weights feed N^j and
//   the resampling plan, formed by k_select (slice_mass), the update stage's
//   last kernel.  The updated weights go to their own buffer: the extraction
//   (Eq. 13, 18) still needs the predicted ones.
//
// Algorithmic work per pair and pass: one ex2 and 7 FP32 operations (linear
// sensor; 10 with the bearing wrap); bytes per particle and pass: 16 B state
// + 4 B weight (+ 4 B weight written in pass 2); per measurement: 8 B (+ 8 B
// of FP64 partial per pass-1 tile).
#include "phd_internal.cuh"

namespace phd {

template <class R, int RB, int MB>
__global__ void __launch_bounds__(kThreads) k_colsum(Dev d, Model m) {
  pdl_enter();
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ int tpref[kMaxPE + 1];   // tiles per slice (pass-1 partial rows)
  __shared__ int ipref[kMaxPE + 1];   // work items per slice (tiles x measurement chunks)
  constexpr int MC = 64 * MB;         // measurements per work item
  const int TP = m.tune.c_tile;
  P4<R>* sp = reinterpret_cast<P4<R>*>(smem_raw);   // [TP]
  R* red = reinterpret_cast<R*>(sp + TP);           // [kThreads * MB]
  const int K = m.K;
  item_prefix(d.n_pred, K, tpref, TP);
  slice_prefix(K, ipref, [&](int j) {
    return ((d.n_pred[j] + TP - 1) / TP) * ((slice_M(d, j) + MC - 1) / MC);
  });
  const int total = ipref[K];
  const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x_alt);
  const R* __restrict__ w = static_cast<const R*>(d.w_alt);
  const P4<R>* __restrict__ geo = static_cast<const P4<R>*>(d.geo);
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);
  const PairQ<R, RB> Q(m);
  const Lik<R> LB = make_lik<R>(m);
  __shared__ R bsh[4 * (kThreads / 32)];
  __shared__ int live[MC];             // the chunk's measurements past no gate
  __shared__ int wcnt[kThreads / 32];
  __shared__ int nlive;
  Box<R> box{0, 0, 0, 0};
  int staged = -1;
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = item_pe(ipref, K, item);
    const int M = slice_M(d, j);
    const V2<R>* __restrict__ Z = slice_Z<R>(d, j);
    const int chunks = (M + MC - 1) / MC;
    const int local = item - ipref[j];
    const int tile = local / chunks, chunk = local - tile * chunks;
    const int titem = tpref[j] + tile;
    const long base = (long)j * m.pe_cap + (long)tile * TP;
    const int cnt = min(TP, d.n_pred[j] - tile * TP);
    if (titem != staged) {   // consecutive items of a CTA can share the tile
      __syncthreads();
      const R inf = (R)INFINITY;
      R lo0 = inf, hi0 = -inf, lo1 = inf, hi1 = -inf;
      for (int i = threadIdx.x; i < TP; i += kThreads) {
        P4<R> q = {0, 0, 0, 0};
        if (i < cnt) {
          if (m.tune.order) {
            q = geo[base + i];   // the spatial order's record: geometry and weight
          } else {
            const H3<R> h = meas_h<R>(m, x[base + i], tab);
            q = P4<R>{h.h0, h.h1, h.h1lo, w[base + i]};
          }
          lo0 = fmin(lo0, q.h0);
          hi0 = fmax(hi0, q.h0);
          lo1 = fmin(lo1, q.h1);
          hi1 = fmax(hi1, q.h1);
        }
        sp[i] = q;
      }
      box = block_box<R>(lo0, hi0, lo1, hi1, bsh);
      __syncthreads();
      staged = titem;
    }
    const int pbeg = chunk * MC;
    const int Mc = min(MC, M - pbeg);
    // the chunk's measurements that can reach the tile, in order (all of them
    // with the gate off); the pair work is spread over the live ones only
    {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      bool keep = false;
      if ((int)threadIdx.x < Mc) {
        const V2<R> z = Z[pbeg + threadIdx.x];
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
      if (keep) live[before + __popc(bal & ((1u << lane) - 1u))] = threadIdx.x;
      if (threadIdx.x == 0) nlive = all;
      __syncthreads();
    }
    const int Ml = nlive;
    if (threadIdx.x == 0 && Ml > 0) atomicAdd(&d.stats[4], (unsigned long long)Ml * (unsigned long long)cnt);
    for (int p = threadIdx.x; p < Mc; p += kThreads) d.colpart[(long)titem * m.m_max + pbeg + p] = 0.0;
    if (Ml > 0) {
      const int G = (Ml + MB - 1) / MB;   // measurement groups (threads per split)
      const int S = kThreads / G;         // splits of the tile
      const int GM = G * MB;
      const int g = threadIdx.x % G, sidx = threadIdx.x / G;
      R acc[MB];
#pragma unroll
      for (int k = 0; k < MB; ++k) acc[k] = 0;
      if (sidx < S) {
        R z0[MB], z1[MB];
#pragma unroll
        for (int k = 0; k < MB; ++k) {
          const int q = g + k * G;
          const V2<R> z = q < Ml ? Z[pbeg + live[q]] : V2<R>{0, 0};
          z0[k] = z.a;
          z1[k] = z.b;
        }
        int i = sidx;
        for (; i + S < cnt; i += 2 * S) {
          const P4<R> qa = sp[i], qb = sp[i + S];
#pragma unroll
          for (int k = 0; k < MB; ++k)
            acc[k] = fma(exp2_neg(Q(z0[k], z1[k], qa.h0, qa.h1, qa.h1lo)), qa.w, acc[k]);
#pragma unroll
          for (int k = 0; k < MB; ++k)
            acc[k] = fma(exp2_neg(Q(z0[k], z1[k], qb.h0, qb.h1, qb.h1lo)), qb.w, acc[k]);
        }
        if (i < cnt) {
          const P4<R> qa = sp[i];
#pragma unroll
          for (int k = 0; k < MB; ++k)
            acc[k] = fma(exp2_neg(Q(z0[k], z1[k], qa.h0, qa.h1, qa.h1lo)), qa.w, acc[k]);
        }
#pragma unroll
        for (int k = 0; k < MB; ++k) red[sidx * GM + g + k * G] = acc[k];
      }
      __syncthreads();
      // the S splits of each measurement: fixed-shape pairwise tree
      for (int width = S; width > 1;) {
        const int half = (width + 1) >> 1;
        for (int t = threadIdx.x; t < (width - half) * GM; t += kThreads) red[t] += red[t + half * GM];
        __syncthreads();
        width = half;
      }
      for (int q = threadIdx.x; q < Ml; q += kThreads)
        d.colpart[(long)titem * m.m_max + pbeg + live[q]] = (double)red[q];
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
  pdl_enter();
  __shared__ int pref[kMaxPE + 1];
  __shared__ int mpref[kMaxPE + 1];
  const int K = m.K;
  item_prefix(d.n_pred, K, pref, m.tune.c_tile);
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
        ginv[j * m.m_max + p] = den > 0.0 ? quot<R>(cs, den) : (R)0;
        d.dwkey[j * m.m_max + p] = order_key(den > 0.0 ? (double)quot<R>(cj, den) : 0.0);
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
        ginv[j * m.m_max + p] = den > 0.0 ? quot<R>(cs, den) : (R)0;
        d.dwkey[j * m.m_max + p] = order_key(den > 0.0 ? (double)quot<R>(c, den) : 0.0);
      }
    }
  }
  if (blockIdx.x == 0) {
    // counters: one slice per thread (K <= blockDim), warp sums, then thread 0
    __shared__ unsigned long long cs[3][8];
    unsigned long long n = 0, pairs = 0, meas = 0;
    if ((int)threadIdx.x < K) {
      const unsigned long long Mj = (unsigned long long)slice_M(d, threadIdx.x);
      n = (unsigned long long)d.n_pred[threadIdx.x];
      pairs = n * Mj;
      meas = Mj;
    }
    for (int o = 16; o > 0; o >>= 1) {
      n += __shfl_down_sync(0xffffffffu, n, o);
      pairs += __shfl_down_sync(0xffffffffu, pairs, o);
      meas += __shfl_down_sync(0xffffffffu, meas, o);
    }
    if ((threadIdx.x & 31) == 0) {
      cs[0][threadIdx.x >> 5] = pairs;
      cs[1][threadIdx.x >> 5] = n;
      cs[2][threadIdx.x >> 5] = meas;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long a = 0, b = 0, c = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        a += cs[0][k];
        b += cs[1][k];
        c += cs[2][k];
      }
      d.stats[0] += a;
      d.stats[1] += b;
      d.stats[2] += d.zshared ? (unsigned long long)*d.M : c;
      d.stats[3] += 1ull;
    }
  }
}

// Pass 2: a thread holds PB particles (k * GR + il of the tile, so loads are
// coalesced) and G consecutive lanes share them, splitting the measurements
// (p = g, g + G, ...); two accumulators per particle for ILP.
template <class R, int RB, int PB, int G>
__global__ void __launch_bounds__(kThreads) k_rowsum(Dev d, Model m) {
  pdl_enter();
  constexpr int GR = kThreads / G;   // particle groups per tile
  constexpr int TPR = GR * PB;       // particles per work item
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ int pref[kMaxPE + 1];
  __shared__ double rs[kThreads / 32];
  __shared__ double rm[kThreads / 32];
  Z4<R>* zs = reinterpret_cast<Z4<R>*>(smem_raw);
  const int K = m.K;
  item_prefix(d.n_pred, K, pref, TPR);
  const int total = pref[K];
  const R* __restrict__ ginv = static_cast<const R*>(d.ginv);
  const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x_alt);
  const R* __restrict__ w = static_cast<const R*>(d.w_alt);
  R* __restrict__ wu = static_cast<R*>(d.wu);
  const P4<R>* __restrict__ geo = static_cast<const P4<R>*>(d.geo);
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);
  const PairQ<R, RB> Q(m);
  const Lik<R> LB = make_lik<R>(m);
  const R miss = consts<R>(m).miss;
  const int il = threadIdx.x / G, g = threadIdx.x % G;
  __shared__ R bsh[4 * (kThreads / 32)];
  __shared__ int wcnt[kThreads / 32];
  int* lidx = reinterpret_cast<int*>(zs + m.m_max);   // [m_max] the gate's survivors
  int staged = -1;
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = item_pe(pref, K, item);
    const int tile = item - pref[j];
    const int M = slice_M(d, j);
    const int n = d.n_pred[j];
    R h0[PB], h1[PB], hl[PB], wi[PB];
    const R inf = (R)INFINITY;
    R lo0 = inf, hi0 = -inf, lo1 = inf, hi1 = -inf;
#pragma unroll
    for (int k = 0; k < PB; ++k) {
      const int i = tile * TPR + k * GR + il;
      h0[k] = h1[k] = hl[k] = wi[k] = 0;
      if (i < n) {
        if (m.tune.order) {
          const P4<R> q = geo[(long)j * m.pe_cap + i];   // sorted position i
          h0[k] = q.h0;
          h1[k] = q.h1;
          hl[k] = q.h1lo;
          wi[k] = q.w;
        } else {
          const long gi = (long)j * m.pe_cap + i;
          const H3<R> h = meas_h<R>(m, x[gi], tab);
          h0[k] = h.h0;
          h1[k] = h.h1;
          hl[k] = h.h1lo;
          wi[k] = w[gi];
        }
        lo0 = fmin(lo0, h0[k]);
        hi0 = fmax(hi0, h0[k]);
        lo1 = fmin(lo1, h1[k]);
        hi1 = fmax(hi1, h1[k]);
      }
    }
    if (j != staged) {
      const V2<R>* __restrict__ Z = slice_Z<R>(d, j);
      __syncthreads();
      for (int p = threadIdx.x; p < M; p += kThreads) {
        const V2<R> z = Z[p];
        zs[p] = Z4<R>{z.a, z.b, ginv[j * m.m_max + p], (R)0};
      }
      __syncthreads();
      staged = j;
    }
    // the measurements that can reach the tile, in order (the gate's survivors)
    const Box<R> box = block_box<R>(lo0, hi0, lo1, hi1, bsh);
    int nl = M;
    if (m.tune.gate) {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      int base_w = 0;
      for (int p0 = 0; p0 < M; p0 += kThreads) {
        const int p = p0 + (int)threadIdx.x;
        const bool keep = p < M && box_qmin<R, RB>(box, LB.b0, LB.b1, zs[p].z0, zs[p].z1) < gate_limit<R>(m);
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wcnt[wid] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int k = 0; k < kThreads / 32; ++k) {
          before += k < wid ? wcnt[k] : 0;
          all += wcnt[k];
        }
        if (keep) lidx[base_w + before + __popc(bal & ((1u << lane) - 1u))] = p;
        base_w += all;
        __syncthreads();
      }
      nl = base_w;
    }
    R a0[PB], a1[PB];
#pragma unroll
    for (int k = 0; k < PB; ++k) a0[k] = a1[k] = 0;
    if (nl == M) {
      int p = g;
      for (; p + G < M; p += 2 * G) {
        const Z4<R> za = zs[p], zb = zs[p + G];
#pragma unroll
        for (int k = 0; k < PB; ++k)
          a0[k] = fma(exp2_neg(Q(za.z0, za.z1, h0[k], h1[k], hl[k])), za.g, a0[k]);
#pragma unroll
        for (int k = 0; k < PB; ++k)
          a1[k] = fma(exp2_neg(Q(zb.z0, zb.z1, h0[k], h1[k], hl[k])), zb.g, a1[k]);
      }
      if (p < M) {
        const Z4<R> za = zs[p];
#pragma unroll
        for (int k = 0; k < PB; ++k)
          a0[k] = fma(exp2_neg(Q(za.z0, za.z1, h0[k], h1[k], hl[k])), za.g, a0[k]);
      }
    } else {
      // the survivors only, each in the lane and accumulator the full loop
      // gives it (p = g mod G, accumulator by the parity of p / G): the sums
      // are those of the full loop without its exact zeros
      for (int e = 0; e < nl; ++e) {
        const int p = lidx[e];
        if (p % G != g) continue;
        const Z4<R> za = zs[p];
        if ((p / G) & 1) {
#pragma unroll
          for (int k = 0; k < PB; ++k)
            a1[k] = fma(exp2_neg(Q(za.z0, za.z1, h0[k], h1[k], hl[k])), za.g, a1[k]);
        } else {
#pragma unroll
          for (int k = 0; k < PB; ++k)
            a0[k] = fma(exp2_neg(Q(za.z0, za.z1, h0[k], h1[k], hl[k])), za.g, a0[k]);
        }
      }
    }
    R sv = 0, mv = 0;
#pragma unroll
    for (int k = 0; k < PB; ++k) {
      R acc = a0[k] + a1[k];
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      const int i = tile * TPR + k * GR + il;
      if (g == 0 && i < n) {
        const R wv = (miss + acc) * wi[k];
        wu[(long)j * m.pe_cap + (m.tune.order ? d.perm[(long)j * m.pe_cap + i] : i)] = wv;
        sv += wv;
        mv = wv > mv ? wv : mv;
      }
    }
    // tile sum and max: the warp's values in the kernel's precision, the
    // warp totals in FP64 by one thread (FP64 is ~1/60 of the FP32 rate)
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

int grid_items(const Model& m) {
  long items = (long)m.K * ((m.pe_cap + kTile - 1) / kTile);
  long g = 152L * 4;
  return (int)(items < g ? (items > 0 ? items : 1) : g);
}

static int grid_cap(long items, long cap) { return (int)(items < cap ? (items > 0 ? items : 1) : cap); }

Tune default_tune(bool fp64) {
  Tune t;
  t.c_tile = 512;
  t.c_mb = fp64 ? 2 : 4;
  t.r_pb = 1;
  t.r_g = 4;
  t.grid1 = 152 * 8;
  t.grid2 = 152 * 8;
  t.gate = 1;
  t.order = fp64 ? 0 : 1;
  return t;
}

bool tune_supported(const Tune& t, bool fp64) {
  if (t.c_tile != 256 && t.c_tile != 512 && t.c_tile != 1024) return false;
  if (t.grid1 < 1 || t.grid2 < 1 || t.grid1 > 152 * 64 || t.grid2 > 152 * 64) return false;
  if (t.gate != 0 && t.gate != 1) return false;
  if (t.order != 0 && t.order != 1) return false;
  if (fp64) return t.c_mb == 2 && t.r_pb == 1 && t.r_g == 4;
  if (t.c_mb != 1 && t.c_mb != 2 && t.c_mb != 4) return false;
  const int pg = t.r_pb * 16 + t.r_g;
  return pg == 16 + 1 || pg == 32 + 1 || pg == 64 + 1 || pg == 16 + 2 || pg == 32 + 2 || pg == 16 + 4 ||
         pg == 16 + 8;
}

template <class R, int RB, int MB>
static void colsum_go(const Dev& d, const Model& m, cudaStream_t s) {
  const long tiles = (long)m.K * ((m.pe_cap + m.tune.c_tile - 1) / m.tune.c_tile);
  const long chunks = (m.m_max + 64 * MB - 1) / (64 * MB);
  const size_t smem = sizeof(P4<R>) * (size_t)m.tune.c_tile + sizeof(R) * kThreads * MB;
  launch_k(k_colsum<R, RB, MB>, dim3(grid_cap(tiles * chunks, m.tune.grid1)), dim3(kThreads), smem, s, d, m);
}

template <class R, int RB, int PB, int G>
static void rowsum_go(const Dev& d, const Model& m, cudaStream_t s) {
  const int tpr = kThreads / G * PB;
  const long tiles = (long)m.K * ((m.pe_cap + tpr - 1) / tpr);
  launch_k(k_rowsum<R, RB, PB, G>, dim3(grid_cap(tiles, m.tune.grid2)), dim3(kThreads),
           (sizeof(Z4<R>) + sizeof(int)) * (size_t)m.m_max, s, d, m);
}

template <class R, int RB>
static cudaError_t prepare_rowsum(size_t sm) {
  cudaError_t e = cudaFuncSetAttribute(k_rowsum<R, RB, 1, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if constexpr (sizeof(R) == 4) {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rowsum<R, RB, 1, 1>, a, (int)sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rowsum<R, RB, 2, 1>, a, (int)sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rowsum<R, RB, 4, 1>, a, (int)sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rowsum<R, RB, 1, 2>, a, (int)sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rowsum<R, RB, 2, 2>, a, (int)sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rowsum<R, RB, 1, 8>, a, (int)sm);
  }
  return e;
}

template <class R>
cudaError_t prepare_kernels(const Model& m) {
  const size_t sm = (sizeof(Z4<R>) + sizeof(int)) * (size_t)m.m_max;
  cudaError_t e = prepare_rowsum<R, 0>(sm);
  if (e == cudaSuccess) e = prepare_rowsum<R, 1>(sm);
  if (e == cudaSuccess) e = prepare_rowsum<R, 2>(sm);
  if (e == cudaSuccess) e = prepare_rowsum<R, 3>(sm);
  if (e == cudaSuccess) e = prepare_extract<R>();
  return e;
}

template <class R, int RB>
static cudaError_t colsum_model(const Dev& d, const Model& m, cudaStream_t s) {
  if constexpr (sizeof(R) == 8) {
    colsum_go<R, RB, 2>(d, m, s);
  } else {
    switch (m.tune.c_mb) {
      case 1: colsum_go<R, RB, 1>(d, m, s); break;
      case 2: colsum_go<R, RB, 2>(d, m, s); break;
      default: colsum_go<R, RB, 4>(d, m, s); break;
    }
  }
  return cudaGetLastError();
}

template <class R, int RB>
static cudaError_t rowsum_model(const Dev& d, const Model& m, cudaStream_t s) {
  if constexpr (sizeof(R) == 8) {
    rowsum_go<R, RB, 1, 4>(d, m, s);
  } else {
    switch (m.tune.r_pb * 16 + m.tune.r_g) {
      case 16 + 1: rowsum_go<R, RB, 1, 1>(d, m, s); break;
      case 32 + 1: rowsum_go<R, RB, 2, 1>(d, m, s); break;
      case 64 + 1: rowsum_go<R, RB, 4, 1>(d, m, s); break;
      case 16 + 2: rowsum_go<R, RB, 1, 2>(d, m, s); break;
      case 32 + 2: rowsum_go<R, RB, 2, 2>(d, m, s); break;
      case 16 + 8: rowsum_go<R, RB, 1, 8>(d, m, s); break;
      default: rowsum_go<R, RB, 1, 4>(d, m, s); break;
    }
  }
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_colsum(const Dev& d, const Model& m, cudaStream_t s) {
  switch (model_flag(m)) {
    case 1: return colsum_model<R, 1>(d, m, s);
    case 2: return colsum_model<R, 2>(d, m, s);
    case 3: return colsum_model<R, 3>(d, m, s);
    default: return colsum_model<R, 0>(d, m, s);
  }
}

template <class R>
cudaError_t launch_finalize(const Dev& d, const Model& m, cudaStream_t s) {
  launch_k(k_finalize<R>, dim3(grid_cap(((long)m.K * m.m_max + 7) / 8, 152L * 8)), dim3(256), 0, s, d, m);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_rowsum(const Dev& d, const Model& m, cudaStream_t s) {
  switch (model_flag(m)) {
    case 1: return rowsum_model<R, 1>(d, m, s);
    case 2: return rowsum_model<R, 2>(d, m, s);
    case 3: return rowsum_model<R, 3>(d, m, s);
    default: return rowsum_model<R, 0>(d, m, s);
  }
}

int n_update_launches(const Model& m) { return (m.tune.order ? n_order_launches() : 0) + 4; }

template <class R>
cudaError_t launch_update(const Dev& d, const Model& m, cudaStream_t s) {
  cudaError_t e = m.tune.order ? launch_order<R>(d, m, s) : cudaSuccess;
  if (e == cudaSuccess) e = launch_colsum<R>(d, m, s);
  if (e == cudaSuccess) e = launch_finalize<R>(d, m, s);
  if (e == cudaSuccess) e = launch_rowsum<R>(d, m, s);
  if (e == cudaSuccess) e = launch_select<R>(d, m, s);   // N^j, the resampling plan, the LT_j labels
  return e;
}

template cudaError_t launch_update<float>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_update<double>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_colsum<float>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_colsum<double>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_finalize<float>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_finalize<double>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_rowsum<float>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_rowsum<double>(const Dev&, const Model&, cudaStream_t);
template cudaError_t prepare_kernels<float>(const Model&);
template cudaError_t prepare_kernels<double>(const Model&);

}  // namespace phd
