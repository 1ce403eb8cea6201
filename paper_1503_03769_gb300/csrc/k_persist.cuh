#pragma once
// Persistent step kernel (the template; k_persist.cu and k_persist_wide.cu
// instantiate it): one cooperative launch runs a whole filter step
// (predict, update, labelled extraction, resampling) for every slice of a
// handle, its phases separated by grid-wide barriers with bounded waits.
//
// It computes what the staged kernels compute (the same helpers, the same
// per-pair arithmetic), for handles without particle exchange or CU fusion:
// one filter (one PE) or a batch of independent runs.  What changes is the
// organisation of the work, which on the gated dense workloads is what the
// staged step's time goes to (a dozen launches of latency-bound kernels):
//  - every phase is one sweep of the grid over work items: chunks of 256
//    particles (prediction, spatial order, CDF, gather), tiles of 512 for the
//    pair passes (two particles per thread, so most CTAs hold one tile of a
//    large slice), or measurements / labels; no launch between phases;
//  - the spatial order of the pair passes (a stable counting sort on a 16 x 16
//    grid over measurement space) is built in three phases (chunk histograms
//    with the prediction, per-bin totals, per-bin starts) and its records
//    (sensor-space geometry and predicted weight) are moved once;
//  - pass 1 records, per sorted tile, which measurements can reach the tile
//    (the exact likelihood gate, a bit per measurement).  Pass 1 writes only
//    those partial sums, the normalisers add only those (in tile order, so C
//    is deterministic), pass 2 walks only those, and the extraction's label
//    sums and their reduction use the same bits: no partial matrix is
//    cleared or read in full.
// Phases (barrier between consecutive ones):
//   A  predict (Eq. 5-6), measurement-space geometry, cell key, chunk
//      histograms and the cell totals per (slice, cell) by integer atomics;
//      measurement staging
//   C  cell starts per (slice, cell)
//   D  stable scatter to the cell order       E  pass 1 (Eq. 7) per tile
//   F  C_p, ginv_p and the dW keys (Eq. 12, 16) per measurement
//   G  pass 2 (Eq. 8) per tile: updated weights, tile sums and maxima;
//      selection ranks (Step 3) per measurement beside it
//   H  (batches) N^j, the resampling plan, LT_j per slice
//   J  CDF chunk totals per chunk; pass 3 (Eq. 18 sums) per tile (one
//      filter: N^j, the plan and LT_j from integer sums kept by F and G)
//   K  estimates per selected label; CDF chunk offsets per slice
//   L  offspring ends per chunk and the children gathered (Sec. 2.2 step 3),
//      counts and step counter advanced
// The barrier is one release atomic per CTA on a 64-bit count that only grows
// and acquire polls; the host passes the count the launch starts from.
#include "phd_internal.cuh"

namespace phd {

constexpr int kPT = 256;      // threads per CTA
constexpr int kPMB = 4;       // pass 1: measurements per warp group
constexpr int kGT = 512;      // particles of a chunk and of a pair-pass tile (two per thread)
// phase clock slots (phd_get_phase_times order)
enum : int { kPhA = 0, kPhC, kPhD, kPhE, kPhF, kPhG, kPhH, kPhJ, kPhK, kPhL };

template <class R> struct PersistArgs {
  const R* Z;                 // one filter: the scan (staged into the workspace in phase A); NULL for a batch
  int M;
  const R* noise;             // injected predict draws or NULL
  const uint32_t* u;          // injected resampling uniforms or NULL
  R* out_states;              // one filter: estimates in ascending label order
  int* out_labels;
  int cap;
  int* d_count;               // one filter: true estimate count (may be NULL)
  unsigned long long base;    // barrier count at launch
  int direct;                 // 1: one filter (write the outputs)
  int advance;                // 1: advance the step counter (0: the exchange kernels after the launch do)
};

// Barrier b (1-based) of the launch, in two halves: every CTA arrives once
// (a release add on the count after a block barrier), may then issue loads
// that do not depend on the phase just finished, and waits until all have
// arrived (count >= base + b G), polling at most `limit` times.  On expiry or
// an error recorded by another CTA the wait returns false in every thread.
__device__ __forceinline__ void pbar_arrive(const Dev& d) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(d.pbar) : "memory");
}
__device__ __forceinline__ bool pbar_wait(const Dev& d, unsigned long long target, long long limit) {
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 0;
    long long it = 0;
    for (;;) {
      unsigned long long c;
      int e;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(c) : "l"(d.pbar) : "memory");
      asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(e) : "l"(d.err) : "memory");
      if (c >= target) {
        ok = 1;
        break;
      }
      if (e & kErrTimeout) break;
      if (++it > limit) {
        atomicOr(d.err, kErrTimeout);
        break;
      }
      __nanosleep(32);
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Warp-wide sum of one value per lane (every lane gets the total).
template <class T> __device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// MB: resident CTAs per SM the registers are budgeted for (3: 80 registers,
// for one filter, where a step's phases are a chain or two per CTA; 4: 64
// registers, for batches, whose CTAs walk tens of items a phase and gain
// from the extra warps in flight)
template <class R, int RB, int MB>
__global__ void __launch_bounds__(kPT, MB) k_step_grid(Dev d, Model m, PersistArgs<R> a) {
  extern __shared__ __align__(32) unsigned char smem[];
  unsigned smem_bytes;   // dynamic shared memory of the launch
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(smem_bytes));
  __shared__ int ipref[kMaxPE + 1];   // chunks (kGT particles) per slice, prefix
  __shared__ int tpref[kMaxPE + 1];   // pair-pass tiles (kGT particles) per slice, prefix
  __shared__ int hpref[kMaxPE + 1];   // chunk-histogram rows per slice: 256 x (items rounded up to 4), prefix
  __shared__ int npred_s[kMaxPE];     // predicted particles per slice
  __shared__ int ncur_s[kMaxPE];      // survivors per slice (the current set)
  __shared__ R bw_s[kMaxPE];          // birth weight per slice
  __shared__ int wcnt[kPT / 32];
  __shared__ R bsh[4 * (kPT / 32)];
  __shared__ double dred[kPT / 32];
  __shared__ unsigned long long dredb[kPT / 32];
  __shared__ int nlive_s;
  const int K = m.K, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nb = gridDim.x, bid = blockIdx.x;
  const long nwarps = ((long)nb * kPT) >> 5;
  // warp-per-unit phases spread consecutive units over CTAs first (unit u on
  // CTA u mod nb), so a few hundred units use every SM's FP64 pipe
  const long sw = (long)wid * nb + bid;
  // when a phase has few units (one filter's measurements or labels), a group
  // of G warps of one CTA shares a unit, its lanes over the unit's loop, and
  // the warps' totals are added in warp order; with G > 1 the loop over units
  // runs in rounds that every warp of the CTA takes (a block barrier between
  // the warps' partials and their sum); groups spread over CTAs first
  struct Grp {
    int G, slot, gl;
    long gid, ng;
  };
  auto groups = [&](long units) {
    Grp g;
    g.G = 1;
    while (g.G < kPT / 32 && units * g.G * 2 <= nwarps) g.G *= 2;
    g.slot = wid / g.G;
    g.gl = (wid % g.G) * 32 + lane;
    g.gid = (long)g.slot * nb + bid;
    g.ng = (long)(kPT / 32 / g.G) * nb;
    return g;
  };
  __shared__ double gred[2][kPT / 32][5];   // group partials, two buffers used in turn
  __shared__ int gcnt[2][kPT / 32][2];
  __shared__ R gredr[2][kPT / 32][5];
  const long long lim = m.spin_limit;
  const unsigned long long G = nb;
  unsigned long long tb = 0ull;   // barriers passed
  unsigned long long t_prev = tid == 0 ? gtimer() : 0ull;   // CTA 0: the last barrier's release
  unsigned long long t_go = t_prev;                          // every CTA: when it left the last barrier
  // phase clock: ptimes[phase] sums CTA 0's time from barrier to barrier;
  // ptimes[16 + phase] keeps the longest time any CTA spent working in the
  // phase (leaving one barrier to arriving at the next) and ptimes[32 + phase]
  // sums those times over CTAs
  // host-injected failure: CTA 0 leaves at its first grid barrier without
  // arriving, as a lost part of the grid would; the others' bounded waits
  // report the timeout
  __shared__ int lost_s;
  if (tid == 0) lost_s = bid == 0 && reinterpret_cast<volatile unsigned int*>(d.bar)[2] != 0u;
  __syncthreads();
  auto arrive = [&](int phase) {
    ++tb;
    if (lost_s) return;   // uniform over the block
    if (tid == 0) {
      const unsigned long long busy = gtimer() - t_go;
      atomicMax(d.ptimes + 16 + phase, busy);
      atomicAdd(d.ptimes + 32 + phase, busy);
    }
    pbar_arrive(d);
  };
  auto wait = [&](int phase) -> bool {
    if (lost_s) return false;
    const bool ok = pbar_wait(d, a.base + tb * G, lim);
    if (ok && tid == 0) {
      const unsigned long long t = gtimer();
      if (bid == 0) atomicAdd(d.ptimes + phase, t - t_prev);
      t_prev = t;
      t_go = t;
    }
    return ok;
  };
  auto barrier = [&](int phase) -> bool {
    arrive(phase);
    return wait(phase);
  };
  // slice sizes after prediction: survivors + births
  for (int j = tid; j < K; j += kPT) {
    ncur_s[j] = d.n_cur[j];
    npred_s[j] = ncur_s[j] + d.Jb[j];
    bw_s[j] = slice_bw<R>(d, j);
  }
  __syncthreads();
  slice_prefix(K, ipref, [&](int j) { return (npred_s[j] + kGT - 1) / kGT; });
  slice_prefix(K, tpref, [&](int j) { return (npred_s[j] + kGT - 1) / kGT; });
  slice_prefix(K, hpref, [&](int j) { return 256 * ((((npred_s[j] + kGT - 1) / kGT) + 3) & ~3); });
  const int nitems = ipref[K];
  const int ntiles = tpref[K];
  const long T = d.max_items;   // row stride of the gate bits [word][tile]
  // chunk histograms: slice j, cell b, chunk c at pchist[hpref[j] + b * hstride(j) + c]
  auto hstride = [&](int j) { return ((ipref[j + 1] - ipref[j]) + 3) & ~3; };
  const unsigned long long step = *d.step;
  const Cst<R> cc = consts<R>(m);
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);

  // ---- A: prediction, geometry, cell keys, chunk histograms; Z staging
  {
    int* hist = reinterpret_cast<int*>(smem);
    const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x);
    const R* __restrict__ w = static_cast<const R*>(d.w);
    St4<R>* __restrict__ xp = static_cast<St4<R>*>(d.x_alt);
    R* __restrict__ wp = static_cast<R*>(d.w_alt);
    P4<R>* __restrict__ geo_s = static_cast<P4<R>*>(d.geo_s);
    if (a.direct) {
      V2<R>* zs = static_cast<V2<R>*>(d.Z);
      for (int p = bid * kPT + tid; p < a.M; p += nb * kPT) {
        const V2<R> z = reinterpret_cast<const V2<R>*>(a.Z)[p];
        if (!isfinite(z.a) || !isfinite(z.b)) atomicOr(d.err, kErrNonFinite);
        if (a.Z != static_cast<const R*>(d.Z)) zs[p] = z;
      }
    }
    if (bid == 0) {
      for (int j = tid; j < K; j += kPT) {
        d.n_pred[j] = npred_s[j];
        // the slice plan's inputs, filled by F and G
        d.pmassq[2 * j] = 0ull;
        d.pmassq[2 * j + 1] = 0ull;
        d.pwmaxb[j] = 0ull;
        d.pnpos[j] = 0;
      }
      if (tid == 0 && a.direct) *d.M = a.M;
    }
    for (int it = bid; it < nitems; it += nb) {
      const int j = item_pe(ipref, K, it);
      hist[tid] = 0;
      __syncthreads();
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {   // the thread's two slots of the chunk
        const int i = (it - ipref[j]) * kGT + hh * kPT + tid;
        int key = kCells;   // none
        if (i < npred_s[j]) {
          const long g = (long)j * m.pe_cap + i;
          const bool surv = i < ncur_s[j];
          St4<R> o;
          R wo;
          if (!surv && m.learned) {
            // a birth of the measurement-driven proposal, drawn into its slot
            // before the launch
            o = xp[g];
            wo = wp[g];
          } else {
            R n1, n2, u1, u2;
            draw_noise<R>(m, a.noise, g, step, n1, n2, u1, u2);
            predict_slot<R>(cc, surv, surv ? x[g] : St4<R>{0, 0, 0, 0}, surv ? w[g] : (R)0, bw_s[j], n1, n2, u1,
                            u2, o, wo);
            xp[g] = o;
            wp[g] = wo;
          }
          const H3<R> h = meas_h<R>(m, o, tab);
          geo_s[g] = P4<R>{h.h0, h.h1, h.h1lo, wo};
          key = cell_key(m, (float)h.h0, (float)h.h1);
          d.ckey[g] = (unsigned char)key;
        }
        // one shared-memory add per distinct cell of the warp (a chunk's slots
        // hold siblings of a few parents, mostly in one cell)
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key < kCells && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&hist[key], __popc(peers));
      }
      __syncthreads();
      // the chunk's count of every cell, and the cell totals of the slice by
      // integer atomics (exact in any order); the totals were cleared by the
      // previous launch after their last use
      const int hv = hist[tid];
      d.pchist[hpref[j] + (long)tid * hstride(j) + (it - ipref[j])] = hv;
      if (hv) atomicAdd(d.bintot + (long)j * 256 + tid, hv);
      __syncthreads();
    }
  }
  if (!barrier(kPhA)) return;

  // ---- C: per (slice, cell): the cell's start (cells before it), then each
  // chunk's start within the cell (chunks before it), in place: rounds of
  // 128 chunks, four per lane, a warp scan of the lane totals
  for (long u = sw; u < (long)K * 256; u += nwarps) {
    const int j = (int)(u >> 8), b = (int)(u & 255);
    int4* row = reinterpret_cast<int4*>(d.pchist + hpref[j] + (long)b * hstride(j));
    const int n4 = hstride(j) >> 2, nc = ipref[j + 1] - ipref[j];
    // the first kCR rounds of the row are fetched with the cell totals
    constexpr int kCR = 8;
    int4 pre[kCR];
#pragma unroll
    for (int r = 0; r < kCR; ++r) pre[r] = 32 * r + lane < n4 ? __ldcg(row + 32 * r + lane) : int4{0, 0, 0, 0};
    int base = 0;
    for (int q = lane; q < b; q += 32) base += __ldcg(d.bintot + (long)j * 256 + q);
    base = warp_sum(base);
    for (int q0 = 0; q0 < n4; q0 += 32) {
      const int q = q0 + lane;
      int4 v = pre[0];
#pragma unroll
      for (int r = 1; r < kCR; ++r) v = q0 == 32 * r ? pre[r] : v;
      if (q0 >= 32 * kCR) v = q < n4 ? __ldcg(row + q) : int4{0, 0, 0, 0};
      const int c = 4 * q;
      if (c >= nc) v.x = 0;
      if (c + 1 >= nc) v.y = 0;
      if (c + 2 >= nc) v.z = 0;
      if (c + 3 >= nc) v.w = 0;
      const int tot = v.x + v.y + v.z + v.w;
      int incl = tot;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int s0 = base + incl - tot;
      if (q < n4) row[q] = int4{s0, s0 + v.x, s0 + v.x + v.y, s0 + v.x + v.y + v.z};
      base += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  arrive(kPhC);
  // the first chunk's keys and records (phase A's) are fetched while the
  // other CTAs finish the cell starts
  int dkey[2] = {kCells, kCells};
  P4<R> drec[2] = {P4<R>{0, 0, 0, 0}, P4<R>{0, 0, 0, 0}};
  if (bid < nitems) {
    const int j = item_pe(ipref, K, bid);
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int i = (bid - ipref[j]) * kGT + hh * kPT + tid;
      if (i < npred_s[j]) {
        const long g = (long)j * m.pe_cap + i;
        dkey[hh] = (int)d.ckey[g];
        drec[hh] = static_cast<const P4<R>*>(d.geo_s)[g];
      }
    }
  }
  if (!wait(kPhC)) return;

  // ---- D: stable scatter: each particle's rank among its chunk's particles
  // with its key gives its sorted position; the geometry record moves there
  {
    int* wc = reinterpret_cast<int*>(smem);   // [16][256]: per (warp of 32 consecutive slots, cell)
    const P4<R>* __restrict__ geo_s = static_cast<const P4<R>*>(d.geo_s);
    P4<R>* __restrict__ geo = static_cast<P4<R>*>(d.geo);
    // the cell totals were last read in C: cleared for the next launch
    for (long u = (long)bid * kPT + tid; u < (long)K * 256; u += (long)nb * kPT) d.bintot[u] = 0;
    for (int it = bid; it < nitems; it += nb) {
      const int j = item_pe(ipref, K, it);
      // the thread's two slots: i[hh] = chunk start + hh 256 + tid, so the
      // 16 groups of 32 consecutive slots are (hh, warp) in slot order
      int key[2], cstart[2], slot[2];
      bool live[2];
      P4<R> rec[2];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        slot[hh] = (it - ipref[j]) * kGT + hh * kPT + tid;
        live[hh] = slot[hh] < npred_s[j];
        const long g = (long)j * m.pe_cap + slot[hh];
        if (it == bid) {
          key[hh] = dkey[hh];
          rec[hh] = drec[hh];
        } else {
          key[hh] = live[hh] ? (int)d.ckey[g] : kCells;
          rec[hh] = live[hh] ? geo_s[g] : P4<R>{0, 0, 0, 0};
        }
        // the (cell, chunk) start is fetched before the ranking
        cstart[hh] = live[hh] ? __ldcg(d.pchist + hpref[j] + (long)key[hh] * hstride(j) + (it - ipref[j])) : 0;
      }
      for (int t = tid; t < 16 * kCells; t += kPT) wc[t] = 0;
      __syncthreads();
      int rank_w[2];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const unsigned peers = __match_any_sync(0xffffffffu, key[hh]);
        rank_w[hh] = __popc(peers & ((1u << lane) - 1u));
        if (live[hh] && rank_w[hh] == 0) wc[(hh * (kPT / 32) + wid) * kCells + key[hh]] = __popc(peers);
      }
      __syncthreads();
      {
        int run = 0;
        for (int w16 = 0; w16 < 16; ++w16) {
          const int v = wc[w16 * kCells + tid];
          wc[w16 * kCells + tid] = run;
          run += v;
        }
      }
      __syncthreads();
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        if (!live[hh]) continue;
        const int dst = cstart[hh] + wc[(hh * (kPT / 32) + wid) * kCells + key[hh]] + rank_w[hh];
        if (dst >= 0 && dst < npred_s[j]) {
          d.perm[(long)j * m.pe_cap + dst] = slot[hh];
          geo[(long)j * m.pe_cap + dst] = rec[hh];
        } else {
          atomicOr(d.err, kErrCapacity);   // inconsistent cell counts: never written out of the slice
        }
      }
      __syncthreads();
    }
  }
  if (!barrier(kPhD)) return;

  const PairQ<R, RB> Q(m);
  const Lik<R> LB = make_lik<R>(m);
  const P4<R>* __restrict__ geo = static_cast<const P4<R>*>(d.geo);
  // the tile's box (every thread loads its two particles' records) and the
  // measurements of slice j that can reach it: live list in smem (lidx, in
  // measurement order) and, when `record`, the tile's gate bits
  auto tile_gate = [&](int it, int j, int cnt, P4<R>& q0, P4<R>& q1, int* lidx, bool record) -> int {
    const R inf = (R)INFINITY;
    R lo0 = inf, hi0 = -inf, lo1 = inf, hi1 = -inf;
    q0 = P4<R>{0, 0, 0, 0};
    q1 = q0;
    const long base = (long)j * m.pe_cap + (long)(it - tpref[j]) * kGT;
    if (tid < cnt) {
      q0 = geo[base + tid];
      lo0 = q0.h0;
      hi0 = q0.h0;
      lo1 = q0.h1;
      hi1 = q0.h1;
    }
    if (tid + kPT < cnt) {
      q1 = geo[base + kPT + tid];
      lo0 = fmin(lo0, q1.h0);
      hi0 = fmax(hi0, q1.h0);
      lo1 = fmin(lo1, q1.h1);
      hi1 = fmax(hi1, q1.h1);
    }
    const Box<R> box = block_box<R>(lo0, hi0, lo1, hi1, bsh);
    const int M = slice_M(d, j);
    const V2<R>* __restrict__ Z = slice_Z<R>(d, j);
    int nl = 0;
    constexpr int kPre = 4;   // rounds whose measurements are fetched up front
    V2<R> zpre[kPre];
#pragma unroll
    for (int r = 0; r < kPre; ++r) zpre[r] = r * kPT + tid < M ? Z[r * kPT + tid] : V2<R>{0, 0};
    for (int p0 = 0; p0 < M; p0 += kPT) {
      const int p = p0 + tid;
      bool keep = false;
      if (p < M) {
        V2<R> z = zpre[0];
#pragma unroll
        for (int r = 1; r < kPre; ++r) z = p0 == r * kPT ? zpre[r] : z;
        if (p0 >= kPre * kPT) z = Z[p];
        keep = !m.tune.gate || box_qmin<R, RB>(box, LB.b0, LB.b1, z.a, z.b) < gate_limit<R>(m);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) {
        wcnt[wid] = __popc(bal);
        if (record && p0 + wid * 32 < M) d.gbits[(long)((p0 >> 5) + wid) * T + it] = bal;
      }
      __syncthreads();
      int before = 0, all = 0;
      for (int k = 0; k < kPT / 32; ++k) {
        before += k < wid ? wcnt[k] : 0;
        all += wcnt[k];
      }
      if (keep) lidx[nl + before + __popc(bal & ((1u << lane) - 1u))] = p;
      nl += all;
      __syncthreads();
    }
    return nl;
  };
  // the live list of a tile from its gate bits (measurement order)
  auto tile_bits = [&](int it, int j, int* lidx) -> int {
    const int M = slice_M(d, j);
    const int nwd = (M + 31) / 32;
    __syncthreads();
    int nl = 0;
    for (int w0 = 0; w0 < nwd; w0 += kPT) {
      const int wd = w0 + tid;
      const unsigned bits = wd < nwd ? __ldcg(d.gbits + (long)wd * T + it) : 0u;
      const int c = __popc(bits);
      int incl = c;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (lane == 31) wcnt[wid] = incl;
      __syncthreads();
      int before = 0, all = 0;
      for (int k = 0; k < kPT / 32; ++k) {
        before += k < wid ? wcnt[k] : 0;
        all += wcnt[k];
      }
      int pos = nl + before + incl - c;
      unsigned b = bits;
      while (b) {
        const int k = __ffs(b) - 1;
        b &= b - 1u;
        lidx[pos++] = wd * 32 + k;
      }
      nl += all;
      __syncthreads();
    }
    return nl;
  };

  // the box of a warp's 64 particles (its lanes' two slots; slots past the
  // tile's end take no part); false if the warp holds none
  auto warp_box = [&](const P4<R>& q0, const P4<R>& q1, bool has0, bool has1, Box<R>& b) -> bool {
    const R inf = (R)INFINITY;
    R lo0 = inf, hi0 = -inf, lo1 = inf, hi1 = -inf;
    if (has0) {
      lo0 = q0.h0;
      hi0 = q0.h0;
      lo1 = q0.h1;
      hi1 = q0.h1;
    }
    if (has1) {
      lo0 = fmin(lo0, q1.h0);
      hi0 = fmax(hi0, q1.h0);
      lo1 = fmin(lo1, q1.h1);
      hi1 = fmax(hi1, q1.h1);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo0 = fmin(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
      hi0 = fmax(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
      lo1 = fmin(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
      hi1 = fmax(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
    }
    b = Box<R>{lo0, hi0, lo1, hi1};
    return __any_sync(0xffffffffu, has0 || has1);
  };
  // the entries e of the tile's live list (measurement points zt2(e)) that
  // can reach the warp's box, in list order, into wl; returns their count.
  // A skipped pair's term is an exact zero, so the sums do not change.
  auto warp_list = [&](const Box<R>& b, bool any, int nl, unsigned short* wl, auto zt2) -> int {
    int nw = 0;
    if (!any) return 0;
    for (int e0 = 0; e0 < nl; e0 += 32) {
      const int e = e0 + lane;
      bool keep = false;
      if (e < nl) {
        const V2<R> z = zt2(e);
        keep = !m.tune.gate || box_qmin<R, RB>(b, LB.b0, LB.b1, z.a, z.b) < gate_limit<R>(m);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) wl[nw + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)e;
      nw += __popc(bal);
    }
    __syncwarp();
    return nw;
  };

  // ---- E: pass 1 (Eq. 7): tile partials of the live measurements, in FP32
  // within the tile, written as FP64
  {
    P4<R>* sp = reinterpret_cast<P4<R>*>(smem);        // [kGT]
    int* lidx = reinterpret_cast<int*>(sp + kGT);     // [m_max]
    for (int it = bid; it < ntiles; it += nb) {
      const int j = item_pe(tpref, K, it);
      const int cnt = min(kGT, npred_s[j] - (it - tpref[j]) * kGT);
      P4<R> q0, q1;
      __syncthreads();
      const int nl = tile_gate(it, j, cnt, q0, q1, lidx, true);
      sp[tid] = q0;
      sp[tid + kPT] = q1;
      if (tid == 0 && nl > 0) atomicAdd(&d.stats[4], (unsigned long long)nl * (unsigned long long)cnt);
      const V2<R>* __restrict__ Z = slice_Z<R>(d, j);
      __syncthreads();
      // a warp per group of kPMB live measurements, its lanes over the tile's
      // particles (lane l: particles l, l + 32, ... in order), FP32 sums per
      // lane, a fixed shuffle tree over the lanes
      const int ngr = (nl + kPMB - 1) / kPMB;
      for (int gi = wid; gi < ngr; gi += kPT / 32) {
        R z0[kPMB], z1[kPMB], acc[kPMB];
#pragma unroll
        for (int k = 0; k < kPMB; ++k) {
          const int qq = gi * kPMB + k;
          const V2<R> z = qq < nl ? Z[lidx[qq]] : V2<R>{0, 0};
          z0[k] = z.a;
          z1[k] = z.b;
          acc[k] = 0;
        }
        for (int i = lane; i < cnt; i += 32) {
          const P4<R> qa = sp[i];
#pragma unroll
          for (int k = 0; k < kPMB; ++k)
            acc[k] = fma(exp2_neg(Q(z0[k], z1[k], qa.h0, qa.h1, qa.h1lo)), qa.w, acc[k]);
        }
#pragma unroll
        for (int k = 0; k < kPMB; ++k)
          for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
        if (lane == 0) {   // the tree's totals are in lane 0
#pragma unroll
          for (int k = 0; k < kPMB; ++k) {
            const int qq = gi * kPMB + k;
            if (qq < nl) d.colpart[(long)it * m.m_max + lidx[qq]] = (double)acc[k];
          }
        }
      }
    }
  }
  if (!barrier(kPhE)) return;

  // ---- F: per (slice, measurement): C = p_D cnorm (sum of the live tile
  // partials in tile order), the normaliser, ginv and the dW order key.
  // PEs on one scan with the global normaliser (Alg. 1 Step 2 with the PE
  // mean): a unit per measurement forms every PE's C^j in PE order, then
  // C_used = their mean, the same for all PEs (not in the FP32 instance at
  // 3 CTAs per SM, which runs one filter only)
  {
    const double cs = m.p_d * m.cnorm;
    R* ginv = static_cast<R*>(d.ginv);
    constexpr bool kMulti = !(sizeof(R) == 4 && MB == 3);
    const bool cglob = kMulti && !a.direct && m.ck_global && K > 1;
    const long units = a.direct ? (long)a.M : cglob ? (long)slice_M(d, 0) : (long)K * m.m_max;
    const Grp g = groups(units);
    int par = 0;
    if (cglob) {
      for (long r0 = 0; r0 < units; r0 += g.ng) {   // CTA-uniform rounds
        const long u = r0 + g.gid;
        const int p = (int)u;
        const bool act = u < units;
        if (g.G == 1 && !act) continue;
        double mean = 0.0;
        for (int j = 0; j < K; ++j) {   // C^j as below, the PEs in order
          double c = 0.0;
          if (act) {   // uniform over the group
            const unsigned* brow = d.gbits + (long)(p >> 5) * T;
            const int t1 = tpref[j + 1];
            for (int t0 = tpref[j]; t0 < t1; t0 += 32 * g.G) {
              const int it = t0 + g.gl;
              const bool live = it < t1 && ((__ldcg(brow + it) >> (p & 31)) & 1u);
              if (__any_sync(0xffffffffu, live) && live) c += __ldcg(d.colpart + (long)it * m.m_max + p);
            }
          }
          for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
          if (g.G > 1) {
            if (lane == 0) gred[par][wid][0] = c;
            __syncthreads();
            if (g.gl == 0) {
              c = 0.0;
              for (int k = 0; k < g.G; ++k) c += gred[par][g.slot * g.G + k][0];
            }
            par ^= 1;
          }
          if (act && g.gl == 0) {
            c *= cs;
            d.C[j * m.m_max + p] = c;
            mean += c;
          }
        }
        if (act && g.gl == 0) {
          const double cu = mean / (double)K;
          for (int j = 0; j < K; ++j) {
            const double c = d.C[j * m.m_max + p];
            d.Cused[j * m.m_max + p] = cu;
            const double den = d.kap[j] + cu;
            ginv[j * m.m_max + p] = den > 0.0 ? quot<R>(cs, den) : (R)0;
            const unsigned long long key = order_key(den > 0.0 ? (double)quot<R>(c, den) : 0.0);
            d.dwkey[j * m.m_max + p] = key;
            if (key > 0ull) atomicAdd(d.pnpos + j, 1);
          }
        }
      }
    } else {
      for (long r0 = 0; r0 < units; r0 += g.ng) {   // CTA-uniform rounds
        const long u = r0 + g.gid;
        int j = 0, p = 0;
        bool act = u < units;
        if (act) {
          j = a.direct ? 0 : (int)(u / m.m_max);
          p = a.direct ? (int)u : (int)(u - (long)j * m.m_max);
          act = p < slice_M(d, j);
        }
        if (g.G == 1 && !act) continue;
        // group lane l takes tiles l, l + 32 G, ... of the slice in order; the
        // bit row of word p / 32 is contiguous over tiles; only the tiles the
        // measurement reaches are loaded and added
        double c = 0.0;
        if (act) {   // uniform over the group
          const unsigned* brow = d.gbits + (long)(p >> 5) * T;
          const int t1 = tpref[j + 1];
  #pragma unroll 4
          for (int t0 = tpref[j]; t0 < t1; t0 += 32 * g.G) {   // group-uniform rounds: every lane runs every round
            const int it = t0 + g.gl;
            const bool live = it < t1 && ((__ldcg(brow + it) >> (p & 31)) & 1u);
            if (__any_sync(0xffffffffu, live) && live) c += __ldcg(d.colpart + (long)it * m.m_max + p);
          }
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (g.G > 1) {
          if (lane == 0) gred[par][wid][0] = c;
          __syncthreads();
          if (g.gl == 0) {
            c = 0.0;
            for (int k = 0; k < g.G; ++k) c += gred[par][g.slot * g.G + k][0];
          }
          par ^= 1;
        }
        if (act && g.gl == 0) {
          c *= cs;
          d.C[j * m.m_max + p] = c;
          d.Cused[j * m.m_max + p] = c;
          const double den = d.kap[j] + c;
          ginv[j * m.m_max + p] = den > 0.0 ? quot<R>(cs, den) : (R)0;
          const unsigned long long key = order_key(den > 0.0 ? (double)quot<R>(c, den) : 0.0);
          d.dwkey[j * m.m_max + p] = key;
          if (key > 0ull) atomicAdd(d.pnpos + j, 1);
        }
      }
    }
    if (bid == 0) {
      // counters: pairs, particles, measurements, updates
      unsigned long long n = 0, pairs = 0, meas = 0;
      for (int j = tid; j < K; j += kPT) {
        const unsigned long long Mj = (unsigned long long)slice_M(d, j);
        n += (unsigned long long)npred_s[j];
        pairs += (unsigned long long)npred_s[j] * Mj;
        meas += Mj;
      }
      n = warp_sum(n);
      pairs = warp_sum(pairs);
      meas = warp_sum(meas);
      __shared__ unsigned long long cst[3][kPT / 32];
      if (lane == 0) {
        cst[0][wid] = pairs;
        cst[1][wid] = n;
        cst[2][wid] = meas;
      }
      __syncthreads();
      if (tid == 0) {
        unsigned long long s0 = 0, s1 = 0, s2 = 0;
        for (int k = 0; k < kPT / 32; ++k) {
          s0 += cst[0][k];
          s1 += cst[1][k];
          s2 += cst[2][k];
        }
        d.stats[0] += s0;
        d.stats[1] += s1;
        d.stats[2] += s2;
        d.stats[3] += 1ull;
      }
    }
  }
  // ---- H: per slice: N^j (tile sums in a fixed order), the resampling plan,
  // LT_j = min(round(N^j), labels with dW > 0).  One filter: every CTA forms
  // them at the start of J from the integer sums F and G kept (N^j as exact
  // fixed-point sums of the tile sums, the largest weight and the count of
  // positive labels), and the barrier between H and J goes.
  __shared__ int nsel_s, rss_s;
  auto slice_plan = [&](int j, bool store) {
    // N^j: the FP64 sum of the tile sums by warp 0 alone (lane l: tiles l,
    // l + 32, ... in order, then a shuffle tree), so one warp per CTA uses
    // the narrow FP64 pipe; the largest weight and the count of positive
    // labels on the integer units (non-negative doubles order as their bit
    // patterns)
    double s = 0.0;
    unsigned long long mxb = 0ull;
    int npos = 0;
    const int M = slice_M(d, j);
    const int nt = tpref[j + 1] - tpref[j];
    // every thread fetches its share of the tile sums into shared memory (one
    // round of loads), then warp 0 adds them
    double* ts = reinterpret_cast<double*>(smem);   // [tiles of the slice] when they fit, else read directly
    const bool staged = (size_t)nt * sizeof(double) <= smem_bytes;
    for (int t = tid; t < nt; t += kPT) {
      const double v = __ldcg(d.rowpart + tpref[j] + t);
      if (staged) ts[t] = v;
      const unsigned long long b = (unsigned long long)__double_as_longlong(__ldcg(d.rowmax + tpref[j] + t));
      mxb = b > mxb ? b : mxb;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll 8
      for (int t = lane; t < nt; t += 32) s += staged ? ts[t] : __ldcg(d.rowpart + tpref[j] + t);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    for (int p = tid; p < M; p += kPT) npos += __ldcg(d.dwkey + j * m.m_max + p) > 0ull ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, mxb, o);
      mxb = t > mxb ? t : mxb;
    }
    npos = warp_sum(npos);
    __syncthreads();
    if (lane == 0) {
      dredb[wid] = mxb;
      wcnt[wid] = npos;
      if (wid == 0) dred[0] = s;
    }
    __syncthreads();
    if (tid == 0) {
      const double t = dred[0];
      unsigned long long tb = 0ull;
      int np = 0;
      for (int k = 0; k < kPT / 32; ++k) {
        tb = dredb[k] > tb ? dredb[k] : tb;
        np += wcnt[k];
      }
      const double tm = __longlong_as_double((long long)tb);
      int L, sc;
      resample_plan(d.rho[j], d.lmax[j], npred_s[j], t, tm, L, sc);
      long long LT = llround(t);
      if (LT > np) LT = np;
      if (LT < 0) LT = 0;
      nsel_s = (int)LT;
      rss_s = sc;
      if (store) {
        d.mass[j] = t;
        d.rs_mass[j] = t;
        d.rs_wn[j] = L > 0 ? t / (double)L : 0.0;
        d.rs_s[j] = sc;
        d.rs_L[j] = L;
        d.nsel[j] = (int)LT;
      }
    }
    __syncthreads();
  };
  arrive(kPhF);
  // the first tile's records and slots (phase D's) are fetched while the
  // other CTAs finish the normalisers
  P4<R> gq0{0, 0, 0, 0}, gq1{0, 0, 0, 0};
  int gs0 = 0, gs1 = 0;
  if (bid < ntiles) {
    const int j = item_pe(tpref, K, bid);
    const int t = bid - tpref[j];
    const int cnt = min(kGT, npred_s[j] - t * kGT);
    const long base = (long)j * m.pe_cap + (long)t * kGT;
    if (tid < cnt) {
      gq0 = geo[base + tid];
      gs0 = d.perm[base + tid];
    }
    if (tid + kPT < cnt) {
      gq1 = geo[base + kPT + tid];
      gs1 = d.perm[base + kPT + tid];
    }
  }
  if (!wait(kPhF)) return;

  // ---- G: pass 2 (Eq. 8) per tile: the live measurements from the gate
  // bits, updated weights to their slots, tile sum and largest weight
  {
    const int mm = (m.m_max + 7) & ~7;
    int* lidx = reinterpret_cast<int*>(smem);                                // [mm]
    Z4<R>* zs = reinterpret_cast<Z4<R>*>(lidx + mm);                         // [mm]
    unsigned short* wl = reinterpret_cast<unsigned short*>(zs + mm);         // [8][mm] warp lists
    const R* __restrict__ ginv = static_cast<const R*>(d.ginv);
    R* __restrict__ wu = static_cast<R*>(d.wu);
    const R miss = cc.miss;
    for (int it = bid; it < ntiles; it += nb) {
      const int j = item_pe(tpref, K, it);
      const int t = it - tpref[j];
      const int cnt = min(kGT, npred_s[j] - t * kGT);
      const long base = (long)j * m.pe_cap + (long)t * kGT;
      // the two particles' records and slots are fetched before the gate bits
      // are read
      P4<R> q0{0, 0, 0, 0}, q1{0, 0, 0, 0};
      int slot0 = 0, slot1 = 0;
      const bool has0 = tid < cnt, has1 = tid + kPT < cnt;
      if (it == bid) {
        q0 = gq0;
        q1 = gq1;
        slot0 = gs0;
        slot1 = gs1;
      } else {
        if (has0) {
          q0 = geo[base + tid];
          slot0 = d.perm[base + tid];
        }
        if (has1) {
          q1 = geo[base + kPT + tid];
          slot1 = d.perm[base + kPT + tid];
        }
      }
      __syncthreads();
      const int nl = tile_bits(it, j, lidx);
      const V2<R>* __restrict__ Z = slice_Z<R>(d, j);
      for (int e = tid; e < nl; e += kPT) {
        const int p = lidx[e];
        const V2<R> z = Z[p];
        zs[e] = Z4<R>{z.a, z.b, ginv[j * m.m_max + p], (R)0};
      }
      Box<R> wb;
      const bool any = warp_box(q0, q1, has0, has1, wb);
      __syncthreads();
      // the live measurements that can reach the warp's 64 particles, walked
      // by each thread for its two particles
      const int nw = warp_list(wb, any, nl, wl + wid * mm, [&](int e) { return V2<R>{zs[e].z0, zs[e].z1}; });
      R wv0 = 0, wv1 = 0;
      if (has0) {
        R a0 = 0, a1 = 0, b0 = 0, b1 = 0;
        for (int k = 0; k < nw; ++k) {
          const int e = wl[wid * mm + k];
          const Z4<R> za = zs[e];
          const R v = exp2_neg(Q(za.z0, za.z1, q0.h0, q0.h1, q0.h1lo)) * za.g;
          const R u = exp2_neg(Q(za.z0, za.z1, q1.h0, q1.h1, q1.h1lo)) * za.g;
          if (lidx[e] & 1) {
            a1 += v;
            b1 += u;
          } else {
            a0 += v;
            b0 += u;
          }
        }
        wv0 = (miss + (a0 + a1)) * q0.w;
        wu[(long)j * m.pe_cap + slot0] = wv0;
        if (has1) {
          wv1 = (miss + (b0 + b1)) * q1.w;
          wu[(long)j * m.pe_cap + slot1] = wv1;
        }
      }
      // tile sum and largest weight: warps in the kernel's precision, warp
      // totals in FP64 in warp order
      R sv = wv0 + wv1, mv = wv1 > wv0 ? wv1 : wv0;
      for (int o = 16; o > 0; o >>= 1) {
        sv += __shfl_down_sync(0xffffffffu, sv, o);
        const R v2 = __shfl_down_sync(0xffffffffu, mv, o);
        mv = v2 > mv ? v2 : mv;
      }
      if (lane == 0) {
        dred[wid] = (double)sv;
        bsh[wid] = mv;
      }
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        R mx = 0;
        for (int k = 0; k < kPT / 32; ++k) {
          s += dred[k];
          mx = bsh[k] > mx ? bsh[k] : mx;
        }
        d.rowpart[it] = s;
        d.rowmax[it] = (double)mx;
        // the slice's mass as exact integer sums (any order gives the same
        // bits): s 2^30 = hi + f with f in [0, 1), lo = floor(f 2^32); the
        // largest weight as an integer max of the bit patterns
        const double s30 = s * 1073741824.0;
        const unsigned long long hi = __double2ull_rz(s30);
        const unsigned long long lo = __double2ull_rz((s30 - (double)hi) * 4294967296.0);
        atomicAdd(d.pmassq + 2 * j, hi);
        atomicAdd(d.pmassq + 2 * j + 1, lo);
        atomicMax(d.pwmaxb + j, (unsigned long long)__double_as_longlong((double)mx));
      }
    }
  }
  // selection ranks (Step 3) beside pass 2: a warp per measurement, on the
  // CTAs from the end of the grid (those past the last pass-2 tile have no
  // other work here); the rank of its dW among the slice's (larger first,
  // ties to the lower label) goes to selrank, the measurement to sel[rank]
  // (the ranks are a permutation); the selection itself, rank < LT, is
  // applied where LT is known (J, K)
  if (a.direct && ntiles < nb) {
    // one filter with CTAs to spare: only those rank, each from a copy of the
    // slice's dW keys in shared memory (one load round per CTA)
    if (bid >= ntiles) {
      const int M = a.M;
      unsigned long long* ks = reinterpret_cast<unsigned long long*>(smem);   // [M]
      for (int p = tid; p < M; p += kPT) ks[p] = __ldcg(d.dwkey + p);
      __syncthreads();
      const long nw = (long)(nb - ntiles) * (kPT / 32);
      for (long u = (long)(bid - ntiles) * (kPT / 32) + wid; u < M; u += nw) {
        const int p = (int)u;
        const unsigned long long v = ks[p];
        int c = 0;
#pragma unroll 8
        for (int q = lane; q < M; q += 32) {
          const unsigned long long w2 = ks[q];
          c += (w2 > v || (w2 == v && q < p)) ? 1 : 0;
        }
        const int rank = warp_sum(c);
        if (lane == 0) {
          d.selrank[p] = rank;
          d.sel[rank] = p;
        }
      }
    }
  } else {
    const long units = a.direct ? (long)a.M : (long)K * m.m_max;
    for (long u = (long)(nb - 1 - bid) * (kPT / 32) + wid; u < units; u += nwarps) {
      const int j = a.direct ? 0 : (int)(u / m.m_max);
      const int p = a.direct ? (int)u : (int)(u - (long)j * m.m_max);
      const int M = slice_M(d, j);
      if (p >= M) continue;   // uniform over the warp
      const unsigned long long* key = d.dwkey + (long)j * m.m_max;
      const unsigned long long v = __ldcg(key + p);
      int c = 0;
#pragma unroll 8
      for (int q = lane; q < M; q += 32) {
        const unsigned long long w2 = __ldcg(key + q);
        c += (w2 > v || (w2 == v && q < p)) ? 1 : 0;
      }
      const int rank = warp_sum(c);
      if (lane == 0) {
        d.selrank[j * m.m_max + p] = rank;
        d.sel[j * m.m_max + rank] = p;
      }
    }
  }
  arrive(kPhG);
  // pass 3's first tile: records and predicted states (phases D and A) are
  // fetched while the other CTAs finish pass 2
  P4<R> jq0{0, 0, 0, 0}, jq1{0, 0, 0, 0};
  St4<R> jx0{0, 0, 0, 0}, jx1{0, 0, 0, 0};
  if (bid < ntiles) {
    const St4<R>* __restrict__ xs = static_cast<const St4<R>*>(d.x_alt);
    const int j = item_pe(tpref, K, bid);
    const int t = bid - tpref[j];
    const int cnt = min(kGT, npred_s[j] - t * kGT);
    const long base = (long)j * m.pe_cap + (long)t * kGT;
    if (tid < cnt) {
      jq0 = geo[base + tid];
      jx0 = xs[(long)j * m.pe_cap + d.perm[base + tid]];
    }
    if (tid + kPT < cnt) {
      jq1 = geo[base + kPT + tid];
      jx1 = xs[(long)j * m.pe_cap + d.perm[base + kPT + tid]];
    }
  }
  if (!wait(kPhG)) return;

  if (!a.direct) {
    for (int j = bid; j < K; j += nb) slice_plan(j, true);
    if (!barrier(kPhH)) return;
  }

  // ---- J: the CDF chunk totals per slot chunk; pass 3 per tile (Eq. 18
  // label sums of the selected labels that can reach the tile, offsets from
  // the label's point)
  {
    const R* wu = static_cast<const R*>(d.wu);
    // the weights of the CTA's first chunk (two slots per thread) are
    // fetched before the plan
    R wpre[2];
    {
      const int it = bid;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        wpre[hh] = 0;
        if (it < nitems) {
          const int j = item_pe(ipref, K, it);
          const int i = (it - ipref[j]) * kGT + hh * kPT + tid;
          if (i < npred_s[j]) wpre[hh] = wu[(long)j * m.pe_cap + i];
        }
      }
    }
    if (a.direct) {
      // one filter: N^j, the resampling plan and LT_j from F's and G's
      // integer sums (every CTA the same; CTA 0 stores them; N^j / L_j in K)
      if (tid == 0) {
        const double t = (double)__ldcg(d.pmassq) * 9.313225746154785e-10 +        // 2^-30
                         (double)__ldcg(d.pmassq + 1) * 2.168404344971009e-19;    // 2^-62
        const double tm = __longlong_as_double((long long)__ldcg(d.pwmaxb));
        const int np = __ldcg(d.pnpos);
        int L, sc;
        resample_plan(d.rho[0], d.lmax[0], npred_s[0], t, tm, L, sc);
        long long LT = llround(t);
        if (LT > np) LT = np;
        if (LT < 0) LT = 0;
        nsel_s = (int)LT;
        rss_s = sc;
        if (bid == 0) {
          d.mass[0] = t;
          d.rs_mass[0] = t;
          d.rs_s[0] = sc;
          d.rs_L[0] = L;
          d.nsel[0] = (int)LT;
        }
      }
      __syncthreads();
    }
    unsigned long long* wt = reinterpret_cast<unsigned long long*>(smem);
    for (int it = bid; it < nitems; it += nb) {
      const int j = item_pe(ipref, K, it);
      const int sj = a.direct ? rss_s : d.rs_s[j];
      unsigned long long q = 0ull;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int i = (it - ipref[j]) * kGT + hh * kPT + tid;
        const R wi = it == bid ? wpre[hh] : (i < npred_s[j] ? wu[(long)j * m.pe_cap + i] : (R)0);
        q += i < npred_s[j] ? scaled_floor(wi, sj) : 0ull;
      }
      // the chunk total: warp sums, then the 8 warp totals in warp order
      const unsigned long long ws = warp_sum(q);
      if (lane == 0) wt[wid] = ws;
      __syncthreads();
      if (tid == 0) {
        unsigned long long t = 0ull;
        for (int w2 = 0; w2 < kPT / 32; ++w2) t += wt[w2];
        d.pcsum[it] = t;
      }
      __syncthreads();
    }
    __syncthreads();
    P4<R>* sp = reinterpret_cast<P4<R>*>(smem);               // [kGT]
    St4<R>* sx = reinterpret_cast<St4<R>*>(sp + kGT);        // [kGT]
    int2* lr = reinterpret_cast<int2*>(sx + kGT);             // [m_max] live selected (rank, measurement)
    int* lidx = reinterpret_cast<int*>(lr + m.m_max);            // [m_max] live measurements
    const St4<R>* __restrict__ xs = static_cast<const St4<R>*>(d.x_alt);
    constexpr int LB = 2;   // labels per thread group
    for (int it = bid; it < ntiles; it += nb) {
      const int j = item_pe(tpref, K, it);
      const int ns = a.direct ? nsel_s : __ldcg(d.nsel + j);
      if (ns <= 0) continue;   // uniform over the block
      const int t = it - tpref[j];
      const int cnt = min(kGT, npred_s[j] - t * kGT);
      const long base = (long)j * m.pe_cap + (long)t * kGT;
      // the tile's records are fetched before its gate bits are read
      P4<R> qg0{0, 0, 0, 0}, qg1{0, 0, 0, 0};
      St4<R> xg0{0, 0, 0, 0}, xg1{0, 0, 0, 0};
      if (it == bid) {
        qg0 = jq0;
        qg1 = jq1;
        xg0 = jx0;
        xg1 = jx1;
      } else {
        if (tid < cnt) {
          qg0 = geo[base + tid];
          xg0 = xs[(long)j * m.pe_cap + d.perm[base + tid]];
        }
        if (tid + kPT < cnt) {
          qg1 = geo[base + kPT + tid];
          xg1 = xs[(long)j * m.pe_cap + d.perm[base + kPT + tid]];
        }
      }
      __syncthreads();
      const int nl = tile_bits(it, j, lidx);
      if (tid < cnt) {
        sp[tid] = qg0;
        sx[tid] = xg0;
      }
      if (tid + kPT < cnt) {
        sp[tid + kPT] = qg1;
        sx[tid + kPT] = xg1;
      }
      // the selected labels among the live measurements (any order: a
      // label's sums do not depend on its place in the list)
      if (tid == 0) nlive_s = 0;
      __syncthreads();
      for (int e = tid; e < nl; e += kPT) {
        const int p = lidx[e];
        const int r = __ldcg(d.selrank + j * m.m_max + p);
        if (r >= 0 && r < ns) lr[atomicAdd(&nlive_s, 1)] = make_int2(r, p);
      }
      __syncthreads();
      const int nr = nlive_s;
      if (nr == 0) continue;   // uniform
      const V2<R>* __restrict__ Z = slice_Z<R>(d, j);
      const int ng = (nr + LB - 1) / LB;
      int nsplit = 1;
      while (nsplit * 2 <= 32 && nsplit * 2 * ng <= kPT) nsplit *= 2;
      const int gpr = kPT / nsplit;
      const int rl = tid / nsplit, split = tid % nsplit;
      for (int g0 = 0; g0 < ng; g0 += gpr) {
        const int g = g0 + rl;
        R s[LB][5];
        R z0[LB], z1[LB], px[LB], py[LB];
#pragma unroll
        for (int k = 0; k < LB; ++k) {
#pragma unroll
          for (int c = 0; c < 5; ++c) s[k][c] = 0;
          const int qq = g * LB + k;
          V2<R> z = {0, 0};
          if (g < ng && qq < nr) z = Z[lr[qq].y];
          z0[k] = z.a;
          z1[k] = z.b;
          meas_point<R>(m, z, px[k], py[k]);
        }
        if (g < ng) {
          for (int i = split; i < cnt; i += nsplit) {
            const P4<R> q = sp[i];
            const St4<R> st = sx[i];
#pragma unroll
            for (int k = 0; k < LB; ++k) {
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
        for (int k = 0; k < LB; ++k)
#pragma unroll
          for (int c = 0; c < 5; ++c)
            for (int o = nsplit >> 1; o > 0; o >>= 1) s[k][c] += __shfl_down_sync(0xffffffffu, s[k][c], o, nsplit);
        if (split == 0 && g < ng) {
#pragma unroll
          for (int k = 0; k < LB; ++k) {
            const int qq = g * LB + k;
            if (qq < nr) {
              R* o = reinterpret_cast<R*>(d.spart) + ((long)it * m.m_max + lr[qq].x) * 5;
#pragma unroll
              for (int c = 0; c < 5; ++c) o[c] = s[k][c];
            }
          }
        }
      }
    }
  }
  arrive(kPhJ);
  // one filter, a label per CTA (the group mapping K uses when labels are
  // few): the label's measurement, its point and its output position (all
  // from G) are fetched while the other CTAs finish pass 3
  const bool kpre = a.direct && (long)nsel_s * 16 <= nwarps && bid < nsel_s;
  int kp_p = 0, kp_below = 0;
  V2<R> kp_z{0, 0};
  if (kpre) {
    kp_p = __ldcg(d.sel + bid);
    if (wid == 0) {
      int b = 0;
      for (int t = lane; t < nsel_s; t += 32) b += __ldcg(d.sel + t) < kp_p ? 1 : 0;
      kp_below = warp_sum(b);
    }
    kp_z = slice_Z<R>(d, 0)[kp_p];
  }
  if (!wait(kPhJ)) return;

  // ---- K: estimates (Eq. 18) per selected label: the live tile partials in
  // tile order, in the kernel's precision (the tile partials are sums of
  // offsets from the label's point, so the ratio keeps the estimate within
  // 1e-4 m in FP32); one filter: the output in ascending label order.  CDF
  // chunk offsets per slice (the last CTAs); selrank of the labels not
  // selected set to -1
  {
    St4<R>* est = static_cast<St4<R>*>(d.est_local);
    // one filter: units are the selected labels
    const long units = a.direct ? (long)nsel_s : (long)K * m.m_max;
    const Grp g = groups(units);
    const long gid0 = g.gid;
    if (a.direct && bid == 0 && tid == 0) {
      *d.out_count = nsel_s;
      if (a.d_count) *a.d_count = nsel_s;
    }
    int par = 0;
    for (long r0 = 0; r0 < units; r0 += g.ng) {   // CTA-uniform rounds
      const long u = r0 + gid0;
      int j = 0, r = 0, nsel = 0;
      bool act = u < units;
      if (act) {
        j = a.direct ? 0 : (int)(u / m.m_max);
        r = a.direct ? (int)u : (int)(u - (long)j * m.m_max);
        nsel = a.direct ? nsel_s : __ldcg(d.nsel + j);
        act = r < nsel;
      }
      if (g.G == 1 && !act) continue;
      int p = 0, below = 0;
      R a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
      const bool pre = kpre && g.G == kPT / 32 && r0 == 0;   // fetched before the wait
      if (act) {   // uniform over the group
        if (pre) {
          p = kp_p;
          below = wid == 0 ? kp_below : 0;   // the group's sum below adds the warps' shares
        } else {
          p = __ldcg(d.sel + j * m.m_max + r);
          if (a.direct) {
            for (int t = g.gl; t < nsel; t += 32 * g.G) below += __ldcg(d.sel + j * m.m_max + t) < p ? 1 : 0;
            below = warp_sum(below);
          }
        }
        const unsigned* brow = d.gbits + (long)(p >> 5) * T;
        const int t1 = tpref[j + 1];
#pragma unroll 4
        for (int t0 = tpref[j]; t0 < t1; t0 += 32 * g.G) {   // group-uniform rounds
          const int it = t0 + g.gl;
          const bool live = it < t1 && ((__ldcg(brow + it) >> (p & 31)) & 1u);
          if (__any_sync(0xffffffffu, live) && live) {
            const R* q = reinterpret_cast<const R*>(d.spart) + ((long)it * m.m_max + r) * 5;
            a0 += __ldcg(q);
            a1 += __ldcg(q + 1);
            a2 += __ldcg(q + 2);
            a3 += __ldcg(q + 3);
            a4 += __ldcg(q + 4);
          }
        }
      }
      if (act) {   // uniform over the warp
        for (int o = 16; o > 0; o >>= 1) {
          a0 += __shfl_down_sync(0xffffffffu, a0, o);
          a1 += __shfl_down_sync(0xffffffffu, a1, o);
          a2 += __shfl_down_sync(0xffffffffu, a2, o);
          a3 += __shfl_down_sync(0xffffffffu, a3, o);
          a4 += __shfl_down_sync(0xffffffffu, a4, o);
        }
      }
      if (g.G > 1) {
        if (lane == 0) {
          gredr[par][wid][0] = a0;
          gredr[par][wid][1] = a1;
          gredr[par][wid][2] = a2;
          gredr[par][wid][3] = a3;
          gredr[par][wid][4] = a4;
          gcnt[par][wid][1] = below;
        }
        __syncthreads();
        if (act && g.gl == 0) {
          a0 = a1 = a2 = a3 = a4 = 0;
          below = 0;
          for (int k = 0; k < g.G; ++k) {
            const int w2 = g.slot * g.G + k;
            a0 += gredr[par][w2][0];
            a1 += gredr[par][w2][1];
            a2 += gredr[par][w2][2];
            a3 += gredr[par][w2][3];
            a4 += gredr[par][w2][4];
            below += gcnt[par][w2][1];
          }
        }
        par ^= 1;
      }
      if (act && g.gl == 0) {
        const V2<R> z = pre ? kp_z : slice_Z<R>(d, j)[p];
        R px, py;
        meas_point<R>(m, z, px, py);
        St4<R> o;
        if (a0 > (R)0) {
          const R inv = (R)1 / a0;
          o.x = px + a1 * inv;
          o.vx = a2 * inv;
          o.y = py + a3 * inv;
          o.vy = a4 * inv;
        } else {
          o = St4<R>{px, (R)0, py, (R)0};
        }
        est[(long)j * m.m_max + r] = o;
        if (a.direct && below < a.cap) {
          a.out_states[4 * below + 0] = o.x;
          a.out_states[4 * below + 1] = o.vx;
          a.out_states[4 * below + 2] = o.y;
          a.out_states[4 * below + 3] = o.vy;
          a.out_labels[below] = p;
        }
      }
    }
    for (int j = nb - 1 - bid; j >= 0 && j < K; j += nb) {
      unsigned long long* wt = reinterpret_cast<unsigned long long*>(smem);
      unsigned long long carry = 0ull;
      constexpr int kCh = 4;   // consecutive chunks per thread and round
      const int cend_j = ipref[j + 1];
      for (int c0 = ipref[j]; c0 < cend_j; c0 += kCh * kPT) {
        const int cb = c0 + kCh * tid;
        unsigned long long v[kCh], sum = 0ull;
#pragma unroll
        for (int k = 0; k < kCh; ++k) {
          v[k] = cb + k < cend_j ? __ldcg(d.pcsum + cb + k) : 0ull;
          sum += v[k];
        }
        unsigned long long tot = 0;
        unsigned long long run = carry + block_scan_u64<R>(sum, wt, &tot) - sum;
#pragma unroll
        for (int k = 0; k < kCh; ++k) {
          if (cb + k < cend_j) d.pcoff[cb + k] = run;
          run += v[k];
        }
        carry += tot;
      }
      if (tid == 0) {
        d.rs_Qn[j] = carry;
        const Recip r = make_recip(carry);
        d.rs_rcp[2 * j] = r.d;
        d.rs_rcp[2 * j + 1] = r.v;
        if (a.direct) {   // the new weight N^j / L_j (batches: formed in H)
          const int L = d.rs_L[j];
          d.rs_wn[j] = L > 0 ? d.rs_mass[j] / (double)L : 0.0;
        }
      }
      __syncthreads();
    }
    {
      const long units = a.direct ? (long)a.M : (long)K * m.m_max;
      for (long x = (long)bid * kPT + tid; x < units; x += (long)nb * kPT) {
        const int j = a.direct ? 0 : (int)(x / m.m_max);
        const int p = a.direct ? (int)x : (int)(x - (long)j * m.m_max);
        if (p >= slice_M(d, j)) continue;
        const int ns = a.direct ? nsel_s : __ldcg(d.nsel + j);
        if (__ldcg(d.selrank + j * m.m_max + p) >= ns) d.selrank[j * m.m_max + p] = -1;
      }
    }
  }
  arrive(kPhK);
  // the first chunk's updated weights (phase G's) are fetched while the other
  // CTAs finish the estimates and the CDF offsets
  R lw0 = 0, lw1 = 0;
  if (bid < nitems) {
    const int j = item_pe(ipref, K, bid);
    const long base = (long)j * m.pe_cap;
    const int i0 = (bid - ipref[j]) * kGT + tid, i1 = i0 + kPT;
    const R* wu = static_cast<const R*>(d.wu);
    if (i0 < npred_s[j]) lw0 = wu[base + i0];
    if (i1 < npred_s[j]) lw1 = wu[base + i1];
  }
  if (!wait(kPhK)) return;

  // ---- L: offspring ends per slot chunk (exact integer CDF: the chunk's
  // offset plus an inclusive scan of its q_i; c = children of slots up to i)
  // and the children gathered from their parents (the chunk's children as
  // one contiguous range, shared by its threads), weight N^j / L_j; counts
  // and the step counter for the next step
  {
    const St4<R>* xp = static_cast<const St4<R>*>(d.x_alt);
    St4<R>* x = static_cast<St4<R>*>(d.x);
    R* w = static_cast<R*>(d.w);
    const R* wu = static_cast<const R*>(d.wu);
    unsigned long long* wt = reinterpret_cast<unsigned long long*>(smem);   // [kPT / 32]
    int* cend = reinterpret_cast<int*>(wt + kPT / 32);                      // [kGT]
    St4<R>* sxs = reinterpret_cast<St4<R>*>(cend + kGT);                    // [kGT] the chunk's parents
    __shared__ int cprev_s;
    if (bid == 0)
      for (int j = tid; j < K; j += kPT) d.n_cur[j] = d.rs_L[j];
    for (int it = bid; it < nitems; it += nb) {
      const int j = item_pe(ipref, K, it);
      const int n = npred_s[j];
      const int L = d.rs_L[j];
      if (L == 0) continue;   // uniform over the block
      const long base = (long)j * m.pe_cap;
      const int c0i = (it - ipref[j]) * kGT;
      const int i0 = c0i + tid, i1 = c0i + kPT + tid;   // the thread's two slots
      const R w0 = it == bid ? lw0 : (i0 < n ? wu[base + i0] : (R)0);
      const R w1 = it == bid ? lw1 : (i1 < n ? wu[base + i1] : (R)0);
      // the chunk's predicted states, staged once for its children
      sxs[tid] = i0 < n ? xp[base + i0] : St4<R>{0, 0, 0, 0};
      sxs[kPT + tid] = i1 < n ? xp[base + i1] : St4<R>{0, 0, 0, 0};
      const unsigned long long q0 = i0 < n ? scaled_floor(w0, d.rs_s[j]) : 0ull;
      const unsigned long long q1 = i1 < n ? scaled_floor(w1, d.rs_s[j]) : 0ull;
      const unsigned long long off = __ldcg(d.pcoff + it);
      const uint32_t U = a.u ? a.u[j] : philox_u32(m, (uint32_t)j, step, kTagResample);
      const unsigned long long Qn = __ldcg(d.rs_Qn + j);
      const Recip rq{__ldcg(d.rs_rcp + 2 * j), __ldcg(d.rs_rcp + 2 * j + 1), Qn ? __clzll((long long)Qn) : 0};
      // inclusive scans in slot order: the first half, then the second after
      // the first's total; slots past the slice's end repeat the last slot's
      // end (q = 0)
      unsigned long long t0 = 0;
      const unsigned long long s0 = block_scan_u64<R>(q0, wt, &t0);
      const unsigned long long s1 = block_scan_u64<R>(q1, wt, nullptr);
      cend[tid] = offspring_end(off + s0, Qn, (unsigned long long)L, U, rq);
      cend[kPT + tid] = offspring_end(off + t0 + s1, Qn, (unsigned long long)L, U, rq);
      if (tid == 0) cprev_s = offspring_end(off, Qn, (unsigned long long)L, U, rq);   // slots before the chunk
      __syncthreads();
      // the chunk's children [cprev_s, cend[kGT - 1]) are shared by all its
      // threads in turn (a parent with many children does not hold back one
      // warp); child t's parent is the first slot i with cend[i] > t
      const int cA = cprev_s, cB = cend[kGT - 1];
      const R wn = (R)d.rs_wn[j];
      for (int t = cA + tid; t < cB; t += kPT) {
        int lo = 0;
#pragma unroll
        for (int st = kGT / 2; st > 0; st >>= 1)
          if (cend[lo + st - 1] <= t) lo += st;
        const int par = c0i + lo;
        x[base + t] = sxs[lo];
        w[base + t] = wn;
        d.parent[base + t] = par;
      }
      __syncthreads();   // cend, sxs and cprev_s are rewritten by the next chunk
    }
    // every reader of this step's counter finished before the last barrier
    if (tid == 0) {
      const unsigned long long t = gtimer();
      if (bid == 0) {
        if (a.advance) *d.step += 1ull;
        atomicAdd(d.ptimes + kPhL, t - t_prev);
      }
      atomicMax(d.ptimes + 16 + kPhL, t - t_go);
      atomicAdd(d.ptimes + 32 + kPhL, t - t_go);
    }
  }
}

}  // namespace phd
