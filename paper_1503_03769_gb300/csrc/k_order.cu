// Spatial order of the predicted set for the update's pair passes.
//
// The exact likelihood gate skips a (tile, measurement) when every particle
// of the tile is far from the measurement; it pays only when a tile's
// particles are close to one another, which slot order does not give (births
// are spread over the region and resampling keeps parents in slot order).
// Before pass 1, every slice's predicted particles are put in the order of a
// 16 x 16 grid over measurement space (Hilbert order of the cells), by a
// stable counting sort: the permutation perm[sorted position] = slot is read
// by passes 1 and 2 (the particles themselves stay where they are, and every
// per-particle result goes to its own slot), so the only effect on results is
// which particles share a pass-1 / pass-2 tile (the grouping of FP32 partial
// sums); the order is deterministic.
//
// k_cell_hist: per chunk of kChunk particles: the cell key of each particle
//   (from its measurement-space point) and the chunk's 256-bin histogram;
//   the CTA that finishes a slice's last chunk then scans the slice: bin
//   totals over its chunks (four threads per bin on quarters of the chunks),
//   exclusive scan over the bins, then every (chunk, bin) start (bin-major,
//   chunk-minor).
// k_cell_scatter: per chunk: each particle's stable rank among the chunk's
//   particles with its key (a warp's peers by match, earlier warps by their
//   per-bin counts) gives its sorted position.
// The histogram kernel keeps each particle's sensor-space geometry and
// predicted weight, (h0, h1, h1lo, w) as computed for its key, and the scatter
// moves that record to the particle's sorted position: passes 1-3 then load
// one coalesced 16-byte record per particle instead of gathering the state
// through the permutation and recomputing the range and the bearing.
#include "phd_internal.cuh"

namespace phd {


static_assert(kChunk == 4 * kCells, "the slice scan uses four threads per bin");

// Scan of slice j's chunk histograms by a whole CTA of kChunk threads (the
// other CTAs' histograms read through L2), in place: chist[c][b] becomes the
// sorted position of chunk c's first particle with key b.
__device__ void scan_slice(const Dev& d, int c0, int nc, int (*part)[kCells], int* wt) {
  const int b = threadIdx.x % kCells, qtr = threadIdx.x / kCells;
  const int q0 = c0 + (nc * qtr) / 4, q1 = c0 + (nc * (qtr + 1)) / 4;
  constexpr int U = 8;   // chunk loads in flight per thread
  int tot = 0;
  for (int c = q0; c < q1; c += U) {
    int v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = c + u < q1 ? __ldcg(d.chist + (long)(c + u) * kCells + b) : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) tot += v[u];
  }
  part[qtr][b] = tot;
  __syncthreads();
  if (qtr == 0) {
    // bin totals, exclusive scan over the bins, then each quarter's start
    const int t0 = part[0][b], t1 = part[1][b], t2 = part[2][b], t3 = part[3][b];
    const int all = t0 + t1 + t2 + t3;
    const int lane = b & 31, wid = b >> 5;
    int incl = all;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wt[wid] = incl;
    asm volatile("bar.sync 1, %0;" ::"r"(kCells));   // the kCells threads of quarter 0
    int base = incl - all;
    for (int k = 0; k < wid; ++k) base += wt[k];
    part[0][b] = base;
    part[1][b] = base + t0;
    part[2][b] = base + t0 + t1;
    part[3][b] = base + t0 + t1 + t2;
  }
  __syncthreads();
  int run = part[qtr][b];
  for (int c = q0; c < q1; c += U) {
    int v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = c + u < q1 ? __ldcg(d.chist + (long)(c + u) * kCells + b) : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c + u < q1) d.chist[(long)(c + u) * kCells + b] = run;
      run += v[u];
    }
  }
}

template <class R>
__global__ void __launch_bounds__(kChunk) k_cell_hist(Dev d, Model m) {
  pdl_enter();
  __shared__ int pref[kMaxPE + 1];
  __shared__ int hist[kCells];
  __shared__ int part[4][kCells];   // scan: per-quarter bin counts, then their starts
  __shared__ int wt[kCells / 32];
  __shared__ int last_chunk;
  item_prefix(d.n_pred, m.K, pref, kChunk);
  const St4<R>* __restrict__ x = static_cast<const St4<R>*>(d.x_alt);
  const R* __restrict__ w = static_cast<const R*>(d.w_alt);
  P4<R>* __restrict__ geo_s = static_cast<P4<R>*>(d.geo_s);
  const Anchor* __restrict__ tab = static_cast<const Anchor*>(d.anchors);
  for (int c = blockIdx.x; c < pref[m.K]; c += gridDim.x) {
    const int j = item_pe(pref, m.K, c);
    const int i = (c - pref[j]) * kChunk + threadIdx.x;
    for (int b = threadIdx.x; b < kCells; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    if (i < d.n_pred[j]) {
      const long g = (long)j * m.pe_cap + i;
      const H3<R> h = meas_h<R>(m, x[g], tab);
      geo_s[g] = P4<R>{h.h0, h.h1, h.h1lo, w[g]};
      const int k = cell_key(m, (float)h.h0, (float)h.h1);
      d.ckey[g] = (unsigned char)k;
      atomicAdd(&hist[k], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kCells; b += blockDim.x) d.chist[(long)c * kCells + b] = hist[b];
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      last_chunk = atomicAdd(d.hdone + j, 1u) == (unsigned)(pref[j + 1] - pref[j] - 1);
    }
    __syncthreads();
    if (last_chunk) {
      __threadfence();
      scan_slice(d, pref[j], pref[j + 1] - pref[j], part, wt);
      if (threadIdx.x == 0) d.hdone[j] = 0u;
    }
    __syncthreads();
  }
}

template <class R>
__global__ void __launch_bounds__(kChunk) k_cell_scatter(Dev d, Model m) {
  pdl_enter();
  const P4<R>* __restrict__ geo_s = static_cast<const P4<R>*>(d.geo_s);
  P4<R>* __restrict__ geo = static_cast<P4<R>*>(d.geo);
  __shared__ int pref[kMaxPE + 1];
  __shared__ int wc[kChunk / 32][kCells];   // per-warp key counts, then their exclusive prefix over warps
  item_prefix(d.n_pred, m.K, pref, kChunk);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = blockIdx.x; c < pref[m.K]; c += gridDim.x) {
    const int j = item_pe(pref, m.K, c);
    const int i = (c - pref[j]) * kChunk + threadIdx.x;
    const bool live = i < d.n_pred[j];
    const long g = (long)j * m.pe_cap + i;
    const int key = live ? (int)d.ckey[g] : kCells;   // dead lanes form their own group
    for (int t = threadIdx.x; t < (kChunk / 32) * kCells; t += blockDim.x) (&wc[0][0])[t] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int rank_w = __popc(peers & ((1u << lane) - 1u));
    if (live && rank_w == 0) wc[wid][key] = __popc(peers);
    __syncthreads();
    // exclusive prefix over warps, one bin per thread
    for (int b = threadIdx.x; b < kCells; b += blockDim.x) {
      int run = 0;
      for (int w = 0; w < kChunk / 32; ++w) {
        const int v = wc[w][b];
        wc[w][b] = run;
        run += v;
      }
    }
    __syncthreads();
    if (live) {
      const int dst = d.chist[(long)c * kCells + key] + wc[wid][key] + rank_w;
      d.perm[(long)j * m.pe_cap + dst] = i;
      geo[(long)j * m.pe_cap + dst] = geo_s[g];
    }
    __syncthreads();
  }
}

template <class R>
cudaError_t launch_order(const Dev& d, const Model& m, cudaStream_t s) {
  const long chunks = (long)m.K * ((m.pe_cap + kChunk - 1) / kChunk);
  const int gc = (int)(chunks < 152 * 4 ? (chunks > 0 ? chunks : 1) : 152 * 4);
  launch_k(k_cell_hist<R>, dim3(gc), dim3(kChunk), 0, s, d, m);
  launch_k(k_cell_scatter<R>, dim3(gc), dim3(kChunk), 0, s, d, m);
  return cudaGetLastError();
}

int n_order_launches() { return 2; }

template cudaError_t launch_order<float>(const Dev&, const Model&, cudaStream_t);
template cudaError_t launch_order<double>(const Dev&, const Model&, cudaStream_t);

}  // namespace phd
