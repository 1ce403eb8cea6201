// Normaliser column sums (Eq. 7) for callers that cannot allocate device
// memory: phd_colsum_static.
//
// The computation is the staged path's pass 1 for a single particle set:
// tiles of kTile particles, FP32 runs per thread, FP64 partial per tile and
// measurement, and a fixed-order FP64 sum of the tile partials.  The per-tile
// partials live in kStaticScratchDoubles doubles of file-scope device memory
// instead of a caller workspace, and the bearing anchor table of the
// range-bearing sensor in a second file-scope array.  Host code reaches those
// arrays only through the device addresses cudaGetSymbolAddress returns (a
// symbol's host-side name is not a device pointer); on the first call made
// with a device current, the addresses are looked up and the anchor table is
// copied in (on the caller's stream, which the call then waits for), and both
// are cached for that device.  The cache is not invalidated by a device reset:
// after cudaDeviceReset the library's device arrays are gone and this entry
// point must not be called again in the process.
#include <cstdint>
#include <mutex>

#include "phd.h"
#include "phd_internal.cuh"

namespace phd {

// 4 MiB: ceil(n / 256) * M partial sums, e.g. 2.2e5 particles x 600 measurements
constexpr size_t kStaticScratchDoubles = 524288;
static __device__ __align__(256) double g_colsum_scratch[kStaticScratchDoubles];
static __device__ __align__(256) Anchor g_colsum_anchors[kAnchors];

constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices];
static void* g_anchor_ptr[kMaxDevices];
static std::mutex g_scratch_mu;

template <class R>
__global__ void __launch_bounds__(kThreads) k_colsum_flat(Model m, const St4<R>* __restrict__ x,
                                                          const R* __restrict__ w, int n,
                                                          const V2<R>* __restrict__ Z, int M,
                                                          const Anchor* __restrict__ tab,
                                                          double* __restrict__ part) {
  __shared__ R sh0[kTile], sh1[kTile], shl[kTile], sw[kTile];
  __shared__ double red[kThreads];
  const Lik<R> L = make_lik<R>(m);
  const R qk = (R)m.qk;
  const bool trunc = m.qk < (double)INFINITY;   // k-sigma truncation variant on
  const int tiles = (n + kTile - 1) / kTile;
  const int mper = M < kThreads ? M : kThreads;
  const int nsplit = kThreads / mper;
  const int pl = threadIdx.x % mper;
  const int split = threadIdx.x / mper;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long base = (long)tile * kTile;
    const int cnt = min(kTile, n - tile * kTile);
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
      if (split < nsplit && p < M) {
        const V2<R> z = Z[p];
        R part_ = 0;
        int k = 0;
        for (int i = split; i < cnt; i += nsplit) {
          const R q = qform<R>(L, z.a, z.b, sh0[i], sh1[i], shl[i]);
          // truncation only when the variant is on, so a NaN exponent (non-finite
          // state or measurement) propagates into C as on the staged path
          const R qq = (trunc && !(q < qk)) ? (R)INFINITY : q;
          part_ = fma(exp2_neg(qq), sw[i], part_);
          if (++k == 32) { acc += part_; part_ = 0; k = 0; }
        }
        acc += part_;
      }
      red[threadIdx.x] = (double)acc;
      __syncthreads();
      if (split == 0 && p < M) {
        double s = red[threadIdx.x];
        for (int k = 1; k < nsplit; ++k) s += red[threadIdx.x + k * mper];
        part[(long)tile * M + p] = s;
      }
      __syncthreads();
    }
  }
}

__global__ void k_colsum_flat_sum(const double* __restrict__ part, int tiles, int M, double cs,
                                  double* __restrict__ C) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < M; p += gridDim.x * blockDim.x) {
    double c = 0.0;
    for (int t = 0; t < tiles; ++t) c += part[(long)t * M + p];
    C[p] = c * cs;
  }
}

// Device addresses of the scratch array and the anchor table for the current
// device; the first call per device looks them up and fills the table with a
// copy on the caller's stream, then waits for that stream alone.
static cudaError_t static_arrays_for_current_device(cudaStream_t s, void** scratch, void** anchors) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev] || !g_anchor_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    e = cudaGetSymbolAddress(&p, g_colsum_scratch);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&q, g_colsum_anchors);
    if (e != cudaSuccess) return e;
    Anchor tab[kAnchors];
    fill_anchor_table(tab);
    e = cudaMemcpyAsync(q, tab, sizeof(tab), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);   // tab is on this stack frame
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
    g_anchor_ptr[dev] = q;
  }
  *scratch = g_scratch_ptr[dev];
  *anchors = g_anchor_ptr[dev];
  return cudaSuccess;
}

template <class R>
static cudaError_t launch_colsum_static(const Model& m, const void* x, const void* w, int n, const void* Z, int M,
                                        double* C, double* scratch, const Anchor* tab, cudaStream_t s) {
  const int tiles = (n + kTile - 1) / kTile;
  if (tiles > 0 && M > 0) {
    const int g = tiles < 152 * 4 ? tiles : 152 * 4;
    k_colsum_flat<R><<<g, kThreads, 0, s>>>(m, static_cast<const St4<R>*>(x), static_cast<const R*>(w), n,
                                            static_cast<const V2<R>*>(Z), M, tab, scratch);
  }
  if (M > 0) k_colsum_flat_sum<<<(M + 255) / 256, 256, 0, s>>>(scratch, tiles, M, m.p_d * m.cnorm, C);
  return cudaGetLastError();
}

}  // namespace phd


extern "C" phd_status phd_colsum_static(const phd_config* cfg, const void* d_x, const void* d_w, int32_t n,
                                        const void* d_Z, int32_t M, double* d_C, void* stream) {
  if (!cfg || n < 0 || M < 0) return PHD_ERR_INVALID_ARG;
  if (phd::config_problem(*cfg)) return PHD_ERR_INVALID_ARG;
  if ((n > 0 && (!d_x || !d_w)) || (M > 0 && (!d_Z || !d_C))) return PHD_ERR_INVALID_ARG;
  {
    // state rows and Z rows are read as vectors (four and two reals)
    const uintptr_t rs = cfg->precision == PHD_FP64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(d_x) % (4 * rs) != 0 || reinterpret_cast<uintptr_t>(d_w) % rs != 0 ||
        reinterpret_cast<uintptr_t>(d_Z) % (2 * rs) != 0 || reinterpret_cast<uintptr_t>(d_C) % 8 != 0)
      return PHD_ERR_INVALID_ARG;
  }
  const size_t tiles = ((size_t)n + phd::kTile - 1) / phd::kTile;
  if (tiles * (size_t)M > phd::kStaticScratchDoubles) return PHD_ERR_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  void* anchors = nullptr;
  if (phd::static_arrays_for_current_device(s, &scratch, &anchors) != cudaSuccess) return PHD_ERR_CUDA;
  const phd::Anchor* tab = static_cast<const phd::Anchor*>(anchors);
  const phd::Model m = phd::model_from_config(*cfg);
  cudaError_t e = cfg->precision == PHD_FP64
      ? phd::launch_colsum_static<double>(m, d_x, d_w, n, d_Z, M, d_C, static_cast<double*>(scratch), tab, s)
      : phd::launch_colsum_static<float>(m, d_x, d_w, n, d_Z, M, d_C, static_cast<double*>(scratch), tab, s);
  return e == cudaSuccess ? PHD_OK : PHD_ERR_CUDA;
}
