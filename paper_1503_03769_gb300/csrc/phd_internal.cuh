// Internal declarations shared by the libphd.so translation units.
//
// Device-resident state lives in one caller-owned workspace carved by
// phd_api.cu; kernels receive a `Dev` (pointers + sizes) and a `Model`
// (constants) by value.  Every per-step size the host does not know without a
// synchronisation (particle counts, |Z_k|) is read by the kernels from device
// memory, so a step's launches do not depend on the data and can be captured
// once in a CUDA graph.
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "phd.h"

namespace phd {

constexpr int kMaxPE = 256;
constexpr int kMaxM = 4096;
constexpr int kTile = 256;        // particles per work item of pass 3; smallest pass-1 tile
constexpr int kRowTileMin = 32;   // smallest pass-2 tile (8 lanes per particle)
constexpr int kChunk = 1024;      // particles per chunk of the resampling scan
constexpr int kThreads = 256;     // threads of the pair kernels

// Launch shape of the two pair passes (picked by phd_autotune or
// phd_set_tuning; results differ between shapes only by FP32 summation order).
struct Tune {
  int c_tile;    // pass 1: particles per work item (256, 512, 1024)
  int c_mb;      // pass 1: measurements per thread (1, 2, 4); 64 * c_mb per item
  int r_pb;      // pass 2: particles per thread (1, 2, 4)
  int r_g;       // pass 2: lanes sharing a particle (1, 2, 4, 8)
  int grid1;     // pass 1: CTA cap
  int grid2;     // pass 2: CTA cap
  int gate;      // 1: skip pairs past the exact likelihood gate (bit-identical results)
  int order;     // 1: passes 1 and 2 walk the particles in spatial (cell) order
};
__host__ __device__ __forceinline__ int row_tile(const Tune& t) { return kThreads / t.r_g * t.r_pb; }

// Real-typed particle state [x, vx, y, vy].
template <class R> struct alignas(4 * sizeof(R)) St4 { R x, vx, y, vy; };
template <class R> struct alignas(2 * sizeof(R)) V2 { R a, b; };

struct Model {
  int meas_model;        // 0 linear, 1 range-bearing
  int K;
  int pe_cap;
  int m_max;
  int J;                 // births per step, all PEs
  int ck_global;         // 1: every PE uses the PE-mean C
  double dt, sigma_a, sigma_ay;   // acceleration noise std per axis
  double sz0, sz1;       // measurement noise std per coordinate
  double sx, sy;         // sensor
  double rx0, rx1, ry0, ry1;
  double p_s, p_d, kappa, birth_mass, birth_vel_sigma;
  int birth_gauss;       // 1: births from N(bmean, diag(bstd^2)); 0: uniform position
  double bmean[4], bstd[4];
  double rho_pe;         // particles per target per PE
  double exchange_frac;
  int xmode;             // 0 ring, 1 all-to-all
  double xthresh;        // adaptive trigger (0: every step)
  double qk;             // likelihood truncation: pairs with exponent q >= qk are 0 (inf: exact)
  float f_qk;
  long long spin_limit;  // polls of a bounded wait on other CTAs before it gives up
  // likelihood in exp2 form: g = cnorm * 2^-(a0^2 d0^2 + a1^2 d1^2)
  double a0, a1;         // sqrt(log2(e) / 2) / sigma per measurement coordinate
  double cnorm;          // 1 / (2 pi s0 s1)
  uint64_t seed;
  // FP32 copies of the per-particle constants (FP64 is ~1/60 of the FP32 rate
  // on this part: no conversion in the FP32 kernels' inner code)
  float f_dt, f_sigma_a, f_ps, f_rx0, f_rw, f_ry0, f_rh, f_bv, f_sx, f_sy, f_miss;
  float f_sigma_ay, f_bmean[4], f_bstd[4];
  float f_bw_lo, f_bw_hi;  // birth weight nu_b / J_j for J_j = J / K and J / K + 1
  double bw_lo, bw_hi;
  Tune tune;
  // measurement-driven birth (Eq. 6 with a learned p_k(.|Z_k)); FP32 handles
  int learned;           // 1: births from the network's mixture proposal
  int jmax;              // most births of one PE (rows of the injected extra draws)
  float f_alpha;         // weight of the plain birth in the defensive mixture
  float f_blog;          // log2(area s_b^2 / (2 pi s_z0 s_z1))
  float f_win0, f_win1;  // feature window: 3 sigma per measurement coordinate
  float f_cx, f_cy, f_ihx, f_ihy;  // region centre and 1 / half-width
  // 16 x 16 cell grid over measurement space (spatial order of the pair passes)
  float f_cell_o0, f_cell_s0, f_cell_o1, f_cell_s1;
};

// Per-particle model constants in the kernel's precision.
template <class R> struct Cst {
  R dt, sa, ps, rx0, rw, ry0, rh, bv, sx, sy, miss, bw_lo, bw_hi;
  R say;              // y-axis acceleration noise std
  int gauss;          // Gaussian birth density
  R bm[4], bs[4];     // its mean and std per state component
};
template <class R> __device__ __forceinline__ Cst<R> consts(const Model& m);
template <> __device__ __forceinline__ Cst<float> consts<float>(const Model& m) {
  return Cst<float>{m.f_dt, m.f_sigma_a, m.f_ps, m.f_rx0, m.f_rw, m.f_ry0, m.f_rh, m.f_bv, m.f_sx, m.f_sy,
                    m.f_miss, m.f_bw_lo, m.f_bw_hi, m.f_sigma_ay, m.birth_gauss,
                    {m.f_bmean[0], m.f_bmean[1], m.f_bmean[2], m.f_bmean[3]},
                    {m.f_bstd[0], m.f_bstd[1], m.f_bstd[2], m.f_bstd[3]}};
}
template <> __device__ __forceinline__ Cst<double> consts<double>(const Model& m) {
  return Cst<double>{m.dt, m.sigma_a, m.p_s, m.rx0, m.rx1 - m.rx0, m.ry0, m.ry1 - m.ry0, m.birth_vel_sigma, m.sx,
                     m.sy, 1.0 - m.p_d, m.bw_lo, m.bw_hi, m.sigma_ay, m.birth_gauss,
                     {m.bmean[0], m.bmean[1], m.bmean[2], m.bmean[3]},
                     {m.bstd[0], m.bstd[1], m.bstd[2], m.bstd[3]}};
}

// Workspace carve (device pointers).  Real-typed arrays are void* and cast by
// the kernels' Real type.
struct Dev {
  void* x;               // St4<R> [K*pe_cap]  current set (after resampling / exchange)
  void* w;               // R [K*pe_cap]
  void* x_alt;           // St4<R> [K*pe_cap]  predicted set (survivors + births)
  void* w_alt;           // R [K*pe_cap]       predicted weights
  void* wu;              // R [K*pe_cap]       updated weights (Eq. 8)
  void* x_out;           // St4<R> [K*pe_cap]  exchange outbox
  void* w_out;           // R [K*pe_cap]
  int* n_cur;            // [K] particles per PE (survivors before predict)
  int* n_pred;           // [K] particles per PE after predict
  void* Z;               // V2<R> [m_max]  measurements (as given)
  const void* anchors;   // Anchor [kAnchors] bearing anchor table
  int* M;                // [1]
  double* colpart;       // [max_items][m_max] pass-1 partial column sums
  double* C;             // [K][m_max] C^j (with p_D cnorm)
  double* Cused;         // [K][m_max] normaliser each PE applies
  void* ginv;            // R [K][m_max]  cnorm p_D / (kappa + Cused)
  double* rowpart;       // [K*ceil(pe_cap/kRowTileMin)] pass-2 sums of updated weights
  double* rowmax;        // same: largest updated weight per tile
  unsigned long long* dwkey; // [K][m_max] order keys of dW^{j,p}
  double* mass;          // [K] updated mass N^j
  int* nsel;             // [K] labels selected per PE
  int* sel;              // [K][m_max] selected labels, selection order
  int* selrank;          // [K][m_max] label -> selection rank or -1
  double* spart;         // [max_items][m_max][5] pass-3 partial labelled sums (the grid step kernel stores reals)
  void* est_local;       // St4<R> [K][m_max] local estimates (selection order)
  int* out_count;        // [1] fused estimate count
  double* rs_mass;       // [K] mass before resampling
  double* rs_wn;         // [K] weight of a resampled particle, N^j / L_j
  int* rs_s;             // [K] CDF scale exponent
  int* rs_L;             // [K] resample counts
  unsigned long long* csum;  // [K*ceil(pe_cap/kChunk)] CDF chunk totals
  unsigned long long* coff;  // same: exclusive chunk offsets
  unsigned long long* rs_Qn; // [K] CDF total
  unsigned long long* rs_rcp;  // [K][2] normalised CDF total and its reciprocal (make_recip)
  int* child_end;        // [K*pe_cap]
  int* parent;           // [K*pe_cap]
  int* xslots;           // [K][pe_cap] exchange slots
  int* lx;               // [1] particles moved per PE
  unsigned int* bar;     // [4] grid barrier: [0..1] 64-bit arrival count, [2] injected lost-PE flag
  // per-slice descriptors (a slice is a PE of one filter, or one run of a
  // batch of independent filters); slot j*pe_cap .. of every [K][pe_cap] array
  int zshared;           // 1: every slice uses Z rows 0 .. *M-1 (one filter)
  int* zoff;             // [K] first measurement row of slice j (zshared == 0)
  int* Mj;               // [K] measurement count of slice j (zshared == 0)
  double* kap;           // [K] clutter intensity kappa of slice j
  double* rho;           // [K] particles per target of slice j
  int* Jb;               // [K] births per step of slice j
  float* bwf;            // [K] birth weight nu_b / J_j (FP32 copy)
  double* bwd;           // [K] birth weight nu_b / J_j
  int* lmax;             // [K] largest resample count of slice j
  unsigned long long* step;  // [1] step counter (Philox counter word)
  unsigned long long* stats; // [5] sums over updates: pairs, particles, measurements, updates,
                             //     pass-1 pairs evaluated (the rest were past the gate)
  int* err;              // [1] device error bits
  int max_items;
  // measurement-driven birth
  void* mlp_w;           // bfloat16 [kNParams] network parameters
  float* bhead;          // [m_max][5] network output per measurement
  float* bcomp;          // [m_max][8] proposal component constants
  float* bcdf;           // [m_max] mixture CDF
  unsigned int* bdone;   // [1] CTAs of k_birth_head finished (the last builds the table)
  // spatial order of the predicted set
  unsigned char* ckey;   // [K*pe_cap] cell key of each predicted particle
  int* chist;            // [chunks][256] per-chunk cell counts, then their starts
  int* perm;             // [K][pe_cap] slot of the particle at each sorted position
  unsigned int* hdone;   // [K] cell-histogram chunks finished per slice (the last scans the slice)
  void* geo_s;           // P4<R> [K*pe_cap] sensor-space geometry and predicted weight, slot order
  void* geo;             // P4<R> [K*pe_cap] the same at each sorted position (read by passes 1-3)
  // persistent step kernel (k_step_grid): items of 256 particles of every slice
  int* pchist;           // [max_items][256] cell counts per slot chunk, then their sorted starts
  int* bintot;           // [K][256] cell totals per slice
  unsigned int* gbits;   // [max_items][gwords] measurements that reach each sorted tile (gate survivors)
  unsigned long long* pcsum;  // [max_items] CDF totals per slot chunk
  unsigned long long* pcoff;  // [max_items] their exclusive offsets within the slice
  unsigned long long* pbar;   // [1] arrival count of the kernel's grid barriers (only grows)
  unsigned long long* pmassq; // [2K] grid path: slice mass as two fixed-point integers (2^-30 and 2^-62 units), integer adds of the tile sums
  unsigned long long* pwmaxb; // [K] grid path: largest updated weight (bit pattern, integer max)
  int* pnpos;                 // [K] grid path: labels with dW > 0
  unsigned long long* ptimes; // [16] phase durations summed over launches, ns
  int gwords;            // words of gbits per tile: ceil(m_max / 32)
};

enum : int { kErrNonFinite = 1, kErrCapacity = 2, kErrTimeout = 4 };
constexpr long long kDefaultSpinLimit = 20000000;   // several seconds of polls (32 ns sleep + an L2 read)

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based RNG.
// ---------------------------------------------------------------------------
struct U4 { uint32_t a, b, c, d; };

__device__ __forceinline__ U4 philox4x32_10(U4 ctr, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, ctr.a), lo0 = M0 * ctr.a;
    uint32_t hi1 = __umulhi(M1, ctr.c), lo1 = M1 * ctr.c;
    ctr = U4{hi1 ^ ctr.b ^ k0, lo1, hi0 ^ ctr.d ^ k1, lo0};
    k0 += W0;
    k1 += W1;
  }
  return ctr;
}

// Stream tags of the Philox counter's third word.
enum : uint32_t {
  kTagPredict = 0x50524544u, kTagResample = 0x52534d50u, kTagExchange = 0x58434847u, kTagBirth = 0x42495254u
};

// u in (0, 1) from 32 random bits, in the kernel's real type.
template <class R> __device__ __forceinline__ R unit_open(uint32_t b);
template <> __device__ __forceinline__ float unit_open<float>(uint32_t b) {
  return ((float)(b >> 8) + 0.5f) * (1.0f / 16777216.0f);
}
template <> __device__ __forceinline__ double unit_open<double>(uint32_t b) {
  return ((double)b + 0.5) * (1.0 / 4294967296.0);
}

// ---------------------------------------------------------------------------
// exp2 of a non-positive argument in the kernel's precision.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float exp2_neg(float q) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-q));
  return r;
}
__device__ __forceinline__ double exp2_neg(double q) { return exp2(-q); }

// ---------------------------------------------------------------------------
// Measurement-space geometry of a particle (Sec. 4 sensor models).
//
// h0, h1 are the particle's noise-free measurement, unscaled: (x, y) for the
// linear sensor, (range, bearing) for the range-bearing sensor.  The pair
// kernels subtract the measurement from h first and scale afterwards, so the
// difference of two close values is exact (Sterbenz) and the FP32 exponent
// carries no rounding of |z| or |h|.
//
// FP32 bearing: atan2f is only good to a few ulp of pi (~7e-7 rad, ~1e-4 of
// the likelihood at 3 sigma for 0.5 deg bearing noise), so the bearing is
// carried as a double-float h1 + h1lo.  An anchor direction (c_k, s_k) close
// to the particle's is taken from a 256-entry table whose exact angles
// theta_k = atan2(s_k, c_k) are precomputed in FP64; rotating (px, py) by the
// anchor with error-free products gives the small residual angle exactly
// enough (|delta| <= pi/256), and theta = theta_k + delta.
// ---------------------------------------------------------------------------
constexpr int kAnchors = 256;
struct Anchor { float c, s, th_hi, th_lo; };

template <class R> struct H3 { R h0, h1, h1lo; };
// a particle's sensor-space geometry and weight, packed for one shared load
template <class R> struct alignas(4 * sizeof(R)) P4 { R h0, h1, h1lo, w; };
// a measurement and its 1 / normaliser, packed for one shared load
template <class R> struct alignas(4 * sizeof(R)) Z4 { R z0, z1, g, pad; };

// Likelihood constants: q = b0 d0^2 + b1 d1^2 with b = log2(e) / (2 sigma^2),
// so g = cnorm 2^-q; the bearing period 2 pi as a double-float.
template <class R> struct Lik {
  int rb;
  R b0, b1, per_hi, per_lo;
};

template <class R> __device__ __forceinline__ Lik<R> make_lik(const Model& m) {
  Lik<R> L;
  L.rb = m.meas_model;
  L.b0 = (R)(m.a0 * m.a0);
  L.b1 = (R)(m.a1 * m.a1);
  const double two_pi = 6.283185307179586476925286766559;
  L.per_hi = (R)two_pi;
  L.per_lo = (R)(two_pi - (double)L.per_hi);
  return L;
}

__device__ __forceinline__ void bearing_df(float px, float py, const Anchor* __restrict__ tab, float& hi, float& lo) {
  const float t0 = atan2f(py, px);
  int k = __float2int_rn(t0 * (kAnchors / 6.283185307179586f));
  k &= (kAnchors - 1);
  const Anchor a = tab[k];
  // v = py c - px s with error-free products (TwoProduct via FMA)
  const float p1 = py * a.c, e1 = fmaf(py, a.c, -p1);
  const float p2 = px * a.s, e2 = fmaf(px, a.s, -p2);
  const float vhi = p1 - p2;            // exact: p1 ~ p2 when the anchor is close
  const float v = vhi + (e1 - e2);
  const float u = fmaf(px, a.c, py * a.s);
  const float t = u != 0.0f ? v / u : 0.0f;   // |t| <= tan(pi/256); 0 at the sensor
  const float delta = t - t * t * t * (1.0f / 3.0f);
  // theta = th_hi + th_lo + delta as a double-float
  const float s = a.th_hi + delta;
  const float bb = s - a.th_hi;
  const float err = (a.th_hi - (s - bb)) + (delta - bb);
  hi = s;
  lo = err + a.th_lo;
}

// FP32 range sqrt(px^2 + py^2) to within about half an ulp: the squares as
// double-floats (error-free products by FMA), their sum by TwoSum, then one
// Newton step r + (s - r^2) / (2 r) on the low parts.  sqrtf(fmaf(px, px,
// py py)) is off by up to ~3 ulp (~1.7e-4 m at 1.4 km), which at several range
// sigmas moves the likelihood by ~1e-4 relative.
__device__ __forceinline__ float range_f32(float px, float py) {
  const float qx = __fmul_rn(px, px), ex = fmaf(px, px, -qx);
  const float qy = __fmul_rn(py, py), ey = fmaf(py, py, -qy);
  const float sh = __fadd_rn(qx, qy);
  const float bb = __fsub_rn(sh, qx);
  const float sl = __fadd_rn(__fsub_rn(qx, __fsub_rn(sh, bb)), __fsub_rn(qy, bb)) + (ex + ey);
  const float r = sqrtf(sh);
  return r > 0.0f ? r + (fmaf(-r, r, sh) + sl) * (0.5f / r) : 0.0f;
}

template <class R>
__device__ __forceinline__ H3<R> meas_h(const Model& m, const St4<R>& st, const Anchor* __restrict__ tab);

template <>
__device__ __forceinline__ H3<float> meas_h<float>(const Model& m, const St4<float>& st, const Anchor* __restrict__ tab) {
  H3<float> h;
  if (m.meas_model == 0) {
    h.h0 = st.x;
    h.h1 = st.y;
    h.h1lo = 0.0f;
  } else {
    const float px = st.x - m.f_sx, py = st.y - m.f_sy;
    h.h0 = range_f32(px, py);
    bearing_df(px, py, tab, h.h1, h.h1lo);
  }
  return h;
}

template <>
__device__ __forceinline__ H3<double> meas_h<double>(const Model& m, const St4<double>& st, const Anchor* __restrict__) {
  H3<double> h;
  if (m.meas_model == 0) {
    h.h0 = st.x;
    h.h1 = st.y;
  } else {
    const double px = st.x - m.sx, py = st.y - m.sy;
    h.h0 = sqrt(fma(px, px, py * py));
    h.h1 = atan2(py, px);
  }
  h.h1lo = 0.0;
  return h;
}

// Bearing residual |z1 - (h1 + h1lo)| wrapped to [0, pi] (the exponent only
// squares it); d1 = z1 - h1 as rounded.  Bearings lie in (-pi, pi]: on the
// same side of the +-pi cut, z1 - h1 is exact for every pair that can matter
// (Sterbenz), and the wrap is not needed.  Across the cut the raw difference
// is near +-2 pi, where FP32 rounds it to 2.4e-7 rad (~1e-4 of the likelihood
// at 3 sigma for 0.5 deg noise); that rare case recovers the rounding error
// (TwoSum) and wraps with 2 pi as a double-float.
__device__ __forceinline__ float bearing_resid(float z1, float h1, float h1lo, float d1, float per_hi,
                                               float per_lo) {
  const float a = fabsf(d1 - h1lo);
  if (a <= 3.14159265f) return a;
  const float bb = d1 - z1;
  const float err = (z1 - (d1 - bb)) + (-h1 - bb);        // z1 - h1 = d1 + err exactly
  const float sg = d1 > 0.0f ? 1.0f : -1.0f;
  return fabsf((per_hi - sg * d1) + (per_lo - sg * (err - h1lo)));
}
__device__ __forceinline__ double bearing_resid(double, double, double h1lo, double d1, double per_hi,
                                                double per_lo) {
  const double a = fabs(d1 - h1lo);
  return fmin(a, (per_hi - a) + per_lo);
}

// Exponent q of the likelihood 2^-q for measurement (z0, z1) and particle h.
template <class R>
__device__ __forceinline__ R qform(const Lik<R>& L, R z0, R z1, R h0, R h1, R h1lo) {
  const R d0 = z0 - h0;
  R d1 = z1 - h1;
  if (L.rb) d1 = bearing_resid(z1, h1, h1lo, d1, L.per_hi, L.per_lo);
  return fma(L.b1 * d1, d1, (L.b0 * d0) * d0);
}

// Exponent q of the likelihood with the sensor model fixed at compile time
// (same arithmetic as qform).
template <class R, int RB>
__device__ __forceinline__ R qform_t(const Lik<R>& L, R z0, R z1, R h0, R h1, R h1lo) {
  const R d0 = z0 - h0;
  R d1 = z1 - h1;
  if (RB & 1) d1 = bearing_resid(z1, h1, h1lo, d1, L.per_hi, L.per_lo);
  return fma(L.b1 * d1, d1, (L.b0 * d0) * d0);
}

// FP32 pair exponent with packed two-lane instructions (f32x2, sm_100 and
// later): (z0 - h0, z1 - h1) in one subtract and (a0 d0, a1 d1) in one
// multiply, a = sqrt(b); q = (a0 d0)^2 + (a1 d1)^2.  Same subtract-then-scale
// order as qform (the bearing's low word and wrap on the second lane).
struct LikP {
  unsigned long long a01;   // packed (a0, a1)
  float per_hi, per_lo;
  float qk;                 // truncation (inf: none)
};
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ LikP make_likp(const Model& m) {
  const double two_pi = 6.283185307179586476925286766559;
  LikP L;
  L.a01 = f2_pack((float)m.a0, (float)m.a1);
  L.per_hi = (float)two_pi;
  L.per_lo = (float)(two_pi - (double)L.per_hi);
  L.qk = m.f_qk;
  return L;
}
template <int RB>
__device__ __forceinline__ float qform_p(const LikP& L, unsigned long long z, unsigned long long h, float h1lo) {
  float d0, d1;
  f2_unpack(f2_sub(z, h), d0, d1);
  if (RB & 1) {
    float z0, z1, h0, h1;
    f2_unpack(z, z0, z1);
    f2_unpack(h, h0, h1);
    d1 = bearing_resid(z1, h1, h1lo, d1, L.per_hi, L.per_lo);
  }
  float e0, e1;
  f2_unpack(f2_mul(f2_pack(d0, d1), L.a01), e0, e1);
  return fmaf(e0, e0, e1 * e1);
}

// ---------------------------------------------------------------------------
// Exact likelihood gate.  ex2.approx.ftz returns exactly 0 for an exponent
// q > 126 (2^-q is below the smallest normal float and is flushed), and the
// FP64 exp2 underflows to 0 beyond q = 1074: a pair with q >= gate_q<R>() adds
// exactly nothing to any sum of the update.  A box around a tile's particles
// in measurement space bounds q from below for every pair of the tile with a
// measurement; pairs are skipped only when that bound reaches the gate (with
// margin over 126 / 1074 for rounding), so every sum is bit-identical to the
// ungated one.
// ---------------------------------------------------------------------------
template <class R> __host__ __device__ constexpr R gate_q();
template <> __host__ __device__ constexpr float gate_q<float>() { return 130.0f; }
template <> __host__ __device__ constexpr double gate_q<double>() { return 1100.0; }

// Box of a tile in measurement space: [lo0, hi0] in the first coordinate;
// the second as an interval [lo1, hi1] (linear sensor) or an arc of centre c1
// and half-width hw1 (bearing; hw1 < 0: the tile spans more than a half
// circle and the bearing gives no bound).
template <class R> struct Box { R lo0, hi0, lo1, hi1; };

// Lower bound of q over the box for measurement (z0, z1); b = log2(e)/(2 s^2).
template <class R, int RB>
__device__ __forceinline__ R box_qmin(const Box<R>& B, R b0, R b1, R z0, R z1) {
  const R d0 = fmax(fmax(B.lo0 - z0, z0 - B.hi0), (R)0);
  R d1;
  if (RB & 1) {
    const R c = (R)0.5 * (B.lo1 + B.hi1), hw = (R)0.5 * (B.hi1 - B.lo1);
    if (hw > (R)1.5707963267948966) {
      d1 = 0;
    } else {
      const R two_pi = (R)6.283185307179586;
      R t = z1 - c;
      t = t - two_pi * rint(t / two_pi);
      d1 = fmax(fabs(t) - hw, (R)0);
    }
  } else {
    d1 = fmax(fmax(B.lo1 - z1, z1 - B.hi1), (R)0);
  }
  return fma(b1 * d1, d1, (b0 * d0) * d0);
}

// Block-wide box of the values each thread passes (threads with none pass
// +inf / -inf); every thread gets the box.  Two barriers; `sh` holds 4 *
// (blockDim / 32) reals.
template <class R>
__device__ __forceinline__ Box<R> block_box(R lo0, R hi0, R lo1, R hi1, R* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    lo0 = fmin(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
    hi0 = fmax(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
    lo1 = fmin(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
    hi1 = fmax(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
  }
  const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    sh[wid] = lo0;
    sh[nw + wid] = hi0;
    sh[2 * nw + wid] = lo1;
    sh[3 * nw + wid] = hi1;
  }
  __syncthreads();
  Box<R> B{sh[0], sh[nw], sh[2 * nw], sh[3 * nw]};
  for (int k = 1; k < nw; ++k) {
    B.lo0 = fmin(B.lo0, sh[k]);
    B.hi0 = fmax(B.hi0, sh[nw + k]);
    B.lo1 = fmin(B.lo1, sh[2 * nw + k]);
    B.hi1 = fmax(B.hi1, sh[3 * nw + k]);
  }
  return B;
}

// Pair exponent in the kernels' precision: packed FP32, or plain FP64.  The
// kernels' compile-time model flag RB carries the sensor (bit 0: range-
// bearing) and the k-sigma truncation (bit 1): with it, an exponent at or
// past qk = k^2 log2(e) / 2 is returned as +inf, whose exp2 is exactly 0;
// without it no per-pair test is compiled in.
template <class R, int RB> struct PairQ;
template <int RB> struct PairQ<float, RB> {
  LikP L;
  __device__ __forceinline__ explicit PairQ(const Model& m) : L(make_likp(m)) {}
  __device__ __forceinline__ float operator()(float z0, float z1, float h0, float h1, float h1lo) const {
    const float q = qform_p<RB>(L, f2_pack(z0, z1), f2_pack(h0, h1), h1lo);
    if constexpr ((RB & 2) != 0) return q < L.qk ? q : INFINITY;
    return q;
  }
};
template <int RB> struct PairQ<double, RB> {
  Lik<double> L;
  double qk;
  __device__ __forceinline__ explicit PairQ(const Model& m) : L(make_lik<double>(m)), qk(m.qk) {}
  __device__ __forceinline__ double operator()(double z0, double z1, double h0, double h1, double h1lo) const {
    const double q = qform_t<double, RB>(L, z0, z1, h0, h1, h1lo);
    if constexpr ((RB & 2) != 0) return q < qk ? q : (double)INFINITY;
    return q;
  }
};

// The compile-time model flag of a handle: sensor bit | truncation bit.
__host__ __device__ __forceinline__ int model_flag(const Model& m) {
  return (m.meas_model ? 1 : 0) | (m.qk < (double)INFINITY ? 2 : 0);
}

// Exponent beyond which a measurement cannot reach a work item's particles:
// the exp2 flush (gate_q) or the truncation, whichever is lower.
template <class R> __device__ __forceinline__ R gate_limit(const Model& m) {
  return fmin(gate_q<R>(), (R)m.qk);
}

// Quotient in the kernel's precision: the FP32 kernels round the operands to
// FP32 and divide in FP32 (the FP64 divide is a long sequence on the ~2
// lanes/clk/SM FP64 pipe and dominated the small per-label phases); the FP64
// kernels divide in FP64.
template <class R> __device__ __forceinline__ R quot(double a, double b);
template <> __device__ __forceinline__ float quot<float>(double a, double b) { return (float)a / (float)b; }
template <> __device__ __forceinline__ double quot<double>(double a, double b) { return a / b; }

// ---------------------------------------------------------------------------
// Programmatic dependent launch (sm_90 and later).  The staged kernels are
// launched with programmatic stream serialisation: a kernel may be scheduled
// while its predecessor's last CTAs still run, and its first statement waits
// (griddepcontrol.wait) until the predecessor has completed and its writes are
// visible, so no dependent read can come early; each kernel then lets its own
// successor be scheduled.  This hides the launch gap between the ~15 kernels
// of a staged step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... KArgs, class... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Work-item decode for the pair kernels: item -> (PE, particle tile), tiles
// of kTile over each PE's count.  pref gets K+1 entries in shared memory; the
// block needs at least kMaxPE threads (tile counts are scanned in parallel).
__device__ __forceinline__ void item_prefix(const int* n, int K, int* pref, int tile = kTile) {
  __shared__ int wt[kMaxPE / 32];
  const int t = threadIdx.x;
  const int v = t < K ? (n[t] + tile - 1) / tile : 0;
  const int lane = t & 31, wid = t >> 5;
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (t < kMaxPE && lane == 31) wt[wid] = incl;
  __syncthreads();
  if (t < K) {
    int off = 0;
    for (int k = 0; k < wid; ++k) off += wt[k];
    pref[t] = off + incl - v;
    if (t == K - 1) pref[K] = off + incl;
  }
  __syncthreads();
}
// Prefix over slices of per-slice item counts computed by cnt(j) (block of
// >= kMaxPE threads); pref gets K+1 entries.
template <class F>
__device__ __forceinline__ void slice_prefix(int K, int* pref, F cnt) {
  __shared__ int wt2[kMaxPE / 32];
  const int t = threadIdx.x;
  const int v = t < K ? cnt(t) : 0;
  const int lane = t & 31, wid = t >> 5;
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (t < kMaxPE && lane == 31) wt2[wid] = incl;
  __syncthreads();
  if (t < K) {
    int off = 0;
    for (int k = 0; k < wid; ++k) off += wt2[k];
    pref[t] = off + incl - v;
    if (t == K - 1) pref[K] = off + incl;
  }
  __syncthreads();
}

__device__ __forceinline__ int item_pe(const int* pref, int K, int item) {
  int lo = 0, hi = K - 1;   // last j with pref[j] <= item
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__host__ __device__ __forceinline__ int births_of(int J, int K, int j) {
  return J / K + (j < J % K ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Prediction of one particle slot (Eq. 5-6), shared by the staged and fused
// paths.  Slot i of PE j: a survivor when i < L (CV transition, weight p_S w),
// else a birth (position U(region), velocity N(0, s_b^2 I), weight nu_b / J_j).
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void draw_noise(const Model& m, const R* noise, long g, unsigned long long step,
                                           R& n1, R& n2, R& u1, R& u2) {
  if (noise) {
    const St4<R> nz = reinterpret_cast<const St4<R>*>(noise)[g];
    n1 = nz.x;
    n2 = nz.vx;
    u1 = nz.y;
    u2 = nz.vy;
  } else {
    const U4 r = philox4x32_10(U4{(uint32_t)g, (uint32_t)step, kTagPredict, (uint32_t)(step >> 32)},
                               (uint32_t)m.seed, (uint32_t)(m.seed >> 32));
    // Box-Muller on two open-interval uniforms
    const R ua = unit_open<R>(r.a), ub = unit_open<R>(r.b);
    const R rad = sqrt((R)-2 * log(ua));
    R sn, cs;
    sincospi((R)2 * ub, &sn, &cs);
    n1 = rad * cs;
    n2 = rad * sn;
    u1 = unit_open<R>(r.c);
    u2 = unit_open<R>(r.d);
  }
}

template <class R>
__device__ __forceinline__ void predict_slot(const Cst<R>& c, bool survivor, const St4<R>& s, R w, R bw, R n1, R n2,
                                             R u1, R u2, St4<R>& o, R& wo) {
  if (survivor) {
    const R T = c.dt;
    const R ax = c.sa * n1, ay = c.say * n2;
    o.x = s.x + T * s.vx + (R)0.5 * T * T * ax;
    o.vx = s.vx + T * ax;
    o.y = s.y + T * s.vy + (R)0.5 * T * T * ay;
    o.vy = s.vy + T * ay;
    wo = c.ps * w;
  } else if (c.gauss) {
    // Gaussian birth density: velocity normals (n1, n2), position normals by
    // Box-Muller from (u1, u2): r = sqrt(-2 ln(1 - u1)), angle 2 pi u2
    const R rad = sqrt((R)-2 * log1p(-u1));
    R sn, cs;
    sincospi((R)2 * u2, &sn, &cs);
    o.x = c.bm[0] + c.bs[0] * (rad * cs);
    o.vx = c.bm[1] + c.bs[1] * n1;
    o.y = c.bm[2] + c.bs[2] * (rad * sn);
    o.vy = c.bm[3] + c.bs[3] * n2;
    wo = bw;
  } else {
    o.x = c.rx0 + u1 * c.rw;
    o.vx = c.bv * n1;
    o.y = c.ry0 + u2 * c.rh;
    o.vy = c.bv * n2;
    wo = bw;
  }
}

// Step 6: the source PE of receiver j's t-th exchanged particle (ring: j - 1;
// all-to-all: j - 1 - (t mod (K - 1)), so for each t the sources are a
// rotation of the PEs and every PE sends and receives one particle).
__device__ __forceinline__ int exchange_source(const Model& m, int j, int t) {
  const int s = m.xmode && m.K > 2 ? 1 + t % (m.K - 1) : 1;
  return (j + m.K - s) % m.K;
}

// Particles each PE sends in this step's exchange, by one whole warp: L_x =
// floor(frac * min_j L_j) over the PEs' resample counts, or 0 when the
// adaptive trigger is on and no PE has degenerated, i.e. unless
// min_j N^j < threshold * (sum_j N^j) / K (N^j the PEs' masses after the
// update, summed in PE order in FP64).  The lanes load the K counts and
// masses at once (sm: K doubles of scratch); every lane returns L_x.
__device__ __forceinline__ int exchange_count_warp(const Dev& d, const Model& m, double* sm) {
  const int lane = threadIdx.x & 31;
  int nmin = INT_MAX;
  for (int k = lane; k < m.K; k += 32) {
    nmin = min(nmin, __ldcg(d.rs_L + k));
    if (m.xthresh > 0.0) sm[k] = __ldcg(d.rs_mass + k);
  }
  nmin = __reduce_min_sync(0xffffffffu, nmin);
  __syncwarp();
  int due = 1;
  if (m.xthresh > 0.0) {
    if (lane == 0) {
      double sum = 0.0, mn = INFINITY;
      for (int k = 0; k < m.K; ++k) {
        sum += sm[k];
        mn = fmin(mn, sm[k]);
      }
      due = mn < m.xthresh * (sum / (double)m.K) ? 1 : 0;
    }
    due = __shfl_sync(0xffffffffu, due, 0);
  }
  return due ? (int)floor(m.exchange_frac * (double)nmin) : 0;
}

// Birth weight nu_b / J_j of PE j.
template <class R> __device__ __forceinline__ R birth_weight(const Cst<R>& c, const Model& m, int j) {
  return (j < m.J % m.K) ? c.bw_hi : c.bw_lo;
}

// floor(w 2^s) for a finite w >= 0, exactly, from the bits of w (the value
// an FP64 multiply by 2^s followed by floor gives; no FP64 instruction).
__device__ __forceinline__ unsigned long long scaled_floor(float w, int s) {
  const unsigned int b = __float_as_uint(w);
  int e = (int)((b >> 23) & 0xffu);
  unsigned long long mant = b & 0x7fffffu;
  if (e == 0) {
    if (mant == 0) return 0ull;
    e = 1;
  } else {
    mant |= 0x800000ull;
  }
  const int sh = e - 150 + s;   // w = mant 2^(e - 150)
  if (sh >= 0) return sh < 64 ? mant << sh : 0ull;
  return -sh < 64 ? mant >> (-sh) : 0ull;
}
__device__ __forceinline__ unsigned long long scaled_floor(double w, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(w);
  int e = (int)((b >> 52) & 0x7ffull);
  unsigned long long mant = b & 0xfffffffffffffull;
  if (e == 0) {
    if (mant == 0) return 0ull;
    e = 1;
  } else {
    mant |= 0x10000000000000ull;
  }
  const int sh = e - 1075 + s;  // w = mant 2^(e - 1075)
  if (sh >= 0) return sh < 64 ? mant << sh : 0ull;
  return -sh < 64 ? mant >> (-sh) : 0ull;
}

// Order key of a non-negative double: its bit pattern as an unsigned integer
// orders exactly as the value (integer compares instead of FP64 compares).
__device__ __forceinline__ unsigned long long order_key(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

// Division of a 128-bit dividend by a fixed 64-bit divisor through a
// precomputed reciprocal of the normalised divisor (Moller & Granlund,
// "Improved division by invariant integers", IEEE Trans. Computers 60(2),
// 2011, Algorithm 4): one 64 x 64 -> 128-bit product and at most two
// corrections per quotient instead of a 128-bit division.
struct Recip {
  unsigned long long d;   // divisor shifted left until its top bit is set
  unsigned long long v;   // floor((2^128 - 1) / d) - 2^64
  int s;                  // the shift
};

__device__ __forceinline__ Recip make_recip(unsigned long long d) {
  Recip r{0ull, 0ull, 0};
  if (d == 0ull) return r;
  r.s = __clzll((long long)d);
  r.d = d << r.s;
  const unsigned __int128 all = ~(unsigned __int128)0;
  r.v = (unsigned long long)(all / r.d);   // the quotient is 2^64 + v; its low word is v
  return r;
}

// floor((u1 2^64 + u0) / d) for a normalised dividend (u1 < r.d).
__device__ __forceinline__ unsigned long long div_2by1(unsigned long long u1, unsigned long long u0, const Recip& r) {
  unsigned long long q0 = r.v * u1;
  unsigned long long q1 = __umul64hi(r.v, u1);
  const unsigned long long t = q0 + u0;
  q1 += u1 + 1ull + (t < q0 ? 1ull : 0ull);
  q0 = t;
  unsigned long long rem = u0 - q1 * r.d;
  if (rem > q0) {
    q1 -= 1ull;
    rem += r.d;
  }
  if (rem >= r.d) q1 += 1ull;
  return q1;
}

// Systematic resampling: number of children whose pointer falls below Q_i,
// c = #{t : floor((t 2^32 + U) Q_n / (L 2^32)) < Q_i}, with 128-bit integers:
// V = floor((Q_i L 2^32 - 1) / Q_n), c = min(L, V < U ? 0 : ((V - U) >> 32) + 1).
// rq is make_recip(Q_n).
__device__ __forceinline__ int offspring_end(unsigned long long Qi, unsigned long long Qn, unsigned long long L,
                                             uint32_t U, const Recip& rq) {
  if (L == 0 || Qn == 0) return 0;
  // X = Q_i L 2^32 as (hi, lo); Q_i < 2^53 and L < 2^31, so X < 2^116
  const unsigned long long ph = __umul64hi(Qi, L), pl = Qi * L;
  unsigned long long hi = (ph << 32) | (pl >> 32), lo = pl << 32;
  if ((hi | lo) == 0ull) return 0;
  if (lo == 0ull) hi -= 1ull;   // X - 1
  lo -= 1ull;
  // normalise: (X - 1) 2^s < Q_n 2^s 2^64 since L 2^32 < 2^64
  if (rq.s > 0) {
    hi = (hi << rq.s) | (lo >> (64 - rq.s));
    lo <<= rq.s;
  }
  const unsigned long long V = div_2by1(hi, lo, rq);
  const unsigned long long cc = V < (unsigned long long)U ? 0ull : ((V - U) >> 32) + 1ull;
  return (int)(cc < L ? cc : L);
}

// Resample count and CDF scale of a slice from its mass, largest weight and size.
__device__ __forceinline__ void resample_plan(double rho, int lmax, int n, double N, double wmax, int& L, int& s) {
  L = 0;
  s = 0;
  if (n > 0 && wmax > 0.0) {
    int e;
    frexp(wmax, &e);
    int c = 0;
    while ((1LL << c) < (long long)n) ++c;
    s = 52 - c - e;
    long long Ll = llround(rho * (N > 1.0 ? N : 1.0));
    if (Ll > lmax) Ll = lmax;
    if (Ll < 0) Ll = 0;
    L = (int)Ll;
  }
}

// N^j = sum of slice j's pass-2 tile sums (the row-tile prefix `pref`) and its
// largest updated weight, by one CTA of exactly 256 threads in a fixed order
// (each thread a stride of 256 tiles, shuffles within the warps, the 8 warp
// totals in warp order); with `plan` the CTA also writes N^j and the
// resampling plan (L_j and the CDF scale).  Every thread gets N^j.
__device__ __forceinline__ double slice_mass(const Dev& d, const Model& m, int j, const int* pref, bool plan,
                                             double* red, double* redm, double* sh) {
  double s = 0.0, mx = 0.0;
  for (int it = pref[j] + threadIdx.x; it < pref[j + 1]; it += 256) {
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
    *sh = t;
    if (plan) {
      d.mass[j] = t;
      int L, sc;
      resample_plan(d.rho[j], d.lmax[j], d.n_pred[j], t, tm, L, sc);
      d.rs_mass[j] = t;
      d.rs_wn[j] = L > 0 ? t / (double)L : 0.0;
      d.rs_s[j] = sc;
      d.rs_L[j] = L;
    }
  }
  __syncthreads();
  return *sh;
}

// Measurements of slice j.
__device__ __forceinline__ int slice_M(const Dev& d, int j) { return d.zshared ? *d.M : d.Mj[j]; }
template <class R> __device__ __forceinline__ const V2<R>* slice_Z(const Dev& d, int j) {
  return static_cast<const V2<R>*>(d.Z) + (d.zshared ? 0 : d.zoff[j]);
}

__device__ __forceinline__ uint32_t philox_u32(const Model& m, uint32_t a, unsigned long long step, uint32_t tag) {
  return philox4x32_10(U4{a, (uint32_t)step, tag, (uint32_t)(step >> 32)}, (uint32_t)m.seed,
                       (uint32_t)(m.seed >> 32)).a;
}

// ---------------------------------------------------------------------------
// Helpers shared by the staged kernels and the persistent step kernel.
// ---------------------------------------------------------------------------
constexpr int kCells = 256;   // 16 x 16 cells over measurement space, Hilbert order

// Position of the particle's cell on the Hilbert curve through the 16 x 16
// grid (Hilbert 1891; the usual quadrant recursion: at each level the
// quadrant's place on the curve, then the sub-square turned into the
// quadrant's frame).  Consecutive keys are edge neighbours, so a run of
// particles in key order stays in a compact patch of cells; the Morton
// (Z) order jumps across the grid at its quadrant boundaries, and a
// 256-particle tile spanning such a jump reaches most measurements.
__device__ __forceinline__ int cell_key(const Model& m, float h0, float h1) {
  int cx = (int)floorf((h0 - m.f_cell_o0) * m.f_cell_s0);
  int cy = (int)floorf((h1 - m.f_cell_o1) * m.f_cell_s1);
  cx = min(max(cx, 0), 15);
  cy = min(max(cy, 0), 15);
  int k = 0;
#pragma unroll
  for (int s = 8; s > 0; s >>= 1) {
    const int rx = (cx & s) ? 1 : 0, ry = (cy & s) ? 1 : 0;
    k += s * s * ((3 * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        cx = 15 - cx;
        cy = 15 - cy;
      }
      const int t = cx;
      cx = cy;
      cy = t;
    }
  }
  return k;
}

// Exact CDF in three passes over chunks of particles (any PE size):
// chunk totals of q_i = floor(w_i 2^s), an exclusive scan of the totals per
// PE, then every chunk rescans its own q_i and turns Q_i into offspring ends.
template <class R>
__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long v, unsigned long long* wt,
                                                             unsigned long long* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wt[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    unsigned long long u = lane < nw ? wt[lane] : 0ull;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, u, o);
      if (lane >= o) u += t;
    }
    if (lane < nw) wt[lane] = u;
  }
  __syncthreads();
  const unsigned long long r = (wid > 0 ? wt[wid - 1] : 0ull) + incl;
  if (total) *total = wt[nw - 1];
  __syncthreads();
  return r;
}

// Cartesian point of a measurement, the offset origin of the labelled sums.
template <class R>
__device__ __forceinline__ void meas_point(const Model& m, V2<R> z, R& rx, R& ry) {
  if (m.meas_model == 0) {
    rx = z.a;
    ry = z.b;
  } else {
    R sn, cs;
    sincos(z.b, &sn, &cs);
    rx = (R)m.sx + z.a * cs;
    ry = (R)m.sy + z.a * sn;
  }
}

// Birth weight nu_b / J_j of slice j in the kernel's precision.
template <class R> __device__ __forceinline__ R slice_bw(const Dev& d, int j);
template <> __device__ __forceinline__ float slice_bw<float>(const Dev& d, int j) { return d.bwf[j]; }
template <> __device__ __forceinline__ double slice_bw<double>(const Dev& d, int j) { return d.bwd[j]; }

// Grid-wide barrier over gridDim.x CTAs with a bounded wait (`limit`
// polls).  Every CTA adds one to a 64-bit arrival count that only grows, so
// barrier b of a launch completes when the count reaches b * gridDim.x: one
// release atomic and the acquire polls are the whole cost (no reset, no
// generation word).  The count is a multiple of gridDim.x between launches; a
// launch that gave up leaves an error word behind and the host clears both
// before the next.  Returns false (in every thread of the CTA) when the wait
// gave up or an error was recorded; the caller then returns from the kernel.
// `lost` (read by thread 0) makes the CTA leave without arriving, as a PE that
// died would: the host's failure injection.
__device__ __forceinline__ bool grid_sync(const Dev& d, long long limit, bool lost) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 0;
    if (!lost) {
      unsigned long long* cnt = reinterpret_cast<unsigned long long*>(d.bar);
      const unsigned long long G = gridDim.x;
      unsigned long long old;
      asm volatile("atom.release.gpu.global.add.u64 %0, [%1], 1;" : "=l"(old) : "l"(cnt) : "memory");
      const unsigned long long target = (old / G + 1ull) * G;
      long long it = 0;
      for (;;) {
        unsigned long long c;
        int e;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(c) : "l"(cnt) : "memory");
        asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(e) : "l"(d.err) : "memory");
        if (e != 0) break;
        if (c >= target) {
          ok = 1;
          break;
        }
        if (++it > limit) {
          atomicOr(d.err, kErrTimeout);
          break;
        }
        __nanosleep(32);
      }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}


// ---------------------------------------------------------------------------
// Launchers (one per stage), instantiated for float and double.
// ---------------------------------------------------------------------------
template <class R> cudaError_t launch_predict(const Dev& d, const Model& m, const R* noise, cudaStream_t s);
template <class R> cudaError_t launch_stage_z(const Dev& d, const Model& m, const R* Z, int M, cudaStream_t s);
template <class R>
cudaError_t launch_stage_zb(const Dev& d, const Model& m, const R* Z, const int* off, cudaStream_t s);
template <class R>
cudaError_t launch_batch_out(const Dev& d, const Model& m, R* out_states, int* out_labels, int* counts, int cap,
                             cudaStream_t s);
template <class R> cudaError_t launch_update(const Dev& d, const Model& m, cudaStream_t s);
template <class R> cudaError_t launch_order(const Dev& d, const Model& m, cudaStream_t s);
int n_update_launches(const Model& m);   // kernels one launch_update enqueues
int n_order_launches();                  // kernels one launch_order enqueues
// the update's passes one at a time (the autotuner times pass 1 and pass 2 alone)
template <class R> cudaError_t launch_colsum(const Dev& d, const Model& m, cudaStream_t s);
template <class R> cudaError_t launch_finalize(const Dev& d, const Model& m, cudaStream_t s);
template <class R> cudaError_t launch_rowsum(const Dev& d, const Model& m, cudaStream_t s);
template <class R> cudaError_t launch_select(const Dev& d, const Model& m, cudaStream_t s);
Tune default_tune(bool fp64);
// measurement-driven birth (FP32): network head per measurement (unless the
// head was supplied), mixture table, births drawn over the plain ones
cudaError_t launch_birth_head(const Dev& d, const Model& m, cudaStream_t s);
cudaError_t launch_birth_table(const Dev& d, const Model& m, cudaStream_t s);
cudaError_t prepare_birth(const Model& m);
cudaError_t launch_birth_draw(const Dev& d, const Model& m, const float* noise, cudaStream_t s);
cudaError_t launch_params_bf16(void* dst, const float* src, cudaStream_t s);
bool tune_supported(const Tune& t, bool fp64);
template <class R> cudaError_t launch_extract(const Dev& d, const Model& m, R* out_states, int* out_labels,
                                              int cap, int* d_count, cudaStream_t s);
template <class R> cudaError_t launch_resample(const Dev& d, const Model& m, const uint32_t* u,
                                               const uint32_t* xu, cudaStream_t s);
template <class R> cudaError_t prepare_kernels(const Model& m);
template <class R> cudaError_t prepare_extract();
cudaError_t prepare_exchange(const Model& m);
template <class R> bool fused_eligible(const Model& m, int device);
// persistent step kernel (k_persist.cu): grid size (0: cannot launch), launch
template <class R> int persist_grid(const Model& m, bool wide);   // wide: batches and PEs
// direct: one filter (the kernel stages the scan and writes the estimates);
// advance: the kernel advances the step counter (PEs with an exchange leave
// it to the exchange kernels launched after it)
template <class R>
cudaError_t launch_persist(const Dev& d, const Model& m, int grid, const R* Z, int M, const R* noise,
                           const uint32_t* u, R* out_states, int* out_labels, int cap, int* d_count,
                           unsigned long long base, bool direct, bool advance, cudaStream_t s);
int persist_barriers(bool direct);   // grid barriers one launch passes (one filter / batches and PEs)
// after the grid step kernel on PEs: the CU fusion of their local estimates
// (Step 4) and the particle exchange (Step 6), as in the staged step
template <class R>
cudaError_t launch_fuse(const Dev& d, const Model& m, R* out_states, int* out_labels, int cap, int* d_count,
                        cudaStream_t s);
template <class R> cudaError_t launch_exchange(const Dev& d, const Model& m, const uint32_t* xu, cudaStream_t s);
void fill_anchor_table(Anchor* tab);
Model model_from_config(const phd_config& c);
const char* config_problem(const phd_config& c);
template <class R>
cudaError_t launch_fused(const Dev& d, const Model& m, const void* Z, const int* zoff, int M1, int S, const R* noise,
                         const uint32_t* u, const uint32_t* xu, R* out_states, int* out_labels, int* out_count,
                         int cap, cudaStream_t s);
int grid_items(const Model& m);

}  // namespace phd
