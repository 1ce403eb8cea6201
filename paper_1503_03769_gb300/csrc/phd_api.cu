// Host side of the C ABI declared in include/phd.h: configuration checks,
// workspace carve, stage ordering, and stream-ordered launches.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <new>
#include <string>
#include <vector>

#include "mlp_device.cuh"
#include "phd_internal.cuh"

using phd::Dev;
using phd::Model;

namespace {

enum Stage { kReady = 0, kPredicted = 1, kUpdated = 2 };

}  // namespace

struct phd_handle {
  phd_config cfg;
  Model m;
  Dev d;
  cudaStream_t stream;
  int device;
  int stage;
  std::string err;
  void* out_states;   // St4<R> [m_max] fused estimates of phd_step / phd_step_host
  int* out_labels;    // [m_max]
  // CUDA graphs of the step body (in-kernel randomness): the whole body, and
  // the same body split around the update for the stage timer
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side = nullptr;          // second capture branch (measurement-driven births)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t g_all = nullptr, g_pre = nullptr, g_upd = nullptr, g_post = nullptr;
  bool timer = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  size_t ev_used = 0;
  double timer_ms = 0.0;
  unsigned long long timer_calls = 0;
  unsigned long long launches = 0;
  bool fused_ok = false;   // the fused step kernel fits this configuration
  int pgrid = 0;           // CTAs of the grid path's step kernel (0: unavailable)
  unsigned long long pbar_count = 0;  // its barrier count after the launches so far
  int path = 0;            // PHD_PATH_AUTO / PHD_PATH_STAGED / PHD_PATH_FUSED / PHD_PATH_GRID
  bool have_update = false;
  int batch_runs = 0;      // > 0: a batch of independent one-PE filters
  std::vector<int> slice_J;  // births per step of each slice (host copy)
  int* pin = nullptr;        // pinned mapped host ints of phd_step_host: [0] count, [1] error word
};

namespace {

size_t real_size(const phd_config& c) { return c.precision == PHD_FP64 ? 8 : 4; }

// The kernels access caller buffers as vectors: measurement rows (two reals),
// state and estimate rows and injected predict draws (four reals), and 32-bit
// words.  Arrays from cudaMalloc, cudaHostAlloc or PyTorch meet these
// alignments; a view at an odd element offset may not, and is refused before
// any launch instead of faulting.
bool misaligned(const void* p, size_t a) { return p && reinterpret_cast<uintptr_t>(p) % a != 0; }

struct Carver {
  char* base;
  size_t off = 0;
  template <class T> T* take(size_t n_elems, size_t elem = sizeof(T)) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n_elems * elem;
    return p;
  }
};

// Lays out the workspace; with base == nullptr only measures it.
size_t carve(const phd_config& c, char* base, Dev* d, void** out_states, int** out_labels, int batch_runs = 0) {
  const size_t rs = real_size(c);
  const size_t K = batch_runs > 0 ? (size_t)batch_runs : (size_t)c.num_pe, P = (size_t)c.pe_cap,
               Mm = (size_t)c.m_max;
  const size_t items = K * ((P + phd::kTile - 1) / phd::kTile);
  Carver cv{base};
  Dev t{};
  t.x = cv.take<char>(K * P, 4 * rs);
  t.w = cv.take<char>(K * P, rs);
  t.wu = cv.take<char>(K * P, rs);
  t.x_alt = cv.take<char>(K * P, 4 * rs);
  t.w_alt = cv.take<char>(K * P, rs);
  t.x_out = cv.take<char>(K * P, 4 * rs);
  t.w_out = cv.take<char>(K * P, rs);
  t.n_cur = cv.take<int>(K);
  t.n_pred = cv.take<int>(K);
  t.Z = cv.take<char>(batch_runs > 0 ? K * Mm : Mm, 2 * rs);
  t.zshared = batch_runs > 0 ? 0 : 1;
  t.zoff = cv.take<int>(K);
  t.Mj = cv.take<int>(K);
  t.kap = cv.take<double>(K);
  t.rho = cv.take<double>(K);
  t.Jb = cv.take<int>(K);
  t.bwf = cv.take<float>(K);
  t.bwd = cv.take<double>(K);
  t.lmax = cv.take<int>(K);
  t.anchors = cv.take<phd::Anchor>(phd::kAnchors);
  t.M = cv.take<int>(1);
  t.colpart = cv.take<double>(items * Mm);
  t.C = cv.take<double>(K * Mm);
  t.Cused = cv.take<double>(K * Mm);
  t.ginv = cv.take<char>(K * Mm, rs);
  const size_t ritems = K * ((P + phd::kRowTileMin - 1) / phd::kRowTileMin);
  const size_t chunks = K * ((P + phd::kChunk - 1) / phd::kChunk);
  t.rowpart = cv.take<double>(ritems);
  t.rowmax = cv.take<double>(ritems);
  t.dwkey = cv.take<unsigned long long>(K * Mm);
  t.mass = cv.take<double>(K);
  t.nsel = cv.take<int>(K);
  t.sel = cv.take<int>(K * Mm);
  t.selrank = cv.take<int>(K * Mm);
  t.spart = cv.take<double>(items * Mm * 5);
  t.est_local = cv.take<char>(K * Mm, 4 * rs);
  t.out_count = cv.take<int>(1);
  t.rs_mass = cv.take<double>(K);
  t.rs_wn = cv.take<double>(K);
  t.rs_s = cv.take<int>(K);
  t.rs_L = cv.take<int>(K);
  t.csum = cv.take<unsigned long long>(chunks);
  t.coff = cv.take<unsigned long long>(chunks);
  t.rs_Qn = cv.take<unsigned long long>(K);
  t.rs_rcp = cv.take<unsigned long long>(2 * K);
  t.child_end = cv.take<int>(K * P);
  t.parent = cv.take<int>(K * P);
  t.xslots = cv.take<int>(K * P);
  t.lx = cv.take<int>(1);
  t.bar = cv.take<unsigned int>(4);
  t.step = cv.take<unsigned long long>(1);
  t.stats = cv.take<unsigned long long>(5);
  t.err = cv.take<int>(1);
  t.mlp_w = cv.take<char>(phd::kNParams, 2);
  t.bhead = cv.take<float>(Mm * 5);
  t.bcomp = cv.take<float>(Mm * 8);
  t.bcdf = cv.take<float>(Mm);
  t.bdone = cv.take<unsigned int>(1);
  t.ckey = cv.take<unsigned char>(K * P);
  t.chist = cv.take<int>(chunks * 256);
  t.perm = cv.take<int>(K * P);
  t.hdone = cv.take<unsigned int>(K);
  t.geo_s = cv.take<char>(K * P, 4 * rs);
  t.geo = cv.take<char>(K * P, 4 * rs);
  t.gwords = (int)((Mm + 31) / 32);
  t.pchist = cv.take<int>(items * 256 + K * 1024);   // rows of each slice rounded up to 4 chunks
  t.bintot = cv.take<int>(K * 256);
  t.gbits = cv.take<unsigned int>(items * (size_t)t.gwords);
  t.pcsum = cv.take<unsigned long long>(items);
  t.pcoff = cv.take<unsigned long long>(items);
  t.pbar = cv.take<unsigned long long>(1);
  t.pmassq = cv.take<unsigned long long>(2 * K);
  t.pwmaxb = cv.take<unsigned long long>(K);
  t.pnpos = cv.take<int>(K);
  t.ptimes = cv.take<unsigned long long>(48);
  void* os = cv.take<char>(Mm, 4 * rs);
  int* ol = cv.take<int>(Mm);
  t.max_items = (int)items;
  if (d) *d = t;
  if (out_states) *out_states = os;
  if (out_labels) *out_labels = ol;
  return (cv.off + 255) & ~(size_t)255;
}

const char* check_config(const phd_config& c) {
  if (c.meas_model != PHD_MEAS_LINEAR && c.meas_model != PHD_MEAS_RANGE_BEARING) return "meas_model";
  if (c.precision != PHD_FP32 && c.precision != PHD_FP64) return "precision";
  if (c.num_pe < 1 || c.num_pe > phd::kMaxPE) return "num_pe must be in 1..256";
  if (c.ck_mode != PHD_CK_LOCAL && c.ck_mode != PHD_CK_GLOBAL) return "ck_mode";
  if (c.pe_cap < 1 || c.pe_cap > (1 << 24)) return "pe_cap must be in 1..2^24";
  if (c.m_max < 1 || c.m_max > phd::kMaxM) return "m_max must be in 1..4096";
  if (c.birth_count < 0) return "birth_count";
  if (phd::births_of(c.birth_count, c.num_pe, 0) >= c.pe_cap) return "birth_count / num_pe must be < pe_cap";
  if (c.birth_model != PHD_BIRTH_UNIFORM && c.birth_model != PHD_BIRTH_GAUSSIAN) return "birth_model";
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(c.birth_mean[k]) || !(c.birth_std[k] >= 0) || !std::isfinite(c.birth_std[k]))
      return "birth_mean / birth_std";
  if (!(c.sigma_a_y >= 0) || !std::isfinite(c.sigma_a_y)) return "sigma_a_y";
  if (c.exchange_mode != PHD_XCHG_RING && c.exchange_mode != PHD_XCHG_ALL) return "exchange_mode";
  if (c.reserved1 != 0) return "reserved1 must be 0";
  if (!(c.exchange_threshold >= 0) || !std::isfinite(c.exchange_threshold)) return "exchange_threshold";
  if (!(c.gate_sigma >= 0) || !std::isfinite(c.gate_sigma)) return "gate_sigma";
  if (!(c.theta_span >= 0 && c.theta_span <= 2.0 * 3.14159265358979323846)) return "theta_span must be in [0, 2 pi]";
  if (!(c.dt > 0) || !std::isfinite(c.dt)) return "dt";
  if (!(c.sigma_a >= 0) || !std::isfinite(c.sigma_a)) return "sigma_a";
  if (!(c.sigma_z[0] > 0) || !(c.sigma_z[1] > 0) || !std::isfinite(c.sigma_z[0]) || !std::isfinite(c.sigma_z[1]))
    return "sigma_z";
  if (!(c.region[1] > c.region[0]) || !(c.region[3] > c.region[2])) return "region";
  if (c.meas_model == PHD_MEAS_RANGE_BEARING && !(c.r_max > 0)) return "r_max";
  if (!(c.p_s >= 0 && c.p_s <= 1)) return "p_s";
  if (!(c.p_d >= 0 && c.p_d <= 1)) return "p_d";
  if (!(c.clutter_rate >= 0) || !std::isfinite(c.clutter_rate)) return "clutter_rate";
  if (!(c.birth_mass >= 0) || !std::isfinite(c.birth_mass)) return "birth_mass";
  if (!(c.birth_vel_sigma >= 0)) return "birth_vel_sigma";
  if (!(c.particles_per_target > 0) || !std::isfinite(c.particles_per_target)) return "particles_per_target";
  if (!(c.exchange_frac >= 0 && c.exchange_frac < 0.5)) return "exchange_frac must be in [0, 0.5)";
  if (c.num_pe > 1 && c.exchange_frac > 0 && c.pe_cap > 24576)
    return "pe_cap must be <= 24576 when the ring exchange is on";
  return nullptr;
}

// Volume of the measurement space the clutter is uniform over (kappa =
// lambda / volume): the region (linear sensor) or [0, r_max] x bearing span.
double meas_volume(const phd_config& c) {
  const double kPi = 3.14159265358979323846;
  if (c.meas_model == PHD_MEAS_LINEAR) return (c.region[1] - c.region[0]) * (c.region[3] - c.region[2]);
  return c.r_max * (c.theta_span > 0 ? c.theta_span : 2.0 * kPi);
}

Model make_model(const phd_config& c) {
  Model m{};
  const double kPi = 3.14159265358979323846;
  const double kLog2e = 1.4426950408889634;
  m.meas_model = c.meas_model;
  m.K = c.num_pe;
  m.pe_cap = c.pe_cap;
  m.m_max = c.m_max;
  m.J = c.birth_count;
  m.ck_global = c.ck_mode == PHD_CK_GLOBAL;
  m.dt = c.dt;
  m.sigma_a = c.sigma_a;
  m.sigma_ay = c.sigma_a_y > 0 ? c.sigma_a_y : c.sigma_a;
  m.birth_gauss = c.birth_model == PHD_BIRTH_GAUSSIAN;
  for (int k = 0; k < 4; ++k) {
    m.bmean[k] = c.birth_mean[k];
    m.bstd[k] = c.birth_std[k];
    m.f_bmean[k] = (float)c.birth_mean[k];
    m.f_bstd[k] = (float)c.birth_std[k];
  }
  m.f_sigma_ay = (float)m.sigma_ay;
  m.sz0 = c.sigma_z[0];
  m.sz1 = c.sigma_z[1];
  m.sx = c.sensor[0];
  m.sy = c.sensor[1];
  m.rx0 = c.region[0];
  m.rx1 = c.region[1];
  m.ry0 = c.region[2];
  m.ry1 = c.region[3];
  m.p_s = c.p_s;
  m.p_d = c.p_d;
  m.kappa = c.clutter_rate / meas_volume(c);
  m.birth_mass = c.birth_mass;
  m.birth_vel_sigma = c.birth_vel_sigma;
  m.rho_pe = c.particles_per_target / (double)c.num_pe;
  m.exchange_frac = c.exchange_frac;
  m.xmode = c.exchange_mode;
  m.xthresh = c.exchange_threshold;
  m.qk = c.gate_sigma > 0 ? 0.5 * kLog2e * c.gate_sigma * c.gate_sigma : (double)INFINITY;
  m.f_qk = (float)m.qk;
  m.spin_limit = phd::kDefaultSpinLimit;
  m.a0 = std::sqrt(0.5 * kLog2e) / c.sigma_z[0];
  m.a1 = std::sqrt(0.5 * kLog2e) / c.sigma_z[1];
  m.cnorm = 1.0 / (2.0 * kPi * c.sigma_z[0] * c.sigma_z[1]);
  m.seed = c.seed;
  m.f_dt = (float)c.dt;
  m.f_sigma_a = (float)c.sigma_a;
  m.f_ps = (float)c.p_s;
  m.f_rx0 = (float)c.region[0];
  m.f_rw = (float)(c.region[1] - c.region[0]);
  m.f_ry0 = (float)c.region[2];
  m.f_rh = (float)(c.region[3] - c.region[2]);
  m.f_bv = (float)c.birth_vel_sigma;
  m.f_sx = (float)c.sensor[0];
  m.f_sy = (float)c.sensor[1];
  m.f_miss = (float)(1.0 - c.p_d);
  const int jlo = c.birth_count / c.num_pe;
  m.bw_lo = jlo > 0 ? c.birth_mass / (double)jlo : 0.0;
  m.bw_hi = c.birth_mass / (double)(jlo + 1);
  m.f_bw_lo = (float)m.bw_lo;
  m.f_bw_hi = (float)m.bw_hi;
  m.tune = phd::default_tune(c.precision == PHD_FP64);
  m.learned = 0;
  m.jmax = (c.birth_count + c.num_pe - 1) / c.num_pe;
  m.f_alpha = 1.0f;
  {
    const double area = (c.region[1] - c.region[0]) * (c.region[3] - c.region[2]);
    const double sb = c.birth_vel_sigma;
    m.f_blog = (float)std::log2(area * sb * sb / (2.0 * kPi * c.sigma_z[0] * c.sigma_z[1]));
  }
  m.f_win0 = (float)(3.0 * c.sigma_z[0]);
  m.f_win1 = (float)(3.0 * c.sigma_z[1]);
  m.f_cx = (float)(0.5 * (c.region[0] + c.region[1]));
  m.f_cy = (float)(0.5 * (c.region[2] + c.region[3]));
  m.f_ihx = (float)(2.0 / (c.region[1] - c.region[0]));
  m.f_ihy = (float)(2.0 / (c.region[3] - c.region[2]));
  if (c.meas_model == PHD_MEAS_LINEAR) {
    m.f_cell_o0 = (float)c.region[0];
    m.f_cell_s0 = (float)(16.0 / (c.region[1] - c.region[0]));
    m.f_cell_o1 = (float)c.region[2];
    m.f_cell_s1 = (float)(16.0 / (c.region[3] - c.region[2]));
  } else {
    m.f_cell_o0 = 0.0f;
    m.f_cell_s0 = (float)(16.0 / c.r_max);
    m.f_cell_o1 = (float)-kPi;
    m.f_cell_s1 = (float)(16.0 / (2.0 * kPi));
  }
  return m;
}

phd_status fail(phd_handle* h, phd_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

phd_status cuda_fail(phd_handle* h, cudaError_t e, const char* where) {
  return fail(h, PHD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PHD_CUDA(h, call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

bool is_fp64(const phd_handle* h) { return h->cfg.precision == PHD_FP64; }

// Per-slice descriptors: one per PE of a filter (each PE a full filter on its
// slice, births split J/K) or one per run of a batch (slice j = run j).
cudaError_t upload_slices(phd_handle* h, const std::vector<phd_config>& cf) {
  const int K = (int)cf.size();
  const bool batch = h->batch_runs > 0;
  std::vector<double> kap(K), rho(K), bwd(K);
  std::vector<float> bwf(K);
  std::vector<int> Jb(K), lmax(K), zero(K, 0);
  for (int j = 0; j < K; ++j) {
    const phd_config& c = cf[j];
    kap[j] = c.clutter_rate / meas_volume(c);
    if (batch) {
      rho[j] = c.particles_per_target;
      Jb[j] = c.birth_count;
      lmax[j] = c.pe_cap - c.birth_count;
    } else {
      rho[j] = c.particles_per_target / (double)c.num_pe;
      Jb[j] = phd::births_of(c.birth_count, c.num_pe, j);
      lmax[j] = c.pe_cap - Jb[j];
    }
    bwd[j] = Jb[j] > 0 ? c.birth_mass / (double)Jb[j] : 0.0;
    bwf[j] = (float)bwd[j];
  }
  h->slice_J = Jb;
  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemcpyAsync(h->d.kap, kap.data(), K * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.rho, rho.data(), K * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.bwd, bwd.data(), K * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.bwf, bwf.data(), K * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.Jb, Jb.data(), K * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.lmax, lmax.data(), K * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.zoff, zero.data(), K * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.Mj, zero.data(), K * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors go out of scope
  return e;
}

// kernels each stage launches (for the launch counter)
constexpr int kNPredict = 1, kNStageZ = 1, kNBirth = 2;
int n_resample(const Model& m) { return (m.K > 1 && m.exchange_frac > 0.0) ? 7 : 4; }
// label sums and local estimates; the fusion kernel only for K > 1 PEs of one filter
int n_extract(const phd_handle* h) { return (h->batch_runs == 0 && h->m.K > 1) ? 3 : 2; }

phd_status check_align(phd_handle* h, const void* Z, const void* rows4a, const void* rows4b,
                       std::initializer_list<const void*> words) {
  const size_t rs = real_size(h->cfg);
  if (misaligned(Z, 2 * rs)) return fail(h, PHD_ERR_INVALID_ARG, "Z is not aligned to a row of two reals");
  if (misaligned(rows4a, 4 * rs) || misaligned(rows4b, 4 * rs))
    return fail(h, PHD_ERR_INVALID_ARG, "a state, estimate or draw buffer is not aligned to a row of four reals");
  for (const void* p : words)
    if (misaligned(p, 4)) return fail(h, PHD_ERR_INVALID_ARG, "a 32-bit buffer is not 4-byte aligned");
  return PHD_OK;
}

phd_status read_device_error(phd_handle* h) {
  int err = 0;
  PHD_CUDA(h, cudaMemcpyAsync(&err, h->d.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  if (err == 0) return PHD_OK;
  PHD_CUDA(h, cudaMemsetAsync(h->d.err, 0, sizeof(int), h->stream));
  // a wait that gave up may have left the grid barriers mid-count (and an
  // injected fault its flag)
  PHD_CUDA(h, cudaMemsetAsync(h->d.bar, 0, 4 * sizeof(unsigned int), h->stream));
  PHD_CUDA(h, cudaMemsetAsync(h->d.pbar, 0, sizeof(unsigned long long), h->stream));
  h->pbar_count = 0;
  // and a grid step that stopped early its running cell totals
  PHD_CUDA(h, cudaMemsetAsync(h->d.bintot, 0, (size_t)h->m.K * 256 * sizeof(int), h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  if (err & phd::kErrTimeout) return fail(h, PHD_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (err & phd::kErrNonFinite) return fail(h, PHD_ERR_INVALID_ARG, "non-finite measurement in Z");
  return fail(h, PHD_ERR_CAPACITY, "device-side capacity check failed");
}

// Prediction; with a birth network loaded the births are then redrawn from
// its proposal, which needs Z_k staged (z_staged) and, unless `head` is given
// ([M][5] network outputs), runs the network on it.
phd_status do_predict(phd_handle* h, const void* noise, bool z_staged = false, const float* head = nullptr,
                      int M = 0) {
  if (h->stage != kReady) return fail(h, PHD_ERR_STATE, "phd_predict: a step is already in progress");
  if (h->m.learned && !z_staged)
    return fail(h, PHD_ERR_STATE, "phd_predict: a birth network is loaded; births need the scan (phd_predict_z)");
  if (phd_status st = check_align(h, nullptr, noise, nullptr, {})) return st;
  cudaError_t e = is_fp64(h) ? phd::launch_predict<double>(h->d, h->m, static_cast<const double*>(noise), h->stream)
                             : phd::launch_predict<float>(h->d, h->m, static_cast<const float*>(noise), h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "predict");
  h->launches += kNPredict;
  if (h->m.learned) {
    if (head) {
      if (M > 0) e = cudaMemcpyAsync(h->d.bhead, head, sizeof(float) * 5 * (size_t)M, cudaMemcpyDeviceToDevice,
                                     h->stream);
      if (e == cudaSuccess) e = phd::launch_birth_table(h->d, h->m, h->stream);
    } else {
      e = phd::launch_birth_head(h->d, h->m, h->stream);   // builds the table too
    }
    if (e == cudaSuccess) e = phd::launch_birth_draw(h->d, h->m, static_cast<const float*>(noise), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "learned birth");
    h->launches += kNBirth;
  }
  h->stage = kPredicted;
  return PHD_OK;
}

phd_status do_update(phd_handle* h, const void* Z, int M, bool z_in_workspace) {
  if (h->batch_runs) return fail(h, PHD_ERR_STATE, "a batch handle updates through phd_batch_step");
  if (h->stage != kPredicted) return fail(h, PHD_ERR_STATE, "phd_update: call phd_predict first");
  if (M < 0) return fail(h, PHD_ERR_INVALID_ARG, "M < 0");
  if (M > h->cfg.m_max) return fail(h, PHD_ERR_CAPACITY, "M > m_max");
  if (M > 0 && !Z && !z_in_workspace) return fail(h, PHD_ERR_INVALID_ARG, "Z is NULL");
  if (!z_in_workspace)
    if (phd_status st = check_align(h, Z, nullptr, nullptr, {})) return st;
  const void* src = z_in_workspace ? h->d.Z : Z;
  cudaError_t e = is_fp64(h) ? phd::launch_stage_z<double>(h->d, h->m, static_cast<const double*>(src), M, h->stream)
                             : phd::launch_stage_z<float>(h->d, h->m, static_cast<const float*>(src), M, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage_z");
  e = is_fp64(h) ? phd::launch_update<double>(h->d, h->m, h->stream) : phd::launch_update<float>(h->d, h->m, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "update");
  h->launches += kNStageZ + phd::n_update_launches(h->m);
  h->stage = kUpdated;
  h->have_update = true;
  return PHD_OK;
}

phd_status do_extract(phd_handle* h, void* states, int* labels, int cap, int* d_count, int* h_count) {
  if (h->stage != kUpdated) return fail(h, PHD_ERR_STATE, "phd_extract: call phd_update first");
  if (cap < 0) return fail(h, PHD_ERR_INVALID_ARG, "cap < 0");
  if (cap > 0 && (!states || !labels)) return fail(h, PHD_ERR_INVALID_ARG, "NULL output buffer");
  if (phd_status st = check_align(h, nullptr, states, nullptr, {labels, d_count})) return st;
  cudaError_t e = is_fp64(h)
      ? phd::launch_extract<double>(h->d, h->m, static_cast<double*>(states), labels, cap, d_count, h->stream)
      : phd::launch_extract<float>(h->d, h->m, static_cast<float*>(states), labels, cap, d_count, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "extract");
  h->launches += n_extract(h);
  if (h_count) {
    phd_status st = read_device_error(h);
    if (st != PHD_OK) return st;
    PHD_CUDA(h, cudaMemcpyAsync(h_count, h->d.out_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PHD_CUDA(h, cudaStreamSynchronize(h->stream));
    if (*h_count > cap) return fail(h, PHD_ERR_CAPACITY, "more estimates than cap");
  }
  return PHD_OK;
}

phd_status do_resample(phd_handle* h, const uint32_t* u, const uint32_t* xu) {
  if (h->stage != kUpdated) return fail(h, PHD_ERR_STATE, "phd_resample: call phd_update first");
  if (phd_status st = check_align(h, nullptr, nullptr, nullptr, {u, xu})) return st;
  cudaError_t e = is_fp64(h) ? phd::launch_resample<double>(h->d, h->m, u, xu, h->stream)
                             : phd::launch_resample<float>(h->d, h->m, u, xu, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "resample");
  h->launches += n_resample(h->m);
  h->stage = kReady;
  return PHD_OK;
}

// Step body with in-kernel randomness, split in three parts around the update.
cudaError_t enq_pre(phd_handle* h, cudaStream_t s) {
  if (!h->m.learned)
    return is_fp64(h) ? phd::launch_predict<double>(h->d, h->m, nullptr, s)
                      : phd::launch_predict<float>(h->d, h->m, nullptr, s);
  // measurement-driven births on a second branch of the graph (network head,
  // mixture table, draws into the birth slots), beside the survivors'
  // prediction (k_predict leaves the birth slots alone on such a handle)
  cudaError_t e = cudaSuccess;
  if (!h->side) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (e == cudaSuccess && !h->ev_fork) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && !h->ev_join) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
  if (e == cudaSuccess) e = phd::launch_birth_head(h->d, h->m, h->side);
  if (e == cudaSuccess) e = phd::launch_birth_draw(h->d, h->m, nullptr, h->side);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->side);
  if (e == cudaSuccess) e = phd::launch_predict<float>(h->d, h->m, nullptr, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_join, 0);
  return e;
}
cudaError_t enq_upd(phd_handle* h, cudaStream_t s) {
  return is_fp64(h) ? phd::launch_update<double>(h->d, h->m, s) : phd::launch_update<float>(h->d, h->m, s);
}
cudaError_t enq_post(phd_handle* h, cudaStream_t s) {
  const int cap = h->cfg.m_max;
  cudaError_t e = is_fp64(h)
      ? phd::launch_extract<double>(h->d, h->m, static_cast<double*>(h->out_states), h->out_labels, cap, nullptr, s)
      : phd::launch_extract<float>(h->d, h->m, static_cast<float*>(h->out_states), h->out_labels, cap, nullptr, s);
  if (e == cudaSuccess)
    e = is_fp64(h) ? phd::launch_resample<double>(h->d, h->m, nullptr, nullptr, s)
                   : phd::launch_resample<float>(h->d, h->m, nullptr, nullptr, s);
  return e;
}
cudaError_t enq_all(phd_handle* h, cudaStream_t s) {
  cudaError_t e = enq_pre(h, s);
  if (e == cudaSuccess) e = enq_upd(h, s);
  if (e == cudaSuccess) e = enq_post(h, s);
  return e;
}

cudaError_t capture(phd_handle* h, cudaError_t (*body)(phd_handle*, cudaStream_t), cudaGraphExec_t* out) {
  if (!h->cap_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t eb = body(h, h->cap_stream);
  e = cudaStreamEndCapture(h->cap_stream, &g);
  if (eb != cudaSuccess) e = eb;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

void destroy_graphs(phd_handle* h) {
  for (cudaGraphExec_t* g : {&h->g_all, &h->g_pre, &h->g_upd, &h->g_post})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
}

// Mean duration in microseconds of `reps` back-to-back launches of one pass
// (after one untimed launch) on the handle's stream.
template <class F>
cudaError_t time_pass(phd_handle* h, int reps, F launch, float* us) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  *us = 1000.0f * ms / (float)reps;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}


// Sum the timer's recorded event pairs into timer_ms (synchronises).
cudaError_t drain_timer(phd_handle* h) {
  if (h->ev_used == 0) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(h->ev[h->ev_used - 1].second);
  for (size_t i = 0; e == cudaSuccess && i < h->ev_used; ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, h->ev[i].first, h->ev[i].second);
    h->timer_ms += ms;
  }
  h->timer_calls += h->ev_used;
  h->ev_used = 0;
  return e;
}

// The step body on h->stream (Z already staged): one graph launch, or three
// with the update bracketed by events when the stage timer is on.
phd_status run_step_body(phd_handle* h) {
  cudaError_t e = cudaSuccess;
  if (!h->timer) {
    if (!h->g_all) e = capture(h, enq_all, &h->g_all);
    if (e == cudaSuccess) e = cudaGraphLaunch(h->g_all, h->stream);
  } else {
    if (!h->g_pre) e = capture(h, enq_pre, &h->g_pre);
    if (e == cudaSuccess && !h->g_upd) e = capture(h, enq_upd, &h->g_upd);
    if (e == cudaSuccess && !h->g_post) e = capture(h, enq_post, &h->g_post);
    if (e == cudaSuccess && h->ev_used >= 4096) e = drain_timer(h);
    if (e == cudaSuccess && h->ev_used == h->ev.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> p{nullptr, nullptr};
      e = cudaEventCreate(&p.first);
      if (e == cudaSuccess) e = cudaEventCreate(&p.second);
      if (e == cudaSuccess) h->ev.push_back(p);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(h->g_pre, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev[h->ev_used].first, h->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(h->g_upd, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev[h->ev_used].second, h->stream);
    if (e == cudaSuccess) ++h->ev_used;
    if (e == cudaSuccess) e = cudaGraphLaunch(h->g_post, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "step graph");
  h->launches += kNPredict + phd::n_update_launches(h->m) + n_extract(h) + n_resample(h->m) +
                 (h->m.learned ? kNBirth : 0);
  return PHD_OK;
}

phd_status stage_z_only(phd_handle* h, const void* Z, int M);
bool use_fused(const phd_handle* h) {
  return h->fused_ok && !h->m.learned && (h->path == PHD_PATH_AUTO || h->path == PHD_PATH_FUSED);
}
// AUTO takes the grid path while the handle's capacity is at most kGridAutoItems
// 256-particle chunks per CTA of the step kernel (capacities run a few times
// the particles a step holds: the dense 100-target filter has 5.4 chunks of
// capacity per CTA and ~2 in use): there each phase is a few latency-bound
// rounds per CTA and the launches and barriers of the staged graph are what
// the step's time goes to.  Past that (batches of tens to hundreds of runs,
// 50-200 chunks per CTA) the phases become long serial chains, and the
// staged graph with the autotuner's launch shapes runs level with the grid
// kernel at its batch register budget (256 runs, ~1e7 particles: 1.05 ms
// per batched step staged, 1.04 ms grid); AUTO keeps the autotuned graph.
// PEs the fused kernel cannot hold (slices past an SM's shared memory, more
// PEs than co-resident CTAs) follow the same rule (16 PEs at 4x the
// particles of the 16-PE workload: 99.8 us per step grid, 102 us staged).
constexpr double kGridAutoItems = 16.0;
bool grid_auto(const phd_handle* h) {
  const double items = (double)h->m.K * (double)((h->cfg.pe_cap + 255) / 256);
  return h->pgrid > 0 && items <= kGridAutoItems * (double)h->pgrid;
}
bool use_grid(const phd_handle* h) {
  return h->pgrid > 0 &&
         (h->path == PHD_PATH_GRID || (h->path == PHD_PATH_AUTO && !use_fused(h) && grid_auto(h)));
}

// One launch of the grid path's step kernel.  One filter (direct): the scan
// at Z, the estimates to states / labels (cap) and the count to d_count;
// PEs on one scan: the scan staged before the launch, the CU fusion into
// states / labels / d_count and the exchange (draws xu) after it; a batch:
// the scans staged by k_stage_zb, the outputs by k_batch_out.
phd_status run_grid(phd_handle* h, const void* Z, int M, const void* noise, const uint32_t* u,
                    const uint32_t* xu, void* states, int* labels, int cap, int* d_count) {
  const bool timed = h->timer;
  const bool direct = h->batch_runs == 0 && h->m.K == 1;
  const bool pes = h->batch_runs == 0 && h->m.K > 1;
  const bool xchg = pes && h->m.exchange_frac > 0.0;
  cudaError_t e = cudaSuccess;
  if (timed) {
    if (h->ev_used >= 4096) e = drain_timer(h);
    if (e == cudaSuccess && h->ev_used == h->ev.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> p{nullptr, nullptr};
      e = cudaEventCreate(&p.first);
      if (e == cudaSuccess) e = cudaEventCreate(&p.second);
      if (e == cudaSuccess) h->ev.push_back(p);
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev[h->ev_used].first, h->stream);
  }
  if (e == cudaSuccess && pes) {   // also in place (Z already in the workspace): it publishes M
    e = is_fp64(h) ? phd::launch_stage_z<double>(h->d, h->m, static_cast<const double*>(Z), M, h->stream)
                   : phd::launch_stage_z<float>(h->d, h->m, static_cast<const float*>(Z), M, h->stream);
    h->launches += kNStageZ;
  }
  if (e == cudaSuccess)
    e = is_fp64(h) ? phd::launch_persist<double>(h->d, h->m, h->pgrid, static_cast<const double*>(Z), M,
                                                 static_cast<const double*>(noise), u, static_cast<double*>(states),
                                                 labels, cap, d_count, h->pbar_count, direct, !xchg, h->stream)
                   : phd::launch_persist<float>(h->d, h->m, h->pgrid, static_cast<const float*>(Z), M,
                                                static_cast<const float*>(noise), u, static_cast<float*>(states),
                                                labels, cap, d_count, h->pbar_count, direct, !xchg, h->stream);
  if (e == cudaSuccess) {
    h->pbar_count += (unsigned long long)phd::persist_barriers(direct) * (unsigned long long)h->pgrid;
    h->launches += 1;
  }
  if (e == cudaSuccess && pes) {
    e = is_fp64(h) ? phd::launch_fuse<double>(h->d, h->m, static_cast<double*>(states), labels, cap, d_count, h->stream)
                   : phd::launch_fuse<float>(h->d, h->m, static_cast<float*>(states), labels, cap, d_count, h->stream);
    h->launches += 1;
    if (e == cudaSuccess && xchg) {
      e = is_fp64(h) ? phd::launch_exchange<double>(h->d, h->m, xu, h->stream)
                     : phd::launch_exchange<float>(h->d, h->m, xu, h->stream);
      h->launches += 3;
    }
  }
  if (e == cudaSuccess && timed) {
    e = cudaEventRecord(h->ev[h->ev_used].second, h->stream);
    if (e == cudaSuccess) ++h->ev_used;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "grid step");
  h->have_update = true;
  return PHD_OK;
}

// One fused launch of S steps.  With zoff == NULL: one step of M rows at Z.
phd_status run_fused(phd_handle* h, const void* Z, const int* zoff, int M, int S, const void* noise,
                     const uint32_t* u, const uint32_t* xu, void* states, int* labels, int* counts, int cap) {
  const bool timed = h->timer;
  cudaError_t e = cudaSuccess;
  if (timed) {
    if (h->ev_used >= 4096) e = drain_timer(h);
    if (e == cudaSuccess && h->ev_used == h->ev.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> p{nullptr, nullptr};
      e = cudaEventCreate(&p.first);
      if (e == cudaSuccess) e = cudaEventCreate(&p.second);
      if (e == cudaSuccess) h->ev.push_back(p);
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev[h->ev_used].first, h->stream);
  }
  if (e == cudaSuccess)
    e = is_fp64(h) ? phd::launch_fused<double>(h->d, h->m, Z, zoff, M, S, static_cast<const double*>(noise), u, xu,
                                               static_cast<double*>(states), labels, counts, cap, h->stream)
                   : phd::launch_fused<float>(h->d, h->m, Z, zoff, M, S, static_cast<const float*>(noise), u, xu,
                                              static_cast<float*>(states), labels, counts, cap, h->stream);
  if (e == cudaSuccess && timed) {
    e = cudaEventRecord(h->ev[h->ev_used].second, h->stream);
    if (e == cudaSuccess) ++h->ev_used;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "fused step");
  h->launches += 1;
  h->have_update = true;
  return PHD_OK;
}

// The output contract of phd_step: estimates into the caller's buffers (or
// the workspace's), the true count on the device.
// Device address of a host buffer the GPU can read and write in place
// (pinned and mapped: cudaHostAlloc / cudaHostRegister memory), else NULL.
void* mapped_ptr(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

phd_status step_common(phd_handle* h, const void* Z, int M, const void* noise, const uint32_t* u,
                       const uint32_t* xu, void* d_states, int* d_labels, int cap, int* d_count) {
  phd_status st;
  const bool fused = use_fused(h);
  const bool grid = !fused && use_grid(h);
  if (fused) {
    // the kernel writes the count to the caller's buffer and the workspace
    const bool direct = cap > 0 && d_states && d_labels;
    st = run_fused(h, Z, nullptr, M, 1, noise, u, xu, direct ? d_states : h->out_states,
                   direct ? d_labels : h->out_labels, d_count ? d_count : h->d.out_count,
                   direct ? cap : h->cfg.m_max);
  } else if (grid) {
    const bool direct = cap > 0 && d_states && d_labels;
    const void* Zk = Z;
    st = PHD_OK;
    if (h->m.learned) {
      // measurement-driven births before the step kernel: the scan staged,
      // the network head and mixture table, the draws into the birth slots
      // (the step kernel's prediction leaves those slots as drawn)
      st = stage_z_only(h, Z, M);
      if (st == PHD_OK) {
        cudaError_t e = phd::launch_birth_head(h->d, h->m, h->stream);
        if (e == cudaSuccess) e = phd::launch_birth_draw(h->d, h->m, static_cast<const float*>(noise), h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "learned birth");
        h->launches += kNBirth;
      }
      Zk = h->d.Z;
    }
    if (st == PHD_OK)
      st = run_grid(h, Zk, M, noise, u, xu, direct ? d_states : h->out_states, direct ? d_labels : h->out_labels,
                    direct ? cap : h->cfg.m_max, d_count);
  } else if (noise || u || xu) {
    if (h->m.learned) {
      st = stage_z_only(h, Z, M);
      if (st == PHD_OK) st = do_predict(h, noise, true);
      if (st == PHD_OK) st = do_update(h, h->d.Z, M, true);
    } else {
      st = do_predict(h, noise);
      if (st == PHD_OK) st = do_update(h, Z, M, Z == h->d.Z);
    }
    if (st == PHD_OK) st = do_extract(h, h->out_states, h->out_labels, h->cfg.m_max, nullptr, nullptr);
    if (st == PHD_OK) st = do_resample(h, u, xu);
    if (st != PHD_OK) h->stage = kReady;
    if (st == PHD_OK && cap > 0) {
      const size_t rs = real_size(h->cfg);
      const int ncp = cap < h->cfg.m_max ? cap : h->cfg.m_max;
      PHD_CUDA(h, cudaMemcpyAsync(d_states, h->out_states, (size_t)ncp * 4 * rs, cudaMemcpyDefault, h->stream));
      PHD_CUDA(h, cudaMemcpyAsync(d_labels, h->out_labels, (size_t)ncp * sizeof(int), cudaMemcpyDefault, h->stream));
    }
  } else {
    st = stage_z_only(h, Z, M);
    if (st == PHD_OK) st = run_step_body(h);
    if (st == PHD_OK && cap > 0) {
      const size_t rs = real_size(h->cfg);
      const int ncp = cap < h->cfg.m_max ? cap : h->cfg.m_max;
      PHD_CUDA(h, cudaMemcpyAsync(d_states, h->out_states, (size_t)ncp * 4 * rs, cudaMemcpyDefault, h->stream));
      PHD_CUDA(h, cudaMemcpyAsync(d_labels, h->out_labels, (size_t)ncp * sizeof(int), cudaMemcpyDefault, h->stream));
    }
  }
  if (st != PHD_OK) return st;
  h->have_update = true;
  if (d_count && !fused && !grid)
    PHD_CUDA(h, cudaMemcpyAsync(d_count, h->d.out_count, sizeof(int), cudaMemcpyDefault, h->stream));
  return PHD_OK;
}

phd_status stage_z_only(phd_handle* h, const void* Z, int M) {
  cudaError_t e = is_fp64(h) ? phd::launch_stage_z<double>(h->d, h->m, static_cast<const double*>(Z), M, h->stream)
                             : phd::launch_stage_z<float>(h->d, h->m, static_cast<const float*>(Z), M, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage_z");
  h->launches += kNStageZ;
  return PHD_OK;
}

}  // namespace

namespace phd {

// Bearing anchors: float directions (c_k, s_k) near angle 2 pi k / 256 and
// their exact angles atan2(s_k, c_k) in FP64, split into two floats.
void fill_anchor_table(Anchor* tab) {
  for (int k = 0; k < kAnchors; ++k) {
    const double ang = 2.0 * 3.14159265358979323846 * k / kAnchors;
    const float c = (float)std::cos(ang), s = (float)std::sin(ang);
    const double th = std::atan2((double)s, (double)c);
    tab[k].c = c;
    tab[k].s = s;
    tab[k].th_hi = (float)th;
    tab[k].th_lo = (float)(th - (double)tab[k].th_hi);
  }
}

Model model_from_config(const phd_config& c) { return make_model(c); }
const char* config_problem(const phd_config& c) { return check_config(c); }

}  // namespace phd

extern "C" {

const char* phd_status_string(phd_status s) {
  switch (s) {
    case PHD_OK: return "ok";
    case PHD_ERR_INVALID_ARG: return "invalid argument";
    case PHD_ERR_CAPACITY: return "capacity exceeded";
    case PHD_ERR_CUDA: return "CUDA error";
    case PHD_ERR_TIMEOUT: return "device wait timed out";
    case PHD_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* phd_last_error_string(const phd_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

phd_status phd_workspace_size(const phd_config* cfg, size_t* bytes) {
  if (!cfg || !bytes) return PHD_ERR_INVALID_ARG;
  if (check_config(*cfg)) return PHD_ERR_INVALID_ARG;
  *bytes = carve(*cfg, nullptr, nullptr, nullptr, nullptr);
  return PHD_OK;
}

phd_status phd_init(phd_handle** out, const phd_config* cfg, void* ws, size_t bytes, void* stream) {
  if (!out || !cfg) return PHD_ERR_INVALID_ARG;
  *out = nullptr;
  if (check_config(*cfg)) return PHD_ERR_INVALID_ARG;
  const size_t need = carve(*cfg, nullptr, nullptr, nullptr, nullptr);
  if (!ws || bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return PHD_ERR_INVALID_ARG;
  phd_handle* h = new (std::nothrow) phd_handle();
  if (!h) return PHD_ERR_INVALID_ARG;
  h->cfg = *cfg;
  h->m = make_model(*cfg);
  h->stream = static_cast<cudaStream_t>(stream);
  h->stage = kReady;
  carve(*cfg, static_cast<char*>(ws), &h->d, &h->out_states, &h->out_labels);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = is_fp64(h) ? phd::prepare_kernels<double>(h->m) : phd::prepare_kernels<float>(h->m);
  if (e == cudaSuccess && h->m.K > 1 && h->m.exchange_frac > 0) e = phd::prepare_exchange(h->m);
  if (e == cudaSuccess)
    h->fused_ok = is_fp64(h) ? phd::fused_eligible<double>(h->m, h->device) : phd::fused_eligible<float>(h->m, h->device);
  // the grid step kernel: one filter, or PEs on one scan (its batch budget,
  // the PEs' fusion and exchange as kernels after it); a birth network runs
  // on one PE only
  if (e == cudaSuccess && (h->m.K == 1 || !h->m.learned))
    h->pgrid = is_fp64(h) ? phd::persist_grid<double>(h->m, h->m.K > 1)
                          : phd::persist_grid<float>(h->m, h->m.K > 1);
  (void)cudaGetLastError();   // an ineligible attribute query leaves no sticky error
  if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, need, h->stream);
  phd::Anchor tab[phd::kAnchors];
  phd::fill_anchor_table(tab);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<void*>(h->d.anchors), tab, sizeof(tab), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = upload_slices(h, std::vector<phd_config>(cfg->num_pe, *cfg));
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return PHD_ERR_CUDA;
  }
  *out = h;
  return PHD_OK;
}

phd_status phd_destroy(phd_handle* h) {
  if (!h) return PHD_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  destroy_graphs(h);
  for (auto& p : h->ev) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->pin) cudaFreeHost(h->pin);
  delete h;
  return e == cudaSuccess ? PHD_OK : PHD_ERR_CUDA;
}

phd_status phd_predict(phd_handle* h, const void* d_noise) {
  if (!h) return PHD_ERR_INVALID_ARG;
  return do_predict(h, d_noise);
}

phd_status phd_update(phd_handle* h, const void* d_Z, int32_t M) {
  if (!h) return PHD_ERR_INVALID_ARG;
  return do_update(h, d_Z, M, false);
}

phd_status phd_set_birth_proposal(phd_handle* h, const float* d_params, double alpha) {
  if (!h) return PHD_ERR_INVALID_ARG;
  if (!d_params) {
    PHD_CUDA(h, cudaStreamSynchronize(h->stream));
    h->m.learned = 0;
    h->m.f_alpha = 1.0f;
    destroy_graphs(h);
    return PHD_OK;
  }
  if (is_fp64(h) || h->batch_runs)
    return fail(h, PHD_ERR_STATE, "phd_set_birth_proposal: FP32 one-filter handles only");
  if (h->m.birth_gauss)
    return fail(h, PHD_ERR_STATE, "phd_set_birth_proposal: the defensive mixture needs the uniform birth density");
  if (!(alpha > 0.0 && alpha <= 1.0)) return fail(h, PHD_ERR_INVALID_ARG, "alpha must be in (0, 1]");
  PHD_CUDA(h, phd::prepare_birth(h->m));
  PHD_CUDA(h, phd::launch_params_bf16(h->d.mlp_w, d_params, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  h->m.learned = 1;
  h->m.f_alpha = (float)alpha;
  destroy_graphs(h);
  return PHD_OK;
}

phd_status phd_predict_z(phd_handle* h, const void* d_Z, int32_t M, const float* d_head, const void* d_noise) {
  if (!h) return PHD_ERR_INVALID_ARG;
  if (h->batch_runs) return fail(h, PHD_ERR_STATE, "a batch handle steps through phd_batch_step");
  if (h->stage != kReady) return fail(h, PHD_ERR_STATE, "phd_predict_z: a step is already in progress");
  if (M < 0) return fail(h, PHD_ERR_INVALID_ARG, "M < 0");
  if (M > h->cfg.m_max) return fail(h, PHD_ERR_CAPACITY, "M > m_max");
  if (M > 0 && !d_Z) return fail(h, PHD_ERR_INVALID_ARG, "Z is NULL");
  if (phd_status sa = check_align(h, d_Z, d_noise, nullptr, {})) return sa;
  phd_status st = stage_z_only(h, d_Z, M);
  if (st != PHD_OK) return st;
  return do_predict(h, d_noise, true, d_head, M);
}

phd_status phd_get_birth_head(phd_handle* h, float* d_out, int32_t cap, int32_t* h_M) {
  if (!h || !h_M || cap < 0 || (cap > 0 && !d_out)) return PHD_ERR_INVALID_ARG;
  if (!h->m.learned) return fail(h, PHD_ERR_STATE, "phd_get_birth_head: no birth network loaded");
  int M = 0;
  PHD_CUDA(h, cudaMemcpyAsync(&M, h->d.M, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  *h_M = M;
  const int n = M < cap ? M : cap;
  if (n > 0) {
    PHD_CUDA(h, cudaMemcpyAsync(d_out, h->d.bhead, sizeof(float) * 5 * (size_t)n, cudaMemcpyDeviceToDevice,
                                h->stream));
    PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return M > cap ? fail(h, PHD_ERR_CAPACITY, "more measurements than cap") : PHD_OK;
}

phd_status phd_extract(phd_handle* h, void* d_states, int32_t* d_labels, int32_t cap, int32_t* d_count,
                       int32_t* h_count) {
  if (!h) return PHD_ERR_INVALID_ARG;
  return do_extract(h, d_states, d_labels, cap, d_count, h_count);
}

phd_status phd_resample(phd_handle* h, const uint32_t* d_u, const uint32_t* d_xu) {
  if (!h) return PHD_ERR_INVALID_ARG;
  return do_resample(h, d_u, d_xu);
}

phd_status phd_step(phd_handle* h, const void* d_Z, int32_t M, void* d_states, int32_t* d_labels, int32_t cap,
                    int32_t* d_count, int32_t* h_count) {
  return phd_step_inject(h, d_Z, M, nullptr, nullptr, nullptr, d_states, d_labels, cap, d_count, h_count);
}

phd_status phd_step_inject(phd_handle* h, const void* d_Z, int32_t M, const void* d_noise, const uint32_t* d_u,
                           const uint32_t* d_xu, void* d_states, int32_t* d_labels, int32_t cap, int32_t* d_count,
                           int32_t* h_count) {
  if (!h) return PHD_ERR_INVALID_ARG;
  if (h->batch_runs) return fail(h, PHD_ERR_STATE, "a batch handle steps through phd_batch_step");
  if (h->stage != kReady) return fail(h, PHD_ERR_STATE, "phd_step: a step is already in progress");
  if (M < 0) return fail(h, PHD_ERR_INVALID_ARG, "M < 0");
  if (M > h->cfg.m_max) return fail(h, PHD_ERR_CAPACITY, "M > m_max");
  if (M > 0 && !d_Z) return fail(h, PHD_ERR_INVALID_ARG, "Z is NULL");
  if (cap < 0 || (cap > 0 && (!d_states || !d_labels))) return fail(h, PHD_ERR_INVALID_ARG, "bad output buffer");
  if (phd_status sa = check_align(h, d_Z, d_states, d_noise, {d_labels, d_count, d_u, d_xu})) return sa;
  phd_status st = step_common(h, d_Z, M, d_noise, d_u, d_xu, d_states, d_labels, cap, d_count);
  if (st != PHD_OK) return st;
  if (h_count) {
    st = read_device_error(h);
    if (st != PHD_OK) return st;
    PHD_CUDA(h, cudaMemcpyAsync(h_count, h->d.out_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PHD_CUDA(h, cudaStreamSynchronize(h->stream));
    if (*h_count > cap) return fail(h, PHD_ERR_CAPACITY, "more estimates than cap");
  }
  return PHD_OK;
}

phd_status phd_step_host(phd_handle* h, const void* h_Z, int32_t M, void* h_states, int32_t* h_labels, int32_t cap,
                         int32_t* h_count) {
  if (!h || !h_count) return PHD_ERR_INVALID_ARG;
  if (h->batch_runs) return fail(h, PHD_ERR_STATE, "a batch handle steps through phd_batch_step");
  if (h->stage != kReady) return fail(h, PHD_ERR_STATE, "phd_step_host: a step is already in progress");
  if (M < 0) return fail(h, PHD_ERR_INVALID_ARG, "M < 0");
  if (M > h->cfg.m_max) return fail(h, PHD_ERR_CAPACITY, "M > m_max");
  if (M > 0 && !h_Z) return fail(h, PHD_ERR_INVALID_ARG, "Z is NULL");
  if (cap < 0 || (cap > 0 && (!h_states || !h_labels))) return fail(h, PHD_ERR_INVALID_ARG, "bad output buffer");
  const size_t rs = real_size(h->cfg);
  for (int i = 0; i < 2 * M; ++i) {
    const double v = rs == 8 ? static_cast<const double*>(h_Z)[i] : (double)static_cast<const float*>(h_Z)[i];
    if (!std::isfinite(v)) return fail(h, PHD_ERR_INVALID_ARG, "non-finite measurement in Z");
  }
  // Pinned (mapped) host buffers: the step reads Z and writes the estimates
  // and the count in host memory itself (over NVLink-C2C on Grace systems),
  // with one synchronisation; otherwise staged copies.
  void* zd = M > 0 ? mapped_ptr(h_Z) : nullptr;
  void* sd = cap > 0 ? mapped_ptr(h_states) : nullptr;
  void* ld = cap > 0 ? mapped_ptr(h_labels) : nullptr;
  // (buffers the kernels cannot access as vectors take the copying path)
  const bool vec_ok = !misaligned(zd, 2 * rs) && !misaligned(sd, 4 * rs) && !misaligned(ld, 4);
  if ((M == 0 || zd) && (cap == 0 || (sd && ld)) && vec_ok) {
    if (!h->pin) PHD_CUDA(h, cudaHostAlloc(reinterpret_cast<void**>(&h->pin), 2 * sizeof(int), cudaHostAllocMapped));
    int* pin_d = static_cast<int*>(mapped_ptr(h->pin));
    if (!pin_d) return fail(h, PHD_ERR_CUDA, "phd_step_host: no device address for the pinned count");
    phd_status st = step_common(h, M > 0 ? zd : h->d.Z, M, nullptr, nullptr, nullptr, sd, static_cast<int*>(ld), cap,
                                pin_d);
    if (st != PHD_OK) return st;
    PHD_CUDA(h, cudaMemcpyAsync(h->pin + 1, h->d.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PHD_CUDA(h, cudaStreamSynchronize(h->stream));
    const int n = h->pin[0];
    *h_count = n;
    if (h->pin[1] != 0) {
      phd_status es = read_device_error(h);
      if (es != PHD_OK) return es;
    }
    return n > cap ? fail(h, PHD_ERR_CAPACITY, "more estimates than cap") : PHD_OK;
  }
  if (M > 0) PHD_CUDA(h, cudaMemcpyAsync(h->d.Z, h_Z, (size_t)M * 2 * rs, cudaMemcpyHostToDevice, h->stream));
  phd_status st = step_common(h, h->d.Z, M, nullptr, nullptr, nullptr, h->out_states, h->out_labels, h->cfg.m_max,
                              nullptr);
  if (st != PHD_OK) return st;
  int n = 0;
  PHD_CUDA(h, cudaMemcpyAsync(&n, h->d.out_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  const int ncp = n < cap ? n : cap;
  if (ncp > 0) {
    PHD_CUDA(h, cudaMemcpyAsync(h_states, h->out_states, (size_t)ncp * 4 * rs, cudaMemcpyDeviceToHost, h->stream));
    PHD_CUDA(h, cudaMemcpyAsync(h_labels, h->out_labels, (size_t)ncp * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  }
  *h_count = n;
  phd_status es = read_device_error(h);
  if (es != PHD_OK) return es;
  return n > cap ? fail(h, PHD_ERR_CAPACITY, "more estimates than cap") : PHD_OK;
}

phd_status phd_run(phd_handle* h, const void* d_Z, const int32_t* d_offsets, int32_t S, void* d_states,
                   int32_t* d_labels, int32_t* d_counts, int32_t cap) {
  if (!h) return PHD_ERR_INVALID_ARG;
  if (h->batch_runs) return fail(h, PHD_ERR_STATE, "a batch handle steps through phd_batch_step");
  if (h->stage != kReady) return fail(h, PHD_ERR_STATE, "phd_run: a step is already in progress");
  if (S < 0 || !d_offsets || (S > 0 && (!d_counts || cap < 1 || !d_states || !d_labels)))
    return fail(h, PHD_ERR_INVALID_ARG, "bad phd_run arguments");
  if (S == 0) return PHD_OK;
  if (phd_status sa = check_align(h, d_Z, d_states, nullptr, {d_offsets, d_labels, d_counts})) return sa;
  const size_t rs = real_size(h->cfg);
  if (use_fused(h)) return run_fused(h, d_Z, d_offsets, 0, S, nullptr, nullptr, nullptr, d_states, d_labels, d_counts, cap);
  // staged path: one graph-launched step per scan
  std::vector<int32_t> off((size_t)S + 1);
  PHD_CUDA(h, cudaMemcpyAsync(off.data(), d_offsets, off.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int s = 0; s < S; ++s) {
    const int M = off[s + 1] - off[s];
    if (M < 0 || M > h->cfg.m_max) return fail(h, PHD_ERR_CAPACITY, "a scan has M > m_max");
    const char* Zs = static_cast<const char*>(d_Z) + (size_t)off[s] * 2 * rs;
    phd_status st = step_common(h, Zs, M, nullptr, nullptr, nullptr, static_cast<char*>(d_states) + (size_t)s * cap * 4 * rs,
                                d_labels + (size_t)s * cap, cap, d_counts + s);
    if (st != PHD_OK) return st;
  }
  return PHD_OK;
}

phd_status phd_set_path(phd_handle* h, int32_t path) {
  if (!h) return PHD_ERR_INVALID_ARG;
  if (path != PHD_PATH_AUTO && path != PHD_PATH_STAGED && path != PHD_PATH_FUSED && path != PHD_PATH_GRID)
    return fail(h, PHD_ERR_INVALID_ARG, "unknown path");
  if (path == PHD_PATH_FUSED && !h->fused_ok)
    return fail(h, PHD_ERR_INVALID_ARG, "the fused step kernel does not fit this configuration");
  if (path == PHD_PATH_GRID && h->pgrid <= 0)
    return fail(h, PHD_ERR_INVALID_ARG, "the grid step kernel does not fit this configuration");
  h->path = path;
  return PHD_OK;
}

phd_status phd_get_path(phd_handle* h, int32_t* path) {
  if (!h || !path) return PHD_ERR_INVALID_ARG;
  *path = use_fused(h) ? PHD_PATH_FUSED : use_grid(h) ? PHD_PATH_GRID : PHD_PATH_STAGED;
  return PHD_OK;
}

phd_status phd_get_predicted(phd_handle* h, void* d_x, void* d_w_pred, void* d_w_upd, int32_t* h_counts) {
  if (!h) return PHD_ERR_INVALID_ARG;
  if (!h->have_update) return fail(h, PHD_ERR_STATE, "phd_get_predicted: no update has run");
  const int K = h->m.K;
  const size_t rs = real_size(h->cfg);
  const size_t n = (size_t)K * h->cfg.pe_cap;
  if (d_x) PHD_CUDA(h, cudaMemcpyAsync(d_x, h->d.x_alt, n * 4 * rs, cudaMemcpyDeviceToDevice, h->stream));
  if (d_w_pred) PHD_CUDA(h, cudaMemcpyAsync(d_w_pred, h->d.w_alt, n * rs, cudaMemcpyDeviceToDevice, h->stream));
  if (d_w_upd) PHD_CUDA(h, cudaMemcpyAsync(d_w_upd, h->d.wu, n * rs, cudaMemcpyDeviceToDevice, h->stream));
  if (h_counts)
    PHD_CUDA(h, cudaMemcpyAsync(h_counts, h->d.n_pred, K * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  return read_device_error(h);
}

phd_status phd_set_state(phd_handle* h, const void* d_x, const void* d_w, const int32_t* h_counts) {
  if (!h || !d_x || !d_w || !h_counts) return PHD_ERR_INVALID_ARG;
  const int K = h->m.K;
  for (int j = 0; j < K; ++j) {
    const int lim = h->cfg.pe_cap - h->slice_J[j];
    if (h_counts[j] < 0 || h_counts[j] > lim) return fail(h, PHD_ERR_CAPACITY, "count exceeds pe_cap - J_j");
  }
  const size_t rs = real_size(h->cfg);
  const size_t n = (size_t)K * h->cfg.pe_cap;
  PHD_CUDA(h, cudaMemcpyAsync(h->d.x, d_x, n * 4 * rs, cudaMemcpyDeviceToDevice, h->stream));
  PHD_CUDA(h, cudaMemcpyAsync(h->d.w, d_w, n * rs, cudaMemcpyDeviceToDevice, h->stream));
  PHD_CUDA(h, cudaMemcpyAsync(h->d.n_cur, h_counts, K * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  h->stage = kReady;
  return PHD_OK;
}

phd_status phd_get_state(phd_handle* h, void* d_x, void* d_w, int32_t* h_counts) {
  if (!h) return PHD_ERR_INVALID_ARG;
  const int K = h->m.K;
  const size_t rs = real_size(h->cfg);
  const size_t n = (size_t)K * h->cfg.pe_cap;
  const void* xs = h->stage == kReady ? h->d.x : h->d.x_alt;
  const void* ws = h->stage == kReady ? h->d.w : (h->stage == kUpdated ? h->d.wu : h->d.w_alt);
  if (d_x) PHD_CUDA(h, cudaMemcpyAsync(d_x, xs, n * 4 * rs, cudaMemcpyDeviceToDevice, h->stream));
  if (d_w) PHD_CUDA(h, cudaMemcpyAsync(d_w, ws, n * rs, cudaMemcpyDeviceToDevice, h->stream));
  if (h_counts)
    PHD_CUDA(h, cudaMemcpyAsync(h_counts, h->stage == kReady ? h->d.n_cur : h->d.n_pred, K * sizeof(int),
                                cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  return read_device_error(h);
}

phd_status phd_get_update(phd_handle* h, double* d_C, double* h_mass) {
  if (!h) return PHD_ERR_INVALID_ARG;
  if (!h->have_update) return fail(h, PHD_ERR_STATE, "phd_get_update: no update has run");
  const size_t K = h->m.K, Mm = h->cfg.m_max;
  if (d_C) PHD_CUDA(h, cudaMemcpyAsync(d_C, h->d.C, K * Mm * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (h_mass) {
    // the updated mass is finalised by the extraction's selection kernel; run
    // the same reduction here when extraction has not run yet
    PHD_CUDA(h, cudaMemcpyAsync(h_mass, h->d.mass, K * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  return read_device_error(h);
}

phd_status phd_get_local_estimates(phd_handle* h, void* d_states, int32_t* d_labels, int32_t* h_counts) {
  if (!h) return PHD_ERR_INVALID_ARG;
  const size_t K = h->m.K, Mm = h->cfg.m_max, rs = real_size(h->cfg);
  if (d_states)
    PHD_CUDA(h, cudaMemcpyAsync(d_states, h->d.est_local, K * Mm * 4 * rs, cudaMemcpyDeviceToDevice, h->stream));
  if (d_labels)
    PHD_CUDA(h, cudaMemcpyAsync(d_labels, h->d.sel, K * Mm * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
  if (h_counts) PHD_CUDA(h, cudaMemcpyAsync(h_counts, h->d.nsel, K * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  return read_device_error(h);
}

phd_status phd_get_resample(phd_handle* h, int32_t* d_parents, int32_t* h_lx) {
  if (!h) return PHD_ERR_INVALID_ARG;
  const size_t n = (size_t)h->m.K * h->cfg.pe_cap;
  if (d_parents)
    PHD_CUDA(h, cudaMemcpyAsync(d_parents, h->d.parent, n * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
  if (h_lx) {
    if (h->m.K > 1 && h->cfg.exchange_frac > 0)
      PHD_CUDA(h, cudaMemcpyAsync(h_lx, h->d.lx, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    else
      *h_lx = 0;
  }
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  return read_device_error(h);
}

phd_status phd_get_step(phd_handle* h, uint64_t* step) {
  if (!h || !step) return PHD_ERR_INVALID_ARG;
  unsigned long long s = 0;
  PHD_CUDA(h, cudaMemcpyAsync(&s, h->d.step, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  *step = s;
  return PHD_OK;
}

phd_status phd_set_step(phd_handle* h, uint64_t step) {
  if (!h) return PHD_ERR_INVALID_ARG;
  unsigned long long s = step;
  PHD_CUDA(h, cudaMemcpyAsync(h->d.step, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  return PHD_OK;
}

phd_status phd_set_stage_timer(phd_handle* h, int32_t on) {
  if (!h) return PHD_ERR_INVALID_ARG;
  h->timer = on != 0;
  return PHD_OK;
}

phd_status phd_set_wait_limit(phd_handle* h, int64_t iterations) {
  if (!h || iterations < 1 || iterations > 1000000000LL) return PHD_ERR_INVALID_ARG;
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  h->m.spin_limit = iterations;
  destroy_graphs(h);
  return PHD_OK;
}

phd_status phd_inject_barrier_fault(phd_handle* h) {
  if (!h) return PHD_ERR_INVALID_ARG;
  // the lost-PE flag: PE 0 leaves the next fused step at its first grid
  // barrier without arriving
  const unsigned int flag = 1u;
  PHD_CUDA(h, cudaMemcpyAsync(h->d.bar + 2, &flag, sizeof(flag), cudaMemcpyHostToDevice, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  return PHD_OK;
}

phd_status phd_get_stats(phd_handle* h, phd_stats* out) {
  if (!h || !out) return PHD_ERR_INVALID_ARG;
  unsigned long long v[5] = {0, 0, 0, 0, 0};
  PHD_CUDA(h, cudaMemcpyAsync(v, h->d.stats, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  PHD_CUDA(h, drain_timer(h));
  out->pairs = v[0];
  out->particles = v[1];
  out->measurements = v[2];
  out->updates = v[3];
  out->pairs_evaluated = v[4];
  out->launches = h->launches;
  out->timed_updates = h->timer_calls;
  out->update_ms = h->timer_ms;
  return read_device_error(h);
}

phd_status phd_get_phase_times(phd_handle* h, double* h_ms, int32_t n) {
  if (!h || !h_ms || n < 0 || n > 36) return PHD_ERR_INVALID_ARG;
  unsigned long long v[48] = {};
  PHD_CUDA(h, cudaMemcpyAsync(v, h->d.ptimes, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k < n; ++k) {
    const int blk = k / 12, ph = k % 12;
    double ms = 1e-6 * (double)v[16 * blk + ph];
    if (blk == 2) ms /= (h->pgrid > 0 ? (double)h->pgrid : 1.0);   // sum over CTAs -> per CTA
    h_ms[k] = ms;
  }
  return PHD_OK;
}

phd_status phd_reset_stats(phd_handle* h) {
  if (!h) return PHD_ERR_INVALID_ARG;
  PHD_CUDA(h, drain_timer(h));
  PHD_CUDA(h, cudaMemsetAsync(h->d.stats, 0, 5 * sizeof(unsigned long long), h->stream));
  PHD_CUDA(h, cudaMemsetAsync(h->d.ptimes, 0, 48 * sizeof(unsigned long long), h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  h->launches = 0;
  h->timer_ms = 0.0;
  h->timer_calls = 0;
  return PHD_OK;
}

// ---------------------------------------------------------------------------
// Launch shapes of the update's pair passes and their autotuner
// ---------------------------------------------------------------------------

phd_status phd_get_tuning(phd_handle* h, phd_tuning* out) {
  if (!h || !out) return PHD_ERR_INVALID_ARG;
  const phd::Tune& t = h->m.tune;
  *out = phd_tuning{t.c_tile, t.c_mb, t.r_pb, t.r_g, t.grid1, t.grid2, t.gate, t.order, 0.0f, 0.0f};
  return PHD_OK;
}

phd_status phd_set_tuning(phd_handle* h, const phd_tuning* t) {
  if (!h || !t) return PHD_ERR_INVALID_ARG;
  const phd::Tune u{t->c_tile, t->c_mb, t->r_pb, t->r_g, t->grid1, t->grid2, t->gate, t->order};
  if (!phd::tune_supported(u, is_fp64(h))) return fail(h, PHD_ERR_INVALID_ARG, "phd_set_tuning: unsupported shape");
  // the extraction's pass 3 walks the order the update built
  if (h->stage == kUpdated && u.order != h->m.tune.order)
    return fail(h, PHD_ERR_STATE, "phd_set_tuning: the spatial order changes only between steps");
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  h->m.tune = u;
  destroy_graphs(h);
  return PHD_OK;
}

phd_status phd_autotune(phd_handle* h, int32_t reps, phd_tuning* out) {
  if (!h || reps < 1 || reps > 1000) return PHD_ERR_INVALID_ARG;
  if (!h->have_update) return fail(h, PHD_ERR_STATE, "phd_autotune: no update has run (nothing to time on)");
  const bool fp64 = is_fp64(h);
  unsigned long long saved[5];
  PHD_CUDA(h, cudaMemcpyAsync(saved, h->d.stats, sizeof(saved), cudaMemcpyDeviceToHost, h->stream));
  PHD_CUDA(h, cudaStreamSynchronize(h->stream));
  const phd::Tune base = h->m.tune;
  const int grids[3] = {152 * 4, 152 * 8, 152 * 16};
  const int tiles[3] = {256, 512, 1024};
  const int mbs[3] = {1, 2, 4};
  const int pgs[7][2] = {{1, 1}, {2, 1}, {4, 1}, {1, 2}, {2, 2}, {1, 4}, {1, 8}};
  phd::Model m = h->m;
  phd::Tune best = base;
  float best1 = 0.0f, best2 = 0.0f;
  bool have1 = false, have2 = false;
  cudaError_t e = cudaSuccess;
  // the passes read the spatial order when it is on: build it once first
  if (base.order) e = fp64 ? phd::launch_order<double>(h->d, m, h->stream) : phd::launch_order<float>(h->d, m, h->stream);
  // pass 1 over its shapes
  for (int ti = 0; ti < 3 && e == cudaSuccess; ++ti)
    for (int mi = 0; mi < 3 && e == cudaSuccess; ++mi)
      for (int gi = 0; gi < 3 && e == cudaSuccess; ++gi) {
        m.tune = base;
        m.tune.c_tile = tiles[ti];
        m.tune.c_mb = mbs[mi];
        m.tune.grid1 = grids[gi];
        if (!phd::tune_supported(m.tune, fp64)) continue;
        float us = 0.0f;
        e = time_pass(h, reps, [&] {
          return fp64 ? phd::launch_colsum<double>(h->d, m, h->stream) : phd::launch_colsum<float>(h->d, m, h->stream);
        }, &us);
        if (e == cudaSuccess && (!have1 || us < best1)) {
          best1 = us;
          have1 = true;
          best.c_tile = m.tune.c_tile;
          best.c_mb = m.tune.c_mb;
          best.grid1 = m.tune.grid1;
        }
      }
  // ginv from the chosen pass 1, then pass 2 over its shapes
  m.tune = best;
  if (e == cudaSuccess)
    e = fp64 ? phd::launch_colsum<double>(h->d, m, h->stream) : phd::launch_colsum<float>(h->d, m, h->stream);
  if (e == cudaSuccess)
    e = fp64 ? phd::launch_finalize<double>(h->d, m, h->stream) : phd::launch_finalize<float>(h->d, m, h->stream);
  for (int pi = 0; pi < 7 && e == cudaSuccess; ++pi)
    for (int gi = 0; gi < 3 && e == cudaSuccess; ++gi) {
      m.tune = best;
      m.tune.r_pb = pgs[pi][0];
      m.tune.r_g = pgs[pi][1];
      m.tune.grid2 = grids[gi];
      if (!phd::tune_supported(m.tune, fp64)) continue;
      float us = 0.0f;
      e = time_pass(h, reps, [&] {
        return fp64 ? phd::launch_rowsum<double>(h->d, m, h->stream) : phd::launch_rowsum<float>(h->d, m, h->stream);
      }, &us);
      if (e == cudaSuccess && (!have2 || us < best2)) {
        best2 = us;
        have2 = true;
        best.r_pb = m.tune.r_pb;
        best.r_g = m.tune.r_g;
        best.grid2 = m.tune.grid2;
      }
    }
  // spatial order on or off: the whole update and the extraction (whose label
  // sums walk the same order) timed both ways
  if (e == cudaSuccess) {
    float t_on = 0.0f, t_off = 0.0f;
    m.tune = best;
    auto upd_ext = [&] {
      cudaError_t r = fp64 ? phd::launch_update<double>(h->d, m, h->stream)
                           : phd::launch_update<float>(h->d, m, h->stream);
      if (r == cudaSuccess)
        r = fp64 ? phd::launch_extract<double>(h->d, m, static_cast<double*>(h->out_states), h->out_labels,
                                               h->cfg.m_max, nullptr, h->stream)
                 : phd::launch_extract<float>(h->d, m, static_cast<float*>(h->out_states), h->out_labels,
                                              h->cfg.m_max, nullptr, h->stream);
      return r;
    };
    m.tune.order = 1;
    e = time_pass(h, reps, upd_ext, &t_on);
    m.tune.order = 0;
    if (e == cudaSuccess) e = time_pass(h, reps, upd_ext, &t_off);
    if (e == cudaSuccess) best.order = t_on < t_off ? 1 : 0;
  }
  // leave the update's outputs as the chosen shapes compute them, and the
  // statistics as they were
  h->m.tune = best;
  if (e == cudaSuccess)
    e = fp64 ? phd::launch_update<double>(h->d, h->m, h->stream) : phd::launch_update<float>(h->d, h->m, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.stats, saved, sizeof(saved), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  destroy_graphs(h);
  if (e != cudaSuccess) {
    h->m.tune = base;
    return cuda_fail(h, e, "phd_autotune");
  }
  if (out)
    *out = phd_tuning{best.c_tile, best.c_mb, best.r_pb, best.r_g, best.grid1,
                      best.grid2, best.gate, best.order, best1, best2};
  return read_device_error(h);
}

}  // extern "C"

namespace {

// Fields every run of a batch must share (the sensor model and dynamics the
// kernels take as constants); per-run fields are clutter, births, rho, sizes.
const char* batch_problem(const phd_config* c, int runs) {
  if (!c || runs < 1 || runs > phd::kMaxPE) return "runs must be in 1..256";
  for (int j = 0; j < runs; ++j) {
    if (check_config(c[j])) return check_config(c[j]);
    if (c[j].num_pe != 1) return "every run of a batch is a one-PE filter";
    const phd_config& a = c[0];
    const phd_config& b = c[j];
    if (b.meas_model != a.meas_model || b.precision != a.precision || b.sigma_z[0] != a.sigma_z[0] ||
        b.sigma_z[1] != a.sigma_z[1] || b.sensor[0] != a.sensor[0] || b.sensor[1] != a.sensor[1] ||
        b.region[0] != a.region[0] || b.region[1] != a.region[1] || b.region[2] != a.region[2] ||
        b.region[3] != a.region[3] || b.r_max != a.r_max || b.dt != a.dt || b.sigma_a != a.sigma_a ||
        b.p_s != a.p_s || b.p_d != a.p_d || b.birth_vel_sigma != a.birth_vel_sigma || b.seed != a.seed ||
        b.sigma_a_y != a.sigma_a_y || b.birth_model != a.birth_model || b.theta_span != a.theta_span ||
        std::memcmp(b.birth_mean, a.birth_mean, sizeof(a.birth_mean)) != 0 ||
        std::memcmp(b.birth_std, a.birth_std, sizeof(a.birth_std)) != 0)
      return "runs of a batch differ in a shared model field";
  }
  return nullptr;
}

phd_config batch_envelope(const phd_config* c, int runs) {
  phd_config e = c[0];
  for (int j = 1; j < runs; ++j) {
    if (c[j].pe_cap > e.pe_cap) e.pe_cap = c[j].pe_cap;
    if (c[j].m_max > e.m_max) e.m_max = c[j].m_max;
  }
  e.num_pe = 1;
  e.ck_mode = PHD_CK_LOCAL;
  e.exchange_frac = 0.0;
  return e;
}

}  // namespace

extern "C" {

phd_status phd_batch_workspace_size(const phd_config* cfgs, int32_t runs, size_t* bytes) {
  if (!bytes || batch_problem(cfgs, runs)) return PHD_ERR_INVALID_ARG;
  const phd_config e = batch_envelope(cfgs, runs);
  *bytes = carve(e, nullptr, nullptr, nullptr, nullptr, runs);
  return PHD_OK;
}

phd_status phd_batch_init(phd_handle** out, const phd_config* cfgs, int32_t runs, void* ws, size_t bytes,
                          void* stream) {
  if (!out) return PHD_ERR_INVALID_ARG;
  *out = nullptr;
  if (batch_problem(cfgs, runs)) return PHD_ERR_INVALID_ARG;
  const phd_config e = batch_envelope(cfgs, runs);
  const size_t need = carve(e, nullptr, nullptr, nullptr, nullptr, runs);
  if (!ws || bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return PHD_ERR_INVALID_ARG;
  phd_handle* h = new (std::nothrow) phd_handle();
  if (!h) return PHD_ERR_INVALID_ARG;
  h->cfg = e;
  h->batch_runs = runs;
  h->m = make_model(e);
  h->m.K = runs;
  h->stream = static_cast<cudaStream_t>(stream);
  h->stage = kReady;
  carve(e, static_cast<char*>(ws), &h->d, &h->out_states, &h->out_labels, runs);
  cudaError_t err = cudaGetDevice(&h->device);
  if (err == cudaSuccess) err = is_fp64(h) ? phd::prepare_kernels<double>(h->m) : phd::prepare_kernels<float>(h->m);
  if (err == cudaSuccess)
    h->pgrid = is_fp64(h) ? phd::persist_grid<double>(h->m, true) : phd::persist_grid<float>(h->m, true);
  (void)cudaGetLastError();
  if (err == cudaSuccess) err = cudaMemsetAsync(ws, 0, need, h->stream);
  phd::Anchor tab[phd::kAnchors];
  phd::fill_anchor_table(tab);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(const_cast<void*>(h->d.anchors), tab, sizeof(tab), cudaMemcpyHostToDevice, h->stream);
  if (err == cudaSuccess) err = upload_slices(h, std::vector<phd_config>(cfgs, cfgs + runs));
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  if (err != cudaSuccess) {
    delete h;
    return PHD_ERR_CUDA;
  }
  h->fused_ok = false;
  *out = h;
  return PHD_OK;
}

phd_status phd_batch_step(phd_handle* h, const void* d_Z, const int32_t* d_offsets, void* d_states,
                          int32_t* d_labels, int32_t* d_counts, int32_t cap) {
  return phd_batch_step_inject(h, d_Z, d_offsets, nullptr, nullptr, d_states, d_labels, d_counts, cap);
}

phd_status phd_batch_step_inject(phd_handle* h, const void* d_Z, const int32_t* d_offsets, const void* d_noise,
                                 const uint32_t* d_u, void* d_states, int32_t* d_labels, int32_t* d_counts,
                                 int32_t cap) {
  if (!h) return PHD_ERR_INVALID_ARG;
  if (!h->batch_runs) return fail(h, PHD_ERR_STATE, "phd_batch_step needs a handle from phd_batch_init");
  if (h->stage != kReady) return fail(h, PHD_ERR_STATE, "phd_batch_step: a step is already in progress");
  if (!d_Z || !d_offsets || !d_counts || cap < 0 || (cap > 0 && (!d_states || !d_labels)))
    return fail(h, PHD_ERR_INVALID_ARG, "bad phd_batch_step arguments");
  if (phd_status sa = check_align(h, d_Z, d_states, d_noise, {d_offsets, d_labels, d_counts, d_u})) return sa;
  cudaError_t e = is_fp64(h)
      ? phd::launch_stage_zb<double>(h->d, h->m, static_cast<const double*>(d_Z), d_offsets, h->stream)
      : phd::launch_stage_zb<float>(h->d, h->m, static_cast<const float*>(d_Z), d_offsets, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage_zb");
  h->launches += 1;
  phd_status st = PHD_OK;
  if (use_grid(h)) {
    st = run_grid(h, nullptr, 0, d_noise, d_u, nullptr, nullptr, nullptr, 0, nullptr);
    if (st != PHD_OK) return st;
  } else if (d_noise || d_u) {
    // caller random numbers: the stages one by one (no graph)
    st = do_predict(h, d_noise);
    if (st == PHD_OK) {
      e = is_fp64(h) ? phd::launch_update<double>(h->d, h->m, h->stream)
                     : phd::launch_update<float>(h->d, h->m, h->stream);
      if (e != cudaSuccess) st = cuda_fail(h, e, "update");
      h->launches += phd::n_update_launches(h->m);
      h->stage = kUpdated;
    }
    if (st == PHD_OK) {
      e = is_fp64(h) ? phd::launch_extract<double>(h->d, h->m, nullptr, nullptr, 0, nullptr, h->stream)
                     : phd::launch_extract<float>(h->d, h->m, nullptr, nullptr, 0, nullptr, h->stream);
      if (e != cudaSuccess) st = cuda_fail(h, e, "extract");
      h->launches += n_extract(h);
    }
    if (st == PHD_OK) st = do_resample(h, d_u, nullptr);
    if (st != PHD_OK) {
      h->stage = kReady;
      return st;
    }
  } else {
    st = run_step_body(h);
    if (st != PHD_OK) return st;
  }
  e = is_fp64(h) ? phd::launch_batch_out<double>(h->d, h->m, static_cast<double*>(d_states), d_labels, d_counts,
                                                 cap, h->stream)
                 : phd::launch_batch_out<float>(h->d, h->m, static_cast<float*>(d_states), d_labels, d_counts, cap,
                                                h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "batch_out");
  h->launches += 1;
  h->have_update = true;
  return PHD_OK;
}

phd_status phd_sync(phd_handle* h) {
  if (!h) return PHD_ERR_INVALID_ARG;
  return read_device_error(h);
}

}  // extern "C"
