/*
 * phd.h -- C ABI of libphd.so: the particle PHD filter step on one GB300 GPU.
 *
 * The library implements one step of the particle PHD filter of
 * "Distributed Computation Particle PHD filter" (arXiv 1503.03769) in two
 * forms: the exact global filter (Sec. 2.2) and the paper's distributed
 * DCPFPHD scheme (Sec. 3, Algorithm 1), where K processing elements (PEs) each
 * own a slice of the particles against the full measurement set, exchange
 * particles on a ring and report measurement-labelled estimates to a central
 * unit (CU) that fuses them.  Every stage runs in hand-written CUDA kernels on
 * the caller's stream; there is no CPU fallback.
 *
 * Conventions (all entry points):
 *  - Every call returns a phd_status; no exception or longjmp crosses the ABI.
 *  - "d_" pointers are device memory, "h_" pointers host memory.  Device
 *    buffers are borrowed for the duration of the call (asynchronous calls:
 *    until the stream reaches the enqueued work).
 *  - Real-typed buffers hold float when cfg.precision == PHD_FP32 and double
 *    when cfg.precision == PHD_FP64 ("real" below).
 *  - A particle state is 4 reals [x, vx, y, vy] (Sec. 4 state vector); a
 *    measurement is 2 reals: (x, y) for PHD_MEAS_LINEAR, (range, bearing in
 *    (-pi, pi]) for PHD_MEAS_RANGE_BEARING.  The measurement's row index in
 *    Z_k is its label p (Sec. 3, Step 3).
 *  - Particle slices are laid out [K][pe_cap]: PE j owns slots
 *    j*pe_cap .. j*pe_cap + n_j - 1.
 *  - Alignment: the kernels access caller buffers as vectors, so a
 *    measurement array (Z) must be aligned to one row of 2 reals (8 bytes
 *    FP32, 16 FP64); an estimate, state-row or injected-draw array to one row
 *    of 4 reals (16 bytes FP32, 32 FP64); int32 / uint32 arrays to 4 bytes.
 *    Allocations from cudaMalloc, cudaHostAlloc or PyTorch qualify; a view at
 *    an odd element offset may not.  A misaligned buffer is refused with
 *    PHD_ERR_INVALID_ARG before anything is launched (phd_step_host instead
 *    copies through the workspace).
 *  - Calls are asynchronous on the stream given to phd_init unless marked
 *    "synchronises"; those wait for the stream before returning.
 *  - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef PHD_H
#define PHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PHD_OK = 0,
    PHD_ERR_INVALID_ARG = 1,  /* bad pointer, size, config value, or non-finite input */
    PHD_ERR_CAPACITY = 2,     /* a count exceeds pe_cap / m_max / the caller's capacity */
    PHD_ERR_CUDA = 3,         /* a CUDA runtime call failed; see phd_last_error_string */
    PHD_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    PHD_ERR_STATE = 5         /* call out of order (e.g. extract before update) */
} phd_status;

enum { PHD_MEAS_LINEAR = 0, PHD_MEAS_RANGE_BEARING = 1 };
enum { PHD_FP32 = 0, PHD_FP64 = 1 };
enum { PHD_CK_LOCAL = 0, PHD_CK_GLOBAL = 1 };
enum { PHD_PATH_AUTO = 0, PHD_PATH_STAGED = 1, PHD_PATH_FUSED = 2, PHD_PATH_GRID = 3 };
enum { PHD_BIRTH_UNIFORM = 0, PHD_BIRTH_GAUSSIAN = 1 };
enum { PHD_XCHG_RING = 0, PHD_XCHG_ALL = 1 };

/* Filter configuration (plain data, copied by phd_init). */
typedef struct phd_config {
    int32_t meas_model;     /* PHD_MEAS_LINEAR | PHD_MEAS_RANGE_BEARING (Sec. 4) */
    int32_t precision;      /* PHD_FP32: FP32 bulk, FP64 normalisers and CDF; PHD_FP64: all FP64 */
    int32_t num_pe;         /* K >= 1 processing elements (1 = global filter), <= 256 */
    int32_t ck_mode;        /* PHD_CK_LOCAL: each PE uses its own C^j (Step 2);
                               PHD_CK_GLOBAL: every PE uses the mean of the C^j */
    int32_t pe_cap;         /* particle slots per PE (survivors + births), <= 2^24 */
    int32_t m_max;          /* largest |Z_k| accepted, 1..4096 */
    int32_t birth_count;    /* J birth particles per step, split J/K per PE (Step 1) */
    int32_t birth_model;    /* birth density of Eq. 6 (drawn from as the proposal, weight
                               nu_b / J_j): PHD_BIRTH_UNIFORM: position U(region), velocity
                               N(0, birth_vel_sigma^2 I); PHD_BIRTH_GAUSSIAN: the state
                               N(birth_mean, diag(birth_std^2)) (Sec. 4's N(.; x_bar, Q)) */
    double dt;              /* sampling period T */
    double sigma_a;         /* acceleration noise std (m/s^2), x axis (both axes if sigma_a_y = 0) */
    double sigma_z[2];      /* linear: (sx, sy) m; range-bearing: (s_r m, s_theta rad) */
    double sensor[2];       /* range-bearing sensor position */
    double region[4];       /* x_min, x_max, y_min, y_max: birth support, linear clutter support */
    double r_max;           /* range-bearing clutter support [0, r_max] x (bearing span) */
    double p_s;             /* survival probability e_{k|k-1} (Eq. 5) */
    double p_d;             /* detection probability P_D (Eq. 4) */
    double clutter_rate;    /* lambda: kappa(z) = lambda / |measurement space| */
    double birth_mass;      /* nu_b: expected births per step; each birth weighs nu_b / J_j */
    double birth_vel_sigma; /* birth velocity std per axis (m/s) */
    double particles_per_target; /* rho: a PE resamples to round((rho/K) max(1, N^j)) */
    double exchange_frac;   /* ring exchange: floor(frac * min_j n_j) particles per PE (Step 6) */
    uint64_t seed;          /* Philox-4x32-10 key for the in-kernel random numbers */
    double sigma_a_y;       /* acceleration noise std of the y axis; 0: sigma_a */
    double theta_span;      /* range-bearing clutter bearing extent in (0, 2 pi]; 0: 2 pi
                               (kappa = lambda / (r_max theta_span)) */
    double birth_mean[4];   /* PHD_BIRTH_GAUSSIAN: mean state [x, vx, y, vy] */
    double birth_std[4];    /* PHD_BIRTH_GAUSSIAN: std per state component (diagonal Q) */
    int32_t exchange_mode;  /* Step 6 pattern: PHD_XCHG_RING: PE j's t-th outgoing particle goes
                               to PE j+1 (the paper's); PHD_XCHG_ALL: to PE j + 1 + (t mod (K-1))
                               (mod K), so every PE receives from all others; either way the
                               receiver's t-th vacated slot takes it */
    int32_t reserved1;      /* must be 0 */
    double exchange_threshold; /* 0: exchange every step (the paper's); > 0: only in steps where
                               some PE has degenerated, min_j N^j < threshold * mean_j N^j */
    double gate_sigma;      /* 0: the exact likelihood; k > 0: a variant (it changes results) that
                               truncates g(z|x) to 0 beyond k standard deviations, i.e. where
                               (d0/s0)^2 + (d1/s1)^2 >= k^2 (the paper's "simplify the update
                               step"); every pass uses the truncated g */
} phd_config;

typedef struct phd_handle phd_handle;

/* ---- lifetime ------------------------------------------------------------ */

/* Bytes of device workspace phd_init needs for cfg (>= 256-byte aligned). */
phd_status phd_workspace_size(const phd_config *cfg, size_t *bytes);

/* Create a filter.  d_workspace: caller-owned device buffer of at least
 * phd_workspace_size bytes, 256-byte aligned, that must outlive the handle;
 * the handle owns host metadata only.  stream: a cudaStream_t (NULL = the
 * legacy default stream), borrowed.  The filter starts empty (no particles,
 * mass 0): targets enter through birth (Eq. 6).  Synchronises. */
phd_status phd_init(phd_handle **h, const phd_config *cfg, void *d_workspace, size_t bytes,
                    void *stream);

/* Release the handle (not the workspace).  Synchronises. */
phd_status phd_destroy(phd_handle *h);

/* Borrowed, NUL-terminated description of the handle's last error. */
const char *phd_last_error_string(const phd_handle *h);
const char *phd_status_string(phd_status s);

/* ---- the step's stages (Algorithm 1 order) -------------------------------- */

/* Prediction, Eq. 5 (survivors: CV transition with accelerations
 * (sigma_a n1, sigma_a_y n2), weight p_S w) and Eq. 6 (births: J_j particles
 * per PE drawn from the birth density, weight birth_mass / J_j).  d_noise:
 * NULL to draw in-kernel (Philox), or real [K][pe_cap][4] rows (n1, n2, u1,
 * u2): survivor slot i uses n1, n2 as its standard normal accelerations;
 * birth slot i uses n1, n2 as standard normal velocity draws and u1, u2 in
 * [0, 1) as the position draws: uniform birth x = x_min + u1 (x_max - x_min),
 * y likewise with u2; Gaussian birth x = mean_x + std_x r cos(2 pi u2),
 * y = mean_y + std_y r sin(2 pi u2), r = sqrt(-2 ln(1 - u1)) (Box-Muller),
 * vx = mean_vx + std_vx n1, vy = mean_vy + std_vy n2.
 * Errors: PHD_ERR_STATE if called twice without an update. */
phd_status phd_predict(phd_handle *h, const void *d_noise);

/* ---- measurement-driven birth (Eq. 6 with a learned proposal) ------------- */

/* Eq. 6 draws the births from a proposal p_k(x | Z_k) that may depend on the
 * current scan and weights them gamma(x) / (J p_k(x | Z_k)).  With a birth
 * network loaded, each PE's J_j births come from the defensive mixture
 *   q(x | Z) = alpha p_plain(x) + (1 - alpha) sum_p pi_p q_p(x),
 * p_plain = U(region) x N(0, birth_vel_sigma^2 I) the plain birth,
 * pi = softmax of the network's logit over the M measurements, q_p the
 * position draw around z_p (linear sensor: z_p + sensor noise; range-bearing:
 * range |z_r + s_r n1|, bearing z_th + s_th n2 around the sensor) times a
 * velocity Gaussian N(s_b (m_x, m_y), diag (s_b e^l)^2) (l clamped to
 * [log 0.05, log 5]; s_b = birth_vel_sigma), and weight
 *   w = (birth_mass / J_j) / (alpha + (1 - alpha) R(x)),
 *   R(x) = sum_p pi_p q_p(x) / p_plain(x),
 * 0 outside the region: the intensity sum_b w_b delta(x_b) is an unbiased
 * estimate of the plain birth intensity (gamma = birth_mass p_plain), so the
 * PHD recursion is unchanged in expectation; alpha = 1 (or M = 0) gives the
 * plain birth exactly.  The network (inputs per measurement: its position in
 * the plane scaled to the region, (p - centre) / half-width, and log1p of the
 * number of other measurements within 3 sigma per measurement coordinate;
 * 3 -> 64 -> 64 -> 5, exact-erf GELU, bfloat16 operands, FP32 sums) is the
 * one of phd_mlp_forward.
 *
 * Random numbers: each birth slot uses its plain-birth row (n1, n2, u1, u2)
 * (velocity normals; position fractions of the plain branch) and an extra
 * row (u_c, nz1, nz2, unused): u_c < alpha takes the plain branch, else the
 * component is the smallest p with CDF_p > (u_c - alpha) / (1 - alpha) and
 * nz1, nz2 are its position normals.  Injected noise then holds K * pe_cap
 * plain rows followed by K * jmax extra rows, jmax = ceil(J / K), PE j's
 * birth b at extra row j * jmax + b; without injected noise Philox draws them.
 *
 * Load (d_params: device FP32 [phd_mlp_nparams()], rounded to bfloat16 into
 * the workspace) or, with d_params NULL, unload the network.  alpha in (0, 1].
 * FP32 one-filter handles with the uniform birth density only (PHD_ERR_STATE
 * otherwise: the defensive part is the plain uniform birth).  With a network
 * loaded: the fused step kernel is not used; phd_predict refuses
 * (PHD_ERR_STATE: use phd_predict_z); phd_step, phd_step_inject,
 * phd_step_host and phd_run draw the births from the scan they are given.
 * Synchronises. */
phd_status phd_set_birth_proposal(phd_handle *h, const float *d_params, double alpha);

/* Prediction with the scan: stages Z (real [M][2] device rows, as for
 * phd_update), runs phd_predict's survivor and plain-birth draws, then, with
 * a network loaded, evaluates it on Z (or takes d_head, device FP32 [M][5]
 * network outputs (m_x, m_y, l_x, l_y, logit), when not NULL) and redraws
 * the births from the mixture.  Without a network it is phd_predict.
 * Asynchronous.  Errors as phd_predict and phd_update's checks of Z. */
phd_status phd_predict_z(phd_handle *h, const void *d_Z, int32_t M, const float *d_head, const void *d_noise);

/* Copy the network outputs [M][5] of the last learned-birth prediction to
 * d_out (at most cap rows); *h_M gets M.  Synchronises.  PHD_ERR_CAPACITY if
 * M > cap (cap rows copied), PHD_ERR_STATE without a network. */
phd_status phd_get_birth_head(phd_handle *h, float *d_out, int32_t cap, int32_t *h_M);

/* ---- the birth network: stateless inference and training ------------------ */

/* The network input per measurement (FP32): X[M][3] = ((p_x - c_x) / h_x,
 * (p_y - c_y) / h_y, log1p(n)) with p the measurement's position in the plane
 * (the measurement itself for the linear sensor; sensor + r (cos th, sin th)
 * for range-bearing), c and h the centre and half-widths of cfg.region, and
 * n the number of other measurements q with |z_q0 - z_p0| <= 3 sigma_z[0]
 * and |wrap(z_q1 - z_p1)| <= 3 sigma_z[1] (bearing wrapped to [-pi, pi]).
 * d_Z FP32 [M][2], device; stream a cudaStream_t or NULL.  Asynchronous.
 * PHD_ERR_INVALID_ARG for a bad cfg (phd_init's checks), M < 0, NULL
 * buffers or a d_Z not aligned to 8 bytes. */
phd_status phd_birth_features(const phd_config *cfg, const float *d_Z, int32_t M, float *d_X, void *stream);

/* Number of parameters (4741): W1[64][3], b1[64], W2[64][64], b2[64],
 * W3[5][64], b3[5], W[j][k] the weight from input k into unit j. */
int32_t phd_mlp_nparams(void);

/* Y[n][5] = network(X[n][3]) with bfloat16 operands (parameters, inputs and
 * hidden activations rounded to nearest even) and FP32 sums; d_params FP32
 * [phd_mlp_nparams()].  All pointers device; stream a cudaStream_t or NULL.
 * Asynchronous.  PHD_ERR_INVALID_ARG for n < 0 or NULL buffers. */
phd_status phd_mlp_forward(const float *d_params, const float *d_X, int32_t n, float *d_Y, void *stream);

/* Scratch bytes phd_mlp_grad needs for n inputs. */
phd_status phd_mlp_grad_scratch_size(int32_t n, size_t *bytes);

/* Mean training loss over n >= 1 inputs and its gradient d_grad
 * [phd_mlp_nparams()] (FP32).  Targets d_T[n][3] = (t, vx, vy): t = 1 when the
 * filter extracted an estimate for the measurement, with its velocity in m/s
 * (ignored when t = 0); vel_scale s_b > 0.  Per input, with v~ = v / s_b and
 * outputs y = (m_x, m_y, l_x, l_y, logit):
 *   L = softplus(logit) - t logit + t sum_d [ l_d + (v~_d - m_d)^2 e^{-2 l_d} / 2 ].
 * The forward pass is phd_mlp_forward's; the backward pass uses its bfloat16
 * weights and activations with FP32 deltas; per-CTA partial sums are added in
 * a fixed order (deterministic).  d_loss may be NULL.  Asynchronous.
 * PHD_ERR_CAPACITY if scratch_bytes is below phd_mlp_grad_scratch_size. */
phd_status phd_mlp_grad(const float *d_params, const float *d_X, const float *d_T, int32_t n, float vel_scale,
                        float *d_grad, float *d_loss, void *d_scratch, size_t scratch_bytes, void *stream);

/* One Adam step (Kingma & Ba, ICLR 2015, Algorithm 1) on the FP32 parameters
 * with moment buffers d_m, d_v (zero before step t = 1), step t >= 1.
 * Asynchronous. */
phd_status phd_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int32_t t, float lr,
                        float beta1, float beta2, float eps, void *stream);

/* Update, Eq. 7-8: C^j_p = sum_i p_D g(z_p|x_i) w_i per PE (FP64 accumulation),
 * w_i <- [(1 - p_D) + sum_p p_D g(z_p|x_i) / (kappa + C_p)] w_i with C_p the
 * PE's own C^j_p (LOCAL) or the PE mean (GLOBAL).  d_Z: real [M][2]; it is
 * copied into the workspace on the stream, so the caller may overwrite it
 * once the stream has passed this call.
 * Errors: PHD_ERR_CAPACITY if M > m_max; PHD_ERR_INVALID_ARG if M < 0;
 * PHD_ERR_STATE unless a predict came first.  Non-finite measurements set the
 * handle's device error word, reported by the next synchronising call. */
phd_status phd_update(phd_handle *h, const void *d_Z, int32_t M);

/* Measurement-labelled extraction (Eq. 10-18, Step 3) and CU fusion (Step 4).
 * Per PE j: LT_j = round(N^j) with N^j the updated mass; the LT_j largest
 * sub-weight masses dW^{j,p} = C^j_p / (kappa + C_p) (ties: lower label;
 * dW = 0 never taken); zeta_p = sum_i dw^{i,p} x_i / dW^p (Eq. 18).  Fusion
 * keeps a label reported by more than K/2 PEs with the mean of their states
 * (for K = 1 every selected label).  Output, ascending label: d_states real
 * [cap][4], d_labels int32 [cap]; d_count (device int32, may be NULL) gets the
 * true count.  If h_count is non-NULL the call synchronises, stores the true
 * count and returns PHD_ERR_CAPACITY when it exceeds cap (the first cap
 * estimates are still written).  Errors: PHD_ERR_STATE unless after update. */
phd_status phd_extract(phd_handle *h, void *d_states, int32_t *d_labels, int32_t cap,
                       int32_t *d_count, int32_t *h_count);

/* Resampling (Sec. 2.2 step 3; Algorithm 1 "Resample") then, for K > 1 and
 * exchange_frac > 0, the ring exchange (Step 6).  Per PE: systematic
 * resampling on the exact integer CDF Q_i = sum_{k<=i} floor(w_k 2^s),
 * s = 52 - ceil(log2 n) - e, max w < 2^e; L_j = min(pe_cap - J_j,
 * round((rho/K) max(1, N^j))); child t's parent is the least i with
 * Q_i > floor((t 2^32 + U_j) Q_n / (L_j 2^32)); new weights N^j / L_j.  Then
 * PE j moves floor(frac min_j L_j) random particles (partial Fisher-Yates,
 * r = t + floor(u_t (L_j - t) / 2^32)) into the same number of slots that
 * PE j+1 vacated.  d_u: NULL (Philox) or uint32 [K]; d_xu: NULL (Philox) or
 * uint32 [K][pe_cap] exchange draws.  Errors: PHD_ERR_STATE unless after update. */
phd_status phd_resample(phd_handle *h, const uint32_t *d_u, const uint32_t *d_xu);

/* One whole step with in-kernel random numbers: predict, update, extract,
 * resample (+ exchange).  Arguments as for phd_update and phd_extract
 * (h_count non-NULL synchronises). */
phd_status phd_step(phd_handle *h, const void *d_Z, int32_t M, void *d_states, int32_t *d_labels,
                    int32_t cap, int32_t *d_count, int32_t *h_count);

/* phd_step with caller-supplied random numbers (layouts as phd_predict and
 * phd_resample; any of them may be NULL for in-kernel Philox draws).  Runs
 * the same kernels phd_step would (see phd_set_path). */
phd_status phd_step_inject(phd_handle *h, const void *d_Z, int32_t M, const void *d_noise, const uint32_t *d_u,
                           const uint32_t *d_xu, void *d_states, int32_t *d_labels, int32_t cap, int32_t *d_count,
                           int32_t *h_count);

/* S consecutive steps in one call (offline replay of recorded scans, Monte
 * Carlo runs).  d_Z: real rows of all scans back to back; d_offsets: device
 * int32 [S+1], scan s is rows d_offsets[s] .. d_offsets[s+1]-1 (each at most
 * m_max rows, else the scan is skipped and PHD_ERR_CAPACITY is reported at the
 * next synchronising call).  Outputs per scan s: d_states real [S][cap][4],
 * d_labels int32 [S][cap], d_counts int32 [S] (true counts).  On the fused
 * path this is one kernel launch for all S steps; on the staged path one
 * graph launch per step (the offsets are read back once).  Asynchronous. */
phd_status phd_run(phd_handle *h, const void *d_Z, const int32_t *d_offsets, int32_t S, void *d_states,
                   int32_t *d_labels, int32_t *d_counts, int32_t cap);

/* Kernel path of phd_step / phd_step_host / phd_step_inject / phd_run (and,
 * for batch handles, phd_batch_step).
 * PHD_PATH_FUSED: one cooperative kernel per call, one CTA per PE with the PE's
 * slice in shared memory (available when the slice of pe_cap particles and
 * m_max measurements fits an SM's shared memory and all K CTAs can be
 * co-resident); PHD_PATH_GRID: one cooperative kernel per step over the
 * whole GPU, its phases (prediction, spatial order, the two pair passes,
 * selection, label sums, resampling) separated by grid-wide barriers with
 * bounded waits, every PE's slice spread over the kernel's CTAs (available
 * when m_max fits its shared memory, for one-PE filters, for K PEs on one
 * scan without a birth network, whose scan is staged before the launch and
 * whose CU fusion (Step 4) and exchange (Step 6) run as kernels after it,
 * and for batches of independent runs; a one-PE filter with a birth network
 * has the scan staged and the network's head, mixture table and draws run
 * as kernels before it; the pair passes always walk the spatial order, the
 * gate setting of phd_set_tuning applies, its launch shapes do not);
 * PHD_PATH_STAGED: the stage kernels of phd_predict .. phd_resample as a
 * CUDA graph; PHD_PATH_AUTO (default): fused when available, else grid when
 * available and the handle holds at most 16 chunks of 256 particle slots
 * per CTA of the step kernel (K x ceil(pe_cap / 256) <= 16 x its CTAs: one
 * filter, PEs whose slices outgrow an SM, small batches), else staged.  phd_set_path returns
 * PHD_ERR_INVALID_ARG for an unavailable path; phd_get_path reports the
 * path in use.  The stage calls (phd_predict, phd_update, phd_extract,
 * phd_resample) always run the staged kernels. */
phd_status phd_set_path(phd_handle *h, int32_t path);
phd_status phd_get_path(phd_handle *h, int32_t *path);

/* phd_step from host memory: h_Z [M][2] in, the estimates out to h_states
 * [cap][4] / h_labels [cap] and their true count to *h_count.  When h_Z and
 * the two output buffers are pinned and mapped (cudaHostAlloc or
 * cudaHostRegister memory) the step's kernels read h_Z and write the outputs
 * in host memory themselves (zero copy; over NVLink-C2C on Grace systems)
 * and the call synchronises once; otherwise (pageable buffers) it copies
 * through the workspace.  Synchronises.  Errors as phd_step;
 * PHD_ERR_INVALID_ARG for non-finite h_Z. */
phd_status phd_step_host(phd_handle *h, const void *h_Z, int32_t M, void *h_states,
                         int32_t *h_labels, int32_t cap, int32_t *h_count);

/* ---- state access (parity tests, checkpoint / resume) --------------------- */

/* Replace the particle set: d_x real [K][pe_cap][4], d_w real [K][pe_cap],
 * h_counts int32 [K] (each <= pe_cap - J_j).  Resets the stage order to
 * "ready to predict".  Synchronises. */
phd_status phd_set_state(phd_handle *h, const void *d_x, const void *d_w, const int32_t *h_counts);

/* Copy the current particle set (layout as phd_set_state; slots beyond n_j
 * are unspecified) and h_counts int32 [K].  Between phd_predict and
 * phd_resample this is the predicted set, with the predicted weights after
 * phd_predict and the updated weights (Eq. 8) after phd_update.
 * Synchronises. */
phd_status phd_get_state(phd_handle *h, void *d_x, void *d_w, int32_t *h_counts);

/* After an update (phd_update or a whole step): d_C double [K][m_max] with
 * C^j_p of Eq. 7 per PE, and h_mass double [K] (may be NULL) with the updated
 * masses N^j of the most recent update.  Synchronises. */
phd_status phd_get_update(phd_handle *h, double *d_C, double *h_mass);

/* After an update: the most recent predicted set d_x real [K][pe_cap][4], its
 * predicted weights d_w_pred and updated weights d_w_upd (real [K][pe_cap];
 * any pointer may be NULL) and h_counts int32 [K].  Synchronises. */
phd_status phd_get_predicted(phd_handle *h, void *d_x, void *d_w_pred, void *d_w_upd, int32_t *h_counts);

/* After phd_extract: per-PE local estimates before fusion, d_states real
 * [K][m_max][4], d_labels int32 [K][m_max] in selection order, h_counts int32
 * [K].  Synchronises. */
phd_status phd_get_local_estimates(phd_handle *h, void *d_states, int32_t *d_labels,
                                   int32_t *h_counts);

/* After phd_resample: d_parents int32 [K][pe_cap] (parent slot of each child
 * before the exchange) and h_lx (may be NULL) = particles moved per PE.
 * Synchronises. */
phd_status phd_get_resample(phd_handle *h, int32_t *d_parents, int32_t *h_lx);

/* Step counter (drives the Philox counters); set it to resume a checkpoint. */
phd_status phd_get_step(phd_handle *h, uint64_t *step);
phd_status phd_set_step(phd_handle *h, uint64_t step);

/* ---- batches of independent filters --------------------------------------- */

/* A batch runs `runs` independent one-PE filters (Monte-Carlo runs, sensors
 * or sectors tracked separately) as one stage-synchronous pipeline: every
 * stage of every run is split into work items (particle tiles x measurement
 * chunks) that the kernels balance over the whole GPU, and a batched step is
 * one CUDA graph for all runs.  cfgs[j] describes run j (num_pe must be 1);
 * the runs must share the sensor model, precision, noise, region, dynamics,
 * p_S, p_D and seed, and may differ in clutter_rate, birth_count,
 * birth_mass, particles_per_target, pe_cap and m_max.  1 <= runs <= 256.
 * The paper's filter is run per run; batching is this library's addition. */
phd_status phd_batch_workspace_size(const phd_config *cfgs, int32_t runs, size_t *bytes);

/* As phd_init for a batch (same workspace and stream ownership).  The state
 * accessors (phd_get_state, phd_set_state, phd_get_update, ...) see the runs
 * as K = runs slices of the largest pe_cap / m_max.  Synchronises. */
phd_status phd_batch_init(phd_handle **h, const phd_config *cfgs, int32_t runs, void *d_workspace, size_t bytes,
                          void *stream);

/* One step of every run with in-kernel random numbers.  d_Z: real rows of all
 * runs' scans back to back; d_offsets: device int32 [runs+1], run j's scan is
 * rows d_offsets[j] .. d_offsets[j+1]-1 (at most the largest m_max of the
 * runs; a run over it is given no measurements and PHD_ERR_CAPACITY is
 * reported at the next synchronising call).  Outputs per run j, ascending label:
 * d_states real [runs][cap][4], d_labels int32 [runs][cap], d_counts int32
 * [runs] (true counts).  Asynchronous.  Errors: PHD_ERR_STATE on a one-filter
 * handle; PHD_ERR_INVALID_ARG for NULL buffers. */
phd_status phd_batch_step(phd_handle *h, const void *d_Z, const int32_t *d_offsets, void *d_states,
                          int32_t *d_labels, int32_t *d_counts, int32_t cap);

/* phd_batch_step with caller random numbers (either may be NULL for Philox):
 * d_noise real [runs][pe_cap][4] as for phd_predict (pe_cap the largest of the
 * runs), d_u uint32 [runs] resampling uniforms.  The stages run one by one
 * instead of as a graph. */
phd_status phd_batch_step_inject(phd_handle *h, const void *d_Z, const int32_t *d_offsets, const void *d_noise,
                                 const uint32_t *d_u, void *d_states, int32_t *d_labels, int32_t *d_counts,
                                 int32_t cap);

/* ---- counters and the update-stage timer ---------------------------------- */

typedef struct phd_stats {
    uint64_t pairs;          /* sum over updates of particles x measurements */
    uint64_t particles;      /* sum over updates of predicted particles (all PEs) */
    uint64_t measurements;   /* sum over updates of |Z_k| */
    uint64_t updates;        /* updates run */
    uint64_t launches;       /* CUDA kernels this handle launched */
    uint64_t timed_updates;  /* updates bracketed by the stage timer */
    double update_ms;        /* their summed device time (CUDA events), ms: the update
                                stage's kernels on the staged path, the whole fused
                                step kernel on the fused path */
    uint64_t pairs_evaluated; /* pass-1 pairs actually evaluated (pairs of a tile with a
                                 measurement past the exact likelihood gate are not) */
} phd_stats;

/* Read the counters accumulated since phd_init / phd_reset_stats.  Synchronises. */
phd_status phd_get_stats(phd_handle *h, phd_stats *out);
phd_status phd_reset_stats(phd_handle *h);

/* Time spent in each phase of the grid path's step kernel since phd_init /
 * phd_reset_stats (device clock, read by one thread per CTA at the phases'
 * barriers), in milliseconds, in 12 slots per figure of which 10 are used,
 * for the phases: prediction + spatial keys + cell totals, cell starts,
 * scatter, pass 1 (Eq. 7), normalisers (Eq. 12), pass 2 (Eq. 8) + selection
 * ranks, mass and plan (batches), plan + CDF chunk sums + label sums
 * (Eq. 18), estimates + CDF offsets, offspring ends + gather (slots 10, 11:
 * zero):
 *   h_ms[0..11]   summed over launches, from the previous barrier's release
 *                 to the phase's own (the phase's wall time);
 *   h_ms[12..23]  the longest time one CTA worked in the phase (from leaving
 *                 the previous barrier to arriving at the next), the largest
 *                 over launches;
 *   h_ms[24..35]  the time a CTA worked in the phase, summed over launches and
 *                 averaged over CTAs.
 * n <= 36 values are written.  Zeros on the other paths.  Synchronises. */
phd_status phd_get_phase_times(phd_handle *h, double *h_ms, int32_t n);

/* on != 0: phd_step / phd_step_host bracket the update stage (Eq. 7-8 pair
 * passes) with CUDA events on the handle's stream; the times add up in
 * phd_stats.update_ms.  The step then runs as three graph launches instead of
 * one.  Does not synchronise. */
phd_status phd_set_stage_timer(phd_handle *h, int32_t on);

/* ---- failure detection ------------------------------------------------------ */

/* Every wait of a CTA on other CTAs (the fused step's grid barriers) polls at
 * most `iterations` times (each poll a ~32 ns sleep and an L2 load; the
 * default 2e7 is several seconds), then records a timeout in the device error
 * word and every CTA of the launch returns: the GPU context stays usable and
 * the next synchronising call returns PHD_ERR_TIMEOUT (and resets the barrier
 * and the error word).  iterations in 1 .. 1e9.  Synchronises. */
phd_status phd_set_wait_limit(phd_handle *h, int64_t iterations);

/* Failure injection for tests (host side; nothing on the GPU faults): sets a
 * flag that makes PE 0 leave the next fused step of a K > 1 filter at its
 * first grid barrier without arriving, as a PE that died would; the other PEs
 * wait out their limit there and the step reports PHD_ERR_TIMEOUT (which
 * clears the flag).  On the grid path CTA 0 of the step kernel leaves the
 * same way and the other CTAs time out.  Synchronises. */
phd_status phd_inject_barrier_fault(phd_handle *h);

/* ---- launch shapes of the update's pair passes, and their autotuner -------- */

/* How the update's two pair passes (Eq. 7 column sums, Eq. 8 row sums) map
 * onto the GPU.  Every supported shape computes the same quantities; results
 * differ between shapes only by FP32 summation order (the FP64 accumulation
 * of C and of the masses stays in a fixed order for a given shape).
 *  c_tile: pass 1 particles per work item: 256, 512 or 1024;
 *  c_mb:   pass 1 measurements per thread: 1, 2 or 4 (64 * c_mb per item);
 *  r_pb:   pass 2 particles per thread: 1, 2 or 4;
 *  r_g:    pass 2 lanes sharing a particle: 1, 2, 4 or 8; (r_pb, r_g) is one
 *          of (1,1) (2,1) (4,1) (1,2) (2,2) (1,4) (1,8);
 *  grid1, grid2: CTA caps of pass 1 and pass 2 (1 .. 9728);
 *  gate:   1 (default) to skip pairs past the exact likelihood gate, 0 to
 *          evaluate every pair.  The FP32 exp2 flushes 2^-q to exactly 0 for
 *          q > 126 (FP64: q > 1074); a box around each work item's particles
 *          in measurement space bounds q from below, and pairs whose bound is
 *          at least 130 (FP64: 1100) are skipped: they add exactly nothing,
 *          so results are bit-identical with the gate on or off;
 *  order:  1 to walk the particles of passes 1 and 2 in the order of a 16 x 16
 *          grid over measurement space (a stable counting sort of each
 *          slice's predicted set before pass 1; the particles stay in their
 *          slots), which keeps a tile's particles close so that the gate
 *          skips most pairs; the extraction's label sums (pass 3) walk the
 *          same tiles.  Only the grouping of FP32 partial sums changes.
 *          Default 1 on FP32 handles, 0 on FP64 handles;
 *  pass1_us, pass2_us: filled by phd_autotune with the measured mean duration
 *          of each pass in the chosen shape (0 elsewhere; ignored on input).
 * FP64 handles support c_mb 2 and (r_pb, r_g) = (1, 4) only.  The default is
 * c_tile 512, c_mb 4 (2 in FP64), (1, 4), grid1 = grid2 = 1216.  The fused
 * step kernel (phd_set_path) does not use these shapes. */
typedef struct phd_tuning {
    int32_t c_tile, c_mb, r_pb, r_g, grid1, grid2, gate, order;
    float pass1_us, pass2_us;
} phd_tuning;

phd_status phd_get_tuning(phd_handle *h, phd_tuning *out);

/* Select a shape.  Synchronises the stream (captured step graphs are rebuilt
 * on the next step).  PHD_ERR_INVALID_ARG for an unsupported shape;
 * PHD_ERR_STATE for a change of `order` between phd_update and the step's
 * phd_resample (the extraction reads the order the update built). */
phd_status phd_set_tuning(phd_handle *h, const phd_tuning *t);

/* Autotuner: times every supported shape of pass 1 (c_tile x c_mb x grid1 in
 * {608, 1216, 2432}) and then of pass 2 ((r_pb, r_g) x grid2), each as the
 * mean of `reps` launches (1 .. 1000) after one untimed launch, then the whole
 * update and the extraction with the spatial order on and off (the gate
 * setting is kept), on the
 * handle's current predicted set and measurements, i.e. the input of the last
 * update (call it after a representative step: the best shape depends on the
 * slices' particle and measurement counts).  Keeps the fastest shape of each
 * pass, re-runs the update with it (so the update's outputs are the chosen
 * shape's), leaves phd_stats unchanged and returns the choice in *out (may be
 * NULL).  Works on one-filter and batch handles.  Synchronous.  Errors:
 * PHD_ERR_STATE when no update has run; PHD_ERR_CUDA (the previous shape is
 * kept). */
phd_status phd_autotune(phd_handle *h, int32_t reps, phd_tuning *out);

/* ---- normaliser column sums without device allocation ---------------------- */

/* C_p = sum_i p_D g(z_p | x_i) w_i for one particle set (the Eq. 7 column sums
 * of phd_update with the same pair arithmetic: FP32 pair terms, FP64 per-tile
 * partials summed in a fixed order, tiles of 256 particles), for callers that may not allocate device memory at all: trackers
 * whose device memory is fixed when they start (cudaMalloc and cudaFree can
 * synchronise the device and take unbounded time, which a real-time loop
 * cannot afford) and plug-ins running inside a host application that owns
 * every device allocation.  It needs no handle and no workspace; the paper has
 * no counterpart of this entry point.
 *  cfg: as for phd_init (must pass its checks); only the sensor model,
 *       sigma_z, sensor, p_d and precision are used.
 *  d_x: real [n][4] states, d_w: real [n] weights, d_Z: real [M][2]
 *       measurements, d_C: double [M] output; stream: a cudaStream_t or NULL.
 * Its scratch (per-tile partial sums) is a 4 MiB array in the library's own
 * device memory, held by every GPU that loads the library until the process
 * exits: ceil(n / 256) * M must not exceed 524288, else PHD_ERR_CAPACITY and
 * nothing runs.  No cudaMalloc, cudaFree or allocating library call is made.
 * The first call on a device, with that device current, looks up the array's
 * device address and copies in a 4 KB lookup table on `stream`, then waits
 * for `stream` (with stream NULL, the legacy default stream, that wait also
 * covers the work of every blocking stream on the device): make that first
 * call before any stream capture.  Later calls are asynchronous.  The looked-up
 * addresses are kept for the life of the process: after cudaDeviceReset the
 * library's device arrays are gone, and this entry point must not be called
 * again in that process.
 * Every call uses the same array; each call writes every partial it reads,
 * so nothing needs clearing, but calls that overlap on the GPU (concurrent
 * streams, several host threads) race on it: order them on one stream.
 * Non-finite states, weights or measurements give NaN column sums (as in
 * phd_update), except that with the gate_sigma truncation on, a pair whose
 * exponent is NaN counts as truncated (0).
 * Errors: PHD_ERR_INVALID_ARG for a bad cfg, negative sizes, NULL buffers or
 * buffers off their row alignment (d_x 4 reals, d_w 1, d_Z 2, d_C 8 bytes);
 * PHD_ERR_CUDA if the set-up or a launch fails. */
phd_status phd_colsum_static(const phd_config *cfg, const void *d_x, const void *d_w, int32_t n,
                             const void *d_Z, int32_t M, double *d_C, void *stream);

/* ---- roofline denominator ------------------------------------------------- */

/* Measured issue rate of the ex2 instruction the pair passes evaluate once per
 * particle x measurement pair (Eq. 7 and Eq. 8 each take g(z|x) through one
 * FP32 exp2 of its exponent): a full-occupancy grid on the current device (8
 * CTAs of 256 threads per SM), each thread running 8 independent chains of
 * 4096 dependent ex2 instructions.  Times `reps` launches (1 .. 10000) with
 * CUDA events on `stream` (a cudaStream_t or NULL) after one untimed launch
 * and returns the fastest as *h_per_s (ex2 instructions per second, the
 * whole device) and *h_best_ms (may be NULL).  The paper has no counterpart;
 * this is the denominator the benchmark's roofline fraction uses.
 * Synchronises.  Errors: PHD_ERR_INVALID_ARG for reps out of range or a NULL
 * h_per_s; PHD_ERR_CUDA if a launch fails. */
phd_status phd_measure_ex2_rate(int32_t reps, double *h_per_s, double *h_best_ms, void *stream);

/* Wait for the stream and report a device-side error (non-finite input,
 * bounded-wait timeout) recorded since the last check.  Synchronises. */
phd_status phd_sync(phd_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* PHD_H */
