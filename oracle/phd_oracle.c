/*
 * FP64 CPU oracle of the particle PHD filter step and of its distributed
 * (DCPFPHD) form, written from "Distributed Computation Particle PHD filter"
 * (arXiv 1503.03769).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it is built and used by the tests, by the package's smoke
 * check and by the benchmark's CPU-baseline leg.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Style: plain loops in IEEE double, in the order the paper states the
 * steps; no blocking, fusion or reordering.  Each function names the passage
 * it follows.  Where the paper is silent or garbled, the reading taken is
 * stated at the function.  The default build is single-threaded.  A second
 * build with OpenMP (used to time the oracle on all host cores and for long
 * reference runs) splits only the marked loops, whose iterations each write
 * their own outputs and keep their inner sums in the serial order, so its
 * results are bit-identical to the single-threaded build's.
 *
 * State layout: a particle is [x, vx, y, vy] (Sec. 4, state vector), stored as
 * 4 consecutive doubles.  A measurement is 2 doubles: (x, y) for the linear
 * position sensor, (range, bearing) for the range-bearing sensor.
 *
 * Parity pins: every function here is pinned by tests (closed forms,
 * invariants, textbook reductions, brute force); see tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "orc_model.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the OpenMP build (no effect in the single-threaded build). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* 1 in the OpenMP build, 0 otherwise. */
int orc_is_parallel(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

static const double ORC_PI = 3.14159265358979323846;

/* Clutter intensity kappa(z) = lambda * c(z) with c uniform over the
 * measurement space (Sec. 4, clutter model): the region's area for the linear
 * sensor; [0, r_max] x the bearing span (2 pi unless given) for the
 * range-bearing sensor. */
double orc_kappa(const orc_model *m)
{
    /* kappa = lambda V_u(z) (Sec. 4): the uniform density over the
     * measurement space, the region (linear) or [0, r_max] x the bearing span */
    double vol;
    if (m->meas_model == ORC_LINEAR)
        vol = (m->region[1] - m->region[0]) * (m->region[3] - m->region[2]);
    else
        vol = m->r_max * (m->theta_span > 0.0 ? m->theta_span : 2.0 * ORC_PI);
    return m->clutter_rate / vol;
}

/* Bearing difference wrapped to (-pi, pi]. */
static double wrap_angle(double a)
{
    while (a > ORC_PI) a -= 2.0 * ORC_PI;
    while (a <= -ORC_PI) a += 2.0 * ORC_PI;
    return a;
}

/* Noise-free measurement h(x) (Sec. 4, measurement model). */
void orc_measure(const orc_model *m, const double *x, double *h)
{
    if (m->meas_model == ORC_LINEAR) {
        h[0] = x[0];
        h[1] = x[2];
    } else {
        double px = x[0] - m->sensor[0], py = x[2] - m->sensor[1];
        h[0] = sqrt(px * px + py * py);
        h[1] = atan2(py, px);
    }
}

/* Single-target likelihood g(z|x): Gaussian in the sensor's coordinates with
 * its normalising constant kept, since kappa is a density over the same space
 * (Eq. 4 with psi_z = p_D g, Sec. 4 sensor model).  The truncation variant
 * (gate_sigma = k > 0; the paper's "simplify the update step") sets g to 0
 * at Mahalanobis distance k and beyond. */
double orc_likelihood(const orc_model *m, const double *z, const double *x)
{
    double h[2], d0, d1;
    orc_measure(m, x, h);
    d0 = z[0] - h[0];
    d1 = z[1] - h[1];
    if (m->meas_model == ORC_RANGE_BEARING) d1 = wrap_angle(d1);
    d0 /= m->sigma_z[0];
    d1 /= m->sigma_z[1];
    if (m->gate_sigma > 0.0 && d0 * d0 + d1 * d1 >= m->gate_sigma * m->gate_sigma) return 0.0;
    return exp(-0.5 * (d0 * d0 + d1 * d1)) / (2.0 * ORC_PI * m->sigma_z[0] * m->sigma_z[1]);
}

/* Prediction, Eq. 5 (survivors) and Eq. 6 (births).
 * Survivors: proposal q = f (the CV transition of Sec. 4), so phi/q = e_{k|k-1}
 * and w~ = p_S w;  x~ = F x + G a with a = (sigma_a n1, sigma_a_y n2).
 * Births: J particles drawn from the birth density itself, so with
 * gamma = nu_b * p_k the weight gamma / p_k / J = nu_b / J:
 *   uniform: p_k = U(region) x N(0, s_b^2 I) for the velocity;
 *   Gaussian (Sec. 4's N(.; x_bar, Q), Q diagonal): every component
 *   x_bar_c + sqrt(Q_cc) n_c, the position normals by the Box-Muller map of
 *   (u1, u2): r = sqrt(-2 ln(1 - u1)), (r cos 2 pi u2, r sin 2 pi u2).
 * noise rows (n1, n2, u1, u2): survivors use n1, n2; births use n1, n2 for the
 * velocity and u1, u2 for the position.  Output: L survivors then J births. */
void orc_predict(const orc_model *m, const double *x_in, const double *w_in, int L, int J,
                 const double *noise, double *x_out, double *w_out)
{
    const double T = m->dt;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < L; ++i) {
        const double *x = x_in + 4 * i;
        double ax = m->sigma_a * noise[4 * i + 0];
        double ay = (m->sigma_a_y > 0.0 ? m->sigma_a_y : m->sigma_a) * noise[4 * i + 1];
        double *y = x_out + 4 * i;
        y[0] = x[0] + T * x[1] + 0.5 * T * T * ax;
        y[1] = x[1] + T * ax;
        y[2] = x[2] + T * x[3] + 0.5 * T * T * ay;
        y[3] = x[3] + T * ay;
        w_out[i] = m->p_s * w_in[i];
    }
#pragma omp parallel for schedule(static)
    for (int b = 0; b < J; ++b) {
        int i = L + b;
        const double *n = noise + 4 * i;
        double *y = x_out + 4 * i;
        if (m->birth_model == ORC_BIRTH_GAUSSIAN) {
            const double r = sqrt(-2.0 * log(1.0 - n[2]));
            y[0] = m->birth_mean[0] + m->birth_std[0] * r * cos(2.0 * ORC_PI * n[3]);
            y[1] = m->birth_mean[1] + m->birth_std[1] * n[0];
            y[2] = m->birth_mean[2] + m->birth_std[2] * r * sin(2.0 * ORC_PI * n[3]);
            y[3] = m->birth_mean[3] + m->birth_std[3] * n[1];
        } else {
            y[0] = m->region[0] + n[2] * (m->region[1] - m->region[0]);
            y[1] = m->birth_vel_sigma * n[0];
            y[2] = m->region[2] + n[3] * (m->region[3] - m->region[2]);
            y[3] = m->birth_vel_sigma * n[1];
        }
        w_out[i] = m->birth_mass / (double)J;
    }
}

/* Eq. 7 read as <psi_z, D>: C(z_p) = sum_j p_D g(z_p|x_j) w_j, for every
 * measurement (the "* x" of the printed equation is a typo). */
void orc_colsum(const orc_model *m, const double *x, const double *w, int N,
                const double *Z, int M, double *C)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < M; ++p) {
        double c = 0.0;
        for (int j = 0; j < N; ++j)
            c += m->p_d * orc_likelihood(m, Z + 2 * p, x + 4 * j) * w[j];
        C[p] = c;
    }
}

/* Eq. 8: w_i <- [nu(x_i) + sum_z psi_z(x_i) / (kappa(z) + C(z))] w_i with
 * nu = 1 - p_D (Eq. 4).  C_used is the normaliser the filter applies (its
 * own column sums, or an exact mean over PEs in the distributed form).
 * A measurement with kappa + C = 0 adds nothing: C = 0 forces every
 * psi_z(x_j) w_j to be 0, so its terms vanish in the limit. */
void orc_weight_update(const orc_model *m, const double *x, const double *w, int N,
                       const double *Z, int M, const double *C_used, double *w_out)
{
    const double kappa = orc_kappa(m);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        double s = 1.0 - m->p_d;
        for (int p = 0; p < M; ++p)
            if (kappa + C_used[p] > 0.0)   /* a zero normaliser has only zero terms */
                s += m->p_d * orc_likelihood(m, Z + 2 * p, x + 4 * i) / (kappa + C_used[p]);
        w_out[i] = s * w[i];
    }
}

/* Measurement-labelled state extraction (STPHD, Eq. 10-18 and the local
 * target count of Step 3).
 *  G^{i,p}  = psi_{z_p}(x_i) / (kappa + C(z_p))           (Eq. 12)
 *  dw^{i,p} = G^{i,p} w~_i                                 (Eq. 13)
 *  dW^p     = sum_i dw^{i,p}                               (Eq. 16)
 *  dW^0     = sum_i (1 - p_D) w~_i                         (Eq. 14, 17)
 *  LT       = round(N_k), N_k = sum of updated weights     (Step 3)
 *  take the LT largest dW^p (ties: lower label first); labels with dW^p = 0
 *  are never taken, and LT is capped at M;
 *  zeta_p   = sum_i dw^{i,p} x_i / dW^p                    (Eq. 18)
 * w_pred are the predicted weights, Nk the updated mass.  Outputs: labels and
 * states in selection order (descending dW, ties by label); returns the count.
 * dW_out (M) and dW0_out (1) receive the sub-weight masses. */
int orc_extract(const orc_model *m, const double *x, const double *w_pred, int N,
                const double *Z, int M, const double *C_used, double Nk,
                int *labels, double *zeta, double *dW_out, double *dW0_out)
{
    const double kappa = orc_kappa(m);
    double dW0 = 0.0;
    for (int i = 0; i < N; ++i) dW0 += (1.0 - m->p_d) * w_pred[i];
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < M; ++p) {
        double s = 0.0;
        if (kappa + C_used[p] > 0.0)
            for (int i = 0; i < N; ++i)
                s += m->p_d * orc_likelihood(m, Z + 2 * p, x + 4 * i) / (kappa + C_used[p]) * w_pred[i];
        dW_out[p] = s;
    }
    if (dW0_out) *dW0_out = dW0;

    long LT = lround(Nk);             /* round half away from zero */
    if (LT > M) LT = M;
    int n = 0;
    char *taken = (char *)calloc((size_t)(M > 0 ? M : 1), 1);
    while (n < LT) {
        int best = -1;
        for (int p = 0; p < M; ++p) {
            if (taken[p] || !(dW_out[p] > 0.0)) continue;
            if (best < 0 || dW_out[p] > dW_out[best]) best = p;   /* strict: lower p wins ties */
        }
        if (best < 0) break;
        taken[best] = 1;
        labels[n] = best;
        ++n;
    }
    /* Eq. 18 for each selected label */
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n; ++r) {
        const int p = labels[r];
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < N; ++i) {
            double dw = m->p_d * orc_likelihood(m, Z + 2 * p, x + 4 * i) / (kappa + C_used[p]) * w_pred[i];
            for (int d = 0; d < 4; ++d) acc[d] += dw * x[4 * i + d];
        }
        for (int d = 0; d < 4; ++d) zeta[4 * r + d] = acc[d] / dW_out[p];
    }
    free(taken);
    return n;
}

/* Resampling step (Sec. 2.2, step 3; Algorithm 1 "Resample"): systematic
 * resampling with an exact, summation-order independent CDF.
 *   N_k = sum_i w_i
 *   e   = the exponent with max w < 2^e (frexp), c = the least c with N <= 2^c
 *   s   = 52 - c - e;  q_i = floor(w_i 2^s);  Q_i = q_0 + ... + q_i  (exact
 *         integers below 2^53, so the order of summation cannot matter)
 *   L   = min(l_max, round(rho * max(1, N_k)))  (paper: N_k(j) R_k particles)
 *   T_t = floor((t 2^32 + U) Q_N / (L 2^32)) for t = 0..L-1 (128-bit integers)
 *   parent(t) = the least j with Q_j > T_t;  new weights all N_k / L.
 * An empty or zero-mass set resamples to L = 0.  Returns L. */
int orc_resample(const double *x, const double *w, int N, double rho, int l_max, uint32_t U,
                 double *x_out, double *w_out, int *parent)
{
    if (N <= 0) return 0;
    double Nk = 0.0, wmax = 0.0;
    for (int i = 0; i < N; ++i) {
        Nk += w[i];
        if (w[i] > wmax) wmax = w[i];
    }
    if (!(wmax > 0.0)) return 0;
    int e;
    frexp(wmax, &e);
    int c = 0;
    while (((int64_t)1 << c) < (int64_t)N) ++c;
    int s = 52 - c - e;
    double *Q = (double *)malloc(sizeof(double) * (size_t)N);
    double run = 0.0;
    for (int i = 0; i < N; ++i) {
        run += floor(ldexp(w[i], s));
        Q[i] = run;
    }
    double lr = rho * (Nk > 1.0 ? Nk : 1.0);
    long L = lround(lr);
    if (L > l_max) L = l_max;
    if (L < 0) L = 0;
    unsigned __int128 QN = (unsigned __int128)(uint64_t)Q[N - 1];
    unsigned __int128 D = ((unsigned __int128)(uint64_t)L) << 32;
    int j = 0;
    for (long t = 0; t < L; ++t) {
        unsigned __int128 pos = ((((unsigned __int128)(uint64_t)t) << 32) + U) * QN;
        uint64_t T = (uint64_t)(pos / D);
        /* least j with Q_j > T; T_t is non-decreasing in t, so scan forward */
        while ((uint64_t)Q[j] <= T) ++j;
        parent[t] = j;
        for (int d = 0; d < 4; ++d) x_out[4 * t + d] = x[4 * j + d];
        w_out[t] = Nk / (double)L;
    }
    free(Q);
    return (int)L;
}

/* Slot choice of the ring exchange for one PE: the first `count` entries of a
 * Fisher-Yates shuffle of 0..n-1 driven by 32-bit uniforms u:
 *   r = t + floor(u_t (n - t) / 2^32),  swap(perm[t], perm[r]). */
void orc_exchange_slots(int n, int count, const uint32_t *u, int *slots)
{
    int *perm = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int t = 0; t < count; ++t) {
        int r = t + (int)(((uint64_t)u[t] * (uint64_t)(n - t)) >> 32);
        int tmp = perm[t];
        perm[t] = perm[r];
        perm[r] = tmp;
        slots[t] = perm[t];
    }
    free(perm);
}

/* Step 6 "Local exchange".  Each PE j picks L_x random slots s_j; its t-th
 * chosen particle-weight couple moves to PE d = j + shift_t (mod K) and lands
 * in the t-th slot s_d that PE d vacated.  The paper's ring has shift_t = 1
 * (PE j sends to PE j+1, PE K-1 to PE 0); the all-to-all pattern (mode 1, a
 * variant the paper leaves to future work) has shift_t = 1 + (t mod (K-1)),
 * so a PE's outgoing particles spread over all other PEs.  For each t the
 * shift is the same for every PE, so every PE sends and receives one
 * particle per t: with L_x = floor(frac * min_j n_j) slice sizes and the
 * union of all particles are unchanged.  Adaptive trigger (threshold > 0):
 * the exchange runs only when some PE has degenerated, i.e. its mass is
 * negligible next to the others': min_j N_j < threshold * (sum_j N_j) / K
 * (the PE masses N_j of this step's update).
 * x, w: K slices of stride `stride` particles; counts: n_j; u: [K][stride]. */
int orc_exchange_ex(int K, double *x, double *w, const int *counts, int stride, double frac, int mode,
                    double threshold, const double *mass, const uint32_t *u, int *slots_out)
{
    if (K <= 1) return 0;
    if (threshold > 0.0) {
        double sum = 0.0, mn = mass[0];
        for (int j = 0; j < K; ++j) {
            sum += mass[j];
            if (mass[j] < mn) mn = mass[j];
        }
        if (!(mn < threshold * (sum / (double)K))) return 0;
    }
    int nmin = counts[0];
    for (int j = 1; j < K; ++j) if (counts[j] < nmin) nmin = counts[j];
    int Lx = (int)floor(frac * (double)nmin);
    if (Lx <= 0) return 0;
    int *slots = (int *)malloc(sizeof(int) * (size_t)K * (size_t)Lx);
    for (int j = 0; j < K; ++j)
        orc_exchange_slots(counts[j], Lx, u + (size_t)j * stride, slots + (size_t)j * Lx);
    double *xs = (double *)malloc(sizeof(double) * 4 * (size_t)K * (size_t)Lx);
    double *ws = (double *)malloc(sizeof(double) * (size_t)K * (size_t)Lx);
    for (int j = 0; j < K; ++j)
        for (int t = 0; t < Lx; ++t) {
            size_t src = (size_t)j * stride + (size_t)slots[(size_t)j * Lx + t];
            for (int d = 0; d < 4; ++d) xs[4 * ((size_t)j * Lx + t) + d] = x[4 * src + d];
            ws[(size_t)j * Lx + t] = w[src];
        }
    for (int j = 0; j < K; ++j) {
        for (int t = 0; t < Lx; ++t) {
            int shift = (mode == 1 && K > 2) ? 1 + t % (K - 1) : 1;
            int k = (j + shift) % K;
            size_t dst = (size_t)k * stride + (size_t)slots[(size_t)k * Lx + t];
            for (int d = 0; d < 4; ++d) x[4 * dst + d] = xs[4 * ((size_t)j * Lx + t) + d];
            w[dst] = ws[(size_t)j * Lx + t];
        }
    }
    if (slots_out) memcpy(slots_out, slots, sizeof(int) * (size_t)K * (size_t)Lx);
    free(slots);
    free(xs);
    free(ws);
    return Lx;
}

/* The paper's ring exchange, every step. */
void orc_exchange(int K, double *x, double *w, const int *counts, int stride, double frac,
                  const uint32_t *u, int *slots_out)
{
    orc_exchange_ex(K, x, w, counts, stride, frac, 0, 0.0, NULL, u, slots_out);
}

/* Step 4 "Global Estimation" at the central unit: a label (measurement index)
 * is valid when more than half of the K PEs report it; its global state is
 * the mean of those PEs' local states.  Valid labels come out in ascending
 * order.  labels/zeta: per PE j, n[j] entries at stride `stride`. */
int orc_fuse(int K, const int *n, const int *labels, const double *zeta, int stride, int M,
             int *out_labels, double *out_zeta)
{
    int cnt = 0;
    for (int p = 0; p < M; ++p) {
        int votes = 0;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = 0; j < K; ++j)
            for (int r = 0; r < n[j]; ++r)
                if (labels[(size_t)j * stride + r] == p) {
                    ++votes;
                    for (int d = 0; d < 4; ++d) acc[d] += zeta[4 * ((size_t)j * stride + r) + d];
                }
        if (2 * votes > K) {
            out_labels[cnt] = p;
            for (int d = 0; d < 4; ++d) out_zeta[4 * cnt + d] = acc[d] / votes;
            ++cnt;
        }
    }
    return cnt;
}
