/*
 * FP64 CPU oracle of the measurement-driven birth proposal: the birth density
 * p_k(. | Z_k) of Eq. 6 taken as a mixture over the current measurements whose
 * per-measurement velocity Gaussian and mixture logit come from a small
 * network, the importance weights that keep the PHD unbiased under it, and
 * the network's loss, gradient and Adam step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it is built and used by the tests, by the package's smoke
 * check and by the benchmark's CPU-baseline leg.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Style: plain loops in IEEE double, no blocking or fusion.  Where the paper
 * is silent (it fixes only that births are drawn from a proposal conditioned
 * on Z_k and weighted by gamma / (J p_k), Eq. 6), the reading taken is stated
 * at the function.
 *
 * Network (reading): input u = (x', y', d) per measurement, where (x', y') is
 * the measurement's position in the plane scaled to the birth region
 * ((p - centre) / half-width per axis) and d = log1p(number of other
 * measurements inside the window |dz_0| <= 3 sigma_0, |wrap dz_1| <= 3
 * sigma_1); 3 -> 64 -> 64 -> 5 with exact-erf GELU after the two hidden
 * layers; outputs y = (m_x, m_y, l_x, l_y, logit).  Parameter vector (4741
 * doubles): W1[64][3], b1[64], W2[64][64], b2[64], W3[5][64], b3[5], W[j][k]
 * the weight from input k into unit j.
 *
 * Head (reading): velocity mean s_b (m_x, m_y), velocity std s_b exp(l) per
 * axis with l clamped to [log 0.05, log 5] in the proposal, mixture weight
 * pi = softmax(logit) over the measurements; s_b is the plain birth's
 * velocity std.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "orc_model.h"

#define NH 64
#define NIN 3
#define NOUT 5
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + NH * NIN)
#define OFF_W2 (OFF_B1 + NH)
#define OFF_B2 (OFF_W2 + NH * NH)
#define OFF_W3 (OFF_B2 + NH)
#define OFF_B3 (OFF_W3 + NOUT * NH)
#define NPARAMS (OFF_B3 + NOUT)

static const double BPI = 3.14159265358979323846;

int orc_mlp_nparams(void) { return NPARAMS; }

/* GELU(a) = a Phi(a), Phi the standard normal CDF (exact erf form). */
double orc_gelu(double a) { return 0.5 * a * (1.0 + erf(a / sqrt(2.0))); }

/* d GELU / da = Phi(a) + a phi(a). */
double orc_gelu_grad(double a)
{
    return 0.5 * (1.0 + erf(a / sqrt(2.0))) + a * exp(-0.5 * a * a) / sqrt(2.0 * BPI);
}

static double wrap_pi(double a)
{
    while (a > BPI) a -= 2.0 * BPI;
    while (a <= -BPI) a += 2.0 * BPI;
    return a;
}

/* Position of a measurement in the plane: z itself for the linear sensor,
 * sensor + r (cos theta, sin theta) for the range-bearing sensor. */
static void meas_position(const orc_model *m, const double *z, double *p)
{
    if (m->meas_model == ORC_LINEAR) {
        p[0] = z[0];
        p[1] = z[1];
    } else {
        p[0] = m->sensor[0] + z[0] * cos(z[1]);
        p[1] = m->sensor[1] + z[0] * sin(z[1]);
    }
}

/* Network input per measurement (see the header for the reading). */
void orc_birth_features(const orc_model *m, const double *Z, int M, double *X)
{
    const double cx = 0.5 * (m->region[0] + m->region[1]), hx = 0.5 * (m->region[1] - m->region[0]);
    const double cy = 0.5 * (m->region[2] + m->region[3]), hy = 0.5 * (m->region[3] - m->region[2]);
    for (int p = 0; p < M; ++p) {
        double pos[2];
        meas_position(m, Z + 2 * p, pos);
        int count = 0;
        for (int q = 0; q < M; ++q) {
            if (q == p) continue;
            double d0 = Z[2 * q] - Z[2 * p];
            double d1 = Z[2 * q + 1] - Z[2 * p + 1];
            if (m->meas_model == ORC_RANGE_BEARING) d1 = wrap_pi(d1);
            if (fabs(d0) <= 3.0 * m->sigma_z[0] && fabs(d1) <= 3.0 * m->sigma_z[1]) ++count;
        }
        X[3 * p + 0] = (pos[0] - cx) / hx;
        X[3 * p + 1] = (pos[1] - cy) / hy;
        X[3 * p + 2] = log1p((double)count);
    }
}

/* Forward pass of one input; keeps the pre-activations for the backward. */
static void forward_one(const double *P, const double *u, double *a1, double *a2, double *y)
{
    double h1[NH], h2[NH];
    for (int j = 0; j < NH; ++j) {
        double s = P[OFF_B1 + j];
        for (int k = 0; k < NIN; ++k) s += P[OFF_W1 + j * NIN + k] * u[k];
        a1[j] = s;
        h1[j] = orc_gelu(s);
    }
    for (int j = 0; j < NH; ++j) {
        double s = P[OFF_B2 + j];
        for (int k = 0; k < NH; ++k) s += P[OFF_W2 + j * NH + k] * h1[k];
        a2[j] = s;
        h2[j] = orc_gelu(s);
    }
    for (int o = 0; o < NOUT; ++o) {
        double s = P[OFF_B3 + o];
        for (int k = 0; k < NH; ++k) s += P[OFF_W3 + o * NH + k] * h2[k];
        y[o] = s;
    }
}

void orc_mlp_forward(const double *P, const double *X, int n, double *Y)
{
    double a1[NH], a2[NH];
    for (int s = 0; s < n; ++s) forward_one(P, X + NIN * s, a1, a2, Y + NOUT * s);
}

/* softplus(a) = log(1 + e^a), evaluated without overflow. */
static double softplus(double a) { return (a > 0.0 ? a : 0.0) + log1p(exp(-fabs(a))); }

/* Training loss (reading) for a sample with target T = (t, vx, vy): t = 1 if
 * the filter extracted an estimate for the measurement (its velocity vx, vy
 * in m/s), else 0.  With v~ = v / s_b:
 *   L = softplus(logit) - t logit
 *     + t sum_d [ l_d + 0.5 (v~_d - m_d)^2 exp(-2 l_d) ]
 * (Bernoulli cross-entropy of the mixture logit, and the Gaussian negative
 * log-likelihood of the extracted velocity up to a constant).  Returns the
 * mean loss over the n samples and its gradient (mean) in G[NPARAMS]. */
double orc_mlp_loss_grad(const double *P, const double *X, const double *T, int n, double vel_scale, double *G)
{
    for (int i = 0; i < NPARAMS; ++i) G[i] = 0.0;
    double total = 0.0;
    for (int s = 0; s < n; ++s) {
        const double *u = X + NIN * s;
        double a1[NH], a2[NH], y[NOUT];
        forward_one(P, u, a1, a2, y);
        const double t = T[3 * s];
        const double vt[2] = {T[3 * s + 1] / vel_scale, T[3 * s + 2] / vel_scale};
        double L = softplus(y[4]) - t * y[4];
        double dy[NOUT];
        dy[4] = 1.0 / (1.0 + exp(-y[4])) - t;
        for (int d = 0; d < 2; ++d) {
            const double r = vt[d] - y[d];
            const double e = exp(-2.0 * y[2 + d]);
            L += t * (y[2 + d] + 0.5 * r * r * e);
            dy[d] = -t * r * e;
            dy[2 + d] = t * (1.0 - r * r * e);
        }
        total += L;
        /* backward through the three layers */
        double h1[NH], h2[NH], d2[NH], d1[NH];
        for (int j = 0; j < NH; ++j) h1[j] = orc_gelu(a1[j]);
        for (int j = 0; j < NH; ++j) h2[j] = orc_gelu(a2[j]);
        for (int o = 0; o < NOUT; ++o) {
            G[OFF_B3 + o] += dy[o];
            for (int k = 0; k < NH; ++k) G[OFF_W3 + o * NH + k] += dy[o] * h2[k];
        }
        for (int k = 0; k < NH; ++k) {
            double g = 0.0;
            for (int o = 0; o < NOUT; ++o) g += P[OFF_W3 + o * NH + k] * dy[o];
            d2[k] = g * orc_gelu_grad(a2[k]);
        }
        for (int j = 0; j < NH; ++j) {
            G[OFF_B2 + j] += d2[j];
            for (int k = 0; k < NH; ++k) G[OFF_W2 + j * NH + k] += d2[j] * h1[k];
        }
        for (int k = 0; k < NH; ++k) {
            double g = 0.0;
            for (int j = 0; j < NH; ++j) g += P[OFF_W2 + j * NH + k] * d2[j];
            d1[k] = g * orc_gelu_grad(a1[k]);
        }
        for (int j = 0; j < NH; ++j) {
            G[OFF_B1 + j] += d1[j];
            for (int k = 0; k < NIN; ++k) G[OFF_W1 + j * NIN + k] += d1[j] * u[k];
        }
    }
    if (n > 0) {
        for (int i = 0; i < NPARAMS; ++i) G[i] /= (double)n;
        total /= (double)n;
    }
    return total;
}

/* Standard normal density. */
static double phi(double x) { return exp(-0.5 * x * x) / sqrt(2.0 * BPI); }

/* Per-component proposal parameters from the network head. */
typedef struct {
    double pi, mu[2], sd[2];
} comp_t;

static void components(const orc_model *m, const double *head, int M, comp_t *c)
{
    const double sb = m->birth_vel_sigma;
    double mx = -INFINITY;
    for (int p = 0; p < M; ++p) mx = head[5 * p + 4] > mx ? head[5 * p + 4] : mx;
    double s = 0.0;
    for (int p = 0; p < M; ++p) s += exp(head[5 * p + 4] - mx);
    for (int p = 0; p < M; ++p) {
        c[p].pi = exp(head[5 * p + 4] - mx) / s;
        for (int d = 0; d < 2; ++d) {
            double l = head[5 * p + 2 + d];
            if (l < log(0.05)) l = log(0.05);
            if (l > log(5.0)) l = log(5.0);
            c[p].mu[d] = sb * head[5 * p + d];
            c[p].sd[d] = sb * exp(l);
        }
    }
}

/* Density of a component's position draw at plane point pos.  Linear:
 * N(pos; z, diag sigma^2).  Range-bearing: the draw is r = |z_r + s_r n1|,
 * theta = z_theta + s_theta n2, pos = sensor + r (cos, sin); its density at
 * (r, theta) is the folded normal in r times the normal of the wrapped
 * bearing difference (principal term), and 1 / r converts (r, theta) to the
 * plane. */
static double pos_density(const orc_model *m, const double *z, const double *pos)
{
    if (m->meas_model == ORC_LINEAR) {
        return phi((pos[0] - z[0]) / m->sigma_z[0]) / m->sigma_z[0] *
               phi((pos[1] - z[1]) / m->sigma_z[1]) / m->sigma_z[1];
    }
    const double px = pos[0] - m->sensor[0], py = pos[1] - m->sensor[1];
    const double r = sqrt(px * px + py * py);
    const double th = atan2(py, px);
    const double fr = (phi((r - z[0]) / m->sigma_z[0]) + phi((r + z[0]) / m->sigma_z[0])) / m->sigma_z[0];
    const double ft = phi(wrap_pi(th - z[1]) / m->sigma_z[1]) / m->sigma_z[1];
    return fr * ft / r;
}

/* R(x) = sum_p pi_p q_p(x) / (U(pos) N(v; 0, s_b^2 I)) for a point inside the
 * region: the learned mixture's density over the plain birth density. */
static double mixture_ratio(const orc_model *m, const double *Z, int M, const comp_t *c, const double *x)
{
    const double area = (m->region[1] - m->region[0]) * (m->region[3] - m->region[2]);
    const double sb = m->birth_vel_sigma;
    const double pos[2] = {x[0], x[2]}, v[2] = {x[1], x[3]};
    const double plain = (1.0 / area) * phi(v[0] / sb) / sb * phi(v[1] / sb) / sb;
    double R = 0.0;
    for (int p = 0; p < M; ++p) {
        const double qv = phi((v[0] - c[p].mu[0]) / c[p].sd[0]) / c[p].sd[0] *
                          phi((v[1] - c[p].mu[1]) / c[p].sd[1]) / c[p].sd[1];
        R += c[p].pi * pos_density(m, Z + 2 * p, pos) * qv;
    }
    return R / plain;
}

/* Births of one PE from the defensive mixture proposal (reading of Eq. 6 with
 * a learned p_k(.|Z_k)):
 *   q(x | Z) = alpha p_plain(x) + (1 - alpha) sum_p pi_p q_p(x),
 * p_plain = U(region) x N(0, s_b^2 I) (the plain birth), q_p the position
 * draw around z_p (pos_density) times N(v; mu_p, diag sd_p^2).  Weight
 * (Eq. 6): gamma(x) / (J q(x | Z)) with gamma = nu_b p_plain, i.e.
 *   w = (nu_b / J) / (alpha + (1 - alpha) R(x))  inside the region, 0 outside.
 * alpha = 1, or M = 0, is the plain birth exactly.
 * Random numbers per birth b: noise[b] = (n1, n2, u1, u2) as for the plain
 * birth (velocity normals; uniform position in the plain branch) and
 * extra[b] = (u_c, nz1, nz2, unused): u_c < alpha takes the plain branch,
 * otherwise the component is the smallest p with CDF_p > (u_c - alpha) /
 * (1 - alpha) (CDF_p = pi_0 + ... + pi_p, summed in order; the last component
 * if rounding leaves none), and nz1, nz2 are its position normals.
 * Outputs x_out[J][4], w_out[J], comp[J] (-1 for the plain branch). */
void orc_birth_learned(const orc_model *m, const double *Z, int M, const double *head, double alpha, int J,
                       const double *noise, const double *extra, double *x_out, double *w_out, int *comp)
{
    comp_t *c = (comp_t *)malloc(sizeof(comp_t) * (M > 0 ? M : 1));
    double *cdf = (double *)malloc(sizeof(double) * (M > 0 ? M : 1));
    const double a = M > 0 ? alpha : 1.0;
    if (M > 0) {
        components(m, head, M, c);
        double s = 0.0;
        for (int p = 0; p < M; ++p) {
            s += c[p].pi;
            cdf[p] = s;
        }
    }
    const double sb = m->birth_vel_sigma;
    for (int b = 0; b < J; ++b) {
        const double *n = noise + 4 * b;
        const double *e = extra + 4 * b;
        double *x = x_out + 4 * b;
        int k = -1;
        if (e[0] >= a) {
            const double uu = (e[0] - a) / (1.0 - a);
            k = M - 1;
            for (int p = 0; p < M; ++p)
                if (cdf[p] > uu) {
                    k = p;
                    break;
                }
        }
        if (k < 0) {
            x[0] = m->region[0] + n[2] * (m->region[1] - m->region[0]);
            x[2] = m->region[2] + n[3] * (m->region[3] - m->region[2]);
            x[1] = sb * n[0];
            x[3] = sb * n[1];
        } else {
            const double *z = Z + 2 * k;
            if (m->meas_model == ORC_LINEAR) {
                x[0] = z[0] + m->sigma_z[0] * e[1];
                x[2] = z[1] + m->sigma_z[1] * e[2];
            } else {
                const double r = fabs(z[0] + m->sigma_z[0] * e[1]);
                const double th = z[1] + m->sigma_z[1] * e[2];
                x[0] = m->sensor[0] + r * cos(th);
                x[2] = m->sensor[1] + r * sin(th);
            }
            x[1] = c[k].mu[0] + c[k].sd[0] * n[0];
            x[3] = c[k].mu[1] + c[k].sd[1] * n[1];
        }
        comp[b] = k;
        const int inside = x[0] >= m->region[0] && x[0] <= m->region[1] && x[2] >= m->region[2] &&
                           x[2] <= m->region[3];
        if (!inside) {
            w_out[b] = 0.0;
        } else if (a >= 1.0) {
            w_out[b] = m->birth_mass / (double)J;
        } else {
            const double R = mixture_ratio(m, Z, M, c, x);
            w_out[b] = (m->birth_mass / (double)J) / (a + (1.0 - a) * R);
        }
    }
    free(c);
    free(cdf);
}

/* The proposal's CDF over the components (for the parity tests' check of
 * component choices that fall within rounding of a boundary). */
void orc_birth_cdf(const orc_model *m, const double *head, int M, double *cdf)
{
    comp_t *c = (comp_t *)malloc(sizeof(comp_t) * (M > 0 ? M : 1));
    if (M > 0) components(m, head, M, c);
    double s = 0.0;
    for (int p = 0; p < M; ++p) {
        s += c[p].pi;
        cdf[p] = s;
    }
    free(c);
}
