"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each check is a closed form, an
invariant, a textbook reduction (GM-PHD / Kalman), exact rational brute force
or a distributional property, chosen so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import math
from fractions import Fraction
from itertools import permutations

import numpy as np
import pytest

import oracle
import scenario

LIN = scenario.workload("linear4_fp64")
RB = scenario.workload("dense_rb_100t")


def _m(w, **kw):
    return oracle.model(w.with_(**kw))


# ----------------------------------------------------------------------------
# Sensor model (Sec. 4): geometry and normalisation
# ----------------------------------------------------------------------------

def test_range_bearing_geometry():
    m = _m(RB, sensor=(10.0, 20.0))
    cases = [((13.0, 24.0), (5.0, math.atan2(4.0, 3.0))),
             ((10.0, 120.0), (100.0, math.pi / 2)),
             ((-90.0, 20.0), (100.0, math.pi)),
             ((10.0, -80.0), (100.0, -math.pi / 2))]
    for (px, py), (r, th) in cases:
        h = oracle.measure(m, [px, 7.0, py, -3.0])[0]
        assert h[0] == pytest.approx(r, rel=1e-14)
        assert h[1] == pytest.approx(th, abs=1e-14)
    # the likelihood peaks at h(x) with the bivariate normal's peak height
    x = [13.0, 0.0, 24.0, 0.0]
    peak = 1.0 / (2 * math.pi * RB.sigma_z[0] * RB.sigma_z[1])
    assert oracle.likelihood(m, [5.0, math.atan2(4.0, 3.0)], x) == pytest.approx(peak, rel=1e-13)


def test_linear_likelihood_integrates_to_one():
    m = _m(LIN, p_d=1.0)
    x = np.array([[123.0, 4.0, -55.0, 2.0]])
    s = LIN.sigma_z[0]
    g = np.linspace(-9 * s, 9 * s, 241)
    dz = g[1] - g[0]
    Z = np.stack(np.meshgrid(123.0 + g, -55.0 + g, indexing="ij"), -1).reshape(-1, 2)
    C = oracle.colsum(m, x, [1.0], Z)
    assert C.sum() * dz * dz == pytest.approx(1.0, abs=1e-9)
    # the x and y axes are not swapped: a displaced peak moves the mass
    Cx = oracle.colsum(m, x, [1.0], Z + np.array([20.0, 0.0]))
    assert Cx.reshape(241, 241).sum(1).argmax() < 120


@pytest.mark.parametrize("theta0", [0.3, math.pi - 2e-3, -math.pi + 1e-3])
def test_range_bearing_likelihood_integrates_to_one_across_the_cut(theta0):
    """Integral over (r, theta) is 1, also for a particle on the +-pi branch cut:
    a missing bearing wrap loses about half of the mass there."""
    m = _m(RB, p_d=1.0)
    r0 = 700.0
    x = np.array([[r0 * math.cos(theta0), 1.0, r0 * math.sin(theta0), -1.0]])
    sr, st = RB.sigma_z
    rr = r0 + np.linspace(-9 * sr, 9 * sr, 181)
    tt = np.linspace(-math.pi, math.pi, 20001)[1:]
    Z = np.stack(np.meshgrid(rr, tt, indexing="ij"), -1).reshape(-1, 2)
    C = oracle.colsum(m, x, [1.0], Z)
    assert C.sum() * (rr[1] - rr[0]) * (tt[1] - tt[0]) == pytest.approx(1.0, abs=2e-6)


@pytest.mark.parametrize("k", [1.5, 3.0])
def test_truncated_likelihood_mass(k):
    """The k-sigma truncation variant: the integral of g(z|x) over z is the
    chi-square (2 dof) CDF at k^2, 1 - exp(-k^2 / 2) (midpoint rule on a
    fine grid around the particle, anisotropic noise); g is 0 just past the
    radius and the full Gaussian's value just inside it."""
    w = LIN.with_(sigma_z=(7.0, 13.0), gate_sigma=k)
    m = oracle.model(w)
    x = np.array([30.0, 0.0, -20.0, 0.0])
    h = 0.05
    gx = np.arange(-7.0 * k, 7.0 * k, h) + h / 2
    gy = np.arange(-13.0 * k, 13.0 * k, h * 13 / 7) + h * 13 / 14
    tot = 0.0
    for dy in gy[::1]:
        row = [oracle.likelihood(m, np.array([30.0 + dx, -20.0 + dy]), x) for dx in gx[::4]]
        tot += sum(row) * (4 * h) * (h * 13 / 7)
    assert tot == pytest.approx(1.0 - math.exp(-0.5 * k * k), rel=2e-3)
    full = oracle.model(LIN.with_(sigma_z=(7.0, 13.0)))
    inside = np.array([30.0 + 7.0 * k * 0.999, -20.0])
    outside = np.array([30.0 + 7.0 * k * 1.001, -20.0])
    assert oracle.likelihood(m, outside, x) == 0.0
    assert oracle.likelihood(m, inside, x) == oracle.likelihood(full, inside, x) > 0.0


def test_kappa_units():
    assert oracle.kappa(_m(LIN, clutter_rate=10.0)) == pytest.approx(10.0 / 4e6, rel=1e-15)
    assert oracle.kappa(_m(RB, clutter_rate=500.0, r_max=1000.0)) == pytest.approx(
        500.0 / (2 * math.pi * 1000.0), rel=1e-15)


# ----------------------------------------------------------------------------
# Prediction, Eq. 5-6 with the CV model of Sec. 4
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [1.0, 2.0])
def test_predict_moments_match_cv_model(dt):
    """Sample mean F x and covariance sigma_a^2 [[T^4/4, T^3/2], [T^3/2, T^2]] per axis."""
    m = _m(LIN, dt=dt)
    n = 200_000
    x0 = np.array([10.0, 2.0, -5.0, 1.0])
    rng = np.random.default_rng(7)
    noise = np.zeros((n, 4))
    noise[:, :2] = rng.standard_normal((n, 2))
    xo, wo = oracle.predict(m, np.tile(x0, (n, 1)), np.full(n, 1.0 / n), 0, noise)
    mean = xo.mean(0)
    F = np.array([[1, dt, 0, 0], [0, 1, 0, 0], [0, 0, 1, dt], [0, 0, 0, 1]], float)
    sa2 = LIN.sigma_a ** 2
    blk = sa2 * np.array([[dt ** 4 / 4, dt ** 3 / 2], [dt ** 3 / 2, dt ** 2]])
    cov_ref = np.zeros((4, 4))
    cov_ref[:2, :2] = blk
    cov_ref[2:, 2:] = blk
    se = np.sqrt(np.diag(cov_ref) / n)
    assert np.all(np.abs(mean - F @ x0) < 5 * se)
    cov = np.cov(xo.T)
    assert np.allclose(cov, cov_ref, rtol=0.02, atol=0.02 * sa2 * dt ** 2)
    assert wo.sum() == pytest.approx(LIN.p_s, rel=1e-12)


def test_birth_distribution_and_mass():
    m = _m(LIN)
    J = 200_000
    rng = np.random.default_rng(3)
    noise = np.concatenate([rng.standard_normal((J, 2)), rng.random((J, 2))], axis=1)
    xo, wo = oracle.predict(m, np.zeros((0, 4)), np.zeros(0), J, noise)
    x0, x1, y0, y1 = LIN.region
    assert xo[:, 0].min() >= x0 and xo[:, 0].max() < x1
    assert xo[:, 2].min() >= y0 and xo[:, 2].max() < y1
    assert xo[:, 0].mean() == pytest.approx((x0 + x1) / 2, abs=5 * (x1 - x0) / math.sqrt(12 * J))
    assert xo[:, 0].var() == pytest.approx((x1 - x0) ** 2 / 12, rel=0.02)
    assert xo[:, 3].std() == pytest.approx(LIN.birth_vel_sigma, rel=0.01)
    # Eq. 6 with gamma = nu_b p_k: the birth particles carry the birth mass
    assert wo.sum() == pytest.approx(LIN.birth_mass, rel=1e-12)
    assert np.all(wo == wo[0])


PAPER = scenario.workload("paper_bot")


def test_kappa_with_a_bearing_field_of_view():
    """kappa = lambda V_u (Sec. 4): the uniform clutter density over [0, r_max]
    x the bearing span, in closed form and against the scenario's clutter
    generator (independent code): the count in a sub-box of measurement space
    over many scans is kappa x the sub-box area per scan."""
    m = oracle.model(PAPER.with_(clutter_rate=20.0))
    assert oracle.kappa(m) == pytest.approx(20.0 / (200.0 * math.pi), rel=1e-15)
    w = PAPER.with_(clutter_rate=20.0, n_targets=0, steps=4000)
    sc = scenario.simulate(w, 3)
    Z = np.concatenate(sc.meas)
    assert np.all(np.abs(Z[:, 1]) <= math.pi / 2 + 1e-6) and np.all((Z[:, 0] >= 0) & (Z[:, 0] <= 200))
    box = (Z[:, 0] > 40) & (Z[:, 0] < 90) & (Z[:, 1] > -0.3) & (Z[:, 1] < 0.5)
    expect = oracle.kappa(m) * 50.0 * 0.8 * w.steps
    assert abs(box.sum() - expect) < 5 * math.sqrt(expect)


def test_gaussian_birth_box_muller_worked_values():
    """Gaussian birth (Sec. 4's N(x_bar, Q)): velocity from the normals, the
    position normals by the Box-Muller map of (u1, u2); u1 = 1 - e^{-1/2}
    gives radius 1, so the angle 2 pi u2 = 0 or pi/2 puts the draw one std
    along x or y; u1 = 0 gives the mean."""
    w = PAPER.with_(birth_mean=(1.0, 2.0, 3.0, 4.0), birth_std=(2.0, 0.5, 3.0, 0.25), birth_mass=0.3)
    m = oracle.model(w)
    u1 = 1.0 - math.exp(-0.5)
    noise = np.array([[0.5, -1.0, u1, 0.0],
                      [0.0, 2.0, u1, 0.25],
                      [1.0, 1.0, 0.0, 0.7]])
    xo, wo = oracle.predict(m, np.zeros((0, 4)), np.zeros(0), 3, noise)
    np.testing.assert_allclose(xo[0], [1.0 + 2.0, 2.0 + 0.25, 3.0, 4.0 - 0.25], atol=1e-12)
    np.testing.assert_allclose(xo[1], [1.0, 2.0, 3.0 + 3.0, 4.0 + 0.5], atol=1e-12)
    np.testing.assert_allclose(xo[2], [1.0, 2.5, 3.0, 4.25], atol=1e-12)
    np.testing.assert_allclose(wo, 0.1, rtol=1e-15)


def test_gaussian_birth_moments():
    """Draws with uniform (u1, u2) and normal (n1, n2) have the birth density's
    mean and std per component and uncorrelated components."""
    m = oracle.model(PAPER)
    J = 200_000
    rng = np.random.default_rng(11)
    noise = np.concatenate([rng.standard_normal((J, 2)), rng.random((J, 2))], axis=1)
    xo, wo = oracle.predict(m, np.zeros((0, 4)), np.zeros(0), J, noise)
    mean, std = np.asarray(PAPER.birth_mean), np.asarray(PAPER.birth_std)
    assert np.all(np.abs(xo.mean(0) - mean) < 5 * std / math.sqrt(J))
    np.testing.assert_allclose(xo.std(0), std, rtol=0.01)
    c = np.corrcoef(xo.T)
    assert np.all(np.abs(c - np.eye(4)) < 5 / math.sqrt(J))
    # a 4-D normal: the squared standardised radius is chi-square with 4 dof
    q = (((xo - mean) / std) ** 2).sum(1)
    assert q.mean() == pytest.approx(4.0, abs=5 * math.sqrt(8.0 / J))
    assert wo.sum() == pytest.approx(PAPER.birth_mass, rel=1e-12)


def test_predict_per_axis_process_noise():
    """Per-axis acceleration noise: each axis follows the CV covariance with
    its own sigma (T = 2 so a wrong power of T shows), no cross-axis terms."""
    dt, sx, sy = 2.0, 0.7, 3.0
    m = oracle.model(PAPER.with_(dt=dt, sigma_a=sx, sigma_a_y=sy))
    n = 200_000
    rng = np.random.default_rng(5)
    noise = np.zeros((n, 4))
    noise[:, :2] = rng.standard_normal((n, 2))
    xo, _ = oracle.predict(m, np.tile([0.0, 1.0, 0.0, -1.0], (n, 1)), np.full(n, 1.0), 0, noise)
    cov = np.cov(xo.T)
    for s, sl in ((sx, slice(0, 2)), (sy, slice(2, 4))):
        ref = s * s * np.array([[dt ** 4 / 4, dt ** 3 / 2], [dt ** 3 / 2, dt ** 2]])
        np.testing.assert_allclose(cov[sl, sl], ref, rtol=0.02)
    assert np.all(np.abs(cov[:2, 2:]) < 0.02 * sx * sy * dt ** 2)


# ----------------------------------------------------------------------------
# Update, Eq. 7-8
# ----------------------------------------------------------------------------

def _cloud(w, n, seed, M=7, spread=25.0):
    rng = np.random.default_rng(seed)
    centres = np.array([[100.0, -200.0], [400.0, 300.0], [-600.0, 50.0]])
    x, wt = scenario.random_particles(rng, w, n, centres=centres, spread=spread, mass=2.3)
    Z = centres[rng.integers(0, 3, M)] + 15.0 * rng.standard_normal((M, 2))
    return x, wt, Z


def _rb_meas(Zxy):
    return np.stack([np.hypot(Zxy[:, 0], Zxy[:, 1]), np.arctan2(Zxy[:, 1], Zxy[:, 0])], 1)


@pytest.mark.parametrize("wname", ["linear", "range_bearing"])
def test_update_mass_closed_form(wname):
    """sum_i w'_i = (1 - p_D) sum_i w_i + sum_p C_p / (kappa + C_p): Eq. 8 summed."""
    w = LIN if wname == "linear" else RB
    m = oracle.model(w)
    x, wt, Z = _cloud(w, 300, 11)
    if wname == "range_bearing":
        Z = _rb_meas(Z)
    C = oracle.colsum(m, x, wt, Z)
    wu = oracle.weight_update(m, x, wt, Z, C)
    k = oracle.kappa(m)
    ref = (1 - w.p_d) * wt.sum() + np.sum(C / (k + C))
    assert wu.sum() == pytest.approx(ref, rel=1e-12)
    assert C.min() > 0 and np.all(wu > 0)


def test_pd1_no_clutter_mass_counts_measurements():
    """p_D = 1 and kappa = 0: each measurement with C > 0 contributes exactly one
    target; a measurement with C = 0 contributes nothing."""
    m = _m(LIN, p_d=1.0, clutter_rate=0.0)
    x, wt, Z = _cloud(LIN, 200, 5, M=1)
    wu = oracle.weight_update(m, x, wt, Z, oracle.colsum(m, x, wt, Z))
    assert wu.sum() == pytest.approx(1.0, rel=1e-12)
    Z3 = np.concatenate([_cloud(LIN, 200, 5, M=3)[2], [[1e7, 1e7]]])
    C3 = oracle.colsum(m, x, wt, Z3)
    assert C3[3] == 0.0 and np.all(C3[:3] > 0)
    wu3 = oracle.weight_update(m, x, wt, Z3, C3)
    assert wu3.sum() == pytest.approx(3.0, rel=1e-12)


def test_no_measurements_leaves_missed_detection_term():
    m = oracle.model(LIN)
    x, wt, _ = _cloud(LIN, 50, 2)
    wu = oracle.weight_update(m, x, wt, np.zeros((0, 2)), np.zeros(0))
    assert np.array_equal(wu, (1 - LIN.p_d) * wt)


def _gauss(z, mu, S):
    d = z - mu
    return math.exp(-0.5 * d @ np.linalg.solve(S, d)) / (2 * math.pi * math.sqrt(np.linalg.det(S)))


def test_gmphd_reduction_linear_gaussian():
    """Gaussian predicted intensity m N(mu, P), linear sensor: the particle update
    converges to the GM-PHD closed form (Vo & Ma): C_z = p_D m N(z; H mu, HPH'+R),
    and the labelled state of a measurement (Eq. 18) is the Kalman posterior mean."""
    w = LIN
    m = oracle.model(w)
    mass = 1.5
    mu = np.array([100.0, 5.0, -200.0, -3.0])
    P = np.diag([400.0, 25.0, 400.0, 25.0])
    P[0, 1] = P[1, 0] = 60.0          # position-velocity correlation
    n = 400_000
    rng = np.random.default_rng(2024)
    x = rng.multivariate_normal(mu, P, size=n)
    wt = np.full(n, mass / n)
    Z = np.array([[110.0, -190.0], [150.0, -250.0], [800.0, 800.0]])
    H = np.array([[1.0, 0, 0, 0], [0, 0, 1.0, 0]])
    R = np.diag([w.sigma_z[0] ** 2, w.sigma_z[1] ** 2])
    S = H @ P @ H.T + R
    k = oracle.kappa(m)
    C = oracle.colsum(m, x, wt, Z)
    for p in range(2):
        g = np.array([oracle.likelihood(m, Z[p], xi) for xi in x[:20000]])
        se = w.p_d * mass * g.std() / math.sqrt(20000) * math.sqrt(20000 / n)
        C_ref = w.p_d * mass * _gauss(Z[p], H @ mu, S)
        assert abs(C[p] - C_ref) < 5 * se, (p, C[p], C_ref, se)
    assert C[2] < 1e-300
    wu = oracle.weight_update(m, x, wt, Z, C)
    Nk = wu.sum()
    ex = oracle.extract(m, x, wt, Z, C, Nk)
    np.testing.assert_allclose(ex.dW, C / (k + C), rtol=1e-12)
    assert ex.dW0 == pytest.approx((1 - w.p_d) * mass, rel=1e-12)
    assert Nk == pytest.approx(ex.dW.sum() + ex.dW0, rel=1e-12)
    # Kalman posterior mean for the first measurement
    Kg = P @ H.T @ np.linalg.inv(S)
    post = mu + Kg @ (Z[0] - H @ mu)
    Ppost = P - Kg @ H @ P
    i0 = list(ex.labels).index(0)
    g0 = np.array([oracle.likelihood(m, Z[0], xi) for xi in x])
    ess = g0.sum() ** 2 / (g0 ** 2).sum()
    tol = 5 * np.sqrt(np.diag(Ppost) / ess)
    assert np.all(np.abs(ex.zeta[i0] - post) < tol), (ex.zeta[i0], post, tol)


# ----------------------------------------------------------------------------
# Extraction (Step 3, Eq. 10-18)
# ----------------------------------------------------------------------------

def test_extract_single_particle_state_and_symmetric_pair():
    m = oracle.model(LIN)
    x1 = np.array([[321.0, 4.0, -12.0, -7.0]])
    Z = np.array([[330.0, -10.0]])
    C = oracle.colsum(m, x1, [0.8], Z)
    ex = oracle.extract(m, x1, [0.8], Z, C, 1.0)
    assert list(ex.labels) == [0]
    np.testing.assert_allclose(ex.zeta[0], x1[0], rtol=1e-14)
    # two equal-weight particles mirrored about the measurement: midpoint position
    z = np.array([50.0, 60.0])
    x2 = np.array([[50.0 + 7.0, 3.0, 60.0 - 4.0, 1.0], [50.0 - 7.0, -5.0, 60.0 + 4.0, 9.0]])
    C2 = oracle.colsum(m, x2, [0.5, 0.5], z[None])
    ex2 = oracle.extract(m, x2, [0.5, 0.5], z[None], C2, 1.0)
    np.testing.assert_allclose(ex2.zeta[0], [50.0, -1.0, 60.0, 5.0], rtol=1e-13)


def test_extract_selection_rules():
    """LT = round(N_k) half away from zero; largest dW first; ties to the lower
    label; labels with dW = 0 are never taken; LT is capped at M."""
    m = oracle.model(LIN)
    # one particle per measurement, identical geometry -> exactly tied dW
    xs = np.array([[0.0, 0, 0.0, 0], [500.0, 0, 0.0, 0], [0.0, 0, 500.0, 0], [-500.0, 0, -500.0, 0]])
    wt = np.array([0.3, 0.9, 0.9, 0.5])
    Z = xs[:, [0, 2]].copy()
    Z = np.concatenate([Z, [[1e7, -1e7]]])      # label 4: far away, dW = 0
    C = oracle.colsum(m, xs, wt, Z)
    for Nk, want in [(2.5, [1, 2, 3]), (2.49, [1, 2]), (0.49, []), (1.5, [1, 2]),
                     (9.0, [1, 2, 3, 0])]:
        ex = oracle.extract(m, xs, wt, Z, C, Nk)
        assert list(ex.labels) == want, (Nk, ex.labels, ex.dW)
    assert ex.dW[1] == ex.dW[2] and ex.dW[4] == 0.0


# ----------------------------------------------------------------------------
# Systematic resampling with the exact integer CDF
# ----------------------------------------------------------------------------

def _exact_parents(w_dyadic, L, U):
    """Systematic resampling in exact rational arithmetic: pointer t sits at
    (t + U / 2^32) / L of the total weight; its parent is the first particle
    whose cumulative weight exceeds it."""
    W = sum(w_dyadic)
    cum, run = [], Fraction(0)
    for wi in w_dyadic:
        run += wi
        cum.append(run)
    out = []
    for t in range(L):
        ptr = (t + Fraction(U, 2 ** 32)) / L * W
        out.append(next(j for j, c in enumerate(cum) if c > ptr))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_resample_matches_exact_rational_brute_force(seed):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(1, 6))
    k = rng.integers(0, 40, N)
    k[rng.integers(0, N)] += 1                  # at least one positive weight
    scale = 2.0 ** int(rng.integers(-30, 10))
    w = k * scale / 64.0
    rho = float(rng.integers(1, 4))
    Us = [0, 1, 2 ** 31, 2 ** 32 - 1] + [int(u) for u in rng.integers(0, 2 ** 32, 40)]
    for U in Us:
        xo, wo, par = oracle.resample(np.arange(4 * N, dtype=float).reshape(N, 4), w, rho, 1000, U)
        Nk = w.sum()
        L = int(math.floor(rho * max(1.0, Nk) + 0.5))
        assert len(par) == L
        assert list(par) == _exact_parents([Fraction(int(a)) for a in k], L, U)
        assert np.all(wo == Nk / L)
        np.testing.assert_array_equal(xo, np.arange(4 * N, dtype=float).reshape(N, 4)[par])


def test_resample_offspring_counts_and_mean():
    """Offspring of parent j is floor or ceil of L w_j / W, and over a uniform
    grid of U the mean offspring count is L w_j / W (unbiasedness)."""
    rng = np.random.default_rng(99)
    k = rng.integers(1, 200, 37)
    w = k / 1024.0
    W = w.sum()
    rho = 40.0
    L = int(math.floor(rho * W + 0.5))
    R = 2048
    acc = np.zeros(len(w))
    x = np.zeros((len(w), 4))
    for r in range(R):
        U = int((r + 0.5) * 2 ** 32 / R)
        _, wo, par = oracle.resample(x, w, rho, 10 ** 6, U)
        cnt = np.bincount(par, minlength=len(w))
        exp = L * w / W
        assert np.all((cnt == np.floor(exp)) | (cnt == np.ceil(exp)))
        assert wo.sum() == pytest.approx(W, rel=1e-13)
        acc += cnt
    np.testing.assert_allclose(acc / R, L * w / W, atol=2.0 / R)


def test_resample_scale_invariance_and_degenerate_cases():
    rng = np.random.default_rng(5)
    w = rng.random(1000) ** 3
    x = rng.standard_normal((1000, 4))
    _, _, p1 = oracle.resample(x, w, 3.0, 10 ** 6, 123456789)
    _, _, p2 = oracle.resample(x, w * 2.0 ** -40, 3.0, 10 ** 6, 123456789)
    _, _, p3 = oracle.resample(x, w * 2.0 ** 40, 3.0, 10 ** 6, 123456789)
    assert len(p1) == round(3.0 * w.sum())
    assert len(p2) == 3                         # mass < 1: rho * max(1, N) particles
    assert len(p3) == 10 ** 6                   # capped at l_max
    # exact scaling by a power of two leaves the integer CDF unchanged
    _, _, q1 = oracle.resample(x, w, 1e-3 / w.sum() * 4000.0, 10 ** 6, 42)
    _, _, q2 = oracle.resample(x, w * 2.0 ** 7, 1e-3 / (w.sum() * 2.0 ** 7) * 4000.0, 10 ** 6, 42)
    assert np.array_equal(q1, q2)
    assert oracle.resample(np.zeros((0, 4)), np.zeros(0), 5.0, 100, 0)[2].size == 0
    assert oracle.resample(x[:3], np.zeros(3), 5.0, 100, 0)[2].size == 0


# ----------------------------------------------------------------------------
# Distributed form: ring exchange (Step 6), CU fusion (Step 4), "global" C
# ----------------------------------------------------------------------------

def test_exchange_is_a_ring_move():
    rng = np.random.default_rng(8)
    K, stride = 5, 64
    counts = [40, 37, 52, 45, 39]
    xs = [rng.standard_normal((n, 4)) for n in counts]
    ws = [rng.random(n) for n in counts]
    u = rng.integers(0, 2 ** 32, size=(K, stride), dtype=np.uint64).astype(np.uint32)
    nx, nw, slots = oracle.exchange(xs, ws, 0.1, u)
    Lx = int(math.floor(0.1 * min(counts)))
    assert slots.shape == (K, Lx) and Lx == 3
    assert [len(a) for a in nx] == counts
    for j in range(K):
        assert len(set(slots[j])) == Lx and slots[j].max() < counts[j]
        k = (j + 1) % K
        np.testing.assert_array_equal(nx[k][slots[k]], xs[j][slots[j]])
        np.testing.assert_array_equal(nw[k][slots[k]], ws[j][slots[j]])
        keep = np.setdiff1d(np.arange(counts[j]), slots[j])
        np.testing.assert_array_equal(nx[j][keep], xs[j][keep])
    before = np.sort(np.concatenate([np.c_[a, b] for a, b in zip(xs, ws)]).view("u8"), axis=0)
    after = np.sort(np.concatenate([np.c_[a, b] for a, b in zip(nx, nw)]).view("u8"), axis=0)
    np.testing.assert_array_equal(before, after)
    assert sum(a.sum() for a in nw) == pytest.approx(sum(a.sum() for a in ws), rel=1e-15)


def _tagged_slices(rng, counts, stride):
    """Slices whose particles carry their PE and slot in the state (x = PE,
    vx = slot) so a move's source can be read off the destination."""
    xs, ws = [], []
    for j, n in enumerate(counts):
        x = rng.standard_normal((n, 4))
        x[:, 0], x[:, 1] = j, np.arange(n)
        xs.append(x)
        ws.append(rng.random(n))
    u = rng.integers(0, 2 ** 32, size=(len(counts), stride), dtype=np.uint64).astype(np.uint32)
    return xs, ws, u


def test_all_to_all_exchange_reaches_every_pe():
    """The all-to-all variant: PE j's t-th chosen particle lands in the t-th
    vacated slot of PE j + 1 + (t mod (K-1)); every PE then holds particles of
    all K-1 others, keeps its count, and the union and the mass are unchanged."""
    rng = np.random.default_rng(21)
    K, stride = 5, 128
    counts = [90, 84, 101, 95, 88]
    xs, ws, u = _tagged_slices(rng, counts, stride)
    nx, nw, slots = oracle.exchange(xs, ws, 0.1, u, "all")
    Lx = int(math.floor(0.1 * min(counts)))
    assert slots.shape == (K, Lx) and Lx == 8
    assert [len(a) for a in nx] == counts
    for d in range(K):
        got = nx[d][slots[d]]
        for t in range(Lx):
            src = (d - 1 - t % (K - 1)) % K
            assert got[t, 0] == src and got[t, 1] == slots[src][t]
            assert nw[d][slots[d][t]] == ws[src][slots[src][t]]
        assert set(got[:, 0].astype(int)) == set(range(K)) - {d}
        keep = np.setdiff1d(np.arange(counts[d]), slots[d])
        np.testing.assert_array_equal(nx[d][keep], xs[d][keep])
    before = np.sort(np.concatenate([np.c_[a, b] for a, b in zip(xs, ws)]).view("u8"), axis=0)
    after = np.sort(np.concatenate([np.c_[a, b] for a, b in zip(nx, nw)]).view("u8"), axis=0)
    np.testing.assert_array_equal(before, after)
    # with two PEs all-to-all is the ring
    a = oracle.exchange(xs[:2], ws[:2], 0.1, u[:2], "all")
    b = oracle.exchange(xs[:2], ws[:2], 0.1, u[:2], "ring")
    for p, q in zip(a[0] + a[1], b[0] + b[1]):
        np.testing.assert_array_equal(p, q)


@pytest.mark.parametrize("mode", ["ring", "all"])
def test_adaptive_exchange_trigger(mode):
    """Adaptive trigger (threshold > 0): nothing moves while every PE's mass
    is at least threshold x the mean; once one PE's mass drops below it the
    exchange is exactly the unconditional one."""
    rng = np.random.default_rng(4)
    K, stride = 4, 64
    counts = [40, 44, 41, 50]
    xs, ws, u = _tagged_slices(rng, counts, stride)
    even = np.array([2.0, 2.1, 1.9, 2.0])
    nx, nw, slots = oracle.exchange(xs, ws, 0.1, u, mode, 0.5, even)
    assert slots.shape == (K, 0)
    for a, b in zip(nx + nw, xs + ws):
        np.testing.assert_array_equal(a, b)
    # mean 1.525, threshold 0.5: 0.76 > 0.1, the exchange runs
    starved = np.array([2.0, 2.1, 0.1, 1.9])
    got = oracle.exchange(xs, ws, 0.1, u, mode, 0.5, starved)
    ref = oracle.exchange(xs, ws, 0.1, u, mode)
    assert got[2].shape == (K, 4)
    for a, b in zip(got[0] + got[1], ref[0] + ref[1]):
        np.testing.assert_array_equal(a, b)
    # the boundary is strict: min == threshold x mean does not trigger
    edge = np.array([1.0, 3.0, 3.0, 1.0])          # mean 2, threshold 0.5 -> 1.0
    assert oracle.exchange(xs, ws, 0.1, u, mode, 0.5, edge)[2].shape == (K, 0)


def test_exchange_slots_are_uniform():
    rng = np.random.default_rng(1)
    n, cnt, R = 10, 3, 20000
    hits = np.zeros(n)
    for _ in range(R):
        s = oracle.exchange_slots(n, cnt, rng.integers(0, 2 ** 32, cnt, dtype=np.uint64).astype(np.uint32))
        assert len(set(s)) == cnt
        hits[s] += 1
    p = cnt / n
    assert np.all(np.abs(hits / R - p) < 5 * math.sqrt(p * (1 - p) / R))


def test_fusion_majority_rule():
    ex = []
    for labs, shift in [([1, 2], 0.0), ([2, 1, 3], 1.0), ([1, 2], 2.0), ([3], 3.0)]:
        z = np.array([[10.0 * l + shift, 1, 2, 3] for l in labs])
        ex.append(oracle.Extraction(np.array(labs, np.int32), z, np.zeros(5), 0.0, len(labs)))
    lab, zet = oracle.fuse(ex, 5)
    assert list(lab) == [1, 2]                  # 3 of 4 > 4/2; label 3 has 2 of 4
    np.testing.assert_allclose(zet[0], [10.0 + 1.0, 1, 2, 3])
    np.testing.assert_allclose(zet[1], [20.0 + 1.0, 1, 2, 3])
    lab5, _ = oracle.fuse(ex[:3] + ex[:2], 5)   # K = 5: needs 3 votes
    assert list(lab5) == [1, 2]


def test_global_ck_mode_reproduces_the_global_update():
    """Slices of a global set with PE weights K x the global ones: the mean of the
    local C^j is the global C, so each PE's update is K x the global update."""
    m = oracle.model(LIN)
    x, wt, Z = _cloud(LIN, 600, 21)
    K = 3
    Cg = oracle.colsum(m, x, wt, Z)
    wg = oracle.weight_update(m, x, wt, Z, Cg)
    sl = np.array_split(np.arange(600), K)
    Cj = [oracle.colsum(m, x[s], K * wt[s], Z) for s in sl]
    Cm = np.mean(Cj, axis=0)
    np.testing.assert_allclose(Cm, Cg, rtol=1e-12)
    for s in sl:
        np.testing.assert_allclose(oracle.weight_update(m, x[s], K * wt[s], Z, Cm), K * wg[s],
                                   rtol=1e-12)


def test_distributed_filter_conserves_particles_and_k1_is_global():
    w = scenario.workload("dist16_10t", num_pe=4, birth_count=400, particles_per_target=200,
                          steps=3, n_targets=3, clutter_rate=5.0)
    sc = scenario.simulate(w, 1)
    f = oracle.OracleFilter(w)
    for k, Z in enumerate(sc.meas):
        f.step(Z, scenario.step_noise(1, k, w.num_pe, w.pe_cap), scenario.resample_u32(1, k, 4),
               scenario.exchange_u32(1, k, 4, w.pe_cap))
        L = [round(f.rho_pe * max(1.0, n)) for n in f.last["Nk"]]
        assert [len(a) for a in f.x] == L
    # K = 1: Algorithm 1 degenerates to the global particle PHD filter
    w1 = scenario.workload("dist16_10t", num_pe=1, exchange_frac=0.0, birth_count=400,
                           particles_per_target=200, steps=3, n_targets=3, clutter_rate=5.0)
    f1 = oracle.OracleFilter(w1)
    f1.step(sc.meas[0], scenario.step_noise(1, 0, 1, w1.pe_cap), [7])
    assert len(f1.x) == 1 and len(f1.x[0]) == round(200 * max(1.0, f1.last["Nk"][0]))


# ----------------------------------------------------------------------------
# OSPA (Sec. 4.1)
# ----------------------------------------------------------------------------

def _ospa_brute(X, Y, c, p):
    m, n = len(X), len(Y)
    if m > n:
        X, Y, m, n = Y, X, n, m
    if n == 0:
        return 0.0
    best = min(sum(min(c, np.linalg.norm(X[i] - Y[pi[i]])) ** p for i in range(m))
               for pi in permutations(range(n), m))
    return ((best + c ** p * (n - m)) / n) ** (1 / p)


def test_ospa():
    rng = np.random.default_rng(4)
    for _ in range(30):
        X = rng.uniform(-150, 150, (rng.integers(0, 6), 2))
        Y = rng.uniform(-150, 150, (rng.integers(0, 6), 2))
        for p in (1.0, 2.0):
            assert oracle.ospa(X, Y, 100.0, p) == pytest.approx(_ospa_brute(X, Y, 100.0, p), rel=1e-12)
    X = rng.uniform(size=(4, 2))
    assert oracle.ospa(X, X) == 0.0
    assert oracle.ospa(np.zeros((0, 2)), X) == 100.0
    assert oracle.ospa([[0.0, 0.0]], [[3.0, 4.0]]) == pytest.approx(5.0)
    assert oracle.ospa([[0.0, 0.0]], [[0.0, 0.0], [1000.0, 0.0]], 100.0, 2.0) == pytest.approx(
        math.sqrt(100.0 ** 2 / 2))


def test_openmp_build_is_bit_identical():
    """The OpenMP build of the oracle (used to time it on all host cores)
    splits only loops whose iterations write their own outputs, so every
    stage's result equals the single-threaded build's bit for bit."""
    if not oracle.openmp_available():
        pytest.skip("no OpenMP in this compiler")
    for w in (RB, LIN):
        m = oracle.model(w)
        x, wt, Z = _cloud(w, 3000, 8, M=40)
        if w is RB:
            Z = _rb_meas(Z)
        noise = scenario.step_noise(8, 0, 1, 3000 + 500)
        out = {}
        try:
            for th in (1, 4):
                oracle.set_threads(th)
                C = oracle.colsum(m, x, wt, Z)
                wu = oracle.weight_update(m, x, wt, Z, C)
                ex = oracle.extract(m, x, wt, Z, C, wu.sum())
                xp, wp = oracle.predict(m, x, wt, 500, noise)
                out[th] = (C, wu, ex.labels, ex.zeta, ex.dW, xp, wp)
        finally:
            oracle.set_threads(1)
        for a, b in zip(out[1], out[4]):
            assert np.array_equal(a, b)
        assert len(out[1][2]) > 0
