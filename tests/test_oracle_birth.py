"""Pins of the FP64 oracle of the measurement-driven birth proposal (Eq. 6
with a learned p_k(.|Z_k)) and of its network, against values and identities
fixed outside the oracle: normal-table values of GELU, a hand-wired network,
the loss and its gradient in closed form for a bias-only network, central
finite differences, Adam's first step, hand-counted features, the plain birth
as the alpha = 1 special case, and Monte-Carlo moments that hold only if the
sampler and the proposal density agree (E_q[gamma / q] = integral of gamma).
"""
import math

import numpy as np
import pytest

import oracle
import scenario

# standard normal CDF, from printed tables (Abramowitz & Stegun 26.2)
PHI_TABLE = {0.5: 0.6914624612740131, 1.0: 0.8413447460685429, 2.0: 0.9772498680518208,
             -1.0: 0.15865525393145707}


def test_gelu_is_x_times_normal_cdf():
    for x, phi in PHI_TABLE.items():
        assert oracle.gelu(x) == pytest.approx(x * phi, rel=1e-15, abs=1e-16)
    assert oracle.gelu(0.0) == 0.0
    assert oracle.gelu(12.0) == pytest.approx(12.0, rel=1e-15)
    assert abs(oracle.gelu(-12.0)) < 1e-30
    assert oracle.gelu_grad(0.0) == 0.5
    for x in (-2.0, -0.3, 0.7, 1.9):
        h = 1e-6
        fd = (oracle.gelu(x + h) - oracle.gelu(x - h)) / (2 * h)
        assert oracle.gelu_grad(x) == pytest.approx(fd, abs=1e-9)


def _zero_params():
    return np.zeros(oracle.mlp_nparams())


def _offsets():
    o = {"W1": 0}
    o["b1"] = o["W1"] + 64 * 3
    o["W2"] = o["b1"] + 64
    o["b2"] = o["W2"] + 64 * 64
    o["W3"] = o["b2"] + 64
    o["b3"] = o["W3"] + 5 * 64
    assert o["b3"] + 5 == oracle.mlp_nparams() == 4741
    return o


def test_hand_wired_network():
    """Unit j of layer 1 copies input j; unit 0 of layer 2 copies unit 0 of
    layer 1; output o reads unit 0 of layer 2 with weight o + 1."""
    o = _offsets()
    P = _zero_params()
    for j in range(3):
        P[o["W1"] + j * 3 + j] = 1.0
    P[o["W2"] + 0] = 1.0
    b3 = np.array([0.5, -0.5, 0.1, 0.2, 0.3])
    for k in range(5):
        P[o["W3"] + k * 64 + 0] = k + 1.0
    P[o["b3"]:o["b3"] + 5] = b3
    u = np.array([[1.0, 2.0, 0.5]])
    g1 = 1.0 * PHI_TABLE[1.0]                                  # GELU(1)
    g2 = g1 * 0.5 * (1.0 + math.erf(g1 / math.sqrt(2.0)))      # GELU(GELU(1))
    want = (np.arange(5) + 1.0) * g2 + b3
    np.testing.assert_allclose(oracle.mlp_forward(P, u)[0], want, rtol=1e-15)


def test_loss_and_gradient_closed_form_bias_only():
    """All weights zero: y = b3 for every sample, so the loss and its gradient
    are written out by hand."""
    o = _offsets()
    P = _zero_params()
    P[o["b3"]:o["b3"] + 5] = [0.5, -0.25, 0.0, math.log(2.0), 0.0]
    X = np.array([[0.1, 0.2, 0.3], [-0.4, 0.5, 0.0]])
    T = np.array([[1.0, 20.0, -10.0], [0.0, 0.0, 0.0]])      # s_b = 20: v~ = (1, -0.5)
    loss, G = oracle.mlp_loss_grad(P, X, T, 20.0)
    ln2 = math.log(2.0)
    L1 = ln2 + (0.0 + 0.5 * 0.25 * 1.0) + (ln2 + 0.5 * 0.0625 * 0.25)
    L2 = ln2
    assert loss == pytest.approx((L1 + L2) / 2, rel=1e-15)
    gb3 = G[o["b3"]:o["b3"] + 5]
    np.testing.assert_allclose(gb3, [-0.25, 0.03125, 0.375, 0.4921875, 0.0], rtol=1e-14, atol=1e-16)
    # hidden activations are GELU(0) = 0 and W3 = 0: nothing else moves
    mask = np.ones(len(G), bool)
    mask[o["b3"]:o["b3"] + 5] = False
    assert np.all(G[mask] == 0.0)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    P = scenario.mlp_params(11, scale=4.0)
    X = rng.standard_normal((7, 3)) * [0.6, 0.6, 1.0]
    T = np.stack([rng.integers(0, 2, 7).astype(float), 25 * rng.standard_normal(7),
                  25 * rng.standard_normal(7)], 1)
    loss, G = oracle.mlp_loss_grad(P, X, T, 20.0)
    o = _offsets()
    idx = np.concatenate([rng.choice(len(P), 150, replace=False), np.arange(o["b3"], o["b3"] + 5),
                          np.arange(o["W1"], o["W1"] + 6)])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (oracle.mlp_loss_grad(Pp, X, T, 20.0)[0] - oracle.mlp_loss_grad(Pm, X, T, 20.0)[0]) / (2 * h)
        assert G[i] == pytest.approx(fd, abs=2e-8 + 1e-6 * abs(fd)), i


def test_adam_first_step_moves_each_parameter_by_lr():
    """After one step m^ = g and v^ = g^2, so the update is lr g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    z = np.zeros(50)
    p1, m1, m2 = oracle.adam(p, g, z, z, 1, lr=1e-3, eps=1e-8)
    np.testing.assert_allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(m2, 0.001 * g * g, rtol=1e-14)


def test_features_hand_counted():
    w = scenario.workload("linear4_fp64")                     # sigma 10 m: window +-30 m
    m = oracle.model(w)
    Z = np.array([[0.0, 0.0], [20.0, 0.0], [0.0, 31.0], [500.0, 500.0], [-1000.0, 1000.0]])
    X = oracle.birth_features(m, Z)
    np.testing.assert_allclose(X[:, 2], np.log1p([1, 1, 0, 0, 0]), rtol=1e-15)
    np.testing.assert_allclose(X[:, :2], [[0, 0], [0.02, 0], [0, 0.031], [0.5, 0.5], [-1, 1]], atol=1e-15)
    wr = scenario.workload("dense_rb_100t")                   # sigma_r 5 m, sigma_theta 0.5 deg
    mr = oracle.model(wr)
    Zr = np.array([[800.0, math.pi - 0.005], [805.0, -math.pi + 0.004], [800.0, 0.0], [816.0, 0.0]])
    Xr = oracle.birth_features(mr, Zr)
    np.testing.assert_allclose(Xr[:, 2], np.log1p([1, 1, 0, 0]), rtol=1e-15)   # wrap across +-pi; 16 m > 15 m
    np.testing.assert_allclose(Xr[0, :2], [0.8 * math.cos(math.pi - 0.005), 0.8 * math.sin(math.pi - 0.005)],
                               rtol=1e-14)


@pytest.mark.parametrize("model_name", ["linear4_fp64", "dense_rb_100t"])
def test_alpha_one_is_the_plain_birth(model_name):
    w = scenario.workload(model_name)
    m = oracle.model(w)
    rng = np.random.default_rng(5)
    J = 300
    noise = scenario.step_noise(5, 0, 1, J)
    extra = scenario.birth_extra_noise(5, 0, 1, J)
    Z = rng.uniform(-500, 500, (4, 2)) if model_name.startswith("linear") else \
        np.stack([rng.uniform(100, 900, 4), rng.uniform(-3, 3, 4)], 1)
    head = rng.standard_normal((4, 5))
    x, wt, comp = oracle.birth_learned(m, Z, head, 1.0, J, noise, extra)
    xp, wp = oracle.predict(m, np.zeros((0, 4)), np.zeros(0), J, noise)
    np.testing.assert_array_equal(x, xp)
    np.testing.assert_array_equal(wt, wp)
    assert np.all(comp == -1)
    # no measurements: the plain birth whatever alpha
    x0, w0, c0 = oracle.birth_learned(m, np.zeros((0, 2)), np.zeros((0, 5)), 0.2, J, noise, extra)
    np.testing.assert_array_equal(x0, xp)
    np.testing.assert_array_equal(w0, wp)


def test_component_choice_follows_the_cdf():
    w = scenario.workload("linear4_fp64")
    m = oracle.model(w)
    head = np.zeros((4, 5))
    head[:, 4] = np.log([1.0, 2.0, 3.0, 4.0])               # pi = 0.1, 0.2, 0.3, 0.4
    cdf = oracle.birth_cdf(m, head)
    np.testing.assert_allclose(cdf, [0.1, 0.3, 0.6, 1.0], rtol=1e-15)
    alpha = 0.5
    uc = np.array([0.25, 0.5 + 0.5 * 0.05, 0.5 + 0.5 * 0.15, 0.5 + 0.5 * 0.45, 0.5 + 0.5 * 0.99])
    extra = np.zeros((5, 4))
    extra[:, 0] = uc
    noise = np.tile([0.0, 0.0, 0.5, 0.5], (5, 1))
    Z = np.array([[-300.0, 0.0], [0.0, 300.0], [300.0, 0.0], [0.0, -300.0]])
    x, wt, comp = oracle.birth_learned(m, Z, head, alpha, 5, noise, extra)
    assert list(comp) == [-1, 0, 1, 2, 3]
    np.testing.assert_allclose(x[1:, [0, 2]], Z, atol=1e-12)   # zero position normals: at z_c
    # adding a constant to every logit changes nothing
    h2 = head.copy()
    h2[:, 4] += 7.25
    x2, w2, c2 = oracle.birth_learned(m, Z, h2, alpha, 5, noise, extra)
    assert list(c2) == list(comp)
    np.testing.assert_allclose(w2, wt, rtol=1e-13)


def _mc_draw(model_name, alpha, Z, head, J, seed):
    w = scenario.workload(model_name)
    m = oracle.model(w)
    rng = np.random.default_rng(seed)
    noise = np.empty((J, 4))
    noise[:, :2] = rng.standard_normal((J, 2))
    noise[:, 2:] = rng.random((J, 2))
    extra = np.zeros((J, 4))
    extra[:, 0] = rng.random(J)
    extra[:, 1:3] = rng.standard_normal((J, 2))
    x, wt, comp = oracle.birth_learned(m, Z, head, alpha, J, noise, extra)
    return w, x, wt, comp


@pytest.mark.parametrize("model_name,alpha", [("linear4_fp64", 0.3), ("linear4_fp64", 0.01),
                                              ("dense_rb_100t", 0.3), ("dense_rb_100t", 0.01)])
def test_importance_weights_are_unbiased(model_name, alpha):
    """E[sum_b w_b f(x_b)] = integral of gamma f, for f = 1, vx, vx^2 over the
    whole region and for f = 1 and vx^2 restricted to a window around each
    measurement (where the mixture, not the defensive uniform part, carries
    the draws).  Holds only if the sampler and the proposal density agree:
    position Gaussian, or the folded polar draw with its 1/r Jacobian;
    velocity Gaussian; mixture and defensive weights.  Five Monte-Carlo
    standard errors."""
    rng = np.random.default_rng(17)
    if model_name.startswith("linear"):
        Z = np.array([[-400.0, 120.0], [10.0, -700.0], [650.0, 640.0], [-900.0, -880.0]])
    else:   # one measurement at 8 m range exercises the folded range draw
        Z = np.array([[8.0, 1.0], [400.0, 0.3], [900.0, -2.5], [1200.0, 0.75]])
    # velocity stds ~1.2 s_b: gamma / q stays bounded in velocity, so the
    # Monte-Carlo standard error is a faithful yardstick
    head = np.column_stack([rng.normal(0, 0.5, 4), rng.normal(0, 0.5, 4), rng.normal(0.2, 0.05, 4),
                            rng.normal(0.2, 0.05, 4), rng.normal(0, 0.5, 4)])
    J = 400_000
    w, x, wt, comp = _mc_draw(model_name, alpha, Z, head, J, seed=23)
    nu, sb = w.birth_mass, w.birth_vel_sigma
    A = (w.region[1] - w.region[0]) * (w.region[3] - w.region[2])
    checks = [(np.ones(J), nu), (x[:, 1], 0.0), (x[:, 1] ** 2, nu * sb * sb),
              ((x[:, 0] > 0).astype(float), nu * 0.5)]
    s0, s1 = w.sigma_z
    for z in Z:
        if model_name.startswith("linear"):
            inside = (np.abs(x[:, 0] - z[0]) <= 3 * s0) & (np.abs(x[:, 2] - z[1]) <= 3 * s1)
            area = 36 * s0 * s1
        else:
            r = np.hypot(x[:, 0] - w.sensor[0], x[:, 2] - w.sensor[1])
            th = np.arctan2(x[:, 2] - w.sensor[1], x[:, 0] - w.sensor[0])
            lo, hi = max(z[0] - 3 * s0, 0.0), z[0] + 3 * s0
            dth = np.angle(np.exp(1j * (th - z[1])))
            inside = (r >= lo) & (r <= hi) & (np.abs(dth) <= 3 * s1)
            area = 0.5 * (hi * hi - lo * lo) * 6 * s1
        checks.append((inside.astype(float), nu * area / A))
        checks.append((inside * x[:, 3] ** 2, nu * sb * sb * area / A))
    if not model_name.startswith("linear"):
        # r <= 6 m in the first measurement's bearing window: reached mostly
        # by folded draws (z_r = 8 m, sigma_r = 5 m)
        r = np.hypot(x[:, 0] - w.sensor[0], x[:, 2] - w.sensor[1])
        th = np.arctan2(x[:, 2] - w.sensor[1], x[:, 0] - w.sensor[0])
        near = (r <= 6.0) & (np.abs(np.angle(np.exp(1j * (th - Z[0, 1])))) <= 3 * s1)
        checks.append((near.astype(float), nu * 0.5 * 36.0 * 6 * s1 / A))
    for k, (f, want) in enumerate(checks):
        vals = J * wt * f
        est, se = vals.mean(), vals.std() / math.sqrt(J)
        assert abs(est - want) <= 5 * se + 1e-15, (model_name, alpha, k, est, want, se)
    assert (comp >= 0).mean() > 0.6                        # most draws used the mixture


@pytest.mark.parametrize("model_name", ["linear4_fp64", "dense_rb_100t"])
def test_one_component_draws_have_the_head_moments(model_name):
    """alpha = 0 and one measurement: velocities ~ N(s_b m, (s_b e^l)^2) per
    axis and positions ~ the measurement's noise around it (linear sensor:
    N(z, sigma^2); range-bearing: range and bearing of the draw ~ N(z, sigma^2)
    away from the fold), whatever the logit."""
    w = scenario.workload(model_name)
    m = oracle.model(w)
    head = np.array([[0.75, -0.5, math.log(0.5), math.log(1.5), 3.0]])
    Z = np.array([[120.0, -340.0]]) if model_name.startswith("linear") else np.array([[600.0, 2.0]])
    J = 200_000
    rng = np.random.default_rng(29)
    noise = np.column_stack([rng.standard_normal((J, 2)), rng.random((J, 2))])
    extra = np.column_stack([rng.random(J), rng.standard_normal((J, 2)), np.zeros(J)])
    x, wt, comp = oracle.birth_learned(m, Z, head, 0.0, J, noise, extra)
    assert np.all(comp == 0)
    sb = w.birth_vel_sigma
    se = 5 / math.sqrt(J)
    for col, mu, sd in [(1, 0.75 * sb, 0.5 * sb), (3, -0.5 * sb, 1.5 * sb)]:
        v = x[:, col]
        assert abs(v.mean() - mu) <= sd * se
        assert abs(v.std() / sd - 1.0) <= 2 * se
    if model_name.startswith("linear"):
        obs = x[:, [0, 2]]
    else:
        px, py = x[:, 0] - w.sensor[0], x[:, 2] - w.sensor[1]
        obs = np.column_stack([np.hypot(px, py), np.arctan2(py, px)])
    for d in range(2):
        assert abs(obs[:, d].mean() - Z[0, d]) <= w.sigma_z[d] * se
        assert abs(obs[:, d].std() / w.sigma_z[d] - 1.0) <= 2 * se
