"""The k-sigma likelihood truncation variant (phd_config.gate_sigma) against
the FP64 oracle.

A pair within FP32 rounding of the truncation radius may be kept on one side
and dropped on the other, so the oracle brackets the GPU: with the radius
shrunk and grown by 1e-5 relative (far wider than FP32's error on the
exponent, ~1e-7) it gives a lower and an upper bound for every column sum
C_p and every updated weight, and the GPU must lie between them (to the
usual FP32 tolerance).  Both sides start from the same generator slices
(dyadic, so the GPU's prediction equals the oracle's exactly).  Staged passes and the fused step kernel, both
sensors."""
import numpy as np
import pytest
import torch

import oracle
import scenario
from gpu_harness import exact_noise, exact_state

pytestmark = pytest.mark.gpu

K_SIGMA = 3.0


def _case(name):
    if name == "linear":
        w = scenario.workload("dist16_10t", num_pe=4, n_targets=6, clutter_rate=30.0, particles_per_target=800,
                              birth_count=400, birth_steps=(1,) * 6, gate_sigma=K_SIGMA)
        seed = 31
    else:
        w = scenario.workload("dense_rb_100t", n_targets=30, clutter_rate=300.0, particles_per_target=200,
                              birth_count=2000, num_pe=4, exchange_frac=0.1, birth_steps=(1,) * 30,
                              gate_sigma=K_SIGMA, pe_cap=4096)
        seed = 32
    return w, seed


@pytest.mark.parametrize("path", ["staged", "fused"])
@pytest.mark.parametrize("case", ["linear", "range_bearing"])
def test_truncated_update_between_oracle_brackets(case, path):
    from paper_1503_03769_gb300 import ParticlePHD
    w, seed = _case(case)
    sc = scenario.simulate(w, seed, steps=1)
    Z = np.asarray(sc.meas[0], np.float32)
    centres = sc.truth[0][:, [0, 2]]
    xs, ws = exact_state(w, seed, [700 + 90 * j for j in range(w.num_pe)], centres=centres)
    f = ParticlePHD(w, seed=seed, device="cuda:0")
    f.set_path(path)
    f.set_state(xs, ws)
    noise = exact_noise(seed, 0, w.num_pe, w.pe_cap, np.float32)
    if path == "staged":
        f.predict(torch.as_tensor(noise).cuda())
        xp, wp = f.get_state()
        f.update(torch.as_tensor(Z).cuda())
        _, wu = f.get_state()
    else:
        f.step_inject(Z, noise, scenario.resample_u32(seed, 0, w.num_pe),
                      scenario.exchange_u32(seed, 0, w.num_pe, w.pe_cap))
        xp, wp, wu = f.get_predicted()
    C, mass = f.get_update()
    f.close()
    lo = oracle.model(w.with_(gate_sigma=K_SIGMA * (1 - 1e-5)))
    hi = oracle.model(w.with_(gate_sigma=K_SIGMA * (1 + 1e-5)))
    full = oracle.model(w.with_(gate_sigma=0.0))
    kap = oracle.kappa(full)
    Zd = Z.astype(np.float64)
    M = len(Z)
    bites = 0.0
    nz = noise.astype(np.float64).reshape(w.num_pe, w.pe_cap, 4)
    J = scenario.births_per_pe(w)
    for j in range(w.num_pe):
        # the oracle's own prediction of the same generator slice (exact in FP32)
        xo, wo = oracle.predict(full, xs[j].astype(np.float64), ws[j].astype(np.float64), J[j], nz[j])
        assert np.array_equal(np.asarray(xp[j], np.float64), xo), j
        c_lo = oracle.colsum(lo, xo, wo, Zd)
        c_hi = oracle.colsum(hi, xo, wo, Zd)
        c_full = oracle.colsum(full, xo, wo, Zd)
        Cg = C[j, :M]
        assert np.all(Cg >= c_lo * (1 - 1e-4) - 1e-7 * kap), j
        assert np.all(Cg <= c_hi * (1 + 1e-4) + 1e-7 * kap), j
        bites = max(bites, float(np.max((c_full - c_hi) / np.maximum(c_full, 1e-300))))
        # Eq. 8 grows with every g and shrinks with every C: the narrow
        # likelihood over the wide normaliser bounds the weights from below,
        # the wide over the narrow from above
        w_lo = oracle.weight_update(lo, xo, wo, Zd, c_hi)
        w_hi = oracle.weight_update(hi, xo, wo, Zd, c_lo)
        floor = 1e-9 * max(w_hi.sum(), 1e-300) / max(len(w_hi), 1)
        g = np.asarray(wu[j], np.float64)
        assert np.all(g >= w_lo * (1 - 1e-4) - floor), j
        assert np.all(g <= w_hi * (1 + 1e-4) + floor), j
        assert abs(mass[j] - g.sum()) <= 1e-5 * max(g.sum(), 1e-12)
    # the truncation changes some column sum by more than the tolerance
    assert bites > 1e-3
