"""phd_colsum_static: the Eq. 7 column sums for callers that may not allocate
device memory (fixed-memory real-time trackers, plug-ins inside a host
application that owns every allocation).  Its scratch is the library's own
file-scope device array, so the test checks, through the C ABI, that two
calls in a row reproduce the normaliser phd_update computes on the same
particle sets (within the C tolerance of the parity tests), and that sizes
beyond the array are refused.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import scenario

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("wname,precision", [("dense_rb_100t", "fp32"), ("linear4_fp64", "fp64")])
def test_colsum_static_matches_update_on_two_calls(wname, precision):
    from paper_1503_03769_gb300 import ParticlePHD, phd
    kw = dict(n_targets=20, clutter_rate=150.0, particles_per_target=300, birth_count=2000,
              birth_steps=(1,) * 20) if wname == "dense_rb_100t" else dict(birth_count=700)
    w = scenario.workload(wname, precision=precision, **kw)
    f = ParticlePHD(w, seed=5, device="cuda:0")
    f.set_path("staged")
    dt = np.float64 if precision == "fp64" else np.float32
    tdt = torch.float64 if precision == "fp64" else torch.float32
    sc = scenario.simulate(w, 5, steps=2)
    rng = np.random.default_rng(5)
    centres = np.concatenate([t[:, [0, 2]] for t in sc.truth if len(t)])
    x, wt = scenario.random_particles(rng, w, 2300, centres=centres, spread=30.0, mass=4.0)
    f.set_state([x.astype(dt)], [wt.astype(dt)])
    kap = 1e-7 * (w.clutter_rate / (2 * np.pi * w.r_max if w.meas_model != "linear" else 4e6))
    for call in range(2):
        Z = sc.meas[call].astype(dt)
        f.predict(torch.as_tensor(scenario.step_noise(5, call, 1, w.pe_cap, dt)).cuda())
        f.update(torch.as_tensor(Z).cuda())
        C_ref, _ = f.get_update()
        xp, wp, _ = f.get_predicted()
        f.resample()
        X = torch.as_tensor(xp[0], dtype=tdt, device="cuda").contiguous()
        W = torch.as_tensor(wp[0], dtype=tdt, device="cuda").contiguous()
        Zt = torch.as_tensor(Z, device="cuda").contiguous()
        C = torch.full((len(Z),), -1.0, dtype=torch.float64, device="cuda")
        assert phd.colsum_static(f.cfg, X, W, Zt, C) == phd.PHD_OK
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        ref = C_ref[0, :len(Z)]
        assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + kap), (call, np.abs(got - ref).max())
    f.close()


def test_colsum_static_refuses_sizes_beyond_its_array():
    from paper_1503_03769_gb300 import phd
    w = scenario.workload("dist16_10t")
    cfg = phd.make_config(w)
    n, M = 256 * 600, 900            # 600 tiles x 900 > 524288 partials
    X = torch.zeros((n, 4), device="cuda")
    W = torch.zeros(n, device="cuda")
    Z = torch.zeros((M, 2), device="cuda")
    C = torch.zeros(M, dtype=torch.float64, device="cuda")
    assert phd.colsum_static(cfg, X, W, Z, C) == phd.PHD_ERR_CAPACITY
    L = phd.lib()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    assert L.phd_colsum_static(ctypes.byref(cfg), ptr(X), ptr(W), 10, None, 5, ptr(C), None) == \
        phd.PHD_ERR_INVALID_ARG
