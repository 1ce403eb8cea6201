"""phd_colsum_static: the Eq. 7 column sums for callers that may not allocate
device memory (fixed-memory real-time trackers, plug-ins inside a host
application that owns every allocation).  Its scratch is the library's own
file-scope device array, shared by every call, so the tests make two calls in
a row through the C ABI and check each against the normaliser phd_update
computes on the same particle set and, on the generator's particle set,
against the FP64 oracle's column sums (within the C tolerance of the parity
tests); they also cover the k-sigma
truncation variant (between oracle brackets), an empty particle set, a scan
with fewer measurements than a CTA has threads, and sizes beyond the array.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import scenario

pytestmark = pytest.mark.gpu


def _kappa_slack(w):
    return 1e-7 * oracle.kappa(oracle.model(w))


def _particles(w, seed, n):
    sc = scenario.simulate(w, seed, steps=2)
    rng = np.random.default_rng(seed)
    centres = np.concatenate([t[:, [0, 2]] for t in sc.truth if len(t)])
    x, wt = scenario.random_particles(rng, w, n, centres=centres, spread=30.0, mass=4.0)
    return sc, x, wt


def _static(w, cfg, x, wt, Z):
    from paper_1503_03769_gb300 import phd
    tdt = torch.float64 if w.precision == "fp64" else torch.float32
    X = torch.as_tensor(np.asarray(x).reshape(-1, 4), dtype=tdt, device="cuda").contiguous()
    W = torch.as_tensor(np.asarray(wt).reshape(-1), dtype=tdt, device="cuda").contiguous()
    Zt = torch.as_tensor(np.asarray(Z).reshape(-1, 2), dtype=tdt, device="cuda").contiguous()
    C = torch.full((max(len(Z), 1),), -1.0, dtype=torch.float64, device="cuda")
    st = phd.colsum_static(cfg, X, W, Zt, C)
    torch.cuda.synchronize()
    return st, C.cpu().numpy()[:len(Z)]


@pytest.mark.parametrize("wname,precision", [("dense_rb_100t", "fp32"), ("linear4_fp64", "fp64")])
def test_colsum_static_matches_oracle_and_update_on_two_calls(wname, precision):
    from paper_1503_03769_gb300 import ParticlePHD, phd
    kw = dict(n_targets=20, clutter_rate=150.0, particles_per_target=300, birth_count=2000,
              birth_steps=(1,) * 20) if wname == "dense_rb_100t" else dict(birth_count=700)
    w = scenario.workload(wname, precision=precision, **kw)
    dt = np.float64 if precision == "fp64" else np.float32
    rel = 1e-10 if precision == "fp64" else 1e-4
    sc, x, wt = _particles(w, 5, 2300)
    f = ParticlePHD(w, seed=5, device="cuda:0")
    f.set_path("staged")
    f.set_state([x.astype(dt)], [wt.astype(dt)])
    kap = _kappa_slack(w)
    m = oracle.model(w)
    for call in range(2):
        Z = sc.meas[call].astype(dt)
        # the existing entry point: phd_update's C on the predicted set
        f.predict(torch.as_tensor(scenario.step_noise(5, call, 1, w.pe_cap, dt)).cuda())
        f.update(torch.as_tensor(Z).cuda())
        C_upd, _ = f.get_update()
        xp, wp, _ = f.get_predicted()
        f.resample()
        st, got = _static(w, f.cfg, xp[0], wp[0], Z)
        assert st == phd.PHD_OK
        ref = C_upd[0, :len(Z)]
        assert np.all(np.abs(got - ref) <= rel * np.abs(ref) + kap), (call, np.abs(got - ref).max())
        # the FP64 oracle, both sides on the generator's particle set
        xg, wg = x.astype(dt), wt.astype(dt)
        st, got = _static(w, f.cfg, xg, wg, Z)
        assert st == phd.PHD_OK
        Co = oracle.colsum(m, xg.astype(np.float64), wg.astype(np.float64), np.asarray(Z, np.float64))
        assert np.all(np.abs(got - Co) <= rel * np.abs(Co) + kap), (call, np.abs(got - Co).max())
    f.close()


def test_colsum_static_truncation_between_oracle_brackets():
    """gate_sigma = 3: a pair within FP32 rounding of the radius may fall on
    either side, so the oracle with the radius shrunk and grown by 1e-5
    bounds every C_p from below and above."""
    from paper_1503_03769_gb300 import phd
    w = scenario.workload("dense_rb_100t", n_targets=12, clutter_rate=80.0, particles_per_target=300,
                          birth_count=2000, birth_steps=(1,) * 12, gate_sigma=3.0)
    sc, x, wt = _particles(w, 9, 3100)
    x32, w32 = x.astype(np.float32), wt.astype(np.float32)
    cfg = phd.make_config(w)
    kap = _kappa_slack(w)
    for call in range(2):
        Z = sc.meas[call].astype(np.float32)
        st, got = _static(w, cfg, x32, w32, Z)
        assert st == phd.PHD_OK
        lo = oracle.colsum(oracle.model(w.with_(gate_sigma=3.0 * (1 - 1e-5))), x32, w32, Z)
        hi = oracle.colsum(oracle.model(w.with_(gate_sigma=3.0 * (1 + 1e-5))), x32, w32, Z)
        assert np.all(got >= lo * (1 - 1e-4) - kap), (call, (lo - got).max())
        assert np.all(got <= hi * (1 + 1e-4) + kap), (call, (got - hi).max())
        # the truncation removes mass: strictly below the exact column sums somewhere
        exact = oracle.colsum(oracle.model(w.with_(gate_sigma=0.0)), x32, w32, Z)
        assert np.any(got < exact * (1 - 1e-3))


def test_colsum_static_empty_set_and_few_measurements():
    """n = 0 gives C = 0 for every measurement; M = 3 (fewer measurements than
    a CTA's threads, so each measurement's particles are split over many
    threads) matches the oracle; both twice in a row."""
    from paper_1503_03769_gb300 import phd
    w = scenario.workload("dist16_10t", num_pe=1, exchange_frac=0.0, birth_steps=(1,) * 10)
    cfg = phd.make_config(w)
    sc, x, wt = _particles(w, 13, 1777)
    x32, w32 = x.astype(np.float32), wt.astype(np.float32)
    kap = _kappa_slack(w)
    m = oracle.model(w)
    for call in range(2):
        Z = sc.meas[call].astype(np.float32)
        st, got = _static(w, cfg, np.zeros((0, 4), np.float32), np.zeros(0, np.float32), Z)
        assert st == phd.PHD_OK
        assert np.array_equal(got, np.zeros(len(Z))), got
        Z3 = Z[:3]
        st, got = _static(w, cfg, x32, w32, Z3)
        assert st == phd.PHD_OK
        Co = oracle.colsum(m, x32, w32, Z3)
        assert np.all(np.abs(got - Co) <= 1e-4 * np.abs(Co) + kap), (call, got, Co)


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
