"""GPU parity: libphd.so (through its C ABI) against the FP64 oracle.

Every compared step starts both sides from the same generator-made particle
set (dyadic values, so FP32 prediction is exact; see gpu_harness) with the
same injected random numbers, and the oracle runs its own chain through the
stages: predict and update elementwise, extraction per PE and after fusion,
resampling by count and offspring validity, the ring exchange bit-exactly
given the resampled slices.  Sizes span several 256-particle tiles with
ragged tails, PEs with unequal counts, M below and above the 256-thread
measurement rounds, both sensors, both precisions and both normaliser modes;
every other compared step starts from a set shaped like a resampling output
(equal weights, duplicated states).
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import scenario
from gpu_harness import StageReport, stage_step, check_weights, npdtype, exact_noise, exact_state

pytestmark = pytest.mark.gpu


def _filter(w, seed=0, path="staged"):
    from paper_1503_03769_gb300 import ParticlePHD
    f = ParticlePHD(w, seed=seed, device="cuda:0")
    f.set_path(path)
    return f


def _run_stages(w, seed, steps, sc=None, warm=0, n_seed=None, centres=None, path="staged"):
    """`steps` compared steps on scans warm .. warm + steps - 1; each starts
    both sides from a generator state around that scan's truth (or around
    `centres`) with n_seed particles per PE (default: rho / K per live
    target)."""
    f = _filter(w, seed, path)
    m = oracle.model(w)
    if sc is None:
        sc = scenario.simulate(w, seed, steps=warm + steps)
    exact = w.birth_model != "gaussian"     # Box-Muller (log, sin, cos) is not bit-identical
    rep = StageReport()
    K = w.num_pe
    for s in range(steps):
        k = warm + s
        tr = sc.truth[k]
        cen = centres if centres is not None else (tr[:, [0, 2]] if len(tr) else None)
        counts = n_seed if n_seed is not None else \
            int(round(w.particles_per_target / K * max(1, len(tr))))
        x0, w0 = exact_state(w, 1000 * seed + s, counts, centres=cen, mass=float(max(1, len(tr))),
                             resampled=(s % 2 == 1))
        noise = exact_noise(seed, k, K, w.pe_cap, npdtype(w))
        u = scenario.resample_u32(seed, k, K)
        xu = scenario.exchange_u32(seed, k, K, w.pe_cap)
        stage_step(f, w, m, x0, w0, sc.meas[k], noise, u, xu, rep, path=path, exact_predict=exact)
    f.close()
    _log_errors(w, path, rep)
    return rep


def _log_errors(w, path, rep):
    """With PHD_PARITY_LOG set, append the largest errors this test saw
    against the oracle (one JSON line per test) to that file."""
    out = os.environ.get("PHD_PARITY_LOG")
    if not out:
        return
    import json
    rec = {"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], "workload": w.name,
           "precision": w.precision, "path": path, "K": w.num_pe, "C_rel": rep.max_c_rel,
           "w_rel": rep.max_w_rel, "mass_rel": rep.max_mass_rel, "state_abs_m": rep.max_state_err,
           "predict_abs_m": rep.max_pred_abs, "labels": rep.compared_labels}
    with open(out, "a") as fh:
        fh.write(json.dumps(rec) + "\n")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("path", ["staged", "fused", "grid"])
def test_global_linear_stages(precision, path):
    """Global filter, linear sensor: a ragged 2600-particle set, 3 steps."""
    w = scenario.workload("linear4_fp64", precision=precision, n_targets=4,
                          birth_steps=(1, 1, 1, 1), clutter_rate=12.0)
    n0 = 2100
    if path == "fused":                     # the PE slice must fit shared memory
        w = w.with_(pe_cap=4096 if precision == "fp32" else 2560)
        n0 = 2100 if precision == "fp32" else 1900
    truth = scenario.simulate(w, 5, steps=3)
    centres = truth.truth[0][:, [0, 2]]
    rep = _run_stages(w, 5, 3, sc=truth, n_seed=[n0], centres=centres, path=path)
    assert rep.compared_labels > 0


@pytest.mark.parametrize("ck_mode", ["local", "global"])
@pytest.mark.parametrize("path", ["staged", "fused", "grid"])
def test_distributed_linear_stages(ck_mode, path):
    """16 PEs (the paper's DCPFPHD form) with exchange, uneven slice sizes;
    on the grid path every PE's slice spreads over the kernel's CTAs."""
    w = scenario.workload("dist16_10t", ck_mode=ck_mode, n_targets=6, clutter_rate=30.0,
                          particles_per_target=800, birth_count=1000, birth_steps=(1,) * 6)
    truth = scenario.simulate(w, 9, steps=3)
    centres = np.concatenate([t[:, [0, 2]] for t in truth.truth if len(t)])[:6]
    counts = [300 + 37 * j for j in range(16)]
    rep = _run_stages(w, 9, 3, sc=truth, n_seed=counts, centres=centres, path=path)
    assert rep.compared_labels > 0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("path", ["staged", "fused", "grid"])
def test_paper_scenario_stages(precision, path):
    """The paper's own simulation shape (Sec. 4): Gaussian birth N(x_bar, Q),
    per-axis process noise, a bearing field of view (kappa over [0, r_max] x
    [-pi/2, pi/2]), p_S 0.9, p_D 1, 4 PEs with exchange; 8 free-running
    scans, then 3 scans compared stage by stage."""
    w = scenario.workload("paper_bot", precision=precision, clutter_rate=20.0)
    truth = scenario.simulate(w, 21, steps=11)
    rep = _run_stages(w, 21, 3, sc=truth, warm=8, path=path)
    assert rep.compared_labels > 0


def test_learned_proposal_needs_the_uniform_birth():
    """The defensive mixture's plain part is the uniform birth: a Gaussian-birth
    handle refuses a network."""
    from paper_1503_03769_gb300 import PhdError, proposal
    w = scenario.workload("paper_bot")
    f = _filter(w, 1)
    with pytest.raises(PhdError):
        f.set_birth_proposal(torch.as_tensor(proposal.init_params(0), device="cuda:0"))
    f.close()


@pytest.mark.parametrize("pe_cap", [64, 128])
def test_fused_many_pes_small_slices(pe_cap):
    """64 PEs with slices of a few dozen particles on the fused path: CU
    fusion is shared over the CTAs in chunks of a few labels (pe_cap 128,
    M ~ 30 spans ~10 chunks) or, when a slice's scratch cannot hold a chunk
    (pe_cap 64), done by CTA 0 alone; both must give the oracle's fusion."""
    w = scenario.workload("dist16_10t", num_pe=64, n_targets=3, clutter_rate=20.0,
                          particles_per_target=640, birth_count=640, birth_steps=(1, 1, 1),
                          pe_cap=pe_cap, exchange_frac=0.1)
    truth = scenario.simulate(w, 13, steps=3)
    centres = np.concatenate([t[:, [0, 2]] for t in truth.truth if len(t)])
    f = _filter(w, 13, "fused")
    assert f.get_path() == "fused"
    f.close()
    rep = _run_stages(w, 13, 3, sc=truth, n_seed=[30 + (j % 7) for j in range(64)], centres=centres,
                      path="fused")
    assert rep.compared_labels > 0


@pytest.mark.parametrize("path", ["staged", "grid"])
def test_maximum_pe_count(path):
    """K = 256 PEs, the most a handle takes: more PEs than SMs, so the fused
    kernel (one co-resident CTA per PE) cannot hold them; AUTO runs the grid
    step kernel (its CTAs take the PEs' tiles), a forced fused path is
    refused, and every stage (ring exchange and CU fusion over 256 voters
    included) matches the oracle on the staged and grid paths."""
    from paper_1503_03769_gb300 import PhdError
    w = scenario.workload("dist16_10t", num_pe=256, n_targets=3, clutter_rate=20.0,
                          particles_per_target=2560, birth_count=2560, birth_steps=(1, 1, 1),
                          pe_cap=64, exchange_frac=0.1)
    truth = scenario.simulate(w, 17, steps=2)
    centres = np.concatenate([t[:, [0, 2]] for t in truth.truth if len(t)])
    f = _filter(w, 17, "auto")
    assert f.get_path() == "grid"
    with pytest.raises(PhdError):
        f.set_path("fused")
    f.close()
    rep = _run_stages(w, 17, 2, sc=truth, n_seed=[20 + (j % 9) for j in range(256)], centres=centres, path=path)
    assert rep.compared_labels > 0


@pytest.mark.parametrize("mode,threshold", [("all", 0.0), ("ring", 1e-9), ("all", 1e9), ("all", 0.97)])
@pytest.mark.parametrize("path", ["staged", "fused", "grid"])
def test_exchange_variants_stages(mode, threshold, path):
    """Step 6 variants on 16 PEs: all-to-all every step; the adaptive trigger
    never firing (threshold 1e-9), always firing (1e9) and deciding from the
    step's PE masses (0.97); the GPU's exchange count must be the oracle's."""
    w = scenario.workload("dist16_10t", n_targets=6, clutter_rate=30.0, particles_per_target=800,
                          birth_count=1000, birth_steps=(1,) * 6, exchange_mode=mode,
                          exchange_threshold=threshold)
    truth = scenario.simulate(w, 9, steps=3)
    centres = np.concatenate([t[:, [0, 2]] for t in truth.truth if len(t)])[:6]
    counts = [300 + 37 * j for j in range(16)]
    rep = _run_stages(w, 9, 3, sc=truth, n_seed=counts, centres=centres, path=path)
    assert rep.compared_labels > 0


@pytest.mark.parametrize("path", ["staged", "fused", "grid"])
def test_range_bearing_stages_many_measurements(path):
    """Range-bearing sensor, M ~ 330 (> one 256-thread round), 4 PEs, FP32."""
    w = scenario.workload("dense_rb_100t", n_targets=30, clutter_rate=300.0,
                          particles_per_target=200, birth_count=2000, num_pe=4,
                          exchange_frac=0.1, birth_steps=(1,) * 30)
    truth = scenario.simulate(w, 4, steps=2)
    if path == "fused":
        w = w.with_(pe_cap=4096)
    rep = _run_stages(w, 4, 2, sc=truth, warm=0, n_seed=[1500, 1700, 1300, 1611],
                      centres=np.concatenate([t[:, [0, 2]] for t in truth.truth if len(t)]), path=path)
    assert rep.compared_labels > 0


@pytest.mark.parametrize("path", ["staged", "grid"])
def test_bearing_branch_cut(path):
    """Particles and measurements on both sides of bearing +-pi: the wrapped
    likelihood must match the oracle's (a missing wrap drops their weights)."""
    w = scenario.workload("dense_rb_100t", n_targets=1, clutter_rate=5.0,
                          particles_per_target=300, birth_count=64)
    f = _filter(w, 1, path)
    m = oracle.model(w)
    rng = np.random.default_rng(1)
    n = 700
    th = math.pi + 0.01 * rng.standard_normal(n)
    r = 800 + 5 * rng.standard_normal(n)
    x = np.stack([r * np.cos(th), np.zeros(n), r * np.sin(th), np.zeros(n)], 1).astype(np.float32)
    wt = np.full(n, 1.0 / n, np.float32)
    Z = np.array([[800.0, math.pi - 0.002], [800.0, -math.pi + 0.003], [810.0, 3.1]], np.float32)
    noise = np.zeros((w.pe_cap, 4), np.float32)
    noise[:, 2:] = 0.5
    rep = StageReport()
    stage_step(f, w, m, [x], [wt], Z, noise, np.array([12345], np.uint32), None, rep, path=path)
    assert rep.compared_labels >= 1


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_resample_bit_exact_on_injected_weights(precision):
    """With identical weights on both sides the parents are bit-exact,
    for heavy-tailed weights, ragged sizes and several U."""
    for n, seed in [(1, 0), (7, 1), (255, 2), (256, 3), (4099, 4), (70001, 5)]:
        w = scenario.workload("linear4_fp64", precision=precision, birth_count=0, p_s=1.0,
                              p_d=0.0, sigma_a=0.0, particles_per_target=max(1, n // 3),
                              pe_cap=n + 64)
        f = _filter(w, seed)
        rng = np.random.default_rng(seed)
        dt = npdtype(w)
        x = rng.standard_normal((n, 4)).astype(dt)
        wt = (rng.random(n) ** 6 * 3.7).astype(dt)
        for U in [0, 1, 2 ** 31, 2 ** 32 - 1, int(rng.integers(0, 2 ** 32))]:
            f.set_state([x], [wt])
            f.predict(torch.zeros((w.pe_cap, 4), dtype=torch.float64 if dt == np.float64 else torch.float32,
                                  device="cuda"))
            f.update(torch.zeros((0, 2), device="cuda"))
            xp, wp = f.get_state()
            np.testing.assert_array_equal(wp[0], wt)     # p_S = 1, p_D = 0: weights unchanged
            f.resample(np.array([U], np.uint32))
            par, _ = f.get_resample()
            xr, wr = f.get_state()
            x_or, _ = oracle.predict(oracle.model(w), x.astype(np.float64), wt.astype(np.float64), 0,
                                     np.zeros((n, 4)))
            xo, wo, po = oracle.resample(x_or, wt.astype(np.float64), w.particles_per_target, w.pe_cap, U)
            assert np.array_equal(par[0, :len(po)], po), (n, U)
            np.testing.assert_allclose(xr[0].astype(np.float64), xo, rtol=0,
                                       atol=1e-14 if dt == np.float64 else 2e-6)
            check_weights(wr[0], wo, dict(w_rel=1e-15 if dt == np.float64 else 1e-7), "new weights")
        f.close()


def test_free_running_fp64_matches_oracle_over_many_steps():
    """The 4-target linear workload in FP64 (one of the published workloads):
    20 steps with the oracle running its own recursion from the same start,
    fed the same random numbers; estimates and particle sets agree."""
    w = scenario.workload("linear4_fp64", steps=20)
    sc = scenario.simulate(w, 0)
    f = _filter(w, 0)
    orc = oracle.OracleFilter(w)
    worst = 0.0
    for k, Z in enumerate(sc.meas):
        noise = scenario.step_noise(0, k, 1, w.pe_cap)
        u = scenario.resample_u32(0, k, 1)
        f.predict(torch.as_tensor(noise).cuda())
        f.update(torch.as_tensor(Z.astype(np.float64)).cuda())
        states, labels = f.extract()
        f.resample(u)
        lab_o, zet_o = orc.step(Z, noise, u)
        assert list(labels.cpu().numpy()) == list(lab_o), k
        if len(lab_o):
            worst = max(worst, float(np.abs(states.cpu().numpy() - zet_o).max()))
        xs, ws = f.get_state()
        assert len(xs[0]) == len(orc.x[0])
        np.testing.assert_allclose(xs[0], orc.x[0], rtol=0, atol=1e-7)
        np.testing.assert_allclose(ws[0], orc.wt[0], rtol=1e-10)
    assert worst < 1e-6


@pytest.mark.parametrize("path", ["staged", "fused", "grid"])
def test_published_distributed_workload_sizes(path):
    """The 16-PE workload at its published sizes (10 targets, lambda = 50,
    1000 particles per target, 1000 births) in the launch configuration the
    benchmark times: stage parity on scans 12 and 13 (all ten targets live),
    from generator slices of rho / K particles per target."""
    w = scenario.workload("dist16_10t")
    rep = _run_stages(w, 2, 2, warm=12, path=path)
    assert rep.max_mass_rel <= 1e-5


@pytest.mark.parametrize("path", ["staged", "fused", "grid"])
def test_dense_workload_64_pes_full_size(path):
    """The dense workload's 64-PE distributed form (config 3) at full size:
    64 generator slices of rho / 64 particles per live target (~3.1e3 each,
    ~2.2e5 in all) against ~600 measurements, one step in the launch
    configuration the benchmark times (staged path autotuned on these
    slices; fused path one CTA per PE; grid path the PEs over the whole
    GPU), every stage of every PE against the oracle (which runs on all host
    cores)."""
    w = scenario.workload("dense_rb_100t_pe64")
    sc = scenario.simulate(w, 6, steps=61)
    tr = sc.truth[60]
    Z = sc.meas[60]
    counts = int(round(w.particles_per_target / w.num_pe * len(tr)))
    x0, w0 = exact_state(w, 66, counts, centres=tr[:, [0, 2]], mass=float(len(tr)))
    noise = exact_noise(6, 60, w.num_pe, w.pe_cap, np.float32)
    u = scenario.resample_u32(6, 60, w.num_pe)
    xu = scenario.exchange_u32(6, 60, w.num_pe, w.pe_cap)
    assert len(Z) > 450 and counts * w.num_pe > 1.5e5
    f = _filter(w, 6, path)
    if path == "staged":
        f.set_state(x0, w0)
        f.predict(torch.as_tensor(noise).cuda())
        f.update(torch.as_tensor(Z).cuda())
        f.autotune(2)
        f.extract()
        f.resample(u, xu)
    oracle.set_threads(os.cpu_count() or 1)
    try:
        rep = StageReport()
        stage_step(f, w, oracle.model(w), x0, w0, Z, noise, u, xu, rep, path=path)
    finally:
        oracle.set_threads(1)
    f.close()
    _log_errors(w, path, rep)
    assert rep.compared_labels > 100


@pytest.mark.parametrize("path", ["fused", "grid"])
def test_barrier_timeout_is_reported_and_recoverable(path):
    """Failure detection without a GPU fault: the host flags PE 0 (on the grid
    path, CTA 0 of the step kernel) as lost, so it leaves the step at the
    first grid barrier without arriving; the others' bounded waits (limit
    lowered to 2e4 polls) give up, the step reports PHD_ERR_TIMEOUT, and the
    same handle then steps normally again (barrier words, flag, error word
    and the grid path's running cell totals reset)."""
    from paper_1503_03769_gb300 import PhdError, phd
    w = scenario.workload("dist16_10t", num_pe=4 if path == "fused" else 1, n_targets=3, clutter_rate=10.0,
                          particles_per_target=200, birth_count=200, exchange_frac=0.1 if path == "fused" else 0.0)
    sc = scenario.simulate(w, 2, steps=6)
    f = _filter(w, 2, path)
    ref = _filter(w, 2, path)
    for k in range(2):
        f.step(sc.meas[k])
        ref.step(sc.meas[k])
    xs, ws = f.get_state()
    step = f.get_step()
    f.set_wait_limit(20_000)
    f.inject_barrier_fault()
    with pytest.raises(PhdError) as ei:
        f.step(sc.meas[2])
    assert ei.value.status == phd.PHD_ERR_TIMEOUT
    # the context is usable: restore the checkpoint (state and step counter)
    # and the default limit; the next steps equal an uninterrupted filter's
    f.set_wait_limit(20_000_000)
    f.set_state(xs, ws)
    f.set_step(step)
    for k in range(2, 6):
        s_f, l_f = f.step(sc.meas[k])
        s_r, l_r = ref.step(sc.meas[k])
        np.testing.assert_array_equal(l_f.cpu().numpy(), l_r.cpu().numpy())
        np.testing.assert_array_equal(s_f.cpu().numpy(), s_r.cpu().numpy())
    f.close()
    ref.close()


def test_edge_cases_and_errors():
    from paper_1503_03769_gb300 import PhdError
    from paper_1503_03769_gb300 import phd as P
    w = scenario.workload("linear4_fp64", precision="fp32", birth_count=50, particles_per_target=20)
    f = _filter(w, 0)
    # empty filter, no measurements: births only, mass = (1 - p_D) nu_b
    f.predict()
    f.update(torch.zeros((0, 2), device="cuda"))
    C, mass = f.get_update()
    assert mass[0] == pytest.approx((1 - w.p_d) * w.birth_mass, rel=1e-6)
    s, l = f.extract()
    assert len(l) == 0
    f.resample()
    xs, ws = f.get_state()
    assert len(xs[0]) == 20          # rho * max(1, N) with N < 1
    # stage order
    with pytest.raises(PhdError) as e:
        f.update(torch.zeros((1, 2), device="cuda"))
    assert e.value.status == P.PHD_ERR_STATE
    with pytest.raises(PhdError) as e:
        f.extract()
    assert e.value.status == P.PHD_ERR_STATE
    # too many measurements
    f.predict()
    with pytest.raises(PhdError) as e:
        f.update(torch.zeros((w.m_max + 1, 2), device="cuda"))
    assert e.value.status == P.PHD_ERR_CAPACITY
    # non-finite measurement: reported at the next synchronising call
    Z = torch.tensor([[1.0, 2.0], [float("nan"), 0.0]], device="cuda")
    f.update(Z)
    with pytest.raises(PhdError) as e:
        f.get_update()
    assert e.value.status == P.PHD_ERR_INVALID_ARG
    f.resample()
    # exactly m_max measurements, extraction capacity overflow reports the count
    rng = np.random.default_rng(0)
    xs = [rng.uniform(-900, 900, (w.pe_cap - 50, 4)).astype(np.float32)]
    xs[0][:, [1, 3]] = 0
    f.set_state(xs, [np.full(len(xs[0]), 0.05, np.float32)])
    f.predict()
    Zf = np.asarray(xs[0][:w.m_max][:, [0, 2]], np.float32)
    f.update(torch.as_tensor(Zf).cuda())
    with pytest.raises(PhdError) as e:
        f.extract(cap=1)
    assert e.value.status == P.PHD_ERR_CAPACITY and e.value.count > 1
    f.resample()
    f.close()


@pytest.mark.parametrize("path", ["grid", "staged"])
def test_whole_step_edge_cases(path):
    """Whole steps (phd_step) at the edges, on the grid path and the staged
    graph: an empty filter with no measurements (births only: the mass is
    (1 - p_D) nu_b, nothing is extracted, rho max(1, N) particles are kept);
    exactly m_max measurements with an estimate count above cap (reported as
    PHD_ERR_CAPACITY with the true count, and the filter steps on); a
    non-finite measurement (reported as PHD_ERR_INVALID_ARG)."""
    from paper_1503_03769_gb300 import PhdError
    from paper_1503_03769_gb300 import phd as P
    w = scenario.workload("linear4_fp64", precision="fp32", birth_count=50, particles_per_target=20)
    f = _filter(w, 0, path)
    assert f.get_path() == path
    s, l = f.step(np.zeros((0, 2), np.float32))
    C, mass = f.get_update()
    assert mass[0] == pytest.approx((1 - w.p_d) * w.birth_mass, rel=1e-6)
    assert len(l) == 0
    xs, ws = f.get_state()
    assert len(xs[0]) == 20          # rho * max(1, N) with N < 1
    rng = np.random.default_rng(0)
    x = rng.uniform(-900, 900, (w.pe_cap - 50, 4)).astype(np.float32)
    x[:, [1, 3]] = 0
    f.set_state([x], [np.full(len(x), 0.05, np.float32)])
    Zf = np.asarray(x[:w.m_max][:, [0, 2]], np.float32)
    with pytest.raises(PhdError) as e:
        f.step(Zf, cap=1)
    assert e.value.status == P.PHD_ERR_CAPACITY and e.value.count > 1
    s, l = f.step(Zf[:10])
    assert np.isfinite(s.cpu().numpy()).all()
    Z = np.array([[1.0, 2.0], [np.nan, 0.0]], np.float32)
    with pytest.raises(PhdError) as e:
        f.step(Z)
    assert e.value.status == P.PHD_ERR_INVALID_ARG
    f.close()


def test_free_running_philox_moments():
    """In-kernel randomness (Philox-4x32-10 + Box-Muller): predicted survivors
    have the CV model's mean and covariance; births cover the region."""
    w = scenario.workload("linear4_fp64", precision="fp32", birth_count=100000,
                          particles_per_target=1, pe_cap=300000)
    f = _filter(w, 11)
    n = 150000
    x0 = np.array([10.0, 2.0, -5.0, 1.0], np.float32)
    f.set_state([np.tile(x0, (n, 1))], [np.full(n, 1.0 / n, np.float32)])
    f.predict()
    xp, wp = f.get_state()
    sv, bi = xp[0][:n].astype(np.float64), xp[0][n:].astype(np.float64)
    sa2 = w.sigma_a ** 2
    blk = sa2 * np.array([[0.25, 0.5], [0.5, 1.0]])
    cov = np.cov(sv.T)
    assert np.allclose(cov[:2, :2], blk, rtol=0.03) and np.allclose(cov[2:, 2:], blk, rtol=0.03)
    assert abs(cov[0, 2]) < 0.05 * sa2
    assert np.allclose(sv.mean(0), [12.0, 2.0, -4.0, 1.0], atol=0.05)
    assert len(bi) == 100000
    assert bi[:, 0].min() >= -1000 and bi[:, 0].max() <= 1000
    assert bi[:, 0].var() == pytest.approx(2000.0 ** 2 / 12, rel=0.02)
    assert bi[:, 1].std() == pytest.approx(20.0, rel=0.02)
    f.update(torch.zeros((0, 2), device="cuda"))
    f.resample()
    f.close()


@pytest.mark.parametrize("path", ["staged", "fused", "grid"])
def test_checkpoint_resume_is_bit_identical(path):
    w = scenario.workload("dist16_10t", num_pe=4, n_targets=4, clutter_rate=20.0,
                          particles_per_target=300, birth_count=400)
    sc = scenario.simulate(w, 6, steps=8)
    a = _filter(w, 6, path)
    for k in range(4):
        a.step(sc.meas[k])
    xs, ws = a.get_state()
    st = a.get_step()
    b = _filter(w, 6, path)
    b.set_state(xs, ws)
    b.set_step(st)
    for k in range(4, 8):
        sa, la = a.step(sc.meas[k])
        sb, lb = b.step(sc.meas[k])
        assert torch.equal(la, lb) and torch.equal(sa, sb)
    xa, wa = a.get_state()
    xb, wb = b.get_state()
    for j in range(4):
        np.testing.assert_array_equal(xa[j], xb[j])
        np.testing.assert_array_equal(wa[j], wb[j])


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("path", ["staged", "fused", "grid"])
def test_step_host_matches_device_step(path, pinned):
    """Host-memory steps equal device steps: pageable buffers (copies through
    the workspace) and pinned ones (the kernels read Z and write the
    estimates and count in host memory), then a too-small cap."""
    from paper_1503_03769_gb300 import PhdError
    w = scenario.workload("dist16_10t", num_pe=4, n_targets=4, clutter_rate=20.0,
                          particles_per_target=300, birth_count=400)
    sc = scenario.simulate(w, 8, steps=8)
    a, b = _filter(w, 8, path), _filter(w, 8, path)

    def host(shape, dt):
        t = torch.zeros(shape, dtype=dt)
        return (t.pin_memory() if pinned else t).numpy()

    # both start from the same generator slices around the targets of scan 2
    # (the first with a live target), so the compared steps have estimates
    x0, w0 = exact_state(w, 81, 300, centres=sc.truth[2][:, [0, 2]], mass=float(len(sc.truth[2])))
    a.set_state(x0, w0)
    b.set_state(x0, w0)
    out_s = host((w.m_max, 4), torch.float32)
    out_l = host(w.m_max, torch.int32)
    compared = 0
    for Z in sc.meas[2:7]:
        Zh = host(Z.shape, torch.float32)
        Zh[:] = Z
        sa, la = a.step(Z)
        n = b.step_host(Zh, out_s, out_l)
        assert n == len(la)
        np.testing.assert_array_equal(out_l[:n], la.cpu().numpy())
        np.testing.assert_array_equal(out_s[:n], sa.cpu().numpy())
        compared += n
    assert compared > 0
    Z = sc.meas[7]
    Zh = host(Z.shape, torch.float32)
    Zh[:] = Z
    sa, la = a.step(Z)
    if len(la) > 0:
        with pytest.raises(PhdError) as ei:
            b.step_host(Zh, out_s[:0], out_l[:0])
        assert ei.value.count == len(la)
    a.close()
    b.close()


def test_fused_run_matches_fused_steps():
    """phd_run (S steps in one launch) gives bit-identical results to S
    single-step launches of the fused kernel."""
    w = scenario.workload("dist16_10t", steps=12)
    sc = scenario.simulate(w, 21)
    a, b = _filter(w, 21, "fused"), _filter(w, 21, "fused")
    outs = [a.step(Z) for Z in sc.meas]
    runs = b.run(sc.meas)
    for (sa, la), (sb, lb) in zip(outs, runs):
        assert torch.equal(la, lb) and torch.equal(sa, sb)
    xa, wa = a.get_state()
    xb, wb = b.get_state()
    for j in range(w.num_pe):
        np.testing.assert_array_equal(xa[j], xb[j])
        np.testing.assert_array_equal(wa[j], wb[j])


@pytest.mark.parametrize("pair", ["fused-staged", "grid-staged", "grid16-staged"])
def test_paths_track_each_other(pair):
    """Free-running with the same seed: the fused (or grid) step kernel and
    the staged kernels draw the same Philox numbers and agree on the
    estimates over a 40-scan run (the 16-PE workload; on the grid path its
    one-PE form and the 16 PEs), up to near-tie selections (and the
    divergence a resampling tie-flip starts)."""
    w = scenario.workload("dist16_10t", steps=40)
    if pair.startswith("grid-"):
        w = w.with_(num_pe=1, exchange_frac=0.0, pe_cap=16 * w.pe_cap)
    sc = scenario.simulate(w, 31)
    a, b = _filter(w, 31, pair.split("-")[0].rstrip("0123456789")), _filter(w, 31, "staged")
    same, diffs, oa, ob = 0, [], [], []
    for k, Z in enumerate(sc.meas):
        sa, la = a.step(Z)
        sb, lb = b.step(Z)
        tr = sc.truth[k][:, [0, 2]] if len(sc.truth[k]) else np.zeros((0, 2))
        oa.append(oracle.ospa(sa.double().cpu().numpy()[:, [0, 2]], tr))
        ob.append(oracle.ospa(sb.double().cpu().numpy()[:, [0, 2]], tr))
        if torch.equal(la, lb):
            same += 1
            if len(la):
                diffs.append(float((sa.double() - sb.double())[:, [0, 2]].abs().max()))
    if pair.startswith("fused"):
        assert same >= 30 and max(diffs) < 1e-2
    else:
        # the grid kernel groups the FP32 partial sums of the pair passes
        # differently (its tiles and live lists): once a resampling boundary
        # flips, the particle sets differ and the two runs are two draws of the
        # same filter; they must track the truth equally well
        assert same >= 20
        assert abs(np.mean(oa) - np.mean(ob)) <= 0.1 * max(np.mean(oa), np.mean(ob)) + 2.0, (np.mean(oa),
                                                                                           np.mean(ob))


@pytest.mark.parametrize("path", ["staged", "fused"])
def test_misaligned_buffers_are_refused(path):
    """The kernels access caller buffers as vectors (a measurement row of two
    reals, an estimate row of four).  Views at an odd float offset are refused
    with PHD_ERR_INVALID_ARG before anything is launched, the handle keeps
    stepping exactly like an untouched one, and phd_step_host takes the
    copying path for misaligned pinned host arrays."""
    import ctypes
    from paper_1503_03769_gb300 import phd as P
    w = scenario.workload("dist16_10t", num_pe=4, n_targets=3, clutter_rate=10.0, particles_per_target=200,
                          birth_count=200)
    sc = scenario.simulate(w, 5, steps=3)
    f, ref = _filter(w, 5, path), _filter(w, 5, path)
    Z = torch.as_tensor(sc.meas[0], dtype=torch.float32, device="cuda").contiguous()
    M, cap = Z.shape[0], w.m_max
    zbuf = torch.zeros(2 * M + 1, dtype=torch.float32, device="cuda")
    zbuf[1:] = Z.reshape(-1)
    sbuf = torch.zeros(4 * cap + 1, dtype=torch.float32, device="cuda")
    lab = torch.zeros(cap + 1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    off = torch.tensor([0, M], dtype=torch.int32, device="cuda")
    vp = ctypes.c_void_p
    hc = ctypes.c_int32(0)
    z_ok, z_bad = vp(Z.data_ptr()), vp(zbuf.data_ptr() + 4)
    s_ok, s_bad = vp(sbuf.data_ptr()), vp(sbuf.data_ptr() + 4)
    l_ok, l_bad = vp(lab.data_ptr()), vp(lab.data_ptr() + 2)
    c_ok = vp(cnt.data_ptr())
    for args in [(z_bad, s_ok, l_ok), (z_ok, s_bad, l_ok), (z_ok, s_ok, l_bad)]:
        st = f.L.phd_step(f.h, args[0], M, args[1], args[2], cap, c_ok, ctypes.byref(hc))
        assert st == P.PHD_ERR_INVALID_ARG
    assert f.L.phd_run(f.h, z_bad, vp(off.data_ptr()), 1, s_ok, l_ok, c_ok, cap) == P.PHD_ERR_INVALID_ARG
    # nothing ran: the next steps equal an untouched filter's
    for k in range(2):
        s_f, l_f = f.step(sc.meas[k])
        s_r, l_r = ref.step(sc.meas[k])
        assert torch.equal(l_f, l_r) and torch.equal(s_f, s_r)
    # stage API: a refused update leaves the predicted stage in place
    f.predict()
    assert f.L.phd_update(f.h, z_bad, M) == P.PHD_ERR_INVALID_ARG
    f.update(sc.meas[2])
    assert f.L.phd_extract(f.h, s_bad, l_ok, cap, None, ctypes.byref(hc)) == P.PHD_ERR_INVALID_ARG
    f.extract()
    f.resample()
    # misaligned pinned host arrays: copied through the workspace instead
    g, gref = _filter(w, 6, path), _filter(w, 6, path)
    zh = torch.zeros(2 * M + 1, dtype=torch.float32).pin_memory().numpy()
    zh[1:] = np.asarray(sc.meas[0], np.float32).reshape(-1)
    sh = torch.zeros(4 * cap + 1, dtype=torch.float32).pin_memory().numpy()
    lh = torch.zeros(cap, dtype=torch.int32).pin_memory().numpy()
    n = g.step_host(zh[1:].reshape(M, 2), sh[1:].reshape(cap, 4), lh)
    s_r, l_r = gref.step(sc.meas[0])
    assert n == len(l_r)
    np.testing.assert_array_equal(lh[:n], l_r.cpu().numpy())
    np.testing.assert_array_equal(sh[1:].reshape(cap, 4)[:n], s_r.cpu().numpy())
    for x in (f, ref, g, gref):
        x.close()
