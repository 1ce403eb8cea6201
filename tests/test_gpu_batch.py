"""GPU parity of the batch of independent filters (phd_batch_*).

Five runs with different clutter rates, birth counts, particles per target
and measurement capacities, uneven particle sets, stepped together; every
run is checked stage by stage against the FP64 oracle of its own
configuration (the harness of the one-filter tests: both sides from the same
generator slices), on injected random numbers."""
import numpy as np
import pytest
import torch

import oracle
import scenario
from gpu_harness import StageReport, check_step_from_inputs, exact_noise, exact_state

pytestmark = pytest.mark.gpu


def _runs():
    base = scenario.workload("linear4_fp64", precision="fp32", birth_steps=(1, 1, 1, 1))
    specs = [dict(clutter_rate=5.0, birth_count=300, particles_per_target=200, n_targets=2),
             dict(clutter_rate=60.0, birth_count=800, particles_per_target=500, n_targets=4),
             dict(clutter_rate=20.0, birth_count=100, particles_per_target=300, n_targets=3),
             dict(clutter_rate=150.0, birth_count=1200, particles_per_target=256, n_targets=1),
             dict(clutter_rate=0.5, birth_count=64, particles_per_target=1000, n_targets=4)]
    ws = [scenario.workload("linear4_fp64", precision="fp32", birth_steps=(1,) * s["n_targets"], **s)
          for s in specs]
    cap = max(w.pe_cap for w in ws)
    return [w.with_(pe_cap=cap) for w in ws]


@pytest.mark.parametrize("path", ["grid", "staged"])
@pytest.mark.parametrize("autotune", [False, True])
def test_batch_runs_match_their_oracles(autotune, path):
    """Three batched steps, each from generator slices (every run's own size;
    the second shaped like a resampling output); with autotune, the pair
    passes' launch shape is re-chosen after the first step (timed on the
    batch's own slices) and the runs stay on their oracles."""
    from paper_1503_03769_gb300 import ParticlePHDBatch
    ws = _runs()
    R = len(ws)
    b = ParticlePHDBatch(ws, seed=2)
    b.set_path(path)
    scs = [scenario.simulate(w, 40 + j, steps=3) for j, w in enumerate(ws)]
    rep = StageReport()
    for k in range(3):
        xs, wts = [], []
        for j, w in enumerate(ws):
            cen = np.concatenate([t[:, [0, 2]] for t in scs[j].truth if len(t)])
            x, wt = exact_state(w, 100 * k + j, [700 + 333 * j], centres=cen, mass=2.0 + j,
                                resampled=(k == 1))
            xs.append(x[0])
            wts.append(wt[0])
        b.set_state(xs, wts)
        Zs = [scs[j].meas[k] for j in range(R)]
        noise = exact_noise(9, k, R, b.pe_cap, np.float32)
        u = scenario.resample_u32(9, k, R)
        outs = b.batch_step(Zs, noise=noise, u=u)
        xp, wp, wu = b.get_predicted()
        C, mass = b.get_update()
        loc_s, loc_l = b.get_local_estimates()
        par, _ = b.get_resample()
        xr, wr = b.get_state()
        nz = np.asarray(noise).reshape(R, b.pe_cap, 4)
        for j, w in enumerate(ws):
            g = dict(xp=[xp[j]], wp=[wp[j]], wu=[wu[j]], C=C[j:j + 1], mass=mass[j:j + 1], loc_s=[loc_s[j]],
                     loc_l=[loc_l[j]], states=outs[j][0], labels=outs[j][1], par=par[j:j + 1], lx=0,
                     xr=[xr[j]], wr=[wr[j]])
            check_step_from_inputs(w, oracle.model(w), [xs[j]], [wts[j]], Zs[j], nz[j], u[j:j + 1], None, g, rep)
        if autotune and k == 0:
            t = b.autotune(2)
            assert t["pass1_us"] > 0 and t["pass2_us"] > 0
    assert rep.compared_labels > 0
    b.close()


def test_batch_free_running_and_capacity_errors():
    from paper_1503_03769_gb300 import ParticlePHDBatch, PhdError
    from paper_1503_03769_gb300 import phd as P
    ws = _runs()
    b = ParticlePHDBatch(ws, seed=4)
    scs = [scenario.simulate(w, 70 + j, steps=6) for j, w in enumerate(ws)]
    for k in range(6):
        outs = b.batch_step([scs[j].meas[k] for j in range(len(ws))])
        assert len(outs) == len(ws)
    st = b.stats()
    assert st["updates"] == 6 and st["pairs"] > 0
    # a run with more measurements than its capacity is reported
    Zs = [scs[j].meas[0] for j in range(len(ws))]
    Zs[2] = np.zeros((b.m_max + 5, 2), np.float32)
    with pytest.raises(PhdError) as e:
        b.batch_step(Zs)
    assert e.value.status == P.PHD_ERR_CAPACITY
    b.close()


@pytest.mark.parametrize("path", ["grid", "staged"])
def test_batch_edge_runs_match_their_oracles(path):
    """Runs at the edges in one batched step, each against its own oracle
    step from generator slices: no particles and no measurements (births
    only), particles and no measurements, no particles and a scan, and an
    ordinary run."""
    from paper_1503_03769_gb300 import ParticlePHDBatch
    ws = _runs()[:4]
    R = len(ws)
    b = ParticlePHDBatch(ws, seed=5)
    b.set_path(path)
    assert b.get_path() == path
    scs = [scenario.simulate(w, 80 + j, steps=2) for j, w in enumerate(ws)]
    n_seed = [0, 600, 0, 900]
    xs, wts = [], []
    for j, w in enumerate(ws):
        if n_seed[j]:
            cen = np.concatenate([t[:, [0, 2]] for t in scs[j].truth if len(t)])
            x, wt = exact_state(w, 300 + j, [n_seed[j]], centres=cen, mass=2.0)
            xs.append(x[0])
            wts.append(wt[0])
        else:
            xs.append(np.zeros((0, 4), np.float32))
            wts.append(np.zeros(0, np.float32))
    b.set_state(xs, wts)
    empty = np.zeros((0, 2), np.float32)
    Zs = [empty, empty, np.asarray(scs[2].meas[1], np.float32), np.asarray(scs[3].meas[1], np.float32)]
    noise = exact_noise(9, 1, R, b.pe_cap, np.float32)
    u = scenario.resample_u32(9, 1, R)
    outs = b.batch_step(Zs, noise=noise, u=u)
    xp, wp, wu = b.get_predicted()
    C, mass = b.get_update()
    loc_s, loc_l = b.get_local_estimates()
    par, _ = b.get_resample()
    xr, wr = b.get_state()
    nz = np.asarray(noise).reshape(R, b.pe_cap, 4)
    rep = StageReport()
    for j, w in enumerate(ws):
        g = dict(xp=[xp[j]], wp=[wp[j]], wu=[wu[j]], C=C[j:j + 1], mass=mass[j:j + 1], loc_s=[loc_s[j]],
                 loc_l=[loc_l[j]], states=outs[j][0], labels=outs[j][1], par=par[j:j + 1], lx=0,
                 xr=[xr[j]], wr=[wr[j]])
        check_step_from_inputs(w, oracle.model(w), [xs[j]], [wts[j]], Zs[j], nz[j], u[j:j + 1], None, g, rep)
    # births only where nothing was measured: the mass is (1 - p_D) nu_b
    assert mass[0] == pytest.approx((1 - ws[0].p_d) * ws[0].birth_mass, rel=1e-6)
    assert len(outs[0][1]) == 0 and len(outs[1][1]) == 0
    b.close()
