"""GPU parity of every launch shape of the update's pair passes (Eq. 7 column
sums, Eq. 8 row sums), and of the autotuner that picks among them.

Each shape is checked stage by stage against the FP64 oracle (the harness of
the one-filter tests: both sides from the same generator state) on a configuration whose slices span several work
items with ragged tails and whose measurement count crosses the pass-1 chunk
of every shape, with CTA caps small enough that every CTA walks several work
items (and restages particles and measurements between slices)."""
import numpy as np
import pytest

import oracle
import scenario
from gpu_harness import StageReport, exact_noise, exact_state, npdtype, stage_step

pytestmark = pytest.mark.gpu

PASS1 = [(t, mb) for t in (256, 512, 1024) for mb in (1, 2, 4)]
PASS2 = [(1, 1), (2, 1), (4, 1), (1, 2), (2, 2), (1, 4), (1, 8)]


def _filter(w, seed, counts, centres, **shape):
    from paper_1503_03769_gb300 import ParticlePHD
    f = ParticlePHD(w, seed=seed, device="cuda:0")
    f.set_path("staged")
    if shape:
        f.set_tuning(**shape)
    f.gen = (seed, counts, centres)
    xs, ws = exact_state(w, seed, counts, centres=centres)
    f.set_state(xs, ws)
    return f


def _step(f, w, sc, seed, k, rep):
    """One step from a generator state (every other one shaped like a
    resampling output), compared stage by stage with the oracle's chain."""
    s0, counts, centres = f.gen
    xs, ws = exact_state(w, 100 * s0 + k, counts, centres=centres, resampled=(k % 2 == 1))
    noise = exact_noise(seed, k, w.num_pe, w.pe_cap, npdtype(w))
    u = scenario.resample_u32(seed, k, w.num_pe)
    xu = scenario.exchange_u32(seed, k, w.num_pe, w.pe_cap)
    return stage_step(f, w, oracle.model(w), xs, ws, sc.meas[k], noise, u, xu, rep)


def _rb_case():
    w = scenario.workload("dense_rb_100t", n_targets=30, clutter_rate=300.0,
                          particles_per_target=200, birth_count=2000, num_pe=4,
                          exchange_frac=0.1, birth_steps=(1,) * 30)
    sc = scenario.simulate(w, 4, steps=2)
    cen = np.concatenate([t[:, [0, 2]] for t in sc.truth if len(t)])
    return w, sc, cen, [1500, 1700, 1300, 1611]


def _lin_case():
    w = scenario.workload("dist16_10t", n_targets=6, clutter_rate=30.0, num_pe=8,
                          particles_per_target=800, birth_count=1000, birth_steps=(1,) * 6)
    sc = scenario.simulate(w, 9, steps=2)
    cen = np.concatenate([t[:, [0, 2]] for t in sc.truth if len(t)])[:6]
    return w, sc, cen, [300 + 97 * j for j in range(8)]


@pytest.mark.parametrize("c_tile,c_mb", PASS1)
def test_pass1_shapes_range_bearing(c_tile, c_mb):
    """M ~ 330 crosses the 64/128/256-measurement chunks; 5 CTAs walk all items."""
    w, sc, cen, counts = _rb_case()
    f = _filter(w, 4, counts, cen, c_tile=c_tile, c_mb=c_mb, grid1=5)
    rep = StageReport()
    _step(f, w, sc, 4, 0, rep)
    f.close()
    assert rep.compared_labels > 0


@pytest.mark.parametrize("r_pb,r_g", PASS2)
@pytest.mark.parametrize("case", ["linear", "range_bearing"])
def test_pass2_shapes(r_pb, r_g, case):
    w, sc, cen, counts = _lin_case() if case == "linear" else _rb_case()
    f = _filter(w, 9, counts, cen, r_pb=r_pb, r_g=r_g, grid2=7, c_mb=1, grid1=11)
    rep = StageReport()
    _step(f, w, sc, 9, 0, rep)
    f.close()
    assert rep.compared_labels > 0


def test_fp64_shapes():
    """FP64 handles: the tile and the CTA caps are free, the lane shapes fixed."""
    from paper_1503_03769_gb300 import PhdError
    w = scenario.workload("linear4_fp64", n_targets=4, birth_steps=(1, 1, 1, 1), clutter_rate=12.0)
    sc = scenario.simulate(w, 5, steps=2)
    cen = sc.truth[0][:, [0, 2]]
    f = _filter(w, 5, [2100], cen, c_tile=1024, grid1=3, grid2=2)
    with pytest.raises(PhdError):
        f.set_tuning(c_mb=4)
    with pytest.raises(PhdError):
        f.set_tuning(r_pb=2, r_g=1)
    assert f.get_tuning()["c_tile"] == 1024
    rep = StageReport()
    _step(f, w, sc, 5, 0, rep)
    f.close()
    assert rep.compared_labels > 0


def test_unsupported_shapes_are_refused():
    from paper_1503_03769_gb300 import PhdError
    w, sc, cen, counts = _lin_case()
    f = _filter(w, 9, counts, cen)
    before = f.get_tuning()
    for bad in [dict(c_tile=128), dict(c_mb=3), dict(r_pb=4, r_g=2), dict(r_g=16), dict(grid1=0),
                dict(grid2=10 ** 6)]:
        with pytest.raises(PhdError):
            f.set_tuning(**bad)
    assert f.get_tuning() == before
    f.close()


def test_autotune_keeps_parity_and_statistics():
    """The autotuner needs an update to time on, returns a supported shape with
    its measured times, leaves the counters alone, and the filter stays on the
    oracle afterwards."""
    from paper_1503_03769_gb300 import PhdError
    w, sc, cen, counts = _rb_case()
    f = _filter(w, 4, counts, cen)
    with pytest.raises(PhdError):
        f.autotune(2)                      # no update yet
    rep = StageReport()
    _step(f, w, sc, 4, 0, rep)
    st0 = f.stats()
    t = f.autotune(2)
    assert t["pass1_us"] > 0 and t["pass2_us"] > 0
    assert (t["c_tile"], t["c_mb"]) in PASS1 and (t["r_pb"], t["r_g"]) in PASS2
    cur = f.get_tuning()
    assert all(cur[k] == t[k] for k in ("c_tile", "c_mb", "r_pb", "r_g", "grid1", "grid2"))
    st1 = f.stats()
    for k in ("pairs", "particles", "measurements", "updates"):
        assert st1[k] == st0[k], k
    _step(f, w, sc, 4, 1, rep)
    f.close()
    assert rep.compared_labels > 0


@pytest.mark.parametrize("case", ["linear", "range_bearing"])
def test_likelihood_gate_is_exact(case):
    """The gate skips only pairs whose FP32 likelihood term is exactly 0 (the
    exp2 result flushed to zero).  Pass 1 spreads the survivors over the
    CTA (a different grouping of FP32 partial sums), so C agrees to FP32
    rounding; pass 2 keeps every surviving term in the lane and accumulator
    of the full loop, so with the same C its weights are bit-identical (the
    FP32 normaliser copies are compared through the weights)."""
    w, sc, cen, counts = _lin_case() if case == "linear" else _rb_case()
    seed = 9 if case == "linear" else 4
    noise = scenario.step_noise(seed, 0, w.num_pe, w.pe_cap, np.float32)
    Z = np.asarray(sc.meas[0], np.float32)
    for r_pb, r_g in [(1, 4), (2, 1), (1, 8)]:
        outs = []
        for gate in (0, 1):
            f = _filter(w, seed, counts, cen, gate=gate, r_pb=r_pb, r_g=r_g, c_mb=2)
            f.predict(noise)
            f.update(Z)
            C, mass = f.get_update()
            _, wu = f.get_state()
            f.extract()
            ls, ll = f.get_local_estimates()
            outs.append((np.asarray(C), np.asarray(mass), [np.asarray(a) for a in wu],
                         [np.asarray(a) for a in ls], [np.asarray(a) for a in ll]))
            f.close()
        (C0, m0, w0, s0, l0), (C1, m1, w1, s1, l1) = outs
        np.testing.assert_allclose(C1, C0, rtol=2e-6, atol=1e-30)
        np.testing.assert_allclose(m1, m0, rtol=2e-6)
        for a, b in zip(w0, w1):
            np.testing.assert_allclose(b, a, rtol=2e-6, atol=1e-12 * max(float(np.abs(a).max()), 1e-30))
        # pass 3 (label sums of the extraction) gates labels per tile as well:
        # same labels, estimates to FP32 summation rounding
        assert sum(len(a) for a in l0) > 0
        for a, b in zip(l0, l1):
            np.testing.assert_array_equal(b, a)
        for a, b in zip(s0, s1):
            np.testing.assert_allclose(b, a, rtol=1e-5, atol=1e-3)


def test_order_change_waits_for_the_step():
    """The extraction walks the order the update built: switching it between
    the update and the resample is refused, and allowed again after."""
    from paper_1503_03769_gb300 import PhdError
    w, sc, cen, counts = _lin_case()
    f = _filter(w, 9, counts, cen, order=1)
    f.predict(scenario.step_noise(9, 0, w.num_pe, w.pe_cap, np.float32))
    f.update(np.asarray(sc.meas[0], np.float32))
    with pytest.raises(PhdError):
        f.set_tuning(order=0)
    f.set_tuning(gate=1, c_tile=1024)   # other fields may change
    f.extract()
    f.resample(scenario.resample_u32(9, 0, w.num_pe), scenario.exchange_u32(9, 0, w.num_pe, w.pe_cap))
    f.set_tuning(order=0)
    assert f.get_tuning()["order"] == 0
    f.close()


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("case", ["linear", "range_bearing"])
def test_spatial_order_on_and_off(order, case):
    """Passes 1 and 2 in slot order or in the cell order of the predicted set:
    the update stays on the oracle either way."""
    w, sc, cen, counts = _lin_case() if case == "linear" else _rb_case()
    seed = 9 if case == "linear" else 4
    f = _filter(w, seed, counts, cen, order=order, c_tile=256, grid1=9, grid2=13)
    rep = StageReport()
    _step(f, w, sc, seed, 0, rep)
    _step(f, w, sc, seed, 1, rep)
    f.close()
    assert rep.compared_labels > 0
