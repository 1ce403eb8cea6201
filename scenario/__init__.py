"""Seeded synthetic inputs for the particle PHD filter: workloads, truth, sensor, noise.

This module is the one piece shared by the CUDA path's tests/benchmarks and the
CPU oracle.  It simulates the *world* (target truth tracks and the sensor's
measurement sets) and draws the random numbers the filter consumes, and it
computes no filter quantity: no likelihood, weight, normaliser, sum or estimate
lives here.

Scenario (paper Sec. 4): targets move by the constant-velocity model with
sampling period T = 1 and zero-mean Gaussian acceleration noise; each live
target is detected with probability p_D; clutter is a Poisson number of points
uniform over the measurement space.  Two sensors: linear position (x, y) with
Gaussian noise, and range-bearing from a sensor position (paper Sec. 4,
measurement model).  Numbers of the five workloads follow the published
workload list; the truth-birth schedule of the larger workloads is not in the
paper and is a reading (births at seeded steps in the first 40 % of the run,
no deaths other than leaving the region).

Noise layout consumed by both implementations (one row of four per particle
slot, survivors first then births, per processing element (PE) slot range):
  row = (n1, n2, u1, u2); survivors use n1, n2 as the standard normal
  acceleration draws; births use n1, n2 as standard normal velocity draws and
  u1, u2 in [0, 1) as the position fractions across the region (uniform
  birth) or as the Box-Muller pair of the position normals (Gaussian birth).
Resampling takes one uint32 per PE per step; the ring exchange takes one
uint32 per selected slot (a partial Fisher-Yates draw), up to pe_cap per PE.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict, replace
from typing import List, Optional, Sequence

import numpy as np

DEG = math.pi / 180.0

LINEAR = "linear"
RANGE_BEARING = "range_bearing"


@dataclass(frozen=True)
class Workload:
    """Parameters of one filter workload (model, sizes and run length)."""
    name: str
    meas_model: str = LINEAR
    dt: float = 1.0
    sigma_a: float = 5.0                    # process (acceleration) noise std, m/s^2
    sigma_z: tuple = (10.0, 10.0)           # linear: (m, m); range-bearing: (m, rad)
    sensor: tuple = (0.0, 0.0)
    region: tuple = (-1000.0, 1000.0, -1000.0, 1000.0)   # x_min, x_max, y_min, y_max
    r_max: float = 1000.0 * math.sqrt(2.0)  # range-bearing clutter range extent
    p_s: float = 0.99
    p_d: float = 0.95
    clutter_rate: float = 10.0              # lambda: expected clutter points per scan
    birth_mass: float = 0.1                 # expected births per step (nu_b)
    birth_count: int = 500                  # J birth particles per step (all PEs)
    birth_vel_sigma: float = 20.0
    particles_per_target: int = 500         # rho
    num_pe: int = 1                         # K processing elements (1 = global filter)
    exchange_frac: float = 0.0
    ck_mode: str = "local"                  # "local" (paper) or "global" (exact mean)
    precision: str = "fp32"
    n_targets: int = 4
    birth_steps: Optional[tuple] = None     # explicit truth birth steps (1-based)
    steps: int = 50
    truth_vel_sigma: float = 20.0
    truth_bounded: bool = False             # truth tracks reflect at the region boundary (the
                                            # configured target count stays present) instead of leaving
    pe_cap: int = 0                         # particle slots per PE (0: derived)
    m_max: int = 0                          # measurement capacity (0: derived)
    sigma_a_y: float = 0.0                  # y-axis acceleration noise std (0: sigma_a)
    theta_span: float = 0.0                 # range-bearing clutter bearing extent (0: 2 pi)
    birth_model: str = "uniform"            # "uniform" or "gaussian" (N(birth_mean, diag birth_std^2))
    birth_mean: tuple = (0.0, 0.0, 0.0, 0.0)
    birth_std: tuple = (0.0, 0.0, 0.0, 0.0)
    exchange_mode: str = "ring"             # Step 6 pattern: "ring" (the paper's) or "all" (all-to-all)
    exchange_threshold: float = 0.0         # > 0: exchange only when min_j N_j < threshold * mean_j N_j
    gate_sigma: float = 0.0                 # > 0: likelihood truncated beyond this many std (a variant)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    def as_dict(self) -> dict:
        return asdict(self)


def _derive_caps(w: Workload) -> Workload:
    """Fill pe_cap / m_max with generous capacities for the workload's sizes."""
    K = w.num_pe
    j_pe = -(-w.birth_count // K)
    # expected mass <= targets + births; keep 3x headroom on the survivor count
    n_t = max(w.n_targets, 1)
    rho_pe = w.particles_per_target / K
    surv = int(math.ceil(rho_pe * (3 * n_t + 8)))
    pe_cap = w.pe_cap or int(-(-(surv + j_pe) // 256) * 256)
    m_exp = w.clutter_rate + w.n_targets
    m_max = w.m_max or int(-(-int(m_exp + 8 * math.sqrt(m_exp) + 32) // 64) * 64)
    return replace(w, pe_cap=pe_cap, m_max=m_max)


def workload(name: str, **overrides) -> Workload:
    """Named workloads: the five published configurations plus small test cases."""
    base = {
        # Plain global particle PHD, linear position sensor, FP64.
        "linear4_fp64": Workload(
            name="linear4_fp64", meas_model=LINEAR, sigma_z=(10.0, 10.0),
            clutter_rate=10.0, n_targets=4, birth_steps=(1, 10, 20, 30),
            particles_per_target=500, birth_count=500, steps=50, precision="fp64"),
        # Paper's distributed scheme: 16 PEs, 10 % ring exchange, CU fusion.
        "dist16_10t": Workload(
            name="dist16_10t", truth_bounded=True, meas_model=LINEAR, sigma_z=(10.0, 10.0),
            clutter_rate=50.0, n_targets=10, particles_per_target=1000,
            birth_count=1000, steps=100, num_pe=16, exchange_frac=0.1,
            precision="fp32"),
        # Dense scale, range-bearing sensor at the origin.
        "dense_rb_100t": Workload(
            name="dense_rb_100t", truth_bounded=True, meas_model=RANGE_BEARING, sigma_z=(5.0, 0.5 * DEG),
            clutter_rate=500.0, n_targets=100, particles_per_target=2000,
            birth_count=20000, steps=100, precision="fp32"),
        # The dense workload's distributed form: 64 PEs.  A PE keeps rho/64 =
        # 31 particles per target it holds plus 312 births: 4096 slots cover
        # ~120 targets per PE, and a slice fits one SM's shared memory.
        "dense_rb_100t_pe64": Workload(
            name="dense_rb_100t_pe64", truth_bounded=True, meas_model=RANGE_BEARING, sigma_z=(5.0, 0.5 * DEG),
            clutter_rate=500.0, n_targets=100, particles_per_target=2000,
            birth_count=20000, steps=100, num_pe=64, exchange_frac=0.1, precision="fp32", pe_cap=4096),
        # Learned-birth evaluation scenario (range-bearing, 50 targets).
        "rb_50t": Workload(
            name="rb_50t", truth_bounded=True, meas_model=RANGE_BEARING, sigma_z=(5.0, 0.5 * DEG),
            clutter_rate=100.0, n_targets=50, particles_per_target=1000,
            birth_count=5000, steps=100, precision="fp32"),
        # The paper's own simulation shape (Sec. 4): bearing-range sensor with
        # a half-plane field of view over 200 m, p_S 0.9, p_D 1, Gaussian
        # birth N(x_bar, Q) near the sensor, 4 PEs with 200 particles per
        # target each, 5 tracks over 50 scans; process noise std as printed
        # (0.025 and 4 per axis; the printed values are garbled).
        "paper_bot": Workload(
            name="paper_bot", meas_model=RANGE_BEARING, sigma_z=(5.0, 0.05),
            sigma_a=0.025, sigma_a_y=4.0, region=(0.0, 200.0, -200.0, 200.0), r_max=200.0,
            theta_span=math.pi, p_s=0.9, p_d=1.0, clutter_rate=10.0, n_targets=5,
            particles_per_target=800, birth_count=800, num_pe=4, exchange_frac=0.1, steps=50,
            birth_model="gaussian", birth_mean=(0.0, 3.0, 0.0, -3.0),
            birth_std=(math.sqrt(10.0), 1.0, math.sqrt(10.0), 1.0), precision="fp32", pe_cap=2048),
    }
    if name not in base:
        raise KeyError(f"unknown workload {name!r}; known: {sorted(base)}")
    w = base[name].with_(**overrides)
    if name != "linear4_fp64" and "birth_mass" not in overrides:
        w = w.with_(birth_mass=matched_birth_mass(w))
    return _derive_caps(w)


def matched_birth_mass(w: Workload) -> float:
    """Expected truth births per scan of a workload whose targets appear at
    seeded scans spread over the first 40 % of the run (the birth intensity
    nu_b the filter is given for it)."""
    return w.n_targets / (0.4 * w.steps)


def batch_workloads(seed: int = 1000, runs: int = 256, steps: int = 60) -> List[Workload]:
    """The batched Monte-Carlo workload: `runs` independent linear-sensor
    filters whose sizes are drawn per run from a seeded generator: targets
    U{1..50}, clutter rate U[5, 200], particles per target U{256..4096}, births
    per step equal to particles per target (a reading; the count is not
    given), `steps` scans.  All runs share one pe_cap (the largest need)."""
    rng = np.random.default_rng(np.random.SeedSequence([0xBA7C, seed]))
    out = []
    for r in range(runs):
        nt = int(rng.integers(1, 51))
        lam = float(rng.uniform(5.0, 200.0))
        rho = int(rng.integers(256, 4097))
        wr = Workload(name=f"batch_run{r}", meas_model=LINEAR, sigma_z=(10.0, 10.0), truth_bounded=True,
                      clutter_rate=lam, n_targets=nt, particles_per_target=rho,
                      birth_count=rho, steps=steps, precision="fp32")
        out.append(wr.with_(birth_mass=matched_birth_mass(wr)))
    caps = []
    for w in out:
        m_exp = w.clutter_rate + w.n_targets
        m_max = int(-(-int(m_exp + 8 * math.sqrt(m_exp) + 32) // 64) * 64)
        caps.append((w.particles_per_target * (2 * w.n_targets + 8) + w.birth_count, m_max))
    pe_cap = int(-(-max(c for c, _ in caps) // 256) * 256)
    return [w.with_(pe_cap=pe_cap, m_max=mm) for w, (_, mm) in zip(out, caps)]


# ----------------------------------------------------------------------------
# Truth and sensor simulation
# ----------------------------------------------------------------------------

@dataclass
class Scenario:
    workload: Workload
    truth: List[np.ndarray] = field(default_factory=list)   # per step: (n_k, 4) float64
    truth_ids: List[np.ndarray] = field(default_factory=list)
    meas: List[np.ndarray] = field(default_factory=list)    # per step: (M_k, 2) float32
    meas_is_target: List[np.ndarray] = field(default_factory=list)


def _reflect(x: np.ndarray, region) -> np.ndarray:
    """Specular reflection of truth tracks at the region boundary: a position
    past an edge is mirrored back inside and that velocity component negated."""
    out = x.copy()
    for pc, vc, lo, hi in ((0, 1, region[0], region[1]), (2, 3, region[2], region[3])):
        below, above = out[:, pc] < lo, out[:, pc] > hi
        out[below, pc] = 2 * lo - out[below, pc]
        out[above, pc] = 2 * hi - out[above, pc]
        out[below | above, vc] = -out[below | above, vc]
    return out


def _cv_move(x: np.ndarray, dt: float, acc: np.ndarray) -> np.ndarray:
    """World motion of the truth tracks (constant velocity + acceleration noise)."""
    out = x.copy()
    out[:, 0] = x[:, 0] + dt * x[:, 1] + 0.5 * dt * dt * acc[:, 0]
    out[:, 1] = x[:, 1] + dt * acc[:, 0]
    out[:, 2] = x[:, 2] + dt * x[:, 3] + 0.5 * dt * dt * acc[:, 1]
    out[:, 3] = x[:, 3] + dt * acc[:, 1]
    return out


def _sense(w: Workload, x: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Sensor output for true states x with noise draws v (world side)."""
    if w.meas_model == LINEAR:
        return np.stack([x[:, 0] + w.sigma_z[0] * v[:, 0],
                         x[:, 2] + w.sigma_z[1] * v[:, 1]], axis=1)
    px, py = x[:, 0] - w.sensor[0], x[:, 2] - w.sensor[1]
    r = np.sqrt(px * px + py * py) + w.sigma_z[0] * v[:, 0]
    th = np.arctan2(py, px) + w.sigma_z[1] * v[:, 1]
    th = np.where(th > math.pi, th - 2 * math.pi, th)
    th = np.where(th <= -math.pi, th + 2 * math.pi, th)
    return np.stack([r, th], axis=1)


def _clutter(w: Workload, rng: np.random.Generator, n: int) -> np.ndarray:
    u = rng.random((n, 2))
    if w.meas_model == LINEAR:
        x0, x1, y0, y1 = w.region
        return np.stack([x0 + u[:, 0] * (x1 - x0), y0 + u[:, 1] * (y1 - y0)], axis=1)
    if w.theta_span > 0:
        # bearing uniform over [-span / 2, span / 2] (the sensor's field of view)
        return np.stack([u[:, 0] * w.r_max, 0.5 * w.theta_span - u[:, 1] * w.theta_span], axis=1)
    return np.stack([u[:, 0] * w.r_max, math.pi - u[:, 1] * 2 * math.pi], axis=1)


def simulate(w: Workload, seed: int, steps: Optional[int] = None) -> Scenario:
    """Truth tracks and measurement sets for `steps` scans (default: w.steps)."""
    steps = w.steps if steps is None else steps
    rng = np.random.default_rng(np.random.SeedSequence([0x5CE4, seed]))
    x0, x1, y0, y1 = w.region
    if w.birth_steps is not None:
        bsteps = list(w.birth_steps)[: w.n_targets]
        bsteps += [1] * (w.n_targets - len(bsteps))
    else:
        hi = max(1, int(0.4 * w.steps))
        bsteps = sorted(int(s) for s in rng.integers(1, hi + 1, size=w.n_targets))
    if w.birth_model == "gaussian":
        # initial states from the birth density N(x_bar, Q) itself
        init = (np.asarray(w.birth_mean, np.float64)
                + np.asarray(w.birth_std, np.float64) * rng.standard_normal((w.n_targets, 4)))
    else:
        # initial states: positions in the inner 80 % of the region
        cx, cy, hx, hy = 0.5 * (x0 + x1), 0.5 * (y0 + y1), 0.4 * (x1 - x0), 0.4 * (y1 - y0)
        init = np.stack([cx + hx * (2 * rng.random(w.n_targets) - 1),
                         w.truth_vel_sigma * rng.standard_normal(w.n_targets),
                         cy + hy * (2 * rng.random(w.n_targets) - 1),
                         w.truth_vel_sigma * rng.standard_normal(w.n_targets)], axis=1)
    acc_std = np.array([w.sigma_a, w.sigma_a_y if w.sigma_a_y > 0 else w.sigma_a])
    sc = Scenario(workload=w)
    live = np.zeros((0, 4))
    ids = np.zeros((0,), dtype=np.int64)
    for k in range(1, steps + 1):
        if len(live):
            live = _cv_move(live, w.dt, rng.standard_normal((len(live), 2)) * acc_std)
            if w.truth_bounded:
                live = _reflect(live, w.region)
            inside = ((live[:, 0] >= x0) & (live[:, 0] <= x1) &
                      (live[:, 2] >= y0) & (live[:, 2] <= y1))
            if w.meas_model == RANGE_BEARING and w.theta_span > 0:
                # a sensor with a field of view: tracks leave it past r_max
                # or outside the bearing span
                px, py = live[:, 0] - w.sensor[0], live[:, 2] - w.sensor[1]
                inside &= (np.hypot(px, py) <= w.r_max) & (np.abs(np.arctan2(py, px)) <= 0.5 * w.theta_span)
            live, ids = live[inside], ids[inside]
        born = [t for t in range(w.n_targets) if bsteps[t] == k]
        if born:
            live = np.concatenate([live, init[born]], axis=0)
            ids = np.concatenate([ids, np.asarray(born, dtype=np.int64)])
        det = rng.random(len(live)) < w.p_d
        zt = _sense(w, live[det], rng.standard_normal((int(det.sum()), 2)))
        nc = int(rng.poisson(w.clutter_rate))
        zc = _clutter(w, rng, nc)
        z = np.concatenate([zt, zc], axis=0)
        is_t = np.concatenate([np.ones(len(zt), bool), np.zeros(nc, bool)])
        perm = rng.permutation(len(z))
        sc.truth.append(live.copy())
        sc.truth_ids.append(ids.copy())
        sc.meas.append(np.ascontiguousarray(z[perm], dtype=np.float32))
        sc.meas_is_target.append(is_t[perm])
    return sc


# ----------------------------------------------------------------------------
# Random numbers consumed by the filter (injected into both implementations)
# ----------------------------------------------------------------------------

def births_per_pe(w: Workload) -> List[int]:
    """Births per PE: J split as evenly as possible, lower PEs take the remainder."""
    K, J = w.num_pe, w.birth_count
    return [J // K + (1 if j < J % K else 0) for j in range(K)]


def step_noise(seed: int, step: int, K: int, pe_cap: int, dtype=np.float64) -> np.ndarray:
    """Per-slot predict/birth draws, shape (K * pe_cap, 4): (n1, n2, u1, u2).

    Values are rounded to `dtype` here so both implementations read identical
    numbers whatever precision they compute in.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0xA11CE, seed, step]))
    n = K * pe_cap
    out = np.empty((n, 4), dtype=np.float64)
    out[:, 0:2] = rng.standard_normal((n, 2))
    out[:, 2:4] = rng.random((n, 2))
    if dtype == np.float32:
        out = out.astype(np.float32)
        # a float32 rounding of u < 1 may round up to 1.0; keep u in [0, 1)
        out[:, 2:4] = np.minimum(out[:, 2:4], np.float32(1.0 - 2.0 ** -24))
    return np.ascontiguousarray(out)


def birth_extra_noise(seed: int, step: int, K: int, jmax: int, dtype=np.float64) -> np.ndarray:
    """Extra draws of the measurement-driven birth, shape (K * jmax, 4):
    (u_c, nz1, nz2, 0) per birth slot of each PE (jmax = most births of a PE)."""
    rng = np.random.default_rng(np.random.SeedSequence([0xB1E7, seed, step]))
    n = K * jmax
    out = np.zeros((n, 4), dtype=np.float64)
    out[:, 0] = rng.random(n)
    out[:, 1:3] = rng.standard_normal((n, 2))
    if dtype == np.float32:
        out = out.astype(np.float32)
        out[:, 0] = np.minimum(out[:, 0], np.float32(1.0 - 2.0 ** -24))
    return np.ascontiguousarray(out)


def mlp_params(seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded parameters of the 3-64-64-5 birth network (4741 values, layout
    W1[64][3], b1[64], W2[64][64], b2[64], W3[5][64], b3[5]), every value an
    integer in [-127, 127] times a power of two, so it is exact in bfloat16,
    float32 and float64 alike.  Magnitudes follow 1/sqrt(fan-in) (times
    `scale`, a power of two)."""
    assert scale > 0 and math.log2(scale) == int(math.log2(scale))
    rng = np.random.default_rng(np.random.SeedSequence([0x3A1E, seed]))
    parts = []
    for shape, e in [((64, 3), -8), ((64,), -9), ((64, 64), -10), ((64,), -9), ((5, 64), -10), ((5,), -8)]:
        k = rng.integers(-127, 128, size=shape).astype(np.float64)
        parts.append((k * 2.0 ** e * scale).ravel())
    return np.concatenate(parts)


def resample_u32(seed: int, step: int, K: int) -> np.ndarray:
    rng = np.random.default_rng(np.random.SeedSequence([0x5E5A, seed, step]))
    return rng.integers(0, 2 ** 32, size=K, dtype=np.uint64).astype(np.uint32)


def exchange_u32(seed: int, step: int, K: int, pe_cap: int) -> np.ndarray:
    rng = np.random.default_rng(np.random.SeedSequence([0xE8C4, seed, step]))
    return rng.integers(0, 2 ** 32, size=(K, pe_cap), dtype=np.uint64).astype(np.uint32)


def random_particles(rng: np.random.Generator, w: Workload, n: int,
                     centres: Optional[np.ndarray] = None, spread: float = 30.0,
                     mass: float = 1.0) -> tuple:
    """A synthetic particle cloud (states, weights) for stage-level tests.

    Positions cluster around `centres` (or spread over the region), velocities
    N(0, 20^2), weights positive with total `mass`.
    """
    x0, x1, y0, y1 = w.region
    if centres is None or len(centres) == 0:
        pos = np.stack([x0 + rng.random(n) * (x1 - x0), y0 + rng.random(n) * (y1 - y0)], 1)
    else:
        c = centres[rng.integers(0, len(centres), size=n)]
        pos = c + spread * rng.standard_normal((n, 2))
    vel = 20.0 * rng.standard_normal((n, 2))
    x = np.stack([pos[:, 0], vel[:, 0], pos[:, 1], vel[:, 1]], axis=1)
    wgt = rng.random(n) + 0.05
    if n > 0:
        wgt *= mass / wgt.sum()
    return x, wgt


__all__ = [
    "Workload", "workload", "batch_workloads", "Scenario", "simulate", "births_per_pe", "step_noise",
    "resample_u32", "exchange_u32", "random_particles", "LINEAR", "RANGE_BEARING", "DEG",
]
