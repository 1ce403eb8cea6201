"""Helpers for the GPU parity tests: stage-by-stage comparison of libphd.so
against the FP64 oracle on the same generator inputs and injected random
numbers.

Both sides start every compared step from the same generator-made particle
set, and the oracle runs its own chain through the step's stages; no oracle
input is ever taken from the GPU.  Tolerances are the ones the filter is
specified to: weights 1e-4 relative (plus a 1e-9 * mean-weight floor for
weights that FP32's exp2 flushes to zero), masses 1e-5 relative, extracted
states 1e-3 m; resampling by its count and offspring validity, the exchange
bit-exact given the resampled slices.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np
import torch

import oracle
import scenario

# C_p carries the same per-pair FP32 likelihood error as the weights (a few
# 1e-5 for pairs several sigma apart), so it is held to the weight tolerance;
# the mass, which is what C feeds, is held to 1e-5.
FP32_TOL = dict(w_rel=1e-4, mass_rel=1e-5, c_rel=1e-4, state_abs=1e-3)
FP64_TOL = dict(w_rel=1e-10, mass_rel=1e-12, c_rel=1e-11, state_abs=1e-8)


def tol_for(w):
    return FP64_TOL if w.precision == "fp64" else FP32_TOL


def npdtype(w):
    return np.float64 if w.precision == "fp64" else np.float32


@dataclass
class StageReport:
    ambiguous_selection: int = 0
    compared_labels: int = 0
    max_w_rel: float = 0.0
    max_mass_rel: float = 0.0
    max_state_err: float = 0.0
    max_c_rel: float = 0.0
    max_pred_abs: float = 0.0
    notes: List[str] = field(default_factory=list)


def check_weights(w_gpu, w_ref, tol, what=""):
    w_gpu = np.asarray(w_gpu, np.float64)
    w_ref = np.asarray(w_ref, np.float64)
    assert w_gpu.shape == w_ref.shape, (what, w_gpu.shape, w_ref.shape)
    if w_ref.size == 0:
        return 0.0
    floor = 1e-9 * max(w_ref.sum(), 1e-300) / w_ref.size
    err = np.abs(w_gpu - w_ref)
    ok = err <= tol["w_rel"] * np.abs(w_ref) + floor
    if not ok.all():
        i = int(np.argmax(err - tol["w_rel"] * np.abs(w_ref)))
        raise AssertionError(f"{what}: weight {i} gpu {w_gpu[i]!r} ref {w_ref[i]!r} "
                             f"({(~ok).sum()} of {ok.size} outside tolerance)")
    nz = np.abs(w_ref) > floor
    return float((err[nz] / np.abs(w_ref[nz])).max()) if nz.any() else 0.0


def gpu_stages(f, w, Z, noise, u, xu, path):
    """Run one step on the GPU and collect its intermediates.

    path "staged": phd_predict / phd_update / phd_extract / phd_resample with
    the intermediates read between the calls; path "fused" or "grid": one
    phd_step_inject on that path's step kernel, intermediates read
    afterwards."""
    dt = npdtype(w)
    g = {}
    g["xs0"], g["ws0"] = f.get_state()
    if path == "staged":
        f.predict(torch.as_tensor(noise).cuda())
        g["xp"], g["wp"] = f.get_state()
        f.update(torch.as_tensor(np.asarray(Z, dt)).cuda())
        g["C"], g["mass"] = f.get_update()
        _, g["wu"] = f.get_state()
        g["states"], g["labels"] = f.extract()
        g["loc_s"], g["loc_l"] = f.get_local_estimates()
        f.resample(u, xu)
    else:
        assert f.get_path() == path
        g["states"], g["labels"] = f.step_inject(np.asarray(Z, dt), noise, u, xu)
        g["xp"], g["wp"], g["wu"] = f.get_predicted()
        g["C"], g["mass"] = f.get_update()
        g["loc_s"], g["loc_l"] = f.get_local_estimates()
    g["par"], g["lx"] = f.get_resample()
    g["xr"], g["wr"] = f.get_state()
    return g


# ----------------------------------------------------------------------------
# One step from generator inputs on both sides
#
# The oracle never sees a GPU intermediate here: both implementations start
# from the same generator-made particle set and draws, and the oracle runs
# its own chain (predict -> update -> extraction -> resampling).  The inputs
# are dyadic (states on a 2^-8 m grid, normals on 2^-8, uniforms on 2^-12),
# for which the CV prediction and the uniform birth are exact in FP32, so the
# GPU's predicted set must equal the oracle's bit for bit and every later
# stage of both sides starts from the same numbers.  Resampling is compared
# by what is unique (the particle count, within the rounding of rho * N_k)
# and by validity (each parent's offspring count is floor or ceil of
# L w_i / W under the oracle's weights, to their tolerance; children are
# gathered copies; new weights N_k / L).
# ----------------------------------------------------------------------------

def dyadic(a, frac_bits):
    s = float(2 ** frac_bits)
    return np.round(np.asarray(a, np.float64) * s) / s


def exact_particles(rng, w, n, centres=None, spread=30.0, mass=1.0):
    x, wt = scenario.random_particles(rng, w, n, centres=centres, spread=spread, mass=mass)
    x = dyadic(x, 8)
    x[:, [1, 3]] = np.clip(x[:, [1, 3]], -127.0, 127.0)
    dt = npdtype(w)
    return x.astype(dt), wt.astype(dt)


def exact_noise(seed, step, K, pe_cap, dtype):
    nz = scenario.step_noise(seed, step, K, pe_cap, np.float64)
    nz[:, :2] = dyadic(np.clip(nz[:, :2], -7.99, 7.99), 8)
    nz[:, 2:] = np.minimum(dyadic(nz[:, 2:], 12), 1.0 - 2.0 ** -12)
    return nz.astype(dtype)


def check_offspring(par, L, w_ref, what=""):
    """Systematic resampling's unique property under the reference weights:
    every parent's offspring count is floor or ceil of L w_i / W (slack for
    the compared weights' tolerance); parents are non-decreasing."""
    par = np.asarray(par[:L])
    w_ref = np.asarray(w_ref, np.float64)
    assert L == 0 or (np.all(np.diff(par) >= 0) and par[0] >= 0 and par[-1] < len(w_ref)), what
    if L == 0:
        return
    o = np.bincount(par, minlength=len(w_ref))
    xexp = L * w_ref / w_ref.sum()
    lo = np.floor(xexp * (1 - 3e-4) - 1e-6)
    hi = np.ceil(xexp * (1 + 3e-4) + 1e-6)
    bad = (o < lo) | (o > hi)
    assert not bad.any(), (what, int(bad.sum()), np.flatnonzero(bad)[:5], o[bad][:5], xexp[bad][:5])


def check_step_from_inputs(w, m, x0, w0, Z, noise, u, xu, g, rep: StageReport, exact_predict=True,
                           check_resample=True):
    """Compare one GPU step (gpu_stages output g) with the oracle's own chain
    from the generator inputs x0, w0 (per PE) and the same draws."""
    tol = tol_for(w)
    K = w.num_pe
    dt = npdtype(w)
    kap = oracle.kappa(m)
    Zd = np.asarray(Z, np.float64)
    M = len(Zd)
    nz = np.asarray(noise, np.float64).reshape(K, w.pe_cap, 4)
    J = scenario.births_per_pe(w)
    # --- predict (Eq. 5-6)
    xo, wo = [], []
    for j in range(K):
        a, b = oracle.predict(m, np.asarray(x0[j], np.float64), np.asarray(w0[j], np.float64), J[j], nz[j])
        xo.append(a)
        wo.append(b)
        assert len(g["xp"][j]) == len(a), ("predicted count", j)
        if exact_predict:
            assert np.array_equal(np.asarray(g["xp"][j], np.float64), a), ("predicted states", j)
        else:
            np.testing.assert_allclose(g["xp"][j], a, rtol=0, atol=1e-3 if dt == np.float32 else 1e-9)
        check_weights(g["wp"][j], b, dict(w_rel=1e-6 if dt == np.float32 else 1e-14), f"predicted weights {j}")
    # --- update (Eq. 7-8)
    Cloc = [oracle.colsum(m, xo[j], wo[j], Zd) for j in range(K)]
    Cu = [np.mean(np.stack(Cloc), axis=0)] * K if (w.ck_mode == "global" and M) else Cloc
    wuo, Nko = [], []
    for j in range(K):
        if M:
            err = np.abs(g["C"][j, :M] - Cloc[j])
            big = Cloc[j] > 1e-3 * kap
            if big.any():
                rep.max_c_rel = max(rep.max_c_rel, float((err[big] / Cloc[j][big]).max()))
            bad = err > tol["c_rel"] * Cloc[j] + 1e-7 * kap
            assert not bad.any(), ("C", j, int(bad.sum()), err[bad][:3], Cloc[j][bad][:3])
        a = oracle.weight_update(m, xo[j], wo[j], Zd, Cu[j])
        wuo.append(a)
        rep.max_w_rel = max(rep.max_w_rel, check_weights(g["wu"][j], a, tol, f"updated weights {j}"))
        Nko.append(float(a.sum()))
        if Nko[j] > 0:
            rel = abs(g["mass"][j] - Nko[j]) / Nko[j]
            rep.max_mass_rel = max(rep.max_mass_rel, rel)
            assert rel <= tol["mass_rel"], ("mass", j, g["mass"][j], Nko[j])
    # --- local estimation (Step 3, Eq. 10-18) and fusion (Step 4)
    exs, ambiguous = [], False
    for j in range(K):
        ex = oracle.extract(m, xo[j], wo[j], Zd, Cu[j], Nko[j])
        exs.append(ex)
        got, want = list(g["loc_l"][j]), list(ex.labels)
        if got != want:
            dW = np.sort(ex.dW)[::-1]
            lt = max(len(got), len(want))
            Nk = Nko[j]
            near_half = abs(Nk - math.floor(Nk) - 0.5) < 1e-5 * max(1.0, Nk)
            near_tie = 0 < lt < len(dW) and abs(dW[lt - 1] - dW[lt]) <= 1e-6 * dW[lt - 1]
            assert near_half or near_tie, ("labels", j, got, want, Nk)
            rep.ambiguous_selection += 1
            ambiguous = True
        for r, p in enumerate(got):
            if p in want:
                e = np.abs(np.asarray(g["loc_s"][j][r], np.float64) - ex.zeta[want.index(p)]).max()
                rep.max_state_err = max(rep.max_state_err, float(e))
                assert e <= tol["state_abs"], ("state", j, p, g["loc_s"][j][r], ex.zeta[want.index(p)])
                rep.compared_labels += 1
    fl, fz = oracle.fuse(exs, M)
    gl = list(np.asarray(g["labels"].cpu()))
    if not ambiguous:
        assert gl == list(fl), (gl, list(fl))
        np.testing.assert_allclose(np.asarray(g["states"].cpu(), np.float64), fz, rtol=0,
                                   atol=tol["state_abs"])
    # --- resampling (Sec. 2.2 step 3; Step 5) and exchange (Step 6): by what
    # is unique (counts) and validity (offspring, gather, weights, union)
    if not check_resample:
        return
    par, lx, xr, wr = g["par"], g["lx"], g["xr"], g["wr"]
    pre, pre_w, Lo_all = [], [], []
    for j in range(K):
        L = len(xr[j])
        lmax = w.pe_cap - J[j]
        Lo = min(lmax, int(math.floor(w.particles_per_target / K * max(1.0, Nko[j]) + 0.5)))
        Lg = min(lmax, int(math.floor(w.particles_per_target / K * max(1.0, float(g["mass"][j])) + 0.5)))
        assert L == Lg and abs(L - Lo) <= 1, ("resample count", j, L, Lg, Lo)
        Lo_all.append(Lo)
        if L != Lo:
            rep.notes.append(f"PE {j}: rho N_k within rounding of a .5 boundary ({L} vs {Lo})")
        check_offspring(par[j], L, wuo[j], f"PE {j}")
        xg = np.asarray(g["xp"][j])[par[j][:L]]
        pre.append(xg)
        # new weights N_j / L_j before the exchange moves some of them
        pre_w.append(np.full(L, float(g["mass"][j]) / L if L else 0.0))

    def check_new_weights(want_w):
        for j in range(K):
            if len(want_w[j]):
                np.testing.assert_allclose(np.asarray(wr[j], np.float64), want_w[j],
                                           rtol=1e-6 if dt == np.float32 else 1e-14)
    if K > 1 and w.exchange_frac > 0:
        # Step 6: the count and the trigger from the oracle's own masses and
        # counts, the slots from the oracle's slot function on the injected
        # draws; PE j's t-th chosen particle lands in the receiver's t-th slot
        counts = Lo_all
        if [len(a) for a in xr] != counts:
            # a count at a rounding boundary: the exchange is checked by its
            # invariants (slice sizes, the union of all particles)
            key = lambda arrs: np.sort(np.concatenate(arrs).view(
                np.dtype((np.void, np.dtype(dt).itemsize * 4))).ravel())
            assert np.array_equal(key([np.ascontiguousarray(a) for a in xr]),
                                  key([np.ascontiguousarray(a) for a in pre]))
            tot = lambda arrs: sum(float(np.sum(np.asarray(a, np.float64))) for a in arrs)
            assert abs(tot(wr) - tot(pre_w)) <= 1e-5 * max(tot(pre_w), 1e-300)
            return
        due = True
        if w.exchange_threshold > 0:
            mn, mean = min(Nko), sum(Nko) / K
            near = abs(mn - w.exchange_threshold * mean) <= 1e-4 * max(mean, 1e-300)
            due = mn < w.exchange_threshold * mean
            if near:
                due = lx > 0
        Lx = int(math.floor(w.exchange_frac * min(counts))) if due else 0
        assert lx == Lx, ("exchange count", lx, Lx)
        slots = [oracle.exchange_slots(counts[j], Lx, np.asarray(xu, np.uint32).reshape(K, -1)[j]) for j in range(K)]
        want = [np.array(a, copy=True) for a in pre]
        want_w = [np.array(a, copy=True) for a in pre_w]
        for j in range(K):
            for t in range(Lx):
                shift = 1 + t % (K - 1) if (w.exchange_mode == "all" and K > 2) else 1
                k = (j + shift) % K
                want[k][slots[k][t]] = pre[j][slots[j][t]]
                want_w[k][slots[k][t]] = pre_w[j][slots[j][t]]
        for j in range(K):
            assert np.array_equal(np.asarray(xr[j]), want[j]), ("exchange", j)
        check_new_weights(want_w)
    else:
        for j in range(K):
            assert np.array_equal(np.asarray(xr[j]), pre[j])
        check_new_weights(pre_w)


def exact_state(w, seed, n_per_pe, centres=None, spread=25.0, mass=3.0, resampled=False):
    """Generator particle slices for K PEs (dyadic, see exact_particles); with
    `resampled` each slice looks like a resampling output: equal weights and
    runs of duplicated states."""
    rng = np.random.default_rng(seed)
    xs, ws = [], []
    for j in range(w.num_pe):
        n = n_per_pe[j] if isinstance(n_per_pe, (list, tuple)) else n_per_pe
        x, wt = exact_particles(rng, w, n, centres=centres, spread=spread, mass=mass)
        if resampled and n > 1:
            src = np.sort(rng.integers(0, max(1, n // 3), size=n))
            x = x[src]
            wt = np.full(n, mass / n, dtype=wt.dtype)
        xs.append(x)
        ws.append(wt)
    return xs, ws


def stage_step(f, w, m, x0, w0, Z, noise, u, xu, rep: StageReport, path="staged", exact_predict=True,
               check_resample=True):
    """Load the generator state (x0, w0) into the GPU filter, run one step with
    the injected draws, and compare every stage with the oracle's own chain
    from the same state."""
    f.set_state(x0, w0)
    g = gpu_stages(f, w, Z, noise, u, xu, path)
    check_step_from_inputs(w, m, x0, w0, Z, noise, u, xu, g, rep, exact_predict, check_resample)
    return g
