"""Helpers for the GPU parity tests: stage-by-stage comparison of libphd.so
against the FP64 oracle on the same injected random numbers.

At every stage the oracle is fed the GPU's own input state (the GPU's
predicted set for the update, the GPU's updated weights for resampling), so
each comparison isolates one stage; tolerances are the ones the filter is
specified to: weights 1e-4 relative (plus a 1e-9 * mean-weight floor for
weights that FP32's exp2 flushes to zero), masses 1e-5 relative, extracted
states 1e-3 m, resampling parents and exchange moves bit-exact.
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
    the intermediates read between the calls; path "fused": one
    phd_step_inject on the fused kernel, intermediates read afterwards."""
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
        assert f.get_path() == "fused"
        g["states"], g["labels"] = f.step_inject(np.asarray(Z, dt), noise, u, xu)
        g["xp"], g["wp"], g["wu"] = f.get_predicted()
        g["C"], g["mass"] = f.get_update()
        g["loc_s"], g["loc_l"] = f.get_local_estimates()
    g["par"], g["lx"] = f.get_resample()
    g["xr"], g["wr"] = f.get_state()
    return g


def check_step(w, m, Z, noise, u, xu, g, rep: StageReport, check_resample=True):
    """Compare one step's GPU intermediates with the oracle, stage by stage,
    the oracle always starting from the GPU's own input to that stage."""
    tol = tol_for(w)
    K = w.num_pe
    dt = npdtype(w)
    kap = oracle.kappa(m)
    xs0, ws0, xp, wp, wu = g["xs0"], g["ws0"], g["xp"], g["wp"], g["wu"]
    # --- predict (Eq. 5-6)
    nz = np.asarray(noise, np.float64).reshape(K, w.pe_cap, 4)
    for j in range(K):
        Jj = scenario.births_per_pe(w)[j]
        xo, wo = oracle.predict(m, xs0[j], ws0[j], Jj, nz[j])
        assert len(xp[j]) == len(xo), ("predicted count", j, len(xs0[j]), Jj, len(xp[j]), len(xo))
        # FP32 rounding of x + T vx + T^2/2 a: a few ulp of |x| <= 2e3 m
        atol = 1e-3 if dt == np.float32 else 1e-9
        np.testing.assert_allclose(xp[j], xo, rtol=0, atol=atol)
        if len(xo):
            rep.max_pred_abs = max(rep.max_pred_abs, float(np.abs(np.asarray(xp[j], np.float64) - xo).max()))
        check_weights(wp[j], wo, tol, f"predict PE {j}")
    # --- update (Eq. 7-8)
    C, mass = g["C"], g["mass"]
    M = len(Z)
    Zd = np.asarray(Z, np.float64)
    Cloc = [oracle.colsum(m, xp[j], wp[j], Zd) for j in range(K)]
    if getattr(w, "ck_mode", "local") == "global" and M:
        Cu = [np.mean(np.stack(Cloc), axis=0)] * K
    else:
        Cu = Cloc
    for j in range(K):
        if M:
            # C matters to the filter through C / (kappa + C): an absolute slack of
            # 1e-7 kappa per measurement moves the mass by at most 1e-7 per label
            err = np.abs(C[j, :M] - Cloc[j])
            big = Cloc[j] > 1e-3 * kap   # relative error where C is not negligible against kappa
            if big.any():
                rep.max_c_rel = max(rep.max_c_rel, float((err[big] / Cloc[j][big]).max()))
            bad = err > tol["c_rel"] * Cloc[j] + 1e-7 * kap
            assert not bad.any(), (j, int(bad.sum()), err[bad][:3], Cloc[j][bad][:3], kap)
        wo = oracle.weight_update(m, xp[j], wp[j], Zd, Cu[j])
        rep.max_w_rel = max(rep.max_w_rel, check_weights(wu[j], wo, tol, f"update PE {j}"))
        Nref = wo.sum()
        if Nref > 0:
            rel = abs(mass[j] - Nref) / Nref
            rep.max_mass_rel = max(rep.max_mass_rel, rel)
            assert rel <= tol["mass_rel"], (j, mass[j], Nref)
    # --- extraction (Eq. 10-18) and fusion (Step 4)
    loc_s, loc_l = g["loc_s"], g["loc_l"]
    for j in range(K):
        Nk = float(wu[j].astype(np.float64).sum())
        ex = oracle.extract(m, xp[j], wp[j], Zd, Cu[j], Nk)
        got = list(loc_l[j])
        want = list(ex.labels)
        if got != want:
            # acceptable only at a genuine tie: LT near a .5 boundary or the
            # boundary dW values within 1e-6 relative
            dW = np.sort(ex.dW)[::-1]
            lt = max(len(got), len(want))
            near_half = abs(Nk - math.floor(Nk) - 0.5) < 1e-5 * max(1.0, Nk)
            near_tie = 0 < lt < len(dW) and abs(dW[lt - 1] - dW[lt]) <= 1e-6 * dW[lt - 1]
            assert near_half or near_tie, (j, got, want, Nk)
            rep.ambiguous_selection += 1
        for r, p in enumerate(got):
            if p in want:
                zi = ex.zeta[want.index(p)]
                e = np.abs(loc_s[j][r].astype(np.float64) - zi).max()
                rep.max_state_err = max(rep.max_state_err, float(e))
                assert e <= tol["state_abs"], (j, p, loc_s[j][r], zi)
                rep.compared_labels += 1
    # fusion of the GPU's own local estimates (identical inputs)
    gl = [oracle.Extraction(np.asarray(loc_l[j], np.int32), np.asarray(loc_s[j], np.float64),
                            np.zeros(M), 0.0, len(loc_l[j])) for j in range(K)]
    fl, fz = oracle.fuse(gl, M)
    assert list(g["labels"].cpu().numpy()) == list(fl), (g["labels"], fl)
    np.testing.assert_allclose(g["states"].cpu().numpy().astype(np.float64), fz,
                               rtol=0, atol=1e-4 if dt == np.float32 else 1e-9)
    # --- resampling (exact CDF) + ring exchange
    if not check_resample:
        return
    par, lx, xr, wr = g["par"], g["lx"], g["xr"], g["wr"]
    rxs, rws = [], []
    for j in range(K):
        rho = w.particles_per_target / K
        lmax = w.pe_cap - scenario.births_per_pe(w)[j]
        xo, wo, po = oracle.resample(xp[j], wu[j].astype(np.float64), rho, lmax, int(u[j]))
        assert np.array_equal(par[j, :len(po)], po), f"resample parents differ on PE {j}"
        rxs.append(xo)
        rws.append(wo)
    if K > 1 and w.exchange_frac > 0:
        # the exchange stage's input: the resampled slices and, for the
        # adaptive trigger, the PE masses the GPU's update produced
        rxs, rws, slots = oracle.exchange(rxs, rws, w.exchange_frac, xu, w.exchange_mode,
                                          w.exchange_threshold, np.asarray(mass, np.float64)[:K])
        assert lx == slots.shape[1]
    for j in range(K):
        assert len(xr[j]) == len(rxs[j])
        np.testing.assert_array_equal(xr[j].astype(np.float64), rxs[j].astype(dt).astype(np.float64))
        check_weights(wr[j], rws[j], tol, f"resampled weights PE {j}")


def stage_step(f, w, m, Z, noise, u, xu, rep: StageReport, check_resample=True, path="staged"):
    """One filter step on the GPU with every stage compared to the oracle."""
    g = gpu_stages(f, w, Z, noise, u, xu, path)
    check_step(w, m, Z, noise, u, xu, g, rep, check_resample)
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
    pre = []
    for j in range(K):
        L = len(xr[j])
        lmax = w.pe_cap - J[j]
        Lo = min(lmax, int(math.floor(w.particles_per_target / K * max(1.0, Nko[j]) + 0.5)))
        Lg = min(lmax, int(math.floor(w.particles_per_target / K * max(1.0, float(g["mass"][j])) + 0.5)))
        assert L == Lg and abs(L - Lo) <= 1, ("resample count", j, L, Lg, Lo)
        check_offspring(par[j], L, wuo[j], f"PE {j}")
        xg = np.asarray(g["xp"][j])[par[j][:L]]
        pre.append(xg)
        nw = float(g["mass"][j]) / L if L else 0.0
        if L:
            np.testing.assert_allclose(np.asarray(wr[j], np.float64), nw, rtol=1e-6 if dt == np.float32 else 1e-14)
    if K > 1 and w.exchange_frac > 0:
        moved = 0
        for j in range(K):
            moved += int((np.asarray(xr[j]) != pre[j]).any(axis=1).sum())
        assert lx == int(math.floor(w.exchange_frac * min(len(a) for a in xr))) or lx == 0
        assert moved <= K * lx
        key = lambda arrs: np.sort(np.concatenate(arrs).view(np.dtype((np.void, np.dtype(dt).itemsize * 4))).ravel())
        assert np.array_equal(key([np.ascontiguousarray(a) for a in xr]), key([np.ascontiguousarray(a) for a in pre]))
    else:
        for j in range(K):
            assert np.array_equal(np.asarray(xr[j]), pre[j])
