"""What the trained birth network gains over the plain birth (Eq. 6 with a
learned, measurement-driven proposal vs the uniform one), end to end on the
GPU: the network is trained by the library's own kernels on (measurement,
extracted estimate) pairs that the plain filter produced on dense
range-bearing runs (100 targets, clutter 500), then three filters track the
50-target range-bearing scenario (clutter 100, 1000 particles per target):
plain birth with 5000 and 20000 birth particles, and the learned proposal
with 5000.  Scored by OSPA (c = 100 m, p = 2) of the extracted positions
against the truth and by the cardinality error, averaged over steps and
seeds.  The birth intensity of both scenarios is matched to their truth
birth rate (the same for every filter)."""
import numpy as np
import pytest
import torch

import oracle
import scenario

pytestmark = pytest.mark.gpu


def _track(w, seeds, params=None, alpha=0.1, steps=None):
    from paper_1503_03769_gb300 import ParticlePHD
    ospa, card = [], []
    for s in seeds:
        sc = scenario.simulate(w, s, steps=steps or w.steps)
        f = ParticlePHD(w, seed=s, device="cuda:0")
        if params is not None:
            f.set_birth_proposal(params, alpha)
        for k in range(len(sc.meas)):
            states, labels = f.step(sc.meas[k])
            est = states.cpu().numpy().astype(np.float64)[:, [0, 2]]
            tru = sc.truth[k][:, [0, 2]] if len(sc.truth[k]) else np.zeros((0, 2))
            ospa.append(oracle.ospa(est, tru, c=100.0, p=2.0))
            card.append(abs(len(est) - len(tru)))
        f.close()
    return float(np.mean(ospa)), float(np.mean(card))


def test_trained_proposal_beats_plain_birth():
    from paper_1503_03769_gb300 import ParticlePHD, proposal
    # birth intensity nu_b matched to each scenario's truth birth rate
    # (targets born uniformly over the first 40 % of the scans)
    nu = lambda w: w.n_targets / (0.4 * w.steps)
    wtrain = scenario.workload("dense_rb_100t")
    wtrain = wtrain.with_(birth_mass=nu(wtrain))
    f = ParticlePHD(wtrain, seed=2000, device="cuda:0")
    Xs, Ts = [], []
    for s in (2000, 2001):
        sc = scenario.simulate(wtrain, s)
        X, T = proposal.collect_pairs(f, sc.meas)
        Xs.append(X)
        Ts.append(T)
    f.close()
    X, T = torch.cat(Xs), torch.cat(Ts)
    pos = float(T[:, 0].mean())
    print(f"training set: {X.shape[0]} measurements, {pos:.4f} extracted")
    assert X.shape[0] > 50_000 and 0.005 < pos < 0.5
    l0 = proposal.full_loss(proposal.init_params(0), X, T)
    params, trace = proposal.train(X, T, steps=1500, batch=4096, lr=2e-3, seed=0, log_every=500)
    l1 = proposal.full_loss(params, X, T)
    assert l1 < 0.9 * l0, (l0, l1)

    w5 = scenario.workload("rb_50t")
    w5 = w5.with_(birth_mass=nu(w5))
    w20 = scenario.workload("rb_50t", birth_count=20000, birth_mass=w5.birth_mass)
    seeds = (3000, 3001, 3002)
    o_plain, c_plain = _track(w5, seeds)
    o_plain4, c_plain4 = _track(w20, seeds)
    o_learn, c_learn = _track(w5, seeds, params=params)
    print(f"OSPA plain 5k {o_plain:.2f} (card err {c_plain:.2f}), plain 20k {o_plain4:.2f} ({c_plain4:.2f}), "
          f"learned 5k {o_learn:.2f} ({c_learn:.2f}); loss {l0:.3f} -> {l1:.3f}")
    assert o_learn < 0.9 * o_plain          # the gain at equal birth count
    assert o_learn <= o_plain4              # at least as good as 4x the plain births
    assert c_learn < c_plain
