"""The learned birth proposal's training loop (Eq. 6 with p_k(.|Z_k) a
mixture over the scan), on the library's own kernels.

The network sees one measurement at a time (its position in the plane scaled
to the birth region and the log1p count of its neighbours, phd_birth_features)
and is fit to what the plain filter itself produces: for every measurement of
every scan, whether the filter extracted an estimate for it (its label was
selected, Eq. 16-18) and, if so, the estimate's velocity.  Training is Adam on
the mean loss of phd_mlp_grad (cross-entropy of the "extracted" flag plus the
Gaussian negative log-likelihood of the extracted velocity), entirely on the
GPU (phd_mlp_grad, phd_mlp_adam); the trained parameters are loaded into a
filter with ParticlePHD.set_birth_proposal.
"""
from __future__ import annotations

import math
from typing import Iterable, Optional, Tuple

import torch

from .phd import MlpTrainer, ParticlePHD, birth_features, mlp_nparams

NH, NIN, NOUT = 64, 3, 5


def init_params(seed: int = 0, device: str = "cuda") -> torch.Tensor:
    """Seeded start for training: fan-in scaled normal weights, zero biases,
    and a near-zero output layer, so the untrained head is about
    (m, l, logit) = 0: velocity N(0, s_b^2) per axis (the plain birth's) and
    equal mixture weights."""
    g = torch.Generator().manual_seed(int(seed))
    W1 = torch.randn(NH, NIN, generator=g) / math.sqrt(NIN)
    W2 = torch.randn(NH, NH, generator=g) / math.sqrt(NH)
    W3 = torch.randn(NOUT, NH, generator=g) * (0.01 / math.sqrt(NH))
    p = torch.cat([W1.ravel(), torch.zeros(NH), W2.ravel(), torch.zeros(NH), W3.ravel(), torch.zeros(NOUT)])
    assert p.numel() == mlp_nparams()
    return p.to(device=device, dtype=torch.float32).contiguous()


def collect_pairs(f: ParticlePHD, scans: Iterable, reset: bool = True) -> Tuple[torch.Tensor, torch.Tensor]:
    """Run the filter (as configured: normally the plain birth) over the scans
    and return the training set on its device: X[n][3] network inputs of
    every measurement, T[n][3] = (t, vx, vy) with t = 1 for the measurements
    whose label the filter extracted (vx, vy its estimate's velocity)."""
    if reset:
        f.set_state([torch.zeros((0, 4))] * f.K, [torch.zeros(0)] * f.K)
    xs, ts = [], []
    for Z in scans:
        Zt = torch.as_tensor(Z, dtype=torch.float32, device=f.device).reshape(-1, 2).contiguous()
        states, labels = f.step(Zt, cap=f.m_max)[:2]
        M = int(Zt.shape[0])
        if M == 0:
            continue
        X = birth_features(f.cfg, Zt)
        T = torch.zeros((M, 3), dtype=torch.float32, device=f.device)
        if labels.numel():
            lab = labels.long()
            T[lab, 0] = 1.0
            T[lab, 1] = states[:, 1].to(torch.float32)
            T[lab, 2] = states[:, 3].to(torch.float32)
        xs.append(X)
        ts.append(T)
    return torch.cat(xs), torch.cat(ts)


def train(X: torch.Tensor, T: torch.Tensor, steps: int = 1500, batch: int = 4096, lr: float = 2e-3,
          vel_scale: float = 20.0, seed: int = 0, params: Optional[torch.Tensor] = None,
          log_every: int = 0) -> Tuple[torch.Tensor, list]:
    """Adam on minibatches drawn (seeded, with replacement) from (X, T);
    returns the trained FP32 parameters and the loss trace (every log_every
    steps, the minibatch loss)."""
    n = int(X.shape[0])
    assert n > 0 and T.shape == (n, 3)
    p0 = init_params(seed, device=str(X.device)) if params is None else params
    b = min(batch, n)
    tr = MlpTrainer(p0, batch_max=b, lr=lr, vel_scale=vel_scale)
    g = torch.Generator(device=X.device).manual_seed(int(seed) + 1)
    trace = []
    for k in range(steps):
        idx = torch.randint(0, n, (b,), generator=g, device=X.device)
        tr.step(X.index_select(0, idx).contiguous(), T.index_select(0, idx).contiguous())
        if log_every and (k % log_every == 0 or k == steps - 1):
            trace.append((k, float(tr.loss.item())))
    return tr.params, trace


def full_loss(params: torch.Tensor, X: torch.Tensor, T: torch.Tensor, vel_scale: float = 20.0,
              chunk: int = 65536) -> float:
    """Mean loss of the parameters over the whole set (phd_mlp_grad in chunks)."""
    n = int(X.shape[0])
    tr = MlpTrainer(params, batch_max=min(chunk, n), vel_scale=vel_scale)
    total = 0.0
    for a in range(0, n, chunk):
        e = min(n, a + chunk)
        tr.grad_of(X[a:e].contiguous(), T[a:e].contiguous())
        total += float(tr.loss.item()) * (e - a)
    return total / n
