"""FP64 CPU oracle of the particle PHD filter (TEST INFRASTRUCTURE ONLY).

Only tests/, the package smoke check and the benchmark's CPU-baseline leg may
import this module.  It shares no code with the CUDA path: the arithmetic is
in `phd_oracle.c` (plain C, IEEE double, built with FMA contraction off so the
results do not depend on the host's instruction set), driven from here with
numpy arrays.  `OracleFilter` strings the stages together in the order of the
paper's Algorithm 1 (predict, update, local estimation and fusion, resample,
exchange); OSPA (the metric of Sec. 4.1) is computed with an optimal
assignment.

Readings of the paper taken here (each also stated in the C source):
 * Eq. 7 is <psi_z, D> (the trailing "* x" is a typo); nu = 1 - p_D.
 * Births: p_k(.|Z) = U(region) x N(0, s_b^2 I), weight nu_b / J.
 * Distributed form: each PE is a full local filter over its slice (births
   split J/K per PE with weight nu_b / J_j), uses its local C^j ("local"
   mode) or the mean of the PEs' C^j ("global" mode), resamples to
   round((rho / K) * max(1, N^j)) particles and sends floor(frac * min_j n_j)
   random particles to the next PE on the ring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "phd_oracle.c"), os.path.join(_HERE, "birth_oracle.c")]
_DEPS = _SRCS + [os.path.join(_HERE, "orc_model.h")]
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}
_threads = 1

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def _build_one(path: str, extra, force: bool) -> str:
    stale = not os.path.exists(path) or any(os.path.getmtime(path) < os.path.getmtime(p) for p in _DEPS)
    if force or stale:
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, *extra, "-I", _HERE, *_SRCS, "-o", tmp, "-lm"])
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into liboracle.so beside them (gcc, no
    CUDA), and the same sources with OpenMP into liboracle_omp.so when the
    compiler supports it (see set_threads)."""
    _build_one(_LIB, [], force)
    try:
        _build_one(_LIB_OMP, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass
    return _LIB


def openmp_available() -> bool:
    try:
        _build_one(_LIB_OMP, ["-fopenmp"], False)
        return True
    except (subprocess.CalledProcessError, OSError):
        return False


def set_threads(n: int) -> int:
    """Run the oracle's stage loops on n host threads (the OpenMP build, whose
    results are bit-identical to the single-threaded build's); n <= 1 selects
    the single-threaded build.  Returns the thread count in effect."""
    global _threads
    n = int(n)
    if n > 1 and openmp_available():
        L = _load(_LIB_OMP)
        L.orc_set_threads(n)
        _threads = n
    else:
        _threads = 1
    return _threads


def threads() -> int:
    return _threads


class _Model(ctypes.Structure):
    _fields_ = [
        ("meas_model", ctypes.c_int), ("birth_model", ctypes.c_int),
        ("dt", ctypes.c_double), ("sigma_a", ctypes.c_double),
        ("sigma_z", ctypes.c_double * 2), ("sensor", ctypes.c_double * 2),
        ("region", ctypes.c_double * 4), ("r_max", ctypes.c_double),
        ("p_s", ctypes.c_double), ("p_d", ctypes.c_double),
        ("clutter_rate", ctypes.c_double), ("birth_mass", ctypes.c_double),
        ("birth_vel_sigma", ctypes.c_double),
        ("sigma_a_y", ctypes.c_double), ("theta_span", ctypes.c_double),
        ("birth_mean", ctypes.c_double * 4), ("birth_std", ctypes.c_double * 4),
        ("gate_sigma", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U = ctypes.POINTER(ctypes.c_uint32)
_M = ctypes.POINTER(_Model)


def lib():
    """The oracle library in use: single-threaded unless set_threads(n > 1)."""
    if _threads > 1:
        return _load(_LIB_OMP)
    if _LIB not in _libs:
        build()
    return _load(_LIB)


def _load(path):
    with _lock:
        if path not in _libs:
            L = ctypes.CDLL(path)
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_is_parallel.restype = ctypes.c_int
            L.orc_kappa.restype = ctypes.c_double
            L.orc_kappa.argtypes = [_M]
            L.orc_measure.argtypes = [_M, _D, _D]
            L.orc_likelihood.restype = ctypes.c_double
            L.orc_likelihood.argtypes = [_M, _D, _D]
            L.orc_predict.argtypes = [_M, _D, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D]
            L.orc_colsum.argtypes = [_M, _D, _D, ctypes.c_int, _D, ctypes.c_int, _D]
            L.orc_weight_update.argtypes = [_M, _D, _D, ctypes.c_int, _D, ctypes.c_int, _D, _D]
            L.orc_extract.restype = ctypes.c_int
            L.orc_extract.argtypes = [_M, _D, _D, ctypes.c_int, _D, ctypes.c_int, _D,
                                      ctypes.c_double, _I, _D, _D, _D]
            L.orc_resample.restype = ctypes.c_int
            L.orc_resample.argtypes = [_D, _D, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_uint32, _D, _D, _I]
            L.orc_exchange_slots.argtypes = [ctypes.c_int, ctypes.c_int, _U, _I]
            L.orc_exchange_ex.restype = ctypes.c_int
            L.orc_exchange_ex.argtypes = [ctypes.c_int, _D, _D, _I, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_double, _D, _U, _I]
            L.orc_exchange.argtypes = [ctypes.c_int, _D, _D, _I, ctypes.c_int, ctypes.c_double,
                                       _U, _I]
            L.orc_fuse.restype = ctypes.c_int
            L.orc_fuse.argtypes = [ctypes.c_int, _I, _I, _D, ctypes.c_int, ctypes.c_int, _I, _D]
            L.orc_mlp_nparams.restype = ctypes.c_int
            L.orc_gelu.restype = ctypes.c_double
            L.orc_gelu.argtypes = [ctypes.c_double]
            L.orc_gelu_grad.restype = ctypes.c_double
            L.orc_gelu_grad.argtypes = [ctypes.c_double]
            L.orc_birth_features.argtypes = [_M, _D, ctypes.c_int, _D]
            L.orc_mlp_forward.argtypes = [_D, _D, ctypes.c_int, _D]
            L.orc_mlp_loss_grad.restype = ctypes.c_double
            L.orc_mlp_loss_grad.argtypes = [_D, _D, _D, ctypes.c_int, ctypes.c_double, _D]
            L.orc_birth_learned.argtypes = [_M, _D, ctypes.c_int, _D, ctypes.c_double, ctypes.c_int,
                                            _D, _D, _D, _D, _I]
            L.orc_birth_cdf.argtypes = [_M, _D, ctypes.c_int, _D]
            _libs[path] = L
    return _libs[path]


def _d(a):
    return a.ctypes.data_as(_D)


def _i(a):
    return a.ctypes.data_as(_I)


def _u(a):
    return a.ctypes.data_as(_U)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def model(w) -> _Model:
    """Oracle model struct from a scenario.Workload (or any object with its fields)."""
    m = _Model()
    m.meas_model = 0 if w.meas_model == "linear" else 1
    m.dt, m.sigma_a = float(w.dt), float(w.sigma_a)
    m.sigma_z[0], m.sigma_z[1] = float(w.sigma_z[0]), float(w.sigma_z[1])
    m.sensor[0], m.sensor[1] = float(w.sensor[0]), float(w.sensor[1])
    for k in range(4):
        m.region[k] = float(w.region[k])
    m.r_max = float(w.r_max)
    m.p_s, m.p_d = float(w.p_s), float(w.p_d)
    m.clutter_rate, m.birth_mass = float(w.clutter_rate), float(w.birth_mass)
    m.birth_vel_sigma = float(w.birth_vel_sigma)
    m.sigma_a_y = float(getattr(w, "sigma_a_y", 0.0))
    m.theta_span = float(getattr(w, "theta_span", 0.0))
    m.birth_model = 1 if getattr(w, "birth_model", "uniform") == "gaussian" else 0
    for k, v in enumerate(getattr(w, "birth_mean", (0.0,) * 4)):
        m.birth_mean[k] = float(v)
    for k, v in enumerate(getattr(w, "birth_std", (0.0,) * 4)):
        m.birth_std[k] = float(v)
    m.gate_sigma = float(getattr(w, "gate_sigma", 0.0))
    return m


# ----------------------------------------------------------------------------
# Stage wrappers (numpy in, numpy out)
# ----------------------------------------------------------------------------

def kappa(m: _Model) -> float:
    return lib().orc_kappa(ctypes.byref(m))


def measure(m: _Model, x) -> np.ndarray:
    x = _f64(x, (-1, 4))
    out = np.empty((len(x), 2))
    for i in range(len(x)):
        lib().orc_measure(ctypes.byref(m), _d(x[i]), _d(out[i]))
    return out


def likelihood(m: _Model, z, x) -> float:
    z, x = _f64(z, (2,)), _f64(x, (4,))
    return lib().orc_likelihood(ctypes.byref(m), _d(z), _d(x))


def predict(m: _Model, x, w, J: int, noise):
    """Eq. 5-6: survivors (len(x)) then J births; noise rows (n1, n2, u1, u2)."""
    x, w = _f64(x, (-1, 4)), _f64(w, (-1,))
    L = len(x)
    noise = _f64(noise, (-1, 4))
    assert len(noise) >= L + J
    xo, wo = np.empty((L + J, 4)), np.empty(L + J)
    lib().orc_predict(ctypes.byref(m), _d(x), _d(w), L, J, _d(noise), _d(xo), _d(wo))
    return xo, wo


def colsum(m: _Model, x, w, Z) -> np.ndarray:
    """Eq. 7: C(z_p) = sum_j p_D g(z_p|x_j) w_j."""
    x, w, Z = _f64(x, (-1, 4)), _f64(w, (-1,)), _f64(Z, (-1, 2))
    C = np.empty(len(Z))
    lib().orc_colsum(ctypes.byref(m), _d(x), _d(w), len(x), _d(Z), len(Z), _d(C))
    return C


def weight_update(m: _Model, x, w, Z, C_used) -> np.ndarray:
    """Eq. 8 with nu = 1 - p_D."""
    x, w, Z, C_used = _f64(x, (-1, 4)), _f64(w, (-1,)), _f64(Z, (-1, 2)), _f64(C_used, (-1,))
    out = np.empty(len(x))
    lib().orc_weight_update(ctypes.byref(m), _d(x), _d(w), len(x), _d(Z), len(Z),
                            _d(C_used), _d(out))
    return out


@dataclass
class Extraction:
    labels: np.ndarray     # selection order: descending dW, ties by label
    zeta: np.ndarray       # (n, 4)
    dW: np.ndarray         # (M,) sub-weight mass per measurement (Eq. 16)
    dW0: float             # missed-detection sub-weight mass (Eq. 17)
    LT: int                # round(N_k) before the caps


def extract(m: _Model, x, w_pred, Z, C_used, Nk: float) -> Extraction:
    """Eq. 10-18 and Step 3: LT = round(N_k), top-LT dW^p, zeta_p (Eq. 18)."""
    x, w_pred, Z, C_used = (_f64(x, (-1, 4)), _f64(w_pred, (-1,)), _f64(Z, (-1, 2)),
                            _f64(C_used, (-1,)))
    M = len(Z)
    labels = np.empty(max(M, 1), dtype=np.int32)
    zeta = np.empty((max(M, 1), 4))
    dW = np.empty(max(M, 1))
    dW0 = np.empty(1)
    n = lib().orc_extract(ctypes.byref(m), _d(x), _d(w_pred), len(x), _d(Z), M, _d(C_used),
                          float(Nk), _i(labels), _d(zeta), _d(dW), _d(dW0))
    return Extraction(labels[:n].copy(), zeta[:n].copy(), dW[:M].copy(), float(dW0[0]),
                      int(np.floor(Nk + 0.5)))


def resample(x, w, rho: float, l_max: int, U: int):
    """Systematic resampling with the exact integer-valued CDF; returns (x, w, parent)."""
    x, w = _f64(x, (-1, 4)), _f64(w, (-1,))
    N = len(x)
    Nk = float(w.sum()) if N else 0.0
    cap = int(min(l_max, max(0, np.floor(rho * max(1.0, Nk) + 0.5) + 1)))
    cap = max(cap, 1)
    xo, wo = np.empty((cap, 4)), np.empty(cap)
    par = np.empty(cap, dtype=np.int32)
    L = lib().orc_resample(_d(x), _d(w), N, float(rho), int(l_max), int(U) & 0xFFFFFFFF,
                           _d(xo), _d(wo), _i(par))
    assert L <= cap
    return xo[:L].copy(), wo[:L].copy(), par[:L].copy()


def exchange_slots(n: int, count: int, u) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.uint32))
    slots = np.empty(max(count, 1), dtype=np.int32)
    lib().orc_exchange_slots(int(n), int(count), _u(u), _i(slots))
    return slots[:count].copy()


def exchange(xs: List[np.ndarray], ws: List[np.ndarray], frac: float, u, mode: str = "ring",
             threshold: float = 0.0, masses=None) -> tuple:
    """Step 6 exchange over K slices (ring, or "all" to all; with threshold > 0
    only when min_j N_j < threshold * mean_j N_j for the PE masses N_j);
    returns new (xs, ws, slots), slots [K][L_x] (L_x = 0 when it did not run)."""
    K = len(xs)
    counts = np.asarray([len(a) for a in xs], dtype=np.int32)
    u = np.ascontiguousarray(np.asarray(u, dtype=np.uint32))
    stride = u.shape[1]
    assert counts.max(initial=0) <= stride
    X = np.zeros((K, stride, 4))
    W = np.zeros((K, stride))
    for j in range(K):
        X[j, :counts[j]] = xs[j]
        W[j, :counts[j]] = ws[j]
    nmin = int(counts.min()) if K else 0
    cap = int(np.floor(frac * nmin)) if K > 1 else 0
    slots = np.zeros((K, max(cap, 1)), dtype=np.int32)
    mass = _f64(masses if masses is not None else np.zeros(max(K, 1)), (-1,))
    Lx = lib().orc_exchange_ex(K, _d(X), _d(W), _i(counts), stride, float(frac), 1 if mode == "all" else 0,
                               float(threshold), _d(mass), _u(u), _i(slots))
    return ([X[j, :counts[j]].copy() for j in range(K)],
            [W[j, :counts[j]].copy() for j in range(K)], slots[:, :Lx].copy())


def fuse(per_pe: Sequence[Extraction], M: int) -> tuple:
    """Step 4 CU fusion: labels reported by more than K/2 PEs, mean state."""
    K = len(per_pe)
    stride = max([len(e.labels) for e in per_pe] + [1])
    n = np.asarray([len(e.labels) for e in per_pe], dtype=np.int32)
    lab = np.full((K, stride), -1, dtype=np.int32)
    zet = np.zeros((K, stride, 4))
    for j, e in enumerate(per_pe):
        lab[j, :len(e.labels)] = e.labels
        zet[j, :len(e.labels)] = e.zeta
    out_l = np.empty(max(M, 1), dtype=np.int32)
    out_z = np.empty((max(M, 1), 4))
    c = lib().orc_fuse(K, _i(n), _i(lab), _d(zet), stride, M, _i(out_l), _d(out_z))
    return out_l[:c].copy(), out_z[:c].copy()


# ----------------------------------------------------------------------------
# Measurement-driven birth proposal (Eq. 6 with a learned p_k(.|Z_k)) and its
# network (birth_oracle.c states the readings)
# ----------------------------------------------------------------------------

def mlp_nparams() -> int:
    return lib().orc_mlp_nparams()


def gelu(a: float) -> float:
    return lib().orc_gelu(float(a))


def gelu_grad(a: float) -> float:
    return lib().orc_gelu_grad(float(a))


def birth_features(m: _Model, Z) -> np.ndarray:
    """Network input per measurement: scaled plane position, log1p(neighbours)."""
    Z = _f64(Z, (-1, 2))
    X = np.empty((len(Z), 3))
    lib().orc_birth_features(ctypes.byref(m), _d(Z), len(Z), _d(X))
    return X


def mlp_forward(params, X) -> np.ndarray:
    P, X = _f64(params, (-1,)), _f64(X, (-1, 3))
    assert len(P) == mlp_nparams()
    Y = np.empty((len(X), 5))
    lib().orc_mlp_forward(_d(P), _d(X), len(X), _d(Y))
    return Y


def mlp_loss_grad(params, X, T, vel_scale: float):
    """Mean training loss and its gradient; T rows (t, vx, vy)."""
    P, X, T = _f64(params, (-1,)), _f64(X, (-1, 3)), _f64(T, (-1, 3))
    assert len(P) == mlp_nparams() and len(X) == len(T)
    G = np.empty(len(P))
    loss = lib().orc_mlp_loss_grad(_d(P), _d(X), _d(T), len(X), float(vel_scale), _d(G))
    return loss, G


def adam(params, grad, m1, m2, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma & Ba, ICLR 2015, Algorithm 1) in FP64; returns
    the new (params, m1, m2)."""
    g = _f64(grad)
    m1 = b1 * _f64(m1) + (1.0 - b1) * g
    m2 = b2 * _f64(m2) + (1.0 - b2) * g * g
    mh = m1 / (1.0 - b1 ** t)
    vh = m2 / (1.0 - b2 ** t)
    return _f64(params) - lr * mh / (np.sqrt(vh) + eps), m1, m2


def birth_learned(m: _Model, Z, head, alpha: float, J: int, noise, extra):
    """Births of one PE from the defensive mixture proposal; noise rows
    (n1, n2, u1, u2), extra rows (u_c, nz1, nz2, -).  Returns (x, w, comp)."""
    Z, head = _f64(Z, (-1, 2)), _f64(head, (-1, 5))
    assert len(head) == len(Z)
    noise, extra = _f64(noise, (-1, 4)), _f64(extra, (-1, 4))
    assert len(noise) >= J and len(extra) >= J
    x, w, comp = np.empty((J, 4)), np.empty(J), np.empty(J, np.int32)
    lib().orc_birth_learned(ctypes.byref(m), _d(Z), len(Z), _d(head), float(alpha), int(J), _d(noise),
                            _d(extra), _d(x), _d(w), _i(comp))
    return x, w, comp


def birth_cdf(m: _Model, head) -> np.ndarray:
    head = _f64(head, (-1, 5))
    out = np.empty(len(head))
    lib().orc_birth_cdf(ctypes.byref(m), _d(head), len(head), _d(out))
    return out


# ----------------------------------------------------------------------------
# OSPA (Schuhmacher, Vo & Vo), on positions
# ----------------------------------------------------------------------------

def ospa(X, Y, c: float = 100.0, p: float = 2.0) -> float:
    """OSPA distance between two point sets (rows are points)."""
    from scipy.optimize import linear_sum_assignment
    X = np.asarray(X, dtype=np.float64).reshape(-1, np.shape(X)[-1] if np.size(X) else 2)
    Y = np.asarray(Y, dtype=np.float64).reshape(-1, np.shape(Y)[-1] if np.size(Y) else 2)
    m, n = len(X), len(Y)
    if m == 0 and n == 0:
        return 0.0
    if m == 0 or n == 0:
        return float(c)
    if m > n:
        X, Y, m, n = Y, X, n, m
    D = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1))
    Dc = np.minimum(D, c) ** p
    r, col = linear_sum_assignment(Dc)
    cost = Dc[r, col].sum() + (c ** p) * (n - m)
    return float((cost / n) ** (1.0 / p))


# ----------------------------------------------------------------------------
# The filter: global (K = 1) and distributed (K > 1) forms
# ----------------------------------------------------------------------------

class OracleFilter:
    """The particle PHD filter (Sec. 2.2) and its DCPFPHD form (Algorithm 1).

    Random numbers are injected: `noise` rows (n1, n2, u1, u2) per particle
    slot laid out [K][pe_cap], one uint32 per PE for resampling, and uint32
    exchange draws [K][pe_cap].
    """

    def __init__(self, w, init_x: Optional[List[np.ndarray]] = None,
                 init_w: Optional[List[np.ndarray]] = None):
        self.w = w
        self.m = model(w)
        self.K = int(w.num_pe)
        self.pe_cap = int(w.pe_cap)
        J = int(w.birth_count)
        self.J = [J // self.K + (1 if j < J % self.K else 0) for j in range(self.K)]
        self.rho_pe = float(w.particles_per_target) / self.K
        self.l_max = [self.pe_cap - self.J[j] for j in range(self.K)]
        self.x = init_x if init_x is not None else [np.zeros((0, 4)) for _ in range(self.K)]
        self.wt = init_w if init_w is not None else [np.zeros(0) for _ in range(self.K)]
        self.last = {}

    def step(self, Z, noise, U, xu=None):
        m, K = self.m, self.K
        Z = _f64(Z, (-1, 2))
        M = len(Z)
        noise = _f64(noise, (K, self.pe_cap, 4))
        # Step 1: predict (survivors + births per PE)
        xp, wp = [], []
        for j in range(K):
            a, b = predict(m, self.x[j], self.wt[j], self.J[j], noise[j])
            xp.append(a)
            wp.append(b)
        # Step 2: update with local C^j (paper) or the PE mean ("global")
        C_loc = [colsum(m, xp[j], wp[j], Z) for j in range(K)]
        if getattr(self.w, "ck_mode", "local") == "global":
            C_mean = np.mean(np.stack(C_loc), axis=0) if M else np.zeros(0)
            C_used = [C_mean] * K
        else:
            C_used = C_loc
        wu = [weight_update(m, xp[j], wp[j], Z, C_used[j]) for j in range(K)]
        Nk = [float(a.sum()) for a in wu]
        # Step 3: local estimation; Step 4: CU fusion (identity for K = 1)
        ex = [extract(m, xp[j], wp[j], Z, C_used[j], Nk[j]) for j in range(K)]
        lab, zet = fuse(ex, M)
        # Step 5: local resampling
        xr, wr, par = [], [], []
        for j in range(K):
            a, b, c = resample(xp[j], wu[j], self.rho_pe, self.l_max[j], int(U[j]))
            xr.append(a)
            wr.append(b)
            par.append(c)
        # Step 6: ring exchange
        slots = None
        if K > 1 and self.w.exchange_frac > 0:
            xr, wr, slots = exchange(xr, wr, self.w.exchange_frac, xu, getattr(self.w, "exchange_mode", "ring"),
                                     getattr(self.w, "exchange_threshold", 0.0), Nk)
        self.x, self.wt = xr, wr
        self.last = dict(x_pred=xp, w_pred=wp, C_local=C_loc, C_used=C_used, w_upd=wu,
                         Nk=Nk, extract=ex, parents=par, slots=slots)
        return lab, zet


__all__ = [
    "build", "lib", "set_threads", "threads", "openmp_available", "model", "kappa", "measure", "likelihood", "predict", "colsum",
    "weight_update", "extract", "Extraction", "resample", "exchange_slots", "exchange",
    "fuse", "ospa", "OracleFilter",
]
