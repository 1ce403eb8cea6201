"""Thin Python binding of libphd.so (the C ABI in include/phd.h).

Argument marshalling only: every stage of the filter runs in the library's
CUDA kernels.  PyTorch supplies device memory (the workspace and the
caller's buffers) and the stream.  If libphd.so is missing the import of this
module fails loudly; there is no CPU path.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libphd.so")

PHD_OK, PHD_ERR_INVALID_ARG, PHD_ERR_CAPACITY, PHD_ERR_CUDA, PHD_ERR_TIMEOUT, PHD_ERR_STATE = range(6)
PHD_MEAS_LINEAR, PHD_MEAS_RANGE_BEARING = 0, 1
PHD_FP32, PHD_FP64 = 0, 1
PHD_CK_LOCAL, PHD_CK_GLOBAL = 0, 1
PHD_PATH_AUTO, PHD_PATH_STAGED, PHD_PATH_FUSED, PHD_PATH_GRID = 0, 1, 2, 3
PHD_BIRTH_UNIFORM, PHD_BIRTH_GAUSSIAN = 0, 1
PHD_XCHG_RING, PHD_XCHG_ALL = 0, 1
_PATHS = {"auto": PHD_PATH_AUTO, "staged": PHD_PATH_STAGED, "fused": PHD_PATH_FUSED, "grid": PHD_PATH_GRID}


class PhdError(RuntimeError):
    def __init__(self, status: int, msg: str, count: Optional[int] = None):
        super().__init__(f"phd status {status}: {msg}")
        self.status = status
        self.count = count


class phd_config(ctypes.Structure):
    _fields_ = [
        ("meas_model", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("num_pe", ctypes.c_int32), ("ck_mode", ctypes.c_int32),
        ("pe_cap", ctypes.c_int32), ("m_max", ctypes.c_int32),
        ("birth_count", ctypes.c_int32), ("birth_model", ctypes.c_int32),
        ("dt", ctypes.c_double), ("sigma_a", ctypes.c_double),
        ("sigma_z", ctypes.c_double * 2), ("sensor", ctypes.c_double * 2),
        ("region", ctypes.c_double * 4), ("r_max", ctypes.c_double),
        ("p_s", ctypes.c_double), ("p_d", ctypes.c_double),
        ("clutter_rate", ctypes.c_double), ("birth_mass", ctypes.c_double),
        ("birth_vel_sigma", ctypes.c_double), ("particles_per_target", ctypes.c_double),
        ("exchange_frac", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("sigma_a_y", ctypes.c_double), ("theta_span", ctypes.c_double),
        ("birth_mean", ctypes.c_double * 4), ("birth_std", ctypes.c_double * 4),
        ("exchange_mode", ctypes.c_int32), ("reserved1", ctypes.c_int32),
        ("exchange_threshold", ctypes.c_double), ("gate_sigma", ctypes.c_double),
    ]


class phd_stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_uint64), ("particles", ctypes.c_uint64),
                ("measurements", ctypes.c_uint64), ("updates", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("timed_updates", ctypes.c_uint64),
                ("update_ms", ctypes.c_double), ("pairs_evaluated", ctypes.c_uint64)]


class phd_tuning(ctypes.Structure):
    _fields_ = [("c_tile", ctypes.c_int32), ("c_mb", ctypes.c_int32), ("r_pb", ctypes.c_int32),
                ("r_g", ctypes.c_int32), ("grid1", ctypes.c_int32), ("grid2", ctypes.c_int32),
                ("gate", ctypes.c_int32), ("order", ctypes.c_int32), ("pass1_us", ctypes.c_float),
                ("pass2_us", ctypes.c_float)]


_P = ctypes.c_void_p
_H = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)

# exported entry points: name -> (restype, argtypes)
ABI = {
    "phd_workspace_size": (ctypes.c_int, [ctypes.POINTER(phd_config), ctypes.POINTER(ctypes.c_size_t)]),
    "phd_init": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.POINTER(phd_config), _P, ctypes.c_size_t, _P]),
    "phd_destroy": (ctypes.c_int, [_H]),
    "phd_last_error_string": (ctypes.c_char_p, [_H]),
    "phd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "phd_predict": (ctypes.c_int, [_H, _P]),
    "phd_update": (ctypes.c_int, [_H, _P, ctypes.c_int32]),
    "phd_extract": (ctypes.c_int, [_H, _P, _P, ctypes.c_int32, _P, _I32P]),
    "phd_resample": (ctypes.c_int, [_H, _P, _P]),
    "phd_step": (ctypes.c_int, [_H, _P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _I32P]),
    "phd_step_host": (ctypes.c_int, [_H, _P, ctypes.c_int32, _P, _P, ctypes.c_int32, _I32P]),
    "phd_set_state": (ctypes.c_int, [_H, _P, _P, _I32P]),
    "phd_get_state": (ctypes.c_int, [_H, _P, _P, _I32P]),
    "phd_get_update": (ctypes.c_int, [_H, _P, ctypes.POINTER(ctypes.c_double)]),
    "phd_get_local_estimates": (ctypes.c_int, [_H, _P, _P, _I32P]),
    "phd_get_resample": (ctypes.c_int, [_H, _P, _I32P]),
    "phd_get_step": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_uint64)]),
    "phd_set_step": (ctypes.c_int, [_H, ctypes.c_uint64]),
    "phd_sync": (ctypes.c_int, [_H]),
    "phd_get_stats": (ctypes.c_int, [_H, ctypes.POINTER(phd_stats)]),
    "phd_reset_stats": (ctypes.c_int, [_H]),
    "phd_set_stage_timer": (ctypes.c_int, [_H, ctypes.c_int32]),
    "phd_set_wait_limit": (ctypes.c_int, [_H, ctypes.c_int64]),
    "phd_inject_barrier_fault": (ctypes.c_int, [_H]),
    "phd_get_tuning": (ctypes.c_int, [_H, ctypes.POINTER(phd_tuning)]),
    "phd_set_tuning": (ctypes.c_int, [_H, ctypes.POINTER(phd_tuning)]),
    "phd_autotune": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.POINTER(phd_tuning)]),
    "phd_step_inject": (ctypes.c_int, [_H, _P, ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.c_int32, _P, _I32P]),
    "phd_run": (ctypes.c_int, [_H, _P, _P, ctypes.c_int32, _P, _P, _P, ctypes.c_int32]),
    "phd_set_path": (ctypes.c_int, [_H, ctypes.c_int32]),
    "phd_get_path": (ctypes.c_int, [_H, _I32P]),
    "phd_get_predicted": (ctypes.c_int, [_H, _P, _P, _P, _I32P]),
    "phd_colsum_static": (ctypes.c_int, [ctypes.POINTER(phd_config), _P, _P, ctypes.c_int32, _P,
                                         ctypes.c_int32, _P, _P]),
    "phd_batch_workspace_size": (ctypes.c_int, [ctypes.POINTER(phd_config), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_size_t)]),
    "phd_batch_init": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.POINTER(phd_config), ctypes.c_int32, _P,
                                      ctypes.c_size_t, _P]),
    "phd_batch_step": (ctypes.c_int, [_H, _P, _P, _P, _P, _P, ctypes.c_int32]),
    "phd_batch_step_inject": (ctypes.c_int, [_H, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int32]),
    "phd_set_birth_proposal": (ctypes.c_int, [_H, _P, ctypes.c_double]),
    "phd_predict_z": (ctypes.c_int, [_H, _P, ctypes.c_int32, _P, _P]),
    "phd_get_birth_head": (ctypes.c_int, [_H, _P, ctypes.c_int32, _I32P]),
    "phd_mlp_nparams": (ctypes.c_int32, []),
    "phd_birth_features": (ctypes.c_int, [ctypes.POINTER(phd_config), _P, ctypes.c_int32, _P, _P]),
    "phd_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P]),
    "phd_mlp_grad_scratch_size": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "phd_mlp_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_float, _P, _P, _P, ctypes.c_size_t, _P]),
    "phd_mlp_adam": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, _P]),
    "phd_get_phase_times": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double), ctypes.c_int32]),
    "phd_measure_ex2_rate": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), _P]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libphd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in ABI.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device buffers must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def make_config(w, seed: int = 0) -> phd_config:
    """phd_config from any object with the workload fields (see scenario.Workload)."""
    c = phd_config()
    c.meas_model = PHD_MEAS_LINEAR if w.meas_model == "linear" else PHD_MEAS_RANGE_BEARING
    c.precision = PHD_FP64 if w.precision == "fp64" else PHD_FP32
    c.num_pe = int(w.num_pe)
    c.ck_mode = PHD_CK_GLOBAL if getattr(w, "ck_mode", "local") == "global" else PHD_CK_LOCAL
    c.pe_cap = int(w.pe_cap)
    c.m_max = int(w.m_max)
    c.birth_count = int(w.birth_count)
    c.dt, c.sigma_a = float(w.dt), float(w.sigma_a)
    c.sigma_z[0], c.sigma_z[1] = float(w.sigma_z[0]), float(w.sigma_z[1])
    c.sensor[0], c.sensor[1] = float(w.sensor[0]), float(w.sensor[1])
    for k in range(4):
        c.region[k] = float(w.region[k])
    c.r_max = float(w.r_max)
    c.p_s, c.p_d = float(w.p_s), float(w.p_d)
    c.clutter_rate, c.birth_mass = float(w.clutter_rate), float(w.birth_mass)
    c.birth_vel_sigma = float(w.birth_vel_sigma)
    c.particles_per_target = float(w.particles_per_target)
    c.exchange_frac = float(w.exchange_frac)
    c.seed = int(seed) & (2 ** 64 - 1)
    c.sigma_a_y = float(getattr(w, "sigma_a_y", 0.0))
    c.theta_span = float(getattr(w, "theta_span", 0.0))
    c.birth_model = PHD_BIRTH_GAUSSIAN if getattr(w, "birth_model", "uniform") == "gaussian" else PHD_BIRTH_UNIFORM
    for k, v in enumerate(getattr(w, "birth_mean", (0.0,) * 4)):
        c.birth_mean[k] = float(v)
    for k, v in enumerate(getattr(w, "birth_std", (0.0,) * 4)):
        c.birth_std[k] = float(v)
    c.exchange_mode = PHD_XCHG_ALL if getattr(w, "exchange_mode", "ring") == "all" else PHD_XCHG_RING
    c.exchange_threshold = float(getattr(w, "exchange_threshold", 0.0))
    c.gate_sigma = float(getattr(w, "gate_sigma", 0.0))
    return c


def _check_colsum_static_args(cfg: phd_config, x, w, Z, C):
    """Shapes, dtypes and device of phd_colsum_static's buffers; returns (n, M)."""
    real = torch.float64 if cfg.precision == PHD_FP64 else torch.float32
    for name, t in (("x", x), ("w", w), ("Z", Z), ("C", C)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
    for name, t in (("x", x), ("w", w), ("Z", Z)):
        if t.dtype != real:
            raise ValueError(f"{name} is {t.dtype}; the config's precision needs {real}")
    if C.dtype != torch.float64:
        raise ValueError(f"C is {C.dtype}; it must be torch.float64")
    if x.dim() != 2 or x.shape[1] != 4:
        raise ValueError(f"x must be (n, 4), got {tuple(x.shape)}")
    if w.dim() != 1 or w.shape[0] != x.shape[0]:
        raise ValueError(f"w must be ({x.shape[0]},), got {tuple(w.shape)}")
    if Z.dim() != 2 or Z.shape[1] != 2:
        raise ValueError(f"Z must be (M, 2), got {tuple(Z.shape)}")
    n, M = int(x.shape[0]), int(Z.shape[0])
    if C.numel() < M:
        raise ValueError(f"C holds {C.numel()} values, fewer than M = {M}")
    devs = {t.device for t in (x, w, Z, C)}
    if len(devs) != 1 or next(iter(devs)).type != "cuda":
        raise ValueError(f"x, w, Z and C must be on one CUDA device, got {sorted(map(str, devs))}")
    for name, t in (("x", x), ("w", w), ("Z", Z), ("C", C)):
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    return n, M


def colsum_static(cfg: phd_config, x: torch.Tensor, w: torch.Tensor, Z: torch.Tensor, C: torch.Tensor,
                  stream: Optional[torch.cuda.Stream] = None) -> int:
    """phd_colsum_static: Eq. 7 column sums into C (double [M]) with no device
    allocation; returns the phd status.

    The library reads x, w and Z as the config's real type and writes M
    doubles into C, so every tensor is checked here first (ValueError, nothing
    launched): x (n, 4), w (n,), Z (M, 2) in float32 (PHD_FP32) or float64
    (PHD_FP64), C float64 with at least M elements, all contiguous on one CUDA
    device."""
    n, M = _check_colsum_static_args(cfg, x, w, Z, C)
    st = stream if stream is not None else torch.cuda.current_stream()
    return lib().phd_colsum_static(ctypes.byref(cfg), _ptr(x) if n else None, _ptr(w) if n else None, n,
                                   _ptr(Z) if M else None, M, _ptr(C) if M else None,
                                   ctypes.c_void_p(st.cuda_stream))


def measure_ex2_rate(reps: int = 20, stream: Optional[torch.cuda.Stream] = None):
    """phd_measure_ex2_rate: (ex2 instructions per second on the current
    device, fastest launch in ms)."""
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = lib().phd_measure_ex2_rate(int(reps), ctypes.byref(rate), ctypes.byref(ms), _stream_ptr(stream))
    _check_status(st, "phd_measure_ex2_rate")
    return rate.value, ms.value


def _stream_ptr(stream: Optional[torch.cuda.Stream]):
    st = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(st.cuda_stream)


def _check_status(st: int, what: str):
    if st != PHD_OK:
        raise PhdError(st, what)


def mlp_nparams() -> int:
    return int(lib().phd_mlp_nparams())


def mlp_forward(params: torch.Tensor, X: torch.Tensor, stream=None) -> torch.Tensor:
    """Birth network outputs Y[n][5] for inputs X[n][3] (phd_mlp_forward)."""
    n = int(X.shape[0])
    Y = torch.empty((n, 5), dtype=torch.float32, device=X.device)
    _check_status(lib().phd_mlp_forward(_ptr(params), _ptr(X) if n else None, n, _ptr(Y) if n else None,
                                        _stream_ptr(stream)), "phd_mlp_forward")
    return Y


def birth_features(cfg: phd_config, Z: torch.Tensor, stream=None) -> torch.Tensor:
    """Birth network inputs X[M][3] of a scan Z[M][2] (FP32, device)."""
    M = int(Z.shape[0])
    X = torch.empty((M, 3), dtype=torch.float32, device=Z.device)
    _check_status(lib().phd_birth_features(ctypes.byref(cfg), _ptr(Z) if M else None, M, _ptr(X) if M else None,
                                           _stream_ptr(stream)), "phd_birth_features")
    return X


class MlpTrainer:
    """Adam training of the birth network through phd_mlp_grad / phd_mlp_adam
    (FP32 master parameters on the device)."""

    def __init__(self, params: torch.Tensor, batch_max: int, lr: float = 1e-3, betas=(0.9, 0.999),
                 eps: float = 1e-8, vel_scale: float = 20.0, stream=None):
        self.L = lib()
        self.params = params.detach().to(torch.float32).contiguous().clone()
        self.m1 = torch.zeros_like(self.params)
        self.m2 = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.params.device)
        nb = ctypes.c_size_t(0)
        _check_status(self.L.phd_mlp_grad_scratch_size(int(batch_max), ctypes.byref(nb)), "scratch_size")
        self.scratch = torch.empty(int(nb.value), dtype=torch.uint8, device=self.params.device)
        self.batch_max = int(batch_max)
        self.lr, self.betas, self.eps, self.vel_scale = float(lr), betas, float(eps), float(vel_scale)
        self.t = 0
        self.stream = stream

    def grad_of(self, X: torch.Tensor, T: torch.Tensor) -> torch.Tensor:
        """Mean-loss gradient for inputs X[n][3], targets T[n][3] into self.grad."""
        n = int(X.shape[0])
        assert 0 < n <= self.batch_max
        _check_status(self.L.phd_mlp_grad(_ptr(self.params), _ptr(X), _ptr(T), n, self.vel_scale,
                                          _ptr(self.grad), _ptr(self.loss), _ptr(self.scratch),
                                          self.scratch.numel(), _stream_ptr(self.stream)), "phd_mlp_grad")
        return self.grad

    def step(self, X: torch.Tensor, T: torch.Tensor):
        self.grad_of(X, T)
        self.t += 1
        _check_status(self.L.phd_mlp_adam(_ptr(self.params), _ptr(self.grad), _ptr(self.m1), _ptr(self.m2),
                                          self.t, self.lr, float(self.betas[0]), float(self.betas[1]),
                                          self.eps, _stream_ptr(self.stream)), "phd_mlp_adam")


class ParticlePHD:
    """One filter (global for num_pe == 1, DCPFPHD for num_pe > 1) on a CUDA device."""

    def __init__(self, workload, seed: int = 0, device: str = "cuda",
                 stream: Optional[torch.cuda.Stream] = None):
        self.L = lib()
        self.w = workload
        self.cfg = make_config(workload, seed)
        self.K = int(self.cfg.num_pe)
        self.pe_cap = int(self.cfg.pe_cap)
        self.m_max = int(self.cfg.m_max)
        self.dtype = torch.float64 if self.cfg.precision == PHD_FP64 else torch.float32
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = ctypes.c_size_t(0)
        self._check(self.L.phd_workspace_size(ctypes.byref(self.cfg), ctypes.byref(nbytes)), "workspace_size")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.L.phd_init(ctypes.byref(h), ctypes.byref(self.cfg), _ptr(self.workspace),
                                 nbytes.value, ctypes.c_void_p(self.stream.cuda_stream))
        self._check(st, "phd_init")
        self.h = h
        self._cnt = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.learned = False
        self.jmax = -(-int(self.cfg.birth_count) // self.K)

    # -- plumbing -----------------------------------------------------------
    def _check(self, st: int, what: str, count: Optional[int] = None):
        if st != PHD_OK:
            msg = what
            if getattr(self, "h", None):
                msg += ": " + (self.L.phd_last_error_string(self.h) or b"").decode()
            raise PhdError(st, msg, count)

    def close(self):
        if getattr(self, "h", None):
            self.L.phd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _real(self, a, shape) -> torch.Tensor:
        t = torch.as_tensor(a, dtype=self.dtype, device=self.device).reshape(shape)
        return t.contiguous()

    # -- stages -------------------------------------------------------------
    def _noise_rows(self) -> int:
        """Rows of injected noise: the plain rows, then (with a birth network)
        the extra rows of the measurement-driven births."""
        return self.K * self.pe_cap + (self.K * self.jmax if self.learned else 0)

    def predict(self, noise=None):
        n = None if noise is None else self._real(noise, (self.K * self.pe_cap, 4))
        self._check(self.L.phd_predict(self.h, _ptr(n)), "phd_predict")
        self._keep = n

    def predict_z(self, Z, noise=None, head=None):
        """phd_predict_z: prediction with the scan (measurement-driven births
        when a birth network is loaded; `head` [M][5] replaces its output)."""
        Zt = self._real(Z, (-1, 2))
        M = int(Zt.shape[0])
        n = None if noise is None else self._real(noise, (self._noise_rows(), 4))
        hd = None if head is None else torch.as_tensor(head, dtype=torch.float32,
                                                       device=self.device).reshape(M, 5).contiguous()
        self._check(self.L.phd_predict_z(self.h, _ptr(Zt) if M else None, M, _ptr(hd) if (hd is not None and M)
                                         else None, _ptr(n)), "phd_predict_z")
        self._keep = (Zt, n, hd)

    def set_birth_proposal(self, params: Optional[torch.Tensor], alpha: float = 0.1):
        """Load the birth network (FP32 device parameters) or unload it (None)."""
        p = None if params is None else params.to(device=self.device, dtype=torch.float32).contiguous()
        self._check(self.L.phd_set_birth_proposal(self.h, _ptr(p), float(alpha)), "phd_set_birth_proposal")
        self.learned = p is not None

    def get_birth_head(self) -> np.ndarray:
        out = torch.empty((self.m_max, 5), dtype=torch.float32, device=self.device)
        M = ctypes.c_int32(0)
        self._check(self.L.phd_get_birth_head(self.h, _ptr(out), self.m_max, ctypes.byref(M)),
                    "phd_get_birth_head")
        return out[:M.value].cpu().numpy()

    def update(self, Z):
        Zt = self._real(Z, (-1, 2))
        self._check(self.L.phd_update(self.h, _ptr(Zt) if Zt.numel() else None, Zt.shape[0]), "phd_update")
        self._keepZ = Zt

    def extract(self, cap: Optional[int] = None):
        cap = self.m_max if cap is None else int(cap)
        states = torch.empty((max(cap, 1), 4), dtype=self.dtype, device=self.device)
        labels = torch.empty(max(cap, 1), dtype=torch.int32, device=self.device)
        hc = ctypes.c_int32(0)
        st = self.L.phd_extract(self.h, _ptr(states), _ptr(labels), cap, _ptr(self._cnt), ctypes.byref(hc))
        self._check(st, "phd_extract", hc.value)
        n = hc.value
        return states[:n], labels[:n]

    def resample(self, u=None, xu=None):
        ut = None if u is None else torch.as_tensor(np.asarray(u, dtype=np.uint32).view(np.int32),
                                                    device=self.device).contiguous()
        xt = None if xu is None else torch.as_tensor(np.asarray(xu, dtype=np.uint32).view(np.int32),
                                                     device=self.device).reshape(-1).contiguous()
        self._check(self.L.phd_resample(self.h, _ptr(ut), _ptr(xt)), "phd_resample")
        self._keepu = (ut, xt)

    def step(self, Z, cap: Optional[int] = None, sync: bool = True):
        """One step (predict, update, extract, resample) with in-kernel randomness."""
        cap = self.m_max if cap is None else int(cap)
        Zt = self._real(Z, (-1, 2))
        if not hasattr(self, "_out") or self._out[0].shape[0] < max(cap, 1):
            self._out = (torch.empty((max(cap, 1), 4), dtype=self.dtype, device=self.device),
                         torch.empty(max(cap, 1), dtype=torch.int32, device=self.device))
        states, labels = self._out
        hc = ctypes.c_int32(0)
        st = self.L.phd_step(self.h, _ptr(Zt) if Zt.numel() else None, Zt.shape[0], _ptr(states),
                             _ptr(labels), cap, _ptr(self._cnt), ctypes.byref(hc) if sync else None)
        self._check(st, "phd_step", hc.value if sync else None)
        self._keepZ = Zt
        if sync:
            return states[:hc.value], labels[:hc.value]
        return states, labels, self._cnt

    def _u32(self, a, shape=None):
        if a is None:
            return None
        t = torch.as_tensor(np.ascontiguousarray(np.asarray(a, dtype=np.uint32)).view(np.int32), device=self.device)
        return t.reshape(-1).contiguous()

    def step_inject(self, Z, noise=None, u=None, xu=None, cap: Optional[int] = None):
        """One step with injected random numbers (phd_step_inject); synchronises."""
        cap = self.m_max if cap is None else int(cap)
        Zt = self._real(Z, (-1, 2))
        nz = None if noise is None else self._real(noise, (self._noise_rows(), 4))
        ut, xt = self._u32(u), self._u32(xu)
        states = torch.empty((max(cap, 1), 4), dtype=self.dtype, device=self.device)
        labels = torch.empty(max(cap, 1), dtype=torch.int32, device=self.device)
        hc = ctypes.c_int32(0)
        st = self.L.phd_step_inject(self.h, _ptr(Zt) if Zt.numel() else None, Zt.shape[0], _ptr(nz), _ptr(ut),
                                    _ptr(xt), _ptr(states), _ptr(labels), cap, _ptr(self._cnt), ctypes.byref(hc))
        self._check(st, "phd_step_inject", hc.value)
        return states[:hc.value], labels[:hc.value]

    def pack(self, Zs):
        """Pack a list of scans into (device rows, device int32 offsets) for run_packed."""
        rows = [torch.as_tensor(z, dtype=self.dtype, device=self.device).reshape(-1, 2) for z in Zs]
        off = np.zeros(len(rows) + 1, dtype=np.int32)
        off[1:] = np.cumsum([r.shape[0] for r in rows])
        Zp = torch.cat(rows).contiguous() if off[-1] else torch.zeros((1, 2), dtype=self.dtype, device=self.device)
        return Zp, torch.as_tensor(off, device=self.device)

    def run_packed(self, Zp, offsets, S: int, cap: Optional[int] = None):
        """phd_run on packed device scans; returns device (states, labels, counts)."""
        cap = self.m_max if cap is None else int(cap)
        states = torch.empty((S, cap, 4), dtype=self.dtype, device=self.device)
        labels = torch.empty((S, cap), dtype=torch.int32, device=self.device)
        counts = torch.empty(S, dtype=torch.int32, device=self.device)
        self._check(self.L.phd_run(self.h, _ptr(Zp), _ptr(offsets), S, _ptr(states), _ptr(labels), _ptr(counts),
                                   cap), "phd_run")
        self._keeprun = (Zp, offsets)
        return states, labels, counts

    def run(self, Zs, cap: Optional[int] = None, sync: bool = True):
        """phd_run over a list of scans; returns per-scan (states, labels)."""
        cap = self.m_max if cap is None else int(cap)
        Zp, offt = self.pack(Zs)
        states, labels, counts = self.run_packed(Zp, offt, len(Zs), cap)
        if not sync:
            return states, labels, counts
        self.sync()
        c = counts.cpu().numpy()
        return [(states[s, :min(c[s], cap)], labels[s, :min(c[s], cap)]) for s in range(len(Zs))]

    def set_path(self, path: str):
        self._check(self.L.phd_set_path(self.h, _PATHS[path]), "phd_set_path")

    def get_path(self) -> str:
        v = ctypes.c_int32(0)
        self._check(self.L.phd_get_path(self.h, ctypes.byref(v)), "phd_get_path")
        return {PHD_PATH_STAGED: "staged", PHD_PATH_FUSED: "fused", PHD_PATH_GRID: "grid"}[v.value]

    def get_predicted(self):
        X = torch.empty((self.K, self.pe_cap, 4), dtype=self.dtype, device=self.device)
        Wp = torch.empty((self.K, self.pe_cap), dtype=self.dtype, device=self.device)
        Wu = torch.empty((self.K, self.pe_cap), dtype=self.dtype, device=self.device)
        counts = (ctypes.c_int32 * self.K)()
        self._check(self.L.phd_get_predicted(self.h, _ptr(X), _ptr(Wp), _ptr(Wu), counts), "phd_get_predicted")
        c = list(counts)
        Xn, Wpn, Wun = X.cpu().numpy(), Wp.cpu().numpy(), Wu.cpu().numpy()
        return ([Xn[j, :c[j]] for j in range(self.K)], [Wpn[j, :c[j]] for j in range(self.K)],
                [Wun[j, :c[j]] for j in range(self.K)])

    def step_host(self, Z: np.ndarray, out_states: np.ndarray, out_labels: np.ndarray) -> int:
        """phd_step_host on host numpy buffers; returns the estimate count."""
        npdt = np.float64 if self.dtype == torch.float64 else np.float32
        Z = np.ascontiguousarray(Z, dtype=npdt)
        assert out_states.dtype == npdt and out_states.flags.c_contiguous
        assert out_labels.dtype == np.int32 and out_labels.flags.c_contiguous
        hc = ctypes.c_int32(0)
        st = self.L.phd_step_host(self.h, Z.ctypes.data_as(ctypes.c_void_p), Z.shape[0],
                                  out_states.ctypes.data_as(ctypes.c_void_p),
                                  out_labels.ctypes.data_as(ctypes.c_void_p), out_labels.shape[0],
                                  ctypes.byref(hc))
        self._check(st, "phd_step_host", hc.value)
        return hc.value

    # -- state access ---------------------------------------------------------
    def set_state(self, xs, ws):
        """xs, ws: per-PE lists of (n_j, 4) and (n_j,) arrays."""
        X = torch.zeros((self.K, self.pe_cap, 4), dtype=self.dtype, device=self.device)
        W = torch.zeros((self.K, self.pe_cap), dtype=self.dtype, device=self.device)
        counts = (ctypes.c_int32 * self.K)()
        for j in range(self.K):
            n = len(ws[j])
            counts[j] = n
            if n:
                X[j, :n] = torch.as_tensor(np.asarray(xs[j]), dtype=self.dtype)
                W[j, :n] = torch.as_tensor(np.asarray(ws[j]), dtype=self.dtype)
        self._check(self.L.phd_set_state(self.h, _ptr(X), _ptr(W), counts), "phd_set_state")

    def get_state(self):
        X = torch.empty((self.K, self.pe_cap, 4), dtype=self.dtype, device=self.device)
        W = torch.empty((self.K, self.pe_cap), dtype=self.dtype, device=self.device)
        counts = (ctypes.c_int32 * self.K)()
        self._check(self.L.phd_get_state(self.h, _ptr(X), _ptr(W), counts), "phd_get_state")
        c = list(counts)
        Xn, Wn = X.cpu().numpy(), W.cpu().numpy()
        return [Xn[j, :c[j]] for j in range(self.K)], [Wn[j, :c[j]] for j in range(self.K)]

    def get_update(self):
        C = torch.empty((self.K, self.m_max), dtype=torch.float64, device=self.device)
        mass = (ctypes.c_double * self.K)()
        self._check(self.L.phd_get_update(self.h, _ptr(C), mass), "phd_get_update")
        return C.cpu().numpy(), np.array(list(mass))

    def get_local_estimates(self):
        S = torch.empty((self.K, self.m_max, 4), dtype=self.dtype, device=self.device)
        Lb = torch.empty((self.K, self.m_max), dtype=torch.int32, device=self.device)
        counts = (ctypes.c_int32 * self.K)()
        self._check(self.L.phd_get_local_estimates(self.h, _ptr(S), _ptr(Lb), counts), "phd_get_local_estimates")
        c = list(counts)
        Sn, Ln = S.cpu().numpy(), Lb.cpu().numpy()
        return [Sn[j, :c[j]] for j in range(self.K)], [Ln[j, :c[j]] for j in range(self.K)]

    def get_resample(self):
        P = torch.empty((self.K, self.pe_cap), dtype=torch.int32, device=self.device)
        lx = ctypes.c_int32(0)
        self._check(self.L.phd_get_resample(self.h, _ptr(P), ctypes.byref(lx)), "phd_get_resample")
        return P.cpu().numpy(), lx.value

    def get_step(self) -> int:
        s = ctypes.c_uint64(0)
        self._check(self.L.phd_get_step(self.h, ctypes.byref(s)), "phd_get_step")
        return s.value

    def set_step(self, step: int):
        self._check(self.L.phd_set_step(self.h, int(step)), "phd_set_step")

    def sync(self):
        self._check(self.L.phd_sync(self.h), "phd_sync")

    def stats(self) -> dict:
        st = phd_stats()
        self._check(self.L.phd_get_stats(self.h, ctypes.byref(st)), "phd_get_stats")
        return {k: getattr(st, k) for k, _ in phd_stats._fields_}

    def reset_stats(self):
        self._check(self.L.phd_reset_stats(self.h), "phd_reset_stats")

    PHASES = ("predict_keys_totals", "cell_starts", "scatter", "pass1", "normalisers", "pass2_ranks",
              "mass_plan", "plan_cdf_pass3", "estimates_offsets", "offspring_gather")

    def phase_times(self, detail: bool = False):
        """Grid path: summed wall time per phase of the step kernel, ms
        (phd_get_phase_times); with detail, also the longest and the mean
        per-CTA working time of each phase."""
        v = (ctypes.c_double * 36)()
        self._check(self.L.phd_get_phase_times(self.h, v, 36), "phd_get_phase_times")
        wall = dict(zip(self.PHASES, list(v)[:12]))
        if not detail:
            return wall
        return wall, dict(zip(self.PHASES, list(v)[12:24])), dict(zip(self.PHASES, list(v)[24:36]))

    def set_stage_timer(self, on: bool):
        self._check(self.L.phd_set_stage_timer(self.h, 1 if on else 0), "phd_set_stage_timer")

    def set_wait_limit(self, iterations: int):
        """Polls of a bounded wait on other CTAs before it reports a timeout."""
        self._check(self.L.phd_set_wait_limit(self.h, int(iterations)), "phd_set_wait_limit")

    def inject_barrier_fault(self):
        """Failure injection for tests: PE 0 leaves the next fused step at its
        first grid barrier without arriving; the other PEs' bounded waits
        report PHD_ERR_TIMEOUT."""
        self._check(self.L.phd_inject_barrier_fault(self.h), "phd_inject_barrier_fault")

    def get_tuning(self) -> dict:
        t = phd_tuning()
        self._check(self.L.phd_get_tuning(self.h, ctypes.byref(t)), "phd_get_tuning")
        return {k: getattr(t, k) for k, _ in phd_tuning._fields_}

    def set_tuning(self, **shape):
        """Select the pair passes' launch shape (keys of phd_tuning; missing
        keys keep their current value)."""
        cur = self.get_tuning()
        cur.update(shape)
        t = phd_tuning(**{k: cur[k] for k, _ in phd_tuning._fields_})
        self._check(self.L.phd_set_tuning(self.h, ctypes.byref(t)), "phd_set_tuning")

    def autotune(self, reps: int = 5) -> dict:
        """Time every supported shape on the current predicted set and keep
        the fastest (phd_autotune); returns the chosen shape and its times."""
        t = phd_tuning()
        self._check(self.L.phd_autotune(self.h, int(reps), ctypes.byref(t)), "phd_autotune")
        return {k: getattr(t, k) for k, _ in phd_tuning._fields_}


class ParticlePHDBatch(ParticlePHD):
    """A batch of independent one-PE filters (phd_batch_*): run j follows workloads[j]."""

    def __init__(self, workloads, seed: int = 0, device: str = "cuda",
                 stream: Optional[torch.cuda.Stream] = None):
        self.L = lib()
        self.ws_list = list(workloads)
        R = len(self.ws_list)
        arr = (phd_config * R)(*[make_config(w, seed) for w in self.ws_list])
        self._cfgs = arr
        self.cfg = arr[0]
        self.K = R
        self.pe_cap = max(int(w.pe_cap) for w in self.ws_list)
        self.m_max = max(int(w.m_max) for w in self.ws_list)
        self.dtype = torch.float64 if self.cfg.precision == PHD_FP64 else torch.float32
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = ctypes.c_size_t(0)
        self._check(self.L.phd_batch_workspace_size(arr, R, ctypes.byref(nbytes)), "phd_batch_workspace_size")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.L.phd_batch_init(ctypes.byref(h), arr, R, _ptr(self.workspace), nbytes.value,
                                       ctypes.c_void_p(self.stream.cuda_stream))
        self._check(st, "phd_batch_init")
        self.h = h
        self._cnt = torch.zeros(1, dtype=torch.int32, device=self.device)

    def pack_batch(self, Zs):
        """Per-run scans -> (device rows, device int32 offsets [runs+1])."""
        return self.pack(Zs)

    def batch_step(self, Zs=None, packed=None, cap: Optional[int] = None, noise=None, u=None, sync: bool = True):
        cap = self.m_max if cap is None else int(cap)
        Zp, offt = packed if packed is not None else self.pack(Zs)
        states = torch.empty((self.K, cap, 4), dtype=self.dtype, device=self.device)
        labels = torch.empty((self.K, cap), dtype=torch.int32, device=self.device)
        counts = torch.empty(self.K, dtype=torch.int32, device=self.device)
        if noise is None and u is None:
            st = self.L.phd_batch_step(self.h, _ptr(Zp), _ptr(offt), _ptr(states), _ptr(labels), _ptr(counts), cap)
        else:
            nz = None if noise is None else self._real(noise, (self.K * self.pe_cap, 4))
            ut = self._u32(u)
            st = self.L.phd_batch_step_inject(self.h, _ptr(Zp), _ptr(offt), _ptr(nz), _ptr(ut), _ptr(states),
                                              _ptr(labels), _ptr(counts), cap)
            self._keepb = (nz, ut)
        self._check(st, "phd_batch_step")
        self._keeprun = (Zp, offt)
        if not sync:
            return states, labels, counts
        self.sync()
        c = counts.cpu().numpy()
        return [(states[j, :min(c[j], cap)], labels[j, :min(c[j], cap)]) for j in range(self.K)]


__all__ = ["lib", "LIB_PATH", "ABI", "ParticlePHDBatch", "phd_config", "phd_stats", "make_config", "colsum_static", "ParticlePHD", "PhdError",
           "PHD_OK", "PHD_ERR_INVALID_ARG", "PHD_ERR_CAPACITY", "PHD_ERR_CUDA", "PHD_ERR_TIMEOUT",
           "PHD_ERR_STATE", "PHD_FP32", "PHD_FP64"]
