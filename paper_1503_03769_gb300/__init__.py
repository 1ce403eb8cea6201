"""GB300-native particle PHD filter (global and DCPFPHD forms).

The compute path is libphd.so (hand-written sm_103a CUDA kernels behind the
C ABI in include/phd.h); `phd` is its thin ctypes binding.
"""
from .phd import (ParticlePHD, ParticlePHDBatch, PhdError, make_config, lib, LIB_PATH, ABI,  # noqa: F401
                  MlpTrainer, mlp_forward, mlp_nparams,
                  PHD_OK, PHD_ERR_INVALID_ARG, PHD_ERR_CAPACITY, PHD_ERR_CUDA,
                  PHD_ERR_TIMEOUT, PHD_ERR_STATE, PHD_FP32, PHD_FP64)
