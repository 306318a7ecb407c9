"""ctypes declarations of the C ABI in include/afqmc.h.

Argument marshalling only: every computation runs in libafqmc.so.  Loading
fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libafqmc.so")

AFQMC_OK, AFQMC_EINVAL, AFQMC_EDOM, AFQMC_ENOMEM, AFQMC_ECUDA, AFQMC_ENOTSUP, AFQMC_ESTATE = range(7)
AFQMC_SPLIT2, AFQMC_SPLIT1, AFQMC_TAYLORPROP, AFQMC_CN = 0, 1, 2, 3
AFQMC_EXPM_TAYLOR, AFQMC_EXPM_KRYLOV, AFQMC_EXPM_BLOCK_KRYLOV, AFQMC_EXPM_CHEBYSHEV, AFQMC_EXPM_LANCZOS = 0, 1, 2, 3, 4
AFQMC_FP64, AFQMC_MIXED = 0, 1
W_FCAP, W_REWEIGHT, W_PHASE, W_NONFINITE, W_SINGULAR = 0x1, 0x2, 0x4, 0x8, 0x10
STATIC_SCRATCH_BYTES = 32 << 20
KERNEL_CLASSES = ("exchange", "field", "expm", "force_bias", "half_step", "overlap", "other")


class Walkers(ctypes.Structure):
    _fields_ = [("n_walkers", ctypes.c_int), ("psi", ctypes.c_void_p),
                ("weight", ctypes.c_void_p), ("logovl", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


class StepParams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("e0", ctypes.c_double),
                ("propagator", ctypes.c_int), ("expm", ctypes.c_int),
                ("order", ctypes.c_int), ("reortho", ctypes.c_int),
                ("measure", ctypes.c_int), ("reuse_bias", ctypes.c_int)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
class WalkAdjointParams(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int), ("order", ctypes.c_int),
                ("reortho_every", ctypes.c_int), ("ckpt_every", ctypes.c_int),
                ("tau", ctypes.c_double), ("e0", ctypes.c_double), ("dJ", ctypes.c_double),
                ("expm", ctypes.c_int)]


SIGNATURES = {
    "afqmc_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _P, _P, _P, _D, _I, _P]),
    "afqmc_set_tau": (_I, [_P, _D]),
    "afqmc_set_stream": (_I, [_P, _P]),
    "afqmc_walkers_init": (_I, [_P, ctypes.POINTER(Walkers)]),
    "afqmc_step": (_I, [_P, ctypes.POINTER(Walkers), _P, ctypes.POINTER(StepParams), _P, _P]),
    "afqmc_local_energy": (_I, [_P, ctypes.POINTER(Walkers), _D, _D, _P, _P]),
    "afqmc_sync": (_I, [_P]),
    "afqmc_launch_count": (ctypes.c_uint64, [_P]),
    "afqmc_destroy": (None, [_P]),
    "afqmc_strerror": (ctypes.c_char_p, [_I]),
    "afqmc_last_cuda_error": (ctypes.c_char_p, []),
    "afqmc_host_eigh": (_I, [_I, _P, _P, _P]),
    "afqmc_profile": (_I, [_P, _I]),
    "afqmc_profile_mask": (_I, [_P, ctypes.c_uint32]),
    "afqmc_wait_probe": (_I, [_P, ctypes.c_longlong]),
    "afqmc_population_control": (_I, [_P, ctypes.POINTER(Walkers), _D, _P]),
    "afqmc_local_energy_static": (_I, [_P, ctypes.POINTER(Walkers), _D, _D, _P, _P]),
    "afqmc_autotune": (_I, [_P, _I, _P]),
    "afqmc_energy_backward": (_I, [_P, ctypes.POINTER(Walkers), _D, _D, _D, _P, _P]),
    "afqmc_walk_backward": (_I, [_P, ctypes.POINTER(Walkers), _P, ctypes.POINTER(WalkAdjointParams),
                                 _P, _P, _P, _P]),
    "afqmc_tune_set": (_I, [_P, _P]),
    "afqmc_tune_get": (_I, [_P, _P]),
    "afqmc_batch_create": (_I, [ctypes.POINTER(_P), _P, _I]),
    "afqmc_batch_step": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "afqmc_batch_destroy": (None, [_P]),
    "afqmc_profile_read": (_I, [_P, _P, _P]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_2403_02542_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


class AfqmcError(RuntimeError):
    def __init__(self, status: int, where: str):
        l = lib()
        msg = l.afqmc_strerror(status).decode()
        if status == AFQMC_ECUDA or status == AFQMC_ENOMEM:
            msg += f" ({l.afqmc_last_cuda_error().decode()})"
        super().__init__(f"{where}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != AFQMC_OK:
        raise AfqmcError(status, where)
