"""ctypes view of libstomsfem.so (the C ABI declared in include/stomsfem.h).

No fallback: if the library is missing, importing a binding that needs it
raises; nothing in this package computes any step of the method in Python.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

OK, EINVAL, ENOMEM, ECUDA, ENOTSPD, ETIMEOUT, EVERSION = 0, -1, -2, -3, -4, -5, -6
FP64, FP32_REFINED, FP32 = 0, 1, 2
FIELD_EXP, FIELD_EXP_SIGMOID, FIELD_AFFINE = 0, 1, 2


class Grid(ctypes.Structure):
    _fields_ = [("nf", ctypes.c_int32), ("nc", ctypes.c_int32), ("f", ctypes.c_double)]


class Field(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nbx", ctypes.c_int32), ("nby", ctypes.c_int32),
                ("width", ctypes.c_double), ("scale", ctypes.c_double),
                ("contrast_log", ctypes.c_double), ("gain", ctypes.c_double)]


class StomsfemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("stomsfem error %d: %s" % (code, msg))
        self.code = code


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int32
_SZ = ctypes.c_size_t
_SIG = {
    "stomsfem_version": (ctypes.c_char_p, []),
    "stomsfem_last_error": (ctypes.c_char_p, []),
    "stomsfem_selftest_wait_timeout": (ctypes.c_int, [_I, ctypes.POINTER(_I)]),
    "stomsfem_selftest_exp": (ctypes.c_int, [_P, _I, _P, _P]),
    "stomsfem_selftest_fma_rate": (ctypes.c_int, [_I, ctypes.POINTER(ctypes.c_float)]),
    "stomsfem_selftest_mma_rate": (ctypes.c_int, [_I, ctypes.POINTER(ctypes.c_float)]),
    "stomsfem_sample_coef": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Field), _P, _I, _P, _P]),
    "stomsfem_sample_coef_precision": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Field), _P, _I,
                                                      _I, _P, _P]),
    "stomsfem_upscale_workspace_size": (ctypes.c_int, [ctypes.POINTER(Grid), _I, _I,
                                                        ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "stomsfem_upscale": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _I, _I, _I, _I, _P, _P, _P, _P,
                                        _P, _SZ, _P]),
    "stomsfem_coarse_workspace_size": (ctypes.c_int, [ctypes.POINTER(Grid), _I, ctypes.POINTER(_SZ)]),
    "stomsfem_coarse_solve": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _I, _P, _P, _P, _P, _P,
                                             _SZ, _P]),
    "stomsfem_upscale_noalloc": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _I, _I, _I, _I, _P, _P,
                                                _P, _P, _P]),
    "stomsfem_upscale_static_scratch_bytes": (ctypes.c_size_t, []),
    "stomsfem_pod_build": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _I, ctypes.c_double, _I, _P,
                                          ctypes.POINTER(_P), _P, _P]),
    "stomsfem_build_pod": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _I, ctypes.c_double, _I, _P,
                                          ctypes.POINTER(_P), _P, _P]),
    "stomsfem_pod_build_per_l": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _I, ctypes.c_double, _I, _P,
                                                ctypes.POINTER(_P), _P, _P]),
    "stomsfem_pod_destroy": (ctypes.c_int, [_P]),
    "stomsfem_pod_eigenvalues": (ctypes.c_int, [_P, _P]),
    "stomsfem_pod_save": (ctypes.c_int, [_P, _P, _SZ, ctypes.POINTER(_SZ)]),
    "stomsfem_pod_load": (ctypes.c_int, [_P, _SZ, ctypes.POINTER(_P)]),
    "stomsfem_pod_workspace_size": (ctypes.c_int, [_P, _I, ctypes.POINTER(_SZ)]),
    "stomsfem_pod_upscale": (ctypes.c_int, [_P, _P, _I, _I, _P, _P, _P, _P, _SZ, _P]),
    "stomsfem_local_vars": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Field), ctypes.c_double,
                                           _P, _P, _P, _P]),
    "stomsfem_surrogate_create": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Field),
                                                 ctypes.c_double, _P, ctypes.POINTER(_P), _P]),
    "stomsfem_surrogate_destroy": (ctypes.c_int, [_P]),
    "stomsfem_surrogate_weights": (ctypes.c_int, [_P, _P]),
    "stomsfem_surrogate_save": (ctypes.c_int, [_P, _P, _SZ, ctypes.POINTER(_SZ)]),
    "stomsfem_surrogate_load": (ctypes.c_int, [_P, _SZ, ctypes.POINTER(_P), _P]),
    "stomsfem_surrogate_train": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _I, _P, _P]),
    "stomsfem_surrogate_grad": (ctypes.c_int, [_P, _P, _P, _I, _P, _P, _P]),
    "stomsfem_surrogate_init_weights": (ctypes.c_int, [_I, ctypes.c_uint64, _P]),
    "stomsfem_surrogate_workspace_size": (ctypes.c_int, [_P, _I, ctypes.POINTER(_SZ)]),
    "stomsfem_surrogate_infer": (ctypes.c_int, [_P, _P, _P, _I, ctypes.c_double, _P, _P, _P, _P, _SZ,
                                                _P]),
    "stomsfem_upscale_pg": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _I, _I, _I, _I, _P, _P, _P, _P, _P,
                                           _SZ, _P]),
    "stomsfem_upscale_bc": (ctypes.c_int, [ctypes.POINTER(Grid), _I, _I, _P, _P, _I, _I, _I, _I, _P, _P, _P, _P,
                                           _P, _SZ, _P]),
    "stomsfem_coarse_pg_workspace_size": (ctypes.c_int, [ctypes.POINTER(Grid), _I, ctypes.POINTER(_SZ)]),
    "stomsfem_coarse_solve_pg": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _I, _P, _P, _P, _P, _P, _SZ,
                                                _P]),
    "stomsfem_coarse_bc_workspace_size": (ctypes.c_int, [ctypes.POINTER(Grid), _I, _I, ctypes.POINTER(_SZ)]),
    "stomsfem_coarse_solve_bc": (ctypes.c_int, [ctypes.POINTER(Grid), _I, _P, _P, _P, _P, _I, _P, _P, _P, _P, _P,
                                                _SZ, _P]),
    "stomsfem_pod_set_affine": (ctypes.c_int, [_P, ctypes.POINTER(Grid), ctypes.POINTER(Field), ctypes.c_double,
                                               _P]),
    "stomsfem_pod_upscale_affine": (ctypes.c_int, [_P, _P, _P, _I, _I, _P, _P, _P, _P]),
    "stomsfem_fine_fem_workspace_size": (ctypes.c_int, [ctypes.POINTER(Grid), _I, ctypes.POINTER(_SZ)]),
    "stomsfem_fine_fem": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _I, _P, _P, _SZ, _P]),
    "stomsfem_restrict_to_coarse": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _I, _P, _P]),
    "stomsfem_mc_moments": (ctypes.c_int, [_I, _I, _P, _P, _P, _P, _P]),
    "stomsfem_plan_create": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Field), _P, _I, _I, _I, _I,
                                            ctypes.POINTER(_P)]),
    "stomsfem_plan_destroy": (ctypes.c_int, [_P]),
    "stomsfem_plan_tune": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "stomsfem_plan_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _I, _P]),
    "stomsfem_plan_info": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "stomsfem_plan_set_choice": (ctypes.c_int, [_P, _I, _I, _I, _I]),
    "stomsfem_plan_upscale_ms": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "stomsfem_mc_merge": (ctypes.c_int, [_I, _P, _P, _P, _P, _P, _P, _P]),
    "stomsfem_pod_set_gemm_split": (ctypes.c_int, [_P, _I]),
    "stomsfem_surrogate_set_partner": (ctypes.c_int, [_P, _P, ctypes.c_double]),
    "stomsfem_upscale_engine": (ctypes.c_int, [ctypes.POINTER(Grid), _P, _P, _I, _I, _I, _I, _I, _I, _P, _P, _P,
                                               _P, _P, _SZ, _P]),
    "stomsfem_local_kl_build": (ctypes.c_int, [ctypes.POINTER(Grid), _I, _I, ctypes.POINTER(Field),
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double, _I,
                                               ctypes.c_double, ctypes.POINTER(_P), _P, _P]),
    "stomsfem_local_kl_destroy": (ctypes.c_int, [_P]),
    "stomsfem_local_kl_modes": (ctypes.c_int, [_P, _P, _P]),
    "stomsfem_local_kl_project": (ctypes.c_int, [_P, _P, _P, _I, _P, _P]),
    "stomsfem_ri_plan": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Field), ctypes.c_double, _I,
                                        _P, _P, _P, _P, _P]),
    "stomsfem_ri_build": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Field), ctypes.c_double, _I,
                                         _I, ctypes.POINTER(_P), _P, _P]),
    "stomsfem_ri_destroy": (ctypes.c_int, [_P]),
    "stomsfem_ri_values": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "stomsfem_ri_save": (ctypes.c_int, [_P, _P, _SZ, ctypes.POINTER(_SZ)]),
    "stomsfem_ri_load": (ctypes.c_int, [_P, _SZ, ctypes.POINTER(_P), _P]),
    "stomsfem_ri_workspace_size": (ctypes.c_int, [_P, _I, ctypes.POINTER(_SZ)]),
    "stomsfem_ri_upscale": (ctypes.c_int, [_P, _P, _P, _I, _P, _P, _P, _P, _SZ, _P]),
}


class SurrogateCfg(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("lr", ctypes.c_double), ("lr_min", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("fp32_products", ctypes.c_int32)]


def lib(path: str | None = None):
    """Load (once) and return the library handle; raises if it is missing."""
    global _lib
    if _lib is None:
        p = path or LIB
        if not os.path.exists(p):
            raise RuntimeError("libstomsfem.so not built (%s); run __graft_entry__.build()" % p)
        L = ctypes.CDLL(p)
        for name, (res, args) in _SIG.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int):
    if rc != OK:
        raise StomsfemError(rc, lib().stomsfem_last_error().decode(errors="replace"))
    return rc
