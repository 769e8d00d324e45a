"""ctypes binding of ``include/sp.h`` (argument marshalling only).

Every computation runs in ``libsp.so``'s CUDA kernels.  If the library is
missing this module raises ImportError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsp.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "sp.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(nvcc, sm_103a). There is no CPU fallback.")

_lib = ctypes.CDLL(LIB_PATH)

# enums (mirrors sp.h)
SP_OK, SP_EINVAL, SP_EUNSTABLE, SP_ENOMEM, SP_EBUDGET, SP_ECUDA, SP_ETIMEOUT, SP_EBUSY, SP_PENDING, SP_ENOTFOUND = range(10)
ALLEN_CAHN, CAHN_HILLIARD, GRAY_SCOTT, MODEL_C, MODEL_H = 0, 1, 2, 3, 4
LAP_DEFAULT, LAP_5, LAP_9BOX, LAP_9CROSS4, LAP_7, LAP_27, LAP_13CROSS4, LAP_GENERATED = -1, 0, 1, 2, 3, 4, 5, 6
F64, F32, BF16_F32 = 0, 1, 2
IC_NOISE, IC_CONSTANT = 0, 1
FLAG_AUTOTUNE = 1
FLAG_BF16_NO_BOUND = 2
SCHEME_FD, SCHEME_SPECTRAL = 0, 1
MASS, FREE_ENERGY, SUM_U, SUM_V, MIN_U, MAX_U, SUMSQ_U = range(7)


class sp_params(ctypes.Structure):
    _fields_ = [("c1", ctypes.c_double), ("c2", ctypes.c_double), ("kappa", ctypes.c_double),
                ("Du", ctypes.c_double), ("Dv", ctypes.c_double), ("F", ctypes.c_double), ("k", ctypes.c_double),
                ("c3", ctypes.c_double), ("stencil", ctypes.c_int), ("dtype", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("ic_kind", ctypes.c_int), ("ic_mean", ctypes.c_double), ("ic_amp", ctypes.c_double),
                ("gs_patches", ctypes.c_int), ("gs_patch", ctypes.c_int),
                ("steps_per_launch", ctypes.c_int), ("scheme", ctypes.c_int), ("stencil_order", ctypes.c_int),
                ("flags", ctypes.c_int)]


class sp_request(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("dims", ctypes.c_int), ("shape", ctypes.c_int64 * 3),
                ("h", ctypes.c_double), ("dt", ctypes.c_double), ("params", sp_params),
                ("nsteps", ctypes.c_int64), ("return_fields", ctypes.c_int), ("fault", ctypes.c_int),
                ("priority", ctypes.c_int)]


class sp_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps_done", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_finish", ctypes.c_double), ("mass", ctypes.c_double),
                ("fields", ctypes.POINTER(ctypes.c_double)), ("n_values", ctypes.c_size_t)]


class sp_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("finished", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("quanta", ctypes.c_uint64), ("resident", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("hbm_in_use", ctypes.c_size_t), ("lups", ctypes.c_double),
                ("busy_s", ctypes.c_double)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_P = ctypes.POINTER

_SIGS = {
    "sp_params_default": (None, [ctypes.c_int, ctypes.c_int, _P(sp_params)]),
    "sp_check_stability": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          _P(sp_params), _P(ctypes.c_double)]),
    "sp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P(_i64), ctypes.c_double, ctypes.c_double,
                                 _P(sp_params), _P(_vp)]),
    "sp_step": (ctypes.c_int, [_vp, _i64, _vp]),
    "sp_read": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int, _vp]),
    "sp_write": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int, _vp]),
    "sp_reduce": (ctypes.c_int, [_vp, ctypes.c_int, _P(ctypes.c_double), _vp]),
    "sp_field_devptr": (ctypes.c_int, [_vp, ctypes.c_int, _P(_vp)]),
    "sp_steps_taken": (ctypes.c_int, [_vp, _P(_i64)]),
    "sp_autotune": (ctypes.c_int, [_vp, _vp, _P(_i64)]),
    "sp_set_launch_config": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "sp_stencil_weights": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P(ctypes.c_double), _P(ctypes.c_double)]),
    "sp_launch_config": (ctypes.c_int, [_vp, _P(ctypes.c_int), _P(ctypes.c_int)]),
    "sp_probe_fp64_rate": (ctypes.c_int, [_vp, _P(ctypes.c_double)]),
    "sp_binary_version": (ctypes.c_int, [_P(ctypes.c_int)]),
    "sp_set_wait_polls": (ctypes.c_int, [ctypes.c_longlong]),
    "sp_destroy": (ctypes.c_int, [_vp]),
    "sp_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, _P(_vp)]),
    "sp_submit": (ctypes.c_int, [_vp, _P(sp_request), _P(ctypes.c_uint64)]),
    "sp_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, _P(sp_result)]),
    "sp_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double, _P(sp_result)]),
    "sp_release": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "sp_admission_order": (ctypes.c_int, [ctypes.c_int, _P(ctypes.c_size_t), _P(ctypes.c_int), ctypes.c_size_t,
                                          ctypes.c_int, _P(ctypes.c_int)]),
    "sp_server_get_stats": (ctypes.c_int, [_vp, _P(sp_server_stats)]),
    "sp_server_destroy": (ctypes.c_int, [_vp]),
    "sp_last_error": (ctypes.c_char_p, []),
    "sp_version": (ctypes.c_int, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions that ``include/sp.h`` declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sp_[a-z0-9_]+)\s*\(", text)))


class SpError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.sp_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def check(code: int, where: str) -> None:
    if code != SP_OK:
        raise SpError(code, where)


def lib() -> ctypes.CDLL:
    return _lib
