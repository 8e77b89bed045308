"""ctypes declarations of the libqmcgb C ABI (include/qmcgb.h).

Loading fails loudly when the library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

QMC_OK, QMC_ERR_INVALID, QMC_ERR_CUDA, QMC_ERR_TIMEOUT, QMC_ERR_CAPACITY, QMC_ERR_NOMEM = 0, -1, -2, -3, -4, -5
STATUS_SINGULAR_UP, STATUS_SINGULAR_DN, STATUS_NONFINITE, STATUS_TIMEOUT = 1, 2, 4, 8
PREC = {"f64": 0, "mixed": 1, "mixed_bf16": 2, "f64_tca4": 3}
DTYPE_F64, DTYPE_F32 = 0, 1

_vp = C.c_void_p
_i = C.c_int


class SystemDesc(C.Structure):
    _fields_ = [
        ("n_atom", _i), ("Z", _vp), ("Q", _vp),
        ("n_shell", _i), ("shell_atom", _vp), ("shell_L", _vp), ("shell_nprim", _vp), ("shell_pstart", _vp),
        ("n_prim", _i), ("prim_gamma", _vp), ("prim_coef", _vp),
        ("n_ao", _i), ("ao_shell", _vp), ("ao_pow", _vp), ("ao_scale", _vp),
        ("n_up", _i), ("n_dn", _i), ("a_dtype", _i), ("A_up", _vp), ("A_dn", _vp),
        ("eps", C.c_double), ("crc32", C.c_uint32),
    ]


class EvalOut(C.Structure):
    _fields_ = [("logpsi", _vp), ("sign", _vp), ("logabs", _vp), ("drift", _vp), ("e_loc", _vp),
                ("e_parts", _vp), ("status", _vp), ("dinv", _vp)]


class Tiles(C.Structure):
    _fields_ = [("gj_panel", _i), ("c15_walkers", _i), ("a4_mode", _i), ("a4_kappa_max", C.c_double),
                ("c15_mode", _i), ("bw_walkers", _i), ("wait_s", C.c_double), ("expire_walker", _i),
                ("expire_kernels", _i), ("f64_kappa_max", C.c_double)]


A4_MODE = {"fp64": 0, "float_float": 1, "tensor": 2}
C15_MODE = {"float_float": 0, "tensor": 1, "cfree": 2}
EXPIRE = {"c15": 1, "a4": 2, "adjoint": 4}


class Jastrow(C.Structure):
    _fields_ = [("enabled", _i), ("a_par", C.c_double), ("a_anti", C.c_double), ("b_ee", C.c_double),
                ("a_en", _vp), ("b_en", _vp)]


class WalkerState(C.Structure):
    _fields_ = [("R", _vp), ("drift", _vp), ("e_loc", _vp), ("logpsi", _vp), ("sign", _vp), ("status", _vp)]


class DmcParams(C.Structure):
    _fields_ = [("tau", C.c_double), ("e_trial", C.c_double), ("seed", C.c_uint64), ("step", C.c_uint64),
                ("precision", _i), ("step_ptr", _vp), ("e_trial_ptr", _vp)]


class Segment(C.Structure):
    _fields_ = [("sys", _vp), ("n_walk", _i), ("R", _vp), ("out", EvalOut)]


class QmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libqmcgb error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libqmcgb (built on first use if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or os.environ.get("QMCGB_NO_AUTOBUILD") != "1":
                path = _build.build()
            L = C.CDLL(path)
            L.qmc_last_error.restype = C.c_char_p
            L.qmc_version.restype = C.c_char_p
            L.qmc_system_load.argtypes = [C.POINTER(SystemDesc), _i, C.POINTER(_vp)]
            L.qmc_system_free.argtypes = [_vp]
            L.qmc_system_shell_r2.argtypes = [_vp, _vp]
            L.qmc_system_set_mo.argtypes = [_vp, _i, _vp, _vp]
            L.qmc_system_crc32.argtypes = [_vp, C.POINTER(C.c_uint32)]
            L.qmc_system_set_jastrow.argtypes = [_vp, C.POINTER(Jastrow)]
            L.qmc_system_set_tiles.argtypes = [_vp, C.POINTER(Tiles)]
            L.qmc_system_get_tiles.argtypes = [_vp, C.POINTER(Tiles)]
            L.qmc_batch_workspace_size.argtypes = [C.POINTER(Segment), _i, _i, C.POINTER(C.c_size_t)]
            L.qmc_batch_eval.argtypes = [C.POINTER(Segment), _i, _i, _vp, C.c_size_t, _vp]
            L.qmc_batch_graph_create.argtypes = [C.POINTER(Segment), _i, _i, _vp, C.c_size_t, C.POINTER(_vp)]
            L.qmc_graph_launch.argtypes = [_vp, _vp]
            L.qmc_graph_free.argtypes = [_vp]
            L.qmc_workspace_size.argtypes = [_vp, _i, _i, C.POINTER(C.c_size_t)]
            L.qmc_walkers_eval.argtypes = [_vp, _i, _vp, _i, C.POINTER(EvalOut), _vp, C.c_size_t, _vp]
            L.qmc_walkers_eval_timed.argtypes = [_vp, _i, _vp, _i, C.POINTER(EvalOut), _vp, C.c_size_t, _vp,
                                                 C.POINTER(C.c_float)]
            L.qmc_walkers_eval_static.argtypes = [_vp, _i, _vp, _i, C.POINTER(EvalOut), _vp]
            L.qmc_logpsi_backward.argtypes = [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp]
            L.qmc_backward_workspace_size.argtypes = [_vp, _i, _i, C.POINTER(C.c_size_t)]
            L.qmc_logpsi_backward_ex.argtypes = [_vp, _i, _vp, _vp, _vp, _i, _vp, _vp, _vp, C.c_size_t, _vp]
            L.qmc_screen_ao.argtypes = [_vp, _i, _vp, _i, _vp, _vp, _vp, _vp]
            L.qmc_shell_masks.argtypes = [_vp, _i, _vp, _vp, C.POINTER(_i), _vp]
            L.qmc_slater_matrices.argtypes = [_vp, _i, _vp, _i, _vp, _vp, C.c_size_t, _vp]
            L.qmc_det_inverse.argtypes = [_i, _i, _vp, _vp, _vp, _vp, _vp, _vp]
            u64 = C.c_uint64
            L.qmc_multidet_workspace_size.argtypes = [_vp, _i, _i, _i, C.POINTER(C.c_size_t)]
            L.qmc_multidet_eval.argtypes = [_vp, _vp, _i, _i, _vp, _i, C.POINTER(EvalOut), _vp, C.c_size_t, _vp]
            L.qmc_dmc_move.argtypes = [_i, _i, _vp, _vp, C.c_double, u64, u64, _vp, _vp, _vp]
            L.qmc_dmc_weight.argtypes = [_i, _vp, _vp, _vp, _vp, _vp, _vp, C.c_double, C.c_double, _vp, _vp, _vp,
                                         _vp]
            L.qmc_srmc_reconfigure.argtypes = [_i, _vp, u64, u64, _vp, _vp, _vp, _vp, C.c_size_t, _vp]
            L.qmc_dmc_workspace_size.argtypes = [_vp, _i, _i, C.POINTER(C.c_size_t)]
            L.qmc_dmc_step.argtypes = [_vp, _i, C.POINTER(WalkerState), C.POINTER(WalkerState),
                                       C.POINTER(DmcParams), _vp, _vp, C.c_size_t, _vp]
            for name in ("qmc_system_load", "qmc_system_free", "qmc_system_shell_r2", "qmc_system_set_mo",
                         "qmc_system_crc32", "qmc_system_set_jastrow",
                         "qmc_system_set_tiles", "qmc_system_get_tiles", "qmc_batch_workspace_size",
                         "qmc_batch_eval", "qmc_batch_graph_create", "qmc_graph_launch", "qmc_graph_free",
                         "qmc_workspace_size",
                         "qmc_walkers_eval", "qmc_walkers_eval_timed", "qmc_walkers_eval_static",
                         "qmc_logpsi_backward", "qmc_backward_workspace_size", "qmc_logpsi_backward_ex",
                         "qmc_screen_ao", "qmc_shell_masks", "qmc_slater_matrices", "qmc_det_inverse",
                         "qmc_dmc_move", "qmc_dmc_weight", "qmc_srmc_reconfigure", "qmc_dmc_workspace_size",
                         "qmc_dmc_step", "qmc_multidet_workspace_size", "qmc_multidet_eval"):
                getattr(L, name).restype = _i
            _lib = L
    return _lib


def check(rc):
    if rc != QMC_OK:
        raise QmcError(rc, lib().qmc_last_error().decode())
    return rc


# every symbol include/qmcgb.h declares
EXPORTED = ("qmc_system_load", "qmc_system_free", "qmc_system_shell_r2", "qmc_system_set_mo", "qmc_system_crc32",
            "qmc_system_set_jastrow",
            "qmc_workspace_size",
            "qmc_system_set_tiles", "qmc_system_get_tiles", "qmc_batch_workspace_size", "qmc_batch_eval",
            "qmc_batch_graph_create", "qmc_graph_launch", "qmc_graph_free",
            "qmc_walkers_eval", "qmc_walkers_eval_timed", "qmc_walkers_eval_static", "qmc_logpsi_backward",
            "qmc_backward_workspace_size", "qmc_logpsi_backward_ex", "qmc_screen_ao", "qmc_shell_masks", "qmc_slater_matrices",
            "qmc_det_inverse", "qmc_dmc_move", "qmc_dmc_weight", "qmc_srmc_reconfigure", "qmc_dmc_workspace_size",
            "qmc_dmc_step", "qmc_multidet_workspace_size", "qmc_multidet_eval", "qmc_last_error", "qmc_version")
