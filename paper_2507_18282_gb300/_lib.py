"""ctypes binding of libew.so: argument marshalling only.

Every function here forwards to the C ABI entry point of the same name in
include/ew.h.  Device buffers are torch CUDA tensors (only their data pointers
cross the ABI); the stream is torch's current stream unless one is given.
There is no fallback: if the compiled library is missing the import fails.
"""
from __future__ import annotations

import ctypes
import os
import platform

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", platform.machine(), "libew.so")

EW_OK, EW_EINVAL, EW_ENOMEM, EW_ECUDA, EW_ENOCONV, EW_EBREAKDOWN, EW_ETIMEOUT, EW_EUNSUPPORTED = range(8)
STATUS_NAMES = ["EW_OK", "EW_EINVAL", "EW_ENOMEM", "EW_ECUDA", "EW_ENOCONV", "EW_EBREAKDOWN",
                "EW_ETIMEOUT", "EW_EUNSUPPORTED"]
EW_FP32, EW_FP64, EW_FP32X2 = 0, 1, 2
EW_BC_DIRICHLET, EW_BC_NEUMANN = 0, 1
EW_EXPLICIT, EW_IMPLICIT = 0, 1


class EWError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libew.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
                          "g.build()\"` first" % LIB_PATH)
    return ctypes.CDLL(LIB_PATH)


lib = _load()


class ew_mg_params(ctypes.Structure):
    _fields_ = [("pre", ctypes.c_int), ("post", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("rtol", ctypes.c_double), ("jacobi_weight", ctypes.c_double),
                ("learned_levels", ctypes.c_int), ("weights_dev", ctypes.c_void_p), ("red_black", ctypes.c_int),
                ("guess", ctypes.c_int)]


class ew_filter_params(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("num_periods", ctypes.c_int),
                ("steps_per_period", ctypes.c_int), ("cfl", ctypes.c_double),
                ("scheme", ctypes.c_int), ("adjust_omega", ctypes.c_int),
                ("temporal_block", ctypes.c_int), ("mg", ctypes.POINTER(ew_mg_params))]


class ew_filter_info(ctypes.Structure):
    _fields_ = [("omega_used", ctypes.c_double), ("final_time", ctypes.c_double),
                ("dt", ctypes.c_double), ("alpha_d", ctypes.c_double),
                ("num_steps", ctypes.c_int64), ("steps_per_period", ctypes.c_int)]


EW_MAX_EIGS = 64


class ew_eigs_params(ctypes.Structure):
    _fields_ = [("n_wanted", ctypes.c_int), ("krylov_dim", ctypes.c_int), ("block", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_wave_solves", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("refine_fp64", ctypes.c_int), ("refine_tol", ctypes.c_double), ("lock", ctypes.c_int)]


class ew_eigs_report(ctypes.Structure):
    _fields_ = [("n_converged", ctypes.c_int), ("wave_solves", ctypes.c_int),
                ("wave_solves_fp64", ctypes.c_int), ("restarts", ctypes.c_int),
                ("seconds", ctypes.c_double), ("beta", ctypes.c_double * EW_MAX_EIGS),
                ("eig_res", ctypes.c_double * EW_MAX_EIGS),
                ("lambda_stage1", ctypes.c_double * EW_MAX_EIGS),
                ("eig_res_stage1", ctypes.c_double * EW_MAX_EIGS),
                ("lambda_rel_change", ctypes.c_double * EW_MAX_EIGS)]


class ew_train_params(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("samples", ctypes.c_int), ("lr", ctypes.c_double),
                ("pre", ctypes.c_int), ("post", ctypes.c_int), ("jacobi_weight", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("accept_cycles", ctypes.c_int)]


class ew_train_report(ctypes.Structure):
    _fields_ = [("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double),
                ("conv_plain", ctypes.c_double), ("conv_learned", ctypes.c_double),
                ("accepted", ctypes.c_int)]


class ew_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("fused_launches", ctypes.c_int64),
                ("fused_ms", ctypes.c_double), ("fused_cell_steps", ctypes.c_int64),
                ("fused_points", ctypes.c_int64), ("mg_cycles", ctypes.c_int64), ("mg_solves", ctypes.c_int64)]


_vp, _i, _d, _i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

lib.ew_last_error.restype = ctypes.c_char_p
lib.ew_grid_create.argtypes = [_i, ctypes.POINTER(_i64), _dp, _i, _ip, _i, ctypes.POINTER(_vp)]
lib.ew_grid_create_mapped.argtypes = [ctypes.POINTER(_i64), _dp, _i, ctypes.POINTER(_vp)]
lib.ew_grid_destroy.argtypes = [_vp]
lib.ew_grid_destroy.restype = None
lib.ew_filter_setup.argtypes = [_vp, ctypes.POINTER(ew_filter_params), ctypes.POINTER(ew_filter_info), _dp, _i64]
lib.ew_filter_apply.argtypes = [_vp, ctypes.POINTER(ew_filter_params), _vp, _vp, _i, _vp]
lib.ew_filter_apply_host.argtypes = [_vp, ctypes.POINTER(ew_filter_params), _vp, _vp, _i, _i, _vp]
lib.ew_choose_num_periods.argtypes = [_vp, ctypes.POINTER(ew_filter_params), _i, _i, _i, _ip, _dp]
lib.ew_apply_L.argtypes = [_vp, _vp, _vp, _i, _vp]
lib.ew_rayleigh.argtypes = [_vp, _vp, _i, _dp, _dp, _vp]
lib.ew_power_iteration.argtypes = [_vp, ctypes.POINTER(ew_filter_params), _vp, _i, _d, _dp, _ip, _dp, _vp]
lib.ew_profile_enable.argtypes = [_i]
lib.ew_profile_read.argtypes = [ctypes.POINTER(ew_profile)]
lib.ew_arnoldi_eigs.argtypes = [_vp, ctypes.POINTER(ew_filter_params), ctypes.POINTER(ew_eigs_params), _vp, _dp,
                                _vp, ctypes.POINTER(ew_eigs_report), _vp]
lib.ew_filter_apply_batched.argtypes = [_i, ctypes.POINTER(_vp), ctypes.POINTER(ew_filter_params),
                                        ctypes.POINTER(_vp), ctypes.POINTER(_vp), _ip, _vp]
lib.ew_filter_apply_batched.restype = ctypes.c_int
lib.ew_arnoldi_eigs_batched.argtypes = [_i, ctypes.POINTER(_vp), ctypes.POINTER(ew_filter_params),
                                        ctypes.POINTER(ew_eigs_params), ctypes.POINTER(_dp), ctypes.POINTER(_vp),
                                        ctypes.POINTER(ew_eigs_report), _ip, _ip, _vp]
lib.ew_arnoldi_eigs_batched.restype = ctypes.c_int
lib.ew_tuned_variant.argtypes = [_vp, _i, ctypes.c_char_p, _i, _ip, _ip, _ip]
lib.ew_tuned_variant.restype = ctypes.c_int
lib.ew_filter_apply_noalloc.argtypes = [_vp, ctypes.POINTER(ew_filter_params), _vp, _vp, _vp]
lib.ew_filter_apply_noalloc.restype = ctypes.c_int
lib.ew_implicit_step_mg.argtypes =[_vp, _d, _vp, _vp, ctypes.POINTER(ew_mg_params), _dp, _ip, _vp]
lib.ew_smoother_forward.argtypes = [_vp, _vp, _vp, _vp, _vp]
lib.ew_smoother_backward.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
lib.ew_smoother_train.argtypes = [_vp, _d, ctypes.POINTER(ew_train_params), _vp, ctypes.POINTER(ew_train_report),
                                  _vp]
for _name in ["ew_grid_create", "ew_grid_create_mapped", "ew_filter_setup", "ew_choose_num_periods", "ew_filter_apply", "ew_filter_apply_host", "ew_apply_L", "ew_rayleigh",
              "ew_power_iteration", "ew_profile_enable", "ew_profile_read", "ew_arnoldi_eigs",
              "ew_implicit_step_mg", "ew_smoother_forward", "ew_smoother_backward", "ew_smoother_train"]:
    getattr(lib, _name).restype = ctypes.c_int


def check(status):
    if status != EW_OK:
        raise EWError(status, lib.ew_last_error().decode(errors="replace"))
    return status


def last_error() -> str:
    return lib.ew_last_error().decode(errors="replace")
