"""ctypes binding of the solver's C ABI (include/hjb.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Importing this module loads ``_build/libhjb.so`` and raises if it is missing --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhjb.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hjb.h")

HJB_OK = 0
HJB_ERR_INVALID_ARG = -1
HJB_ERR_CUDA = -2
HJB_ERR_OOM = -3
HJB_ERR_STATE = -4
HJB_ERR_NOT_CONVERGED = -5
HJB_ERR_TIMEOUT = -6


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_controls", ctypes.c_int32),
                ("h", ctypes.c_double), ("lam", ctypes.c_double), ("sigma", ctypes.c_double),
                ("cost", ctypes.c_double), ("coarse_n", ctypes.c_int32),
                ("n_patches", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("band_width", ctypes.c_double), ("band_window", ctypes.c_int32),
                ("band_group", ctypes.c_int32), ("wave_warps", ctypes.c_int32),
                ("resort_passes", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("tile_waves", ctypes.c_int32), ("tile_period", ctypes.c_int32),
                ("local_sweeps", ctypes.c_int32), ("tile_shape", ctypes.c_int32),
                ("visit", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("status", ctypes.c_int32),
                ("node_updates", ctypes.c_int64), ("node_control_updates", ctypes.c_int64),
                ("residual", ctypes.c_double), ("increment", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_stage", ctypes.c_double * 8),
                ("fp32_passes", ctypes.c_int32), ("fp64_passes", ctypes.c_int32),
                ("fp64_node_updates", ctypes.c_int64), ("residual_evals", ctypes.c_int32),
                ("corr_sweeps", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "ms_stage"}
        d["ms_stage"] = list(self.ms_stage)
        return d


class RegimeInfo(ctypes.Structure):
    _fields_ = [("upsilon", ctypes.c_double), ("omega", ctypes.c_double),
                ("alpha_lower", ctypes.c_double), ("alpha_upper", ctypes.c_double),
                ("alpha", ctypes.c_double), ("tau_dx", ctypes.c_double),
                ("eps_threshold", ctypes.c_double), ("h", ctypes.c_double),
                ("holds", ctypes.c_int32), ("upper_ok", ctypes.c_int32),
                ("lower_ok", ctypes.c_int32), ("reach_cells", ctypes.c_int32)]


class Terms(ctypes.Structure):
    _fields_ = [("sigma_field", ctypes.c_void_p), ("diffusion", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("cost_field", ctypes.c_void_p),
                ("control_cost", ctypes.c_void_p)]


class BatchInst(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("coarse_n", ctypes.c_int32), ("n_patches", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("h", ctypes.c_double), ("lam", ctypes.c_double),
                ("sigma", ctypes.c_double)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("n_controls", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("tile_shape", ctypes.c_int32), ("tile_waves", ctypes.c_int32),
                ("tile_period", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("cost", ctypes.c_double), ("band_width", ctypes.c_double)]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_D = ctypes.c_double
_PTR = ctypes.c_void_p

_SIGNATURES = {
    "hjb_regime": (ctypes.c_int, [_D, _D, _D, _D, ctypes.POINTER(RegimeInfo)]),
    "hjb_create_problem": (ctypes.c_int, [ctypes.POINTER(Desc), _PTR, _PTR, _PTR, _PTR, _PTR, _PTR,
                                          ctypes.POINTER(_P)]),
    "hjb_create_problem_device": (ctypes.c_int, [ctypes.POINTER(Desc), _PTR, _PTR, _PTR, _PTR, _PTR,
                                                 _PTR, ctypes.POINTER(_P)]),
    "hjb_trim_memory": (ctypes.c_int, []),
    "hjb_create_problem_general": (ctypes.c_int, [ctypes.POINTER(Desc), _PTR, _PTR, _PTR, _PTR, _PTR,
                                                  ctypes.POINTER(Terms), _PTR, ctypes.POINTER(_P)]),
    "hjb_coarse_solve": (ctypes.c_int, [_P, _D, _I32, ctypes.POINTER(Stats)]),
    "hjb_build_patches": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
    "hjb_set_feedback": (ctypes.c_int, [_P, _PTR]),
    "hjb_set_uhat": (ctypes.c_int, [_P, _PTR]),
    "hjb_solve_patches": (ctypes.c_int, [_P, _D, _D, _I32, ctypes.POINTER(Stats)]),
    "hjb_solve_full": (ctypes.c_int, [_P, _I32, _D, _D, _I32, ctypes.POINTER(Stats)]),
    "hjb_apply_operator": (ctypes.c_int, [_P, _I32, _I32, _PTR, _PTR, _PTR]),
    "hjb_residual": (ctypes.c_int, [_P, ctypes.POINTER(_D)]),
    "hjb_set_value": (ctypes.c_int, [_P, _PTR]),
    "hjb_get_value": (ctypes.c_int, [_P, _PTR]),
    "hjb_get_coarse_value": (ctypes.c_int, [_P, _PTR]),
    "hjb_get_uhat": (ctypes.c_int, [_P, _PTR]),
    "hjb_get_feedback": (ctypes.c_int, [_P, _PTR]),
    "hjb_get_successors": (ctypes.c_int, [_P, _PTR]),
    "hjb_get_labels": (ctypes.c_int, [_P, _PTR]),
    "hjb_get_order": (ctypes.c_int, [_P, _PTR, _PTR, _PTR, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "hjb_device_info": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                       ctypes.POINTER(_I32)]),
    "hjb_destroy": (None, [_P]),
    "hjb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "hjb_last_error": (ctypes.c_char_p, []),
    "hjb_kernel_launches": (ctypes.c_longlong, []),
    "hjb_residual_noalloc": (ctypes.c_int, [ctypes.POINTER(Desc), _PTR, _PTR, _PTR, _PTR, _PTR, _PTR,
                                            _PTR]),
    "hjb_batch_create": (ctypes.c_int, [ctypes.POINTER(BatchDesc), _I32, _PTR, _PTR, _PTR, _PTR, _PTR,
                                        _PTR, ctypes.POINTER(_P)]),
    "hjb_batch_create_lists": (ctypes.c_int, [ctypes.POINTER(BatchDesc), _I32, _PTR, _PTR, _PTR, _PTR, _PTR,
                                        _PTR, ctypes.POINTER(_P)]),
    "hjb_batch_solve": (ctypes.c_int, [_P, _D, _D, _D, _I32, ctypes.POINTER(Stats), _PTR]),
    "hjb_batch_solve_full": (ctypes.c_int, [_P, _D, _D, _I32, ctypes.POINTER(Stats), _PTR]),
    "hjb_batch_autotune": (ctypes.c_int, [_P, _D, _D, ctypes.POINTER(_I32), ctypes.POINTER(_I32), _PTR]),
    "hjb_batch_get_value": (ctypes.c_int, [_P, _I32, _PTR]),
    "hjb_batch_get_values": (ctypes.c_int, [_P, _PTR]),
    "hjb_batch_get_feedback": (ctypes.c_int, [_P, _I32, _PTR]),
    "hjb_batch_get_labels": (ctypes.c_int, [_P, _I32, _PTR]),
    "hjb_batch_get_uhat": (ctypes.c_int, [_P, _I32, _PTR]),
    "hjb_batch_destroy": (None, [_P]),
    "hjb_batch_coarse_solve": (ctypes.c_int, [_P, _D, _I32, ctypes.POINTER(Stats), _PTR, _PTR]),
    "hjb_batch_precompute": (ctypes.c_int, [_P, _D, ctypes.POINTER(Stats)]),
    "hjb_batch_get_coarse_value": (ctypes.c_int, [_P, _I32, _PTR]),
    "hjb_batch_net_inputs": (ctypes.c_int, [_P, _PTR]),
    "hjb_batch_net_targets": (ctypes.c_int, [_P, _PTR, _PTR, _PTR]),
    "hjb_net_output_device": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "hjb_batch_coarse_warm": (ctypes.c_int, [_P, _PTR, _I32, _I32, _I32, _D]),
    "hjb_net_param_count": (ctypes.c_longlong, []),
    "hjb_net_create": (ctypes.c_int, [_I32, _I32, _I32, _PTR, ctypes.POINTER(_P)]),
    "hjb_net_set_params": (ctypes.c_int, [_P, _PTR]),
    "hjb_net_get_params": (ctypes.c_int, [_P, _PTR]),
    "hjb_net_get_grads": (ctypes.c_int, [_P, _PTR]),
    "hjb_net_forward": (ctypes.c_int, [_P, _I32, _PTR, _PTR]),
    "hjb_net_train_step": (ctypes.c_int, [_P, _I32, _PTR, _PTR, _PTR, _PTR, ctypes.c_int64, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_float, _PTR]),
    "hjb_net_warm_values": (ctypes.c_int, [_P, _I32, _PTR, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                           _PTR]),
    "hjb_net_destroy": (None, [_P]),
    "hjb_conv3x3_forward": (ctypes.c_int, [_I32, _I32, _I32, _I32, _I32, _I32, _PTR, _PTR, _PTR, _I32, _PTR]),
    "hjb_conv3x3_dgrad": (ctypes.c_int, [_I32, _I32, _I32, _I32, _I32, _I32, _PTR, _PTR, _PTR, _PTR]),
    "hjb_conv3x3_wgrad": (ctypes.c_int, [_I32, _I32, _I32, _I32, _I32, _I32, _PTR, _PTR, _PTR, _PTR]),
}

_LIB = None


def lib() -> ctypes.CDLL:
    """The loaded C library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA solver library not found at {LIB_PATH}; build it with "
                "`python -m paper_1502_01629_gb300.build` (requires nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def header_functions() -> list:
    """Names of every function declared in include/hjb.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hjb_[a-z0-9_]+)\s*\(", txt)))


class HJBError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = lib()
        msg = L.hjb_last_error().decode() or L.hjb_status_string(code).decode()
        super().__init__(f"{where}: {L.hjb_status_string(code).decode()} ({code}): {msg}")
        self.code = code


def check(code: int, where: str) -> int:
    if code != HJB_OK:
        raise HJBError(code, where)
    return code
