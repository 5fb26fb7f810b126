"""ctypes declarations of the C ABI in include/mh.h (argument marshalling only).

The shared library is built in-tree (paper_2006_02501_gb300/lib/libmh.so) by
paper_2006_02501_gb300.build.  Loading fails loudly if it is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmh.so")

MH_OK = 0
MH_EINVAL = -1
MH_ENOMEM = -2
MH_ECUDA = -3
MH_ENONFINITE = -4
MH_ETIMEOUT = -5
MH_ENOTCONV = 1

MH_BETA_MODIFIED, MH_BETA_STANDARD = 0, 1
MH_PREC_FP64, MH_PREC_FP32PAIR = 0, 1
MH_STEP_SHARED, MH_STEP_BLOCK, MH_STEP_TIMESYM = 0, 1, 2

# Every entry point declared in include/mh.h (checked by the CPU test suite).
EXPORTS = [
    "mh_config_default", "mh_create", "mh_destroy", "mh_step", "mh_sync", "mh_set_state",
    "mh_diagnostics", "mh_info", "mh_last_error", "mh_pair_eval", "mh_release_scratch",
    "mh_set_timing", "mh_pair_eval_noalloc", "mh_create_batch", "mh_step_batch", "mh_batch_tune",
    "mh_batch_energy", "mh_step_converge", "mh_set_predictor", "mh_collect_samples", "mh_mlp_create",
    "mh_mlp_destroy", "mh_mlp_num_params", "mh_mlp_get_params", "mh_mlp_set_params", "mh_mlp_forward",
    "mh_mlp_loss_grad", "mh_mlp_train", "mh_predict", "mh_step_timesym", "mh_measure_peaks",
    "mh_dd_create", "mh_dd_destroy", "mh_dd_step", "mh_dd_sync", "mh_dd_set_state", "mh_dd_diagnostics",
    "mh_dd_info", "mh_dd_pair_eval", "mh_dd_sym_check", "mh_dd_create_batch", "mh_dd_step_batch", "mh_dd_batch_energy", "mh_restore",
    "mh_sym_schedule_check",
]


class Config(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("beta_mode", ctypes.c_int), ("precision", ctypes.c_int),
                ("step_mode", ctypes.c_int), ("G", ctypes.c_double), ("eta", ctypes.c_double),
                ("dt_max", ctypes.c_double), ("k_max", ctypes.c_int), ("split_j", ctypes.c_int),
                ("heavy_frac", ctypes.c_double), ("symmetric", ctypes.c_int),
                ("fp32_variant", ctypes.c_int), ("compensated", ctypes.c_int)]


class StateC(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("x", ctypes.POINTER(ctypes.c_double)),
                ("v", ctypes.POINTER(ctypes.c_double)), ("derivs", ctypes.POINTER(ctypes.c_double)),
                ("level", ctypes.POINTER(ctypes.c_int32))]


class Counters(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("evaluations", ctypes.c_int64),
                ("pair_interactions", ctypes.c_double), ("particle_steps", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("pair_kernel_ms", ctypes.c_double),
                ("pair_kernel_timed", ctypes.c_int64), ("pair_variant", ctypes.c_int32),
                ("pair_tune_ms_x1000", ctypes.c_int32 * 3)]


class MHError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mh error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run python -m paper_2006_02501_gb300.build)")
            L = ctypes.CDLL(LIB_PATH)
            P, D, I, I64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
            DP = ctypes.POINTER(ctypes.c_double)
            L.mh_config_default.argtypes = [ctypes.POINTER(Config)]
            L.mh_config_default.restype = None
            L.mh_create.argtypes = [ctypes.POINTER(P), I64, I, DP, DP, DP, D, ctypes.POINTER(Config), P]
            L.mh_restore.argtypes = [ctypes.POINTER(P), I64, I, DP, ctypes.POINTER(StateC), D,
                                     ctypes.POINTER(Config), P]
            L.mh_destroy.argtypes = [P]
            L.mh_destroy.restype = None
            L.mh_mlp_destroy.restype = None
            L.mh_step.argtypes = [P, D, I]
            L.mh_step_timesym.argtypes = [P, I64, I, I]
            L.mh_measure_peaks.argtypes = [DP]
            L.mh_sync.argtypes = [P, ctypes.POINTER(StateC)]
            L.mh_set_state.argtypes = [P, ctypes.POINTER(StateC)]
            L.mh_diagnostics.argtypes = [P, DP, DP, I]
            L.mh_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I), ctypes.POINTER(Counters)]
            L.mh_last_error.argtypes = []
            L.mh_last_error.restype = ctypes.c_char_p
            L.mh_pair_eval.argtypes = [I, I, I64, P, P, D, D, I64, I64, P, P]
            L.mh_release_scratch.argtypes = []
            L.mh_set_timing.argtypes = [P, I]
            L.mh_pair_eval_noalloc.argtypes = [I, I, I64, P, P, D, D, I64, I64, P, P]
            I64P = ctypes.POINTER(ctypes.c_int64)
            IP = ctypes.POINTER(ctypes.c_int)
            L.mh_sym_schedule_check.argtypes = [I64, I, I, IP]
            L.mh_create_batch.argtypes = [ctypes.POINTER(P), I64, I64P, DP, DP, DP, DP, D, I,
                                          ctypes.POINTER(Config), P]
            L.mh_step_batch.argtypes = [P, I64, I]
            L.mh_batch_tune.argtypes = [P, I, I, IP, IP]
            L.mh_batch_energy.argtypes = [P, DP]
            FP = ctypes.POINTER(ctypes.c_float)
            U64 = ctypes.c_uint64
            L.mh_step_converge.argtypes = [P, D, D, I, IP]
            L.mh_set_predictor.argtypes = [P, P]
            L.mh_collect_samples.argtypes = [P, D, I, P, P]
            L.mh_predict.argtypes = [P, D, DP, DP]
            L.mh_mlp_create.argtypes = [ctypes.POINTER(P), I, I, I, U64]
            L.mh_mlp_destroy.argtypes = [P]
            L.mh_mlp_num_params.argtypes = [P, I64P]
            L.mh_mlp_get_params.argtypes = [P, FP, I64]
            L.mh_mlp_set_params.argtypes = [P, FP, I64]
            L.mh_mlp_forward.argtypes = [P, P, P, I64, P]
            L.mh_mlp_loss_grad.argtypes = [P, P, P, I64, DP, FP, P]
            L.mh_mlp_train.argtypes = [P, P, P, I64, I, I, ctypes.c_float, U64, DP, P]
            L.mh_dd_create.argtypes = [ctypes.POINTER(P), I64, I, DP, DP, DP, D, ctypes.POINTER(Config), P]
            L.mh_dd_destroy.argtypes = [P]
            L.mh_dd_destroy.restype = None
            L.mh_dd_step.argtypes = [P, D, I, I64]
            L.mh_dd_sync.argtypes = [P, DP, DP, DP, DP]
            L.mh_dd_set_state.argtypes = [P, DP, DP, DP, DP]
            L.mh_dd_diagnostics.argtypes = [P, DP, DP, I]
            L.mh_dd_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I), ctypes.POINTER(Counters)]
            L.mh_dd_pair_eval.argtypes = [I, I64, DP, DP, D, D, I64, I64, I, DP]
            L.mh_dd_sym_check.argtypes = [I64, IP]
            L.mh_dd_create_batch.argtypes = [ctypes.POINTER(P), I64, I64P, DP, DP, DP, DP, D, I,
                                             ctypes.POINTER(Config), P]
            L.mh_dd_step_batch.argtypes = [P, I64, I]
            L.mh_dd_batch_energy.argtypes = [P, DP]
            for name in EXPORTS:
                if name not in ("mh_destroy", "mh_config_default", "mh_last_error", "mh_mlp_destroy",
                                "mh_dd_destroy"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def check(rc: int, allow=(MH_OK,)) -> int:
    if rc not in allow:
        msg = lib().mh_last_error().decode(errors="replace")
        raise MHError(rc, msg)
    return rc
