"""ctypes binding of libarnold.so (include/arnold.h): argument marshalling only.

The library is loaded from this package directory.  There is no fallback:
if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libarnold.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED, ESTATE, ERANGE = 0, -1, -2, -3, -4, -5, -6, -7, -8
SCHEMES = {"yoshida6a": 0, "triplejump6": 1, "leapfrog2": 2}
PRECISIONS = {"fp64": 0, "fp32c": 1, "df64": 2, "df64f": 3}
HOST, DEVICE = 0, 1
IND = {"chi": 0, "V": 1, "dE": 2, "dE_max": 3, "class": 4, "X": 5, "P": 6, "dX": 7, "tangent": 8, "logsum": 9,
       "left": 10, "megno": 11, "megno_y": 12, "vdev": 13}
IND_SHAPE = {"chi": 1, "V": 3, "dE": 1, "dE_max": 1, "class": 1, "X": 3, "P": 3, "dX": 3, "tangent": 6, "logsum": 1,
             "left": 1, "megno": 1, "megno_y": 1, "vdev": 1}
SHELL_DIRECTION, SHELL_PZ = 1, 2
HIST_BINS = 200
NOALLOC_MAX_N = 1 << 40


class ArnoldError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


class Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("h", ctypes.c_double), ("scheme", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("tangent", ctypes.c_int32), ("renorm_every", ctypes.c_int32),
                ("window", ctypes.c_int64), ("chaos_kappa", ctypes.c_double), ("block_size", ctypes.c_int32),
                ("launch_steps", ctypes.c_int32), ("megno", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("hist", ctypes.c_uint64 * HIST_BINS), ("under", ctypes.c_uint64), ("over", ctypes.c_uint64),
                ("chaotic", ctypes.c_uint64), ("n", ctypes.c_uint64), ("dE_max", ctypes.c_double),
                ("p_mean", ctypes.c_double * 3), ("p_var", ctypes.c_double * 3), ("t", ctypes.c_double)]


class BatchSet(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("h", ctypes.c_double), ("E", ctypes.c_double), ("G", ctypes.c_int64),
                ("n_steps", ctypes.c_int64), ("seed", ctypes.c_uint64)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int32), ("traj_per_thread", ctypes.c_int32),
                ("renorm_every", ctypes.c_int32), ("epoch_ms", ctypes.c_int32)]


_lib = None
vp = ctypes.c_void_p
i64 = ctypes.c_int64
SIGNATURES = {
    "arnold_params_default": (None, [ctypes.POINTER(Params)]),
    "arnold_create": (ctypes.c_int, [ctypes.POINTER(Params), i64, ctypes.c_int, vp, ctypes.POINTER(vp)]),
    "arnold_destroy": (None, [vp]),
    "arnold_set_state": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int]),
    "arnold_init_grid": (ctypes.c_int, [vp, i64, i64, ctypes.c_double, ctypes.c_uint64, vp]),
    "arnold_iterate": (ctypes.c_int, [vp, i64]),
    "arnold_set_snapshots": (ctypes.c_int, [vp, vp, i64]),
    "arnold_set_state_shell": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
    "arnold_init_sphere": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_uint64, i64] + [ctypes.c_double] * 4),
    "arnold_init_gaussian": (ctypes.c_int, [vp] + [ctypes.c_double] * 4 + [ctypes.c_uint64, i64,
                                                                          ctypes.POINTER(i64)]),
    "arnold_track_patch": (ctypes.c_int, [vp] + [ctypes.c_double] * 4),
    "arnold_velocity_histogram": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 +
                                  [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int]),
    "arnold_steps_done": (i64, [vp]),
    "arnold_indicator": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
    "arnold_stats_compute": (ctypes.c_int, [vp, ctypes.POINTER(Stats)]),
    "arnold_stats_arrays": (ctypes.c_int, [vp, i64, vp, vp, vp, ctypes.c_double, ctypes.c_double,
                                           ctypes.POINTER(Stats)]),
    "arnold_stats_arrays_noalloc": (ctypes.c_int, [ctypes.c_int, vp, i64, vp, vp, vp, ctypes.c_double,
                                                   ctypes.c_double, ctypes.POINTER(Stats)]),
    "arnold_forward_ckpt": (ctypes.c_int, [vp, i64, i64]),
    "arnold_grad": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, ctypes.c_int]),
    "arnold_batch_tuning_default": (None, [ctypes.POINTER(BatchTuning)]),
    "arnold_batch_create": (ctypes.c_int, [ctypes.POINTER(BatchSet), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.POINTER(BatchTuning), ctypes.c_int, vp,
                                           ctypes.POINTER(vp)]),
    "arnold_batch_init": (ctypes.c_int, [vp]),
    "arnold_batch_run": (ctypes.c_int, [vp]),
    "arnold_batch_indicator": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int]),
    "arnold_batch_stats": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(Stats)]),
    "arnold_batch_info": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
    "arnold_batch_sync": (ctypes.c_int, [vp]),
    "arnold_batch_launch_count": (i64, [vp]),
    "arnold_batch_destroy": (None, [vp]),
    "arnold_checkpoint_size": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_size_t)]),
    "arnold_checkpoint_save": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
    "arnold_checkpoint_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
    "arnold_sync": (ctypes.c_int, [vp]),
    "arnold_launch_count": (i64, [vp]),
    "arnold_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "arnold_debug_sincos": (ctypes.c_int, [vp, ctypes.c_int, i64, vp, vp, vp]),
    "arnold_probe_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
}


def lib():
    """Load libarnold.so (once).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libarnold.so is not built ({LIB_PATH}); run python -m paper_1107_4107_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().arnold_strerror(status).decode()


def check(status: int, what: str) -> None:
    if status != OK:
        raise ArnoldError(status, what)
