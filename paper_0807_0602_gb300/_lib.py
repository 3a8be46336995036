"""ctypes declarations of the C ABI in include/lbm.h (argument marshalling only).

The library must have been built (``paper_0807_0602_gb300.build.build()`` or
``__graft_entry__.build()``); loading fails loudly otherwise: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB, LIB_CHECKED

c_int32, c_int64, c_double, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                  ctypes.c_void_p, ctypes.c_size_t)
P = ctypes.POINTER

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ESTATE, LBM_EIO, LBM_EBOUNDS = range(9)
LBM_F64, LBM_F32, LBM_F16S = 0, 1, 2
LBM_INIT_SLAB, LBM_INIT_DROPLET, LBM_INIT_FIELDS = 0, 1, 2

ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_void_p, c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, c_size_t, c_void_p)


class Geometry(ctypes.Structure):
    _fields_ = [
        ("nx", c_int32), ("ny", c_int32), ("cap_x0", c_int32), ("cap_x1", c_int32),
        ("y_bot", c_int32), ("y_top", c_int32), ("init_kind", c_int32), ("reserved0", c_int32),
        ("solid_mask", P(ctypes.c_uint8)),
        ("x_lo", c_double), ("x_hi", c_double), ("drop_cx", c_double), ("drop_cy", c_double),
        ("drop_r", c_double), ("rho_major", c_double), ("rho_minor", c_double),
        ("init_nA", P(c_double)), ("init_nB", P(c_double)),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", c_int32), ("log_every", c_int32), ("log_capacity", c_int32), ("autotune", c_int32),
        ("tile_w", c_int32), ("tile_h", c_int32), ("graph_chunk", c_int32), ("reserved0", c_int32),
        ("rho_ref", c_double * 2), ("rho_bulk", c_double), ("body", c_double * 2),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", c_void_p), ("stream", c_void_p),
        ("alpha", c_double * 2), ("molecular_mass", c_double * 2),
    ]


class RunInfo(ctypes.Structure):
    _fields_ = [
        ("nx", c_int32), ("ny", c_int32), ("pitch", c_int32), ("precision", c_int32),
        ("current", c_int32), ("elem_bytes", c_int32), ("time", c_int64), ("base", c_void_p * 2),
    ]


# name -> (restype, argtypes); every function declared in include/lbm.h
SIGNATURES = {
    "lbm_get_columns": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_void_p, ctypes.c_int]),
    "lbm_set_columns": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_void_p, ctypes.c_int]),
    "lbm_selftest_fp64_rate": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), c_void_p]),
    "lbm_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_longlong, c_void_p]),
    "lbm_default_options": (None, [P(Options)]),
    "lbm_create": (ctypes.c_int, [P(Geometry), c_double, P(c_double), c_double, c_double, P(Options),
                                  P(c_void_p)]),
    "lbm_create_batch": (ctypes.c_int, [ctypes.c_int, P(Geometry), P(c_double), P(c_double), P(c_double),
                                        P(c_double), P(Options), P(c_void_p)]),
    "lbm_step": (ctypes.c_int, [c_void_p, c_int64]),
    "lbm_sync": (ctypes.c_int, [c_void_p]),
    "lbm_time": (c_int64, [c_void_p]),
    "lbm_num_runs": (ctypes.c_int, [c_void_p]),
    "lbm_run_info_get": (ctypes.c_int, [c_void_p, ctypes.c_int, P(RunInfo)]),
    "lbm_densities": (ctypes.c_int, [c_void_p, ctypes.c_int, c_void_p, c_void_p, ctypes.c_int]),
    "lbm_velocity": (ctypes.c_int, [c_void_p, ctypes.c_int, c_void_p, c_void_p, ctypes.c_int]),
    "lbm_interface_positions": (ctypes.c_int, [c_void_p, ctypes.c_int, P(c_double), P(c_double)]),
    "lbm_get_log": (ctypes.c_int, [c_void_p, ctypes.c_int, P(c_double), ctypes.c_int, P(ctypes.c_int)]),
    "lbm_mass": (ctypes.c_int, [c_void_p, ctypes.c_int, P(c_double)]),
    "lbm_populations": (ctypes.c_int, [c_void_p, ctypes.c_int, c_void_p, ctypes.c_int]),
    "lbm_get_tiling": (ctypes.c_int, [c_void_p, P(ctypes.c_int), P(ctypes.c_int)]),
    "lbm_set_tiling": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int]),
    "lbm_get_schedule": (ctypes.c_int, [c_void_p, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                                        P(ctypes.c_int)]),
    "lbm_set_schedule": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lbm_get_tuning": (ctypes.c_int, [c_void_p, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_float),
                                      P(ctypes.c_int)]),
    "lbm_save": (ctypes.c_int, [c_void_p, ctypes.c_char_p]),
    "lbm_load": (ctypes.c_int, [ctypes.c_char_p, P(Options), P(c_void_p)]),
    "lbm_mass_noalloc": (ctypes.c_int, [P(Geometry), ctypes.c_int, c_void_p, ctypes.c_int, P(c_double), c_void_p,
                                        c_void_p]),
    "lbm_status": (ctypes.c_int, [c_void_p]),
    "lbm_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_destroy": (None, [c_void_p]),
}

_lock = threading.Lock()
_lib = None


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load().lbm_error_string(code).decode() if code < 64 else "unknown"
        super().__init__(f"{where}: {msg} (code {code})")


def load():
    """Loads the in-tree library; raises if it has not been built.  With the
    environment variable LBM_CHECKED=1 the process loads the checked build
    (build(checked=True)) instead."""
    global _lib
    with _lock:
        if _lib is None:
            path = LIB_CHECKED if os.environ.get("LBM_CHECKED") == "1" else LIB
            if not os.path.exists(path):
                raise RuntimeError(
                    f"CUDA library {path} is missing: build it with paper_0807_0602_gb300.build.build() "
                    "(there is no CPU fallback)")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(code: int, where: str) -> None:
    if code != LBM_OK:
        raise LbmError(code, where)
