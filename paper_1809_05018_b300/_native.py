"""ctypes declarations of the C ABI in include/pmrf.h.

Loading fails loudly when lib/libpmrf.so is missing: there is no fallback
implementation of any step.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libpmrf.so")

PMRF_OK = 0
STATUS_NAMES = {0: "PMRF_OK", 1: "PMRF_ERR_ARG", 2: "PMRF_ERR_CUDA", 3: "PMRF_ERR_OOM", 4: "PMRF_ERR_NONFINITE",
                5: "PMRF_ERR_TIMEOUT", 6: "PMRF_ERR_UNSUPPORTED", 7: "PMRF_ERR_DEVICE"}
MAX_LABELS = 8
MAX_DEGREE = 4096

# array ids of pmrf_graph_get
ARR = dict(VERT_OFF=0, HOOD_SLICE_OFF=1, Y=2, NPIX=3, ADJ_OFF=4, ADJ=5, CLQ_OFF=6, CLQ=7, HOOD_OFF=8, HOOD=9,
           REP_OFF=10, REP_HOOD=11, RANK_OFF=12, RANK=13)


class PmrfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("n_labels", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("conv_window", ctypes.c_int32),
                ("init_from_labels", ctypes.c_int32), ("potts_scope", ctypes.c_int32),
                ("replica_rule", ctypes.c_int32), ("beta", ctypes.c_double), ("conv_tol", ctypes.c_double),
                ("sigma_min", ctypes.c_double), ("init_lo", ctypes.c_double), ("init_hi", ctypes.c_double)]


class BuildOptions(ctypes.Structure):
    _fields_ = [("hood_depth", ctypes.c_int32), ("volume_depth", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("hood_tile", ctypes.c_int32), ("hood_lanes", ctypes.c_int32), ("use_cuda_graph", ctypes.c_int32),
                ("profile", ctypes.c_int32)]


# (name, argtypes); every function returns int except where noted
_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_GP = ctypes.c_void_p
SIGNATURES = {
    "pmrf_config_default": [ctypes.POINTER(Config)],
    "pmrf_build_graph": [_P, _P, _I32, _P, _P, _P, ctypes.POINTER(_GP)],
    "pmrf_build_graph_ex": [_P, _P, _I32, _P, _P, _P, _P, ctypes.POINTER(_GP)],
    "pmrf_build_options_default": [_P],
    "pmrf_graph_destroy": [_GP],
    "pmrf_graph_stats": [_GP, _P, _P, _P, _P, _P],
    "pmrf_graph_len": [_GP, _I32, ctypes.POINTER(_I64)],
    "pmrf_graph_get": [_GP, _I32, _P, ctypes.c_size_t, _I32, _P],
    "pmrf_init_labels": [_GP, ctypes.POINTER(Config), _P, _P],
    "pmrf_params": [_GP, ctypes.POINTER(Config), _P, _P, _P, _P, _P],
    "pmrf_map_sweep": [_GP, ctypes.POINTER(Config), _P, _P, _P, _P, _P, _P],
    "pmrf_em": [_GP, ctypes.POINTER(Config), _P, _P, _P, _P, _P, _P],
    "pmrf_pll": [_GP, _I32, _P, _P, _P, _D, _P, _P],
    "pmrf_pll_grad": [_GP, _I32, _P, _P, _P, _D, _P, _P, _P, _P, _P],
    "pmrf_pll_value_and_grad": [_GP, _I32, _P, _P, _P, _D, _P, _P, _P, _P, _P, _P],
    "pmrf_pll_grad_noalloc": [_GP, _I32, _P, _P, _P, _D, _P, _P, _P, _P, _P],
    "pmrf_label_image": [_GP, _P, _P, _P, _P],
    "pmrf_quality": [_GP, ctypes.c_int32, _P, _P, _P, _P, _P],
    "pmrf_random_init": [_GP, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double, _P, _P, _P],
    "pmrf_sync_status": [_GP, _P, ctypes.POINTER(_I64)],
    "pmrf_get_tuning": [_GP, ctypes.POINTER(Tuning)],
    "pmrf_set_tuning": [_GP, ctypes.POINTER(Tuning)],
    "pmrf_autotune": [_GP, ctypes.POINTER(Config), _P, ctypes.POINTER(Tuning)],
    "pmrf_em_kernel_times": [_GP, _I32, _P, _P, ctypes.POINTER(_I32), _P],
    "pmrf_launch_count": [],
    "pmrf_trim_memory": [_I64],
    "pmrf_memory_usage": [ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "pmrf_last_error": [],
    "pmrf_version": [],
}

_lib = None


def load(path: str | None = None):
    """Load the shared library (once).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"PMRF CUDA library not built: {path} is missing "
                          f"(run `python -m paper_1809_05018_b300.build`)")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        if name in ("pmrf_last_error", "pmrf_version"):
            fn.restype = ctypes.c_char_p
        elif name == "pmrf_launch_count":
            fn.restype = ctypes.c_int64
        else:
            fn.restype = ctypes.c_int
    _lib = lib
    return lib


def check(rc: int, what: str):
    if rc != PMRF_OK:
        msg = _lib.pmrf_last_error().decode() if _lib is not None else ""
        raise PmrfError(rc, f"{what}: {msg}")


def exported_symbols():
    return list(SIGNATURES)
