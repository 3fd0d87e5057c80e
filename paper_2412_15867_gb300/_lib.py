"""ctypes view of libirgs.so (include/irgs.h). Loads the in-tree library and
fails loudly when it is missing: there is no fallback implementation."""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_obj", "libirgs.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "irgs.h")

STATUS = {0: "IRGS_OK", 1: "IRGS_ERR_INVALID_ARG", 2: "IRGS_ERR_OOM", 3: "IRGS_ERR_CUDA",
          4: "IRGS_ERR_NONFINITE", 5: "IRGS_ERR_TIMEOUT", 6: "IRGS_ERR_UNSUPPORTED",
          7: "IRGS_ERR_DEVICE"}


class IrgsError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class Surfels(C.Structure):
    _fields_ = [("means", C.c_void_p), ("quats", C.c_void_p), ("scales", C.c_void_p),
                ("opacity", C.c_void_p), ("features", C.c_void_p), ("n", C.c_int64),
                ("num_features", C.c_int32)]


class TraceParamsC(C.Structure):
    _fields_ = [("k", C.c_int32), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("T_min", C.c_float), ("t_min", C.c_float), ("t_max", C.c_float),
                ("feat_offset", C.c_int32), ("feat_count", C.c_int32), ("flags", C.c_uint32)]


_lock = threading.Lock()
_lib = None

P = C.c_void_p
_SIGS = {
    "irgs_status_string": (C.c_char_p, [C.c_int]),
    "irgs_abi_version": (C.c_int32, []),
    "irgs_refit_scene": (C.c_int, [P, C.POINTER(Surfels), P]),
    "irgs_envmap_create": (C.c_int, [P, C.c_int32, C.c_int32, P, C.POINTER(C.c_void_p)]),
    "irgs_rasterize": (C.c_int, [P, P, C.POINTER(TraceParamsC), P, P, P, P, P]),
    "irgs_envmap_destroy": (C.c_int, [P]),
    "irgs_envmap_export": (C.c_int, [P, P, P, P, P, P, P]),
    "irgs_relight": (C.c_int, [P, P, P, P, P, P, P, C.c_int64, C.c_int32, C.c_uint64, C.POINTER(TraceParamsC),
                               P, P, P, P]),
    "irgs_kernel_launches": (C.c_uint64, []),
    "irgs_shade_sample_rays": (C.c_int, [P, P, P, C.c_int64, C.c_int32, C.c_int32, C.c_uint64, C.c_uint32, P, P,
                                         P]),
    "irgs_relight_sample_rays": (C.c_int, [P, C.c_int64, C.c_int32, C.c_uint64, P, P, P, P]),
    "irgs_probe_fma": (C.c_int, [C.c_int64, P, C.POINTER(C.c_double)]),
    "irgs_build_scene": (C.c_int, [C.POINTER(Surfels), C.c_float, P, C.POINTER(P)]),
    "irgs_build_scene_ex": (C.c_int, [C.POINTER(Surfels), C.c_float, C.c_uint32, P, C.POINTER(P)]),
    "irgs_update_scene": (C.c_int, [P, C.POINTER(Surfels), P]),
    "irgs_destroy_scene": (C.c_int, [P]),
    "irgs_scene_info": (C.c_int, [P, P, P, P, P]),
    "irgs_scene_status": (C.c_int, [P, P, P]),
    "irgs_scene_export": (C.c_int, [P, P, P, P, P]),
    "irgs_scene_export_wide": (C.c_int, [P, P, C.c_int64, P]),
    "irgs_trace_forward": (C.c_int, [P, P, P, C.c_int64, C.POINTER(TraceParamsC), P, P, P, P, P,
                                     C.c_int32, P]),
    "irgs_trace_stats": (C.c_int, [P, P, P, C.c_int64, C.POINTER(TraceParamsC), P, P]),
    "irgs_trace_backward": (C.c_int, [P, P, P, C.c_int64, C.POINTER(TraceParamsC), P, P, P, P, P,
                                      C.c_int32, P, P, P, P, P, P, P, P, P]),
    "irgs_build_lbvh_noalloc": (C.c_int, [C.POINTER(Surfels), C.c_float, P, P, P, P, P]),
    "irgs_build_lbvh_noalloc_status": (C.c_int, [C.c_int32, P, C.POINTER(C.c_uint32)]),
    "irgs_shade_mc": (C.c_int, [P, P, P, P, P, P, C.c_int64, P, C.c_int32, C.c_int32, C.c_int32,
                                C.c_int32, C.c_uint64, C.POINTER(TraceParamsC), P, P, P, P]),
    "irgs_shade_mc_backward": (C.c_int, [P, P, P, P, P, P, C.c_int64, P, C.c_int32, C.c_int32, C.c_int32,
                                         C.c_int32, C.c_uint64, C.POINTER(TraceParamsC), P, P, P, P, P, P, P,
                                         P, P, P]),
}


def declared_symbols() -> list[str]:
    """Function names declared in include/irgs.h."""
    text = re.sub(r"/\*.*?\*/", " ", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(irgs_[a-z_0-9]+)\s*\(", text)))


def lib() -> C.CDLL:
    """The loaded libirgs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libirgs.so is not built ({LIB_PATH}); run "
                              "`python -m paper_2412_15867_gb300._build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int, what: str) -> None:
    if status != 0:
        raise IrgsError(status, what)
