"""ctypes declarations of the libfbcorr C ABI (include/fbcorr.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libfbcorr.so.  The library is built in-tree (``build.py``); if it is
missing, loading fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libfbcorr.so")

FBCORR_OK = 0
STATUS_NAMES = {
    0: "FBCORR_OK", 1: "FBCORR_ERR_INVALID_ARG", 2: "FBCORR_ERR_SHAPE",
    3: "FBCORR_ERR_UNSUPPORTED", 4: "FBCORR_ERR_ALIGNMENT", 5: "FBCORR_ERR_WORKSPACE",
    6: "FBCORR_ERR_CUDA", 7: "FBCORR_ERR_NVRTC", 8: "FBCORR_ERR_OOM", 9: "FBCORR_ERR_TIMEOUT",
    10: "FBCORR_ERR_INTERNAL",
}
DTYPES = {"f32": 0, "bf16": 1, "bf16x3": 2}
EPI_NONE, EPI_CLAMP, EPI_SNIPPET = 0, 1, 2


class FbcorrError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.status_name = STATUS_NAMES.get(status, f"status {status}")
        super().__init__(f"{where}: {self.status_name}: {detail}")


class Epilogue(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("lo", ctypes.c_float), ("hi", ctypes.c_float)]


def epilogue(clamp=None) -> Epilogue:
    if clamp is None:
        return Epilogue(EPI_NONE, 0.0, 0.0)
    lo, hi = clamp
    return Epilogue(EPI_CLAMP, float(lo), float(hi))


I64_3 = ctypes.c_int64 * 3
I64_4 = ctypes.c_int64 * 4
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_st = ctypes.c_int

# name -> (restype, argtypes); same names as include/fbcorr.h
PROTOTYPES = {
    "fbcorr_plan_create": (_st, [ctypes.POINTER(_vp), I64_3, I64_4, ctypes.c_int, Epilogue]),
    "fbcorr_plan_destroy": (_st, [_vp]),
    "fbcorr_plan_out_shape": (_st, [_vp, I64_3]),
    "fbcorr_plan_workspace_size": (_st, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "fbcorr_forward": (_st, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "fbcorr_forward_host": (_st, [_vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "fbcorr_plan_create_snippet": (_st, [ctypes.POINTER(_vp), I64_3, I64_4, ctypes.c_int, Epilogue, ctypes.c_char_p]),
    "fbcorr_snippet_check": (_st, [I64_3, I64_4, ctypes.c_int, ctypes.c_char_p, ctypes.c_char_p, _sz]),
    "fbcorr_plan_candidates": (_st, [_vp, ctypes.c_char_p, _sz]),
    "fbcorr_nn_plan_create": (_st, [ctypes.POINTER(_vp), ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]),
    "fbcorr_nn_plan_destroy": (_st, [_vp]),
    "fbcorr_nn_workspace_size": (_st, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "fbcorr_nn_search": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "fbcorr_nn_plan_device_status": (_st, [_vp, ctypes.c_int]),
    "fbcorr_nn_last_fallbacks": (_st, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "fbcorr_nn_rtcg_check": (_st, [ctypes.c_int64, ctypes.c_int, ctypes.c_char_p, _sz]),
    "fbcorr_backward": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "fbcorr_autotune": (_st, [_vp, _vp]),
    "fbcorr_plan_set_variant": (_st, [_vp, ctypes.c_char_p]),
    "fbcorr_plan_info": (_st, [_vp, ctypes.c_char_p, _sz]),
    "fbcorr_plan_device_status": (_st, [_vp, ctypes.c_int]),
    "fbcorr_forward_noalloc": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "fbcorr_plan_profile": (_st, [_vp, ctypes.c_int]),
    "fbcorr_plan_profile_read": (_st, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
    "fbcorr_batch_plan_create": (_st, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_int, Epilogue]),
    "fbcorr_batch_plan_destroy": (_st, [_vp]),
    "fbcorr_batch_plan_workspace_size": (_st, [_vp, ctypes.POINTER(_sz)]),
    "fbcorr_batch_plan_info": (_st, [_vp, ctypes.c_char_p, _sz]),
    "fbcorr_forward_batched": (_st, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                     _vp, _sz, _vp]),
    "fbcorr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fbcorr_last_error": (ctypes.c_char_p, []),
    "fbcorr_version": (ctypes.c_char_p, []),
    "fbcorr_fp32_fma_probe": (_st, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]),
    "fbcorr_rtcg_check": (_st, [I64_3, I64_4, Epilogue, ctypes.c_char_p, ctypes.c_char_p, _sz]),
    "fbcorr_batch_rtcg_check": (_st, [ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64), Epilogue, ctypes.c_char_p, _sz]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load the in-tree libfbcorr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfbcorr.so is not built ({LIB_PATH}); run "
                               "`python -m paper_0911_3456_gb300.build` (or __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def last_error() -> str:
    return load().fbcorr_last_error().decode(errors="replace")


def check(status: int, where: str) -> None:
    if status != FBCORR_OK:
        raise FbcorrError(status, where, last_error())


def call(name: str, *args):
    """Call C function `name` and raise FbcorrError on a non-OK status."""
    check(getattr(load(), name)(*args), name)
