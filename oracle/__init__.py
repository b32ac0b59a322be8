"""FP64 CPU oracle for 3D filter-bank correlation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never imports, links or
calls it, and the two share no code.

The operation (the paper's vision case study, Sec. 6.2, and its Table
"Performance of RTCG auto-tuning on 3D filter-bank convolutions"): an
H x W x D input correlated 'valid' against N filters of fh x fw x D,

    y[p, q, n] = sum_{i, j, d} x[p+i, q+j, d] * w[n, i, j, d],

optionally clamped, plus the two gradients of <y, g>; and the exact
nearest-neighbour search of the paper's second case study (Sec. 6.4): for every
target vector the index and squared Euclidean distance of its nearest neighbour
(lowest index on ties) and the runner-up distance.  The arithmetic lives in
``fbcorr_oracle.c`` and ``nn_oracle.c`` as FP64 loops; this module only widens
the inputs to FP64 (exactly) and marshals arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fbcorr_oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "nn_oracle.c"))
_LIB = os.path.join(_HERE, "liboracle.so")

EPI_NONE = 0
EPI_CLAMP = 1

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(map(os.path.getmtime, _SRCS)):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lp = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_fbcorr_fwd.argtypes = [dp, i64, i64, i64, dp, i64, i64, i64,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_fbcorr_fwd_points.argtypes = [dp, i64, i64, i64, dp, i64, i64, i64,
                                                 ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                 i64, lp, dp]
        lib.oracle_fbcorr_bwd_input.argtypes = [dp, dp, i64, i64, i64, dp, i64, i64, i64,
                                                ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_fbcorr_bwd_input_points.argtypes = [dp, dp, i64, i64, i64, dp, i64, i64, i64,
                                                       ctypes.c_int, ctypes.c_double,
                                                       ctypes.c_double, i64, lp, dp]
        lib.oracle_fbcorr_bwd_filt.argtypes = [dp, dp, dp, i64, i64, i64, i64, i64, i64,
                                               ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        for f in ("oracle_fbcorr_fwd", "oracle_fbcorr_fwd_points", "oracle_fbcorr_bwd_input",
                  "oracle_fbcorr_bwd_input_points", "oracle_fbcorr_bwd_filt"):
            getattr(lib, f).restype = ctypes.c_int
        lib.oracle_nn.argtypes = [dp, i64, dp, i64, i64, lp, dp, dp]
        lib.oracle_nn.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Thread count for the OpenMP loops (0 = OpenMP default)."""
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _f64(a) -> np.ndarray:
    a = np.asarray(a)
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _epi(epilogue):
    if epilogue is None:
        return EPI_NONE, 0.0, 0.0
    lo, hi = epilogue
    return EPI_CLAMP, float(lo), float(hi)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (code {rc})")


def fwd(x, w, epilogue=None) -> np.ndarray:
    """y[H', W', N] in FP64.  ``epilogue`` is None or a (lo, hi) clamp."""
    x = _f64(x)
    w = _f64(w)
    H, W, D = x.shape
    N, fh, fw, Dw = w.shape
    if Dw != D:
        raise ValueError("filter depth must equal input depth")
    kind, lo, hi = _epi(epilogue)
    y = np.empty((H - fh + 1, W - fw + 1, N), dtype=np.float64)
    _check(_load().oracle_fbcorr_fwd(_ptr(x), H, W, D, _ptr(w), N, fh, fw, kind, lo, hi, _ptr(y)),
           "fwd")
    return y


def fwd_points(x, w, idx, epilogue=None) -> np.ndarray:
    """y at the (p, q, n) triples in ``idx`` (shape [k, 3])."""
    x = _f64(x)
    w = _f64(w)
    idx = np.ascontiguousarray(idx, dtype=np.int64).reshape(-1, 3)
    H, W, D = x.shape
    N, fh, fw, _ = w.shape
    kind, lo, hi = _epi(epilogue)
    out = np.empty(idx.shape[0], dtype=np.float64)
    _check(_load().oracle_fbcorr_fwd_points(
        _ptr(x), H, W, D, _ptr(w), N, fh, fw, kind, lo, hi, idx.shape[0],
        idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(out)), "fwd_points")
    return out


def bwd_input(g, w, in_shape, y=None, epilogue=None) -> np.ndarray:
    """dL/dx for L = <y, g>; ``y`` (the clamped forward output) is needed with a clamp."""
    g = _f64(g)
    w = _f64(w)
    H, W, D = in_shape
    N, fh, fw, _ = w.shape
    kind, lo, hi = _epi(epilogue)
    yp = None
    if y is not None:
        y = _f64(y)
        yp = _ptr(y)
    dx = np.empty((H, W, D), dtype=np.float64)
    _check(_load().oracle_fbcorr_bwd_input(_ptr(g), yp, H, W, D, _ptr(w), N, fh, fw,
                                           kind, lo, hi, _ptr(dx)), "bwd_input")
    return dx


def bwd_input_points(g, w, in_shape, idx, y=None, epilogue=None) -> np.ndarray:
    g = _f64(g)
    w = _f64(w)
    idx = np.ascontiguousarray(idx, dtype=np.int64).reshape(-1, 3)
    H, W, D = in_shape
    N, fh, fw, _ = w.shape
    kind, lo, hi = _epi(epilogue)
    yp = None
    if y is not None:
        y = _f64(y)
        yp = _ptr(y)
    out = np.empty(idx.shape[0], dtype=np.float64)
    _check(_load().oracle_fbcorr_bwd_input_points(
        _ptr(g), yp, H, W, D, _ptr(w), N, fh, fw, kind, lo, hi, idx.shape[0],
        idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(out)), "bwd_input_points")
    return out


def bwd_filt(x, g, filt_shape, y=None, epilogue=None) -> np.ndarray:
    """dL/dw[N, fh, fw, D] for L = <y, g>."""
    x = _f64(x)
    g = _f64(g)
    H, W, D = x.shape
    N, fh, fw, _ = filt_shape
    kind, lo, hi = _epi(epilogue)
    yp = None
    if y is not None:
        y = _f64(y)
        yp = _ptr(y)
    dw = np.empty((N, fh, fw, D), dtype=np.float64)
    _check(_load().oracle_fbcorr_bwd_filt(_ptr(x), _ptr(g), yp, H, W, D, N, fh, fw,
                                          kind, lo, hi, _ptr(dw)), "bwd_filt")
    return dw


def nn(targets, neighbors):
    """Exact nearest neighbours (Sec. 6.4): for targets [nt, dim] and neighbors
    [nn, dim], returns (idx [nt] int64, dist [nt], dist2 [nt]) -- the index of the
    nearest neighbour (lowest on ties), its squared Euclidean distance and the
    runner-up squared distance, all in FP64."""
    t = _f64(targets)
    n = _f64(neighbors)
    if t.ndim != 2 or n.ndim != 2 or t.shape[1] != n.shape[1]:
        raise ValueError("targets [nt, dim] and neighbors [nn, dim] must share dim")
    nt, dim = t.shape
    idx = np.empty(nt, dtype=np.int64)
    dist = np.empty(nt, dtype=np.float64)
    dist2 = np.empty(nt, dtype=np.float64)
    _check(_load().oracle_nn(_ptr(t), nt, _ptr(n), n.shape[0], dim,
                             idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(dist), _ptr(dist2)),
           "nn")
    return idx, dist, dist2
