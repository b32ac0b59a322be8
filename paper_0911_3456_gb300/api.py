"""PyTorch-facing binding of libfbcorr: plans, forward/backward, batches and a
``torch.autograd.Function``.

PyTorch supplies only device memory and the current stream; every arithmetic
step runs in libfbcorr's CUDA kernels through the C ABI (``_capi``).  Tensors
use the library's layouts: x [H, W, D], w [N, fh, fw, D], y [H', W', N]; all
contiguous FP32 on a CUDA device.
"""
from __future__ import annotations

import ctypes
import json
import threading
from typing import Optional, Sequence, Tuple

import torch

from . import _capi as C

Clamp = Optional[Tuple[float, float]]


def _check_tensor(t: torch.Tensor, name: str, shape=None) -> None:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device (libfbcorr has no CPU path)")
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def _check_host_tensor(t: torch.Tensor, name: str, shape) -> None:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a CPU torch.Tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous float32")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def _vp(t: Optional[torch.Tensor]) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A single-image correlation plan (``fbcorr_plan_create``)."""

    def __init__(self, in_shape: Sequence[int], filt_shape: Sequence[int], dtype: str = "f32",
                 clamp: Clamp = None, snippet: Optional[str] = None,
                 snippet_params: Tuple[float, float] = (0.0, 0.0)):
        """``snippet``: a C expression of float y (the accumulator), int n (the
        filter index) and float lo, hi (= ``snippet_params``) compiled into the
        forward kernels as the epilogue (fbcorr_plan_create_snippet); forward
        only.  Excludes ``clamp``."""
        if dtype not in C.DTYPES:
            raise ValueError(f"dtype must be one of {sorted(C.DTYPES)}")
        if snippet is not None and clamp is not None:
            raise ValueError("a plan has one epilogue: clamp or snippet")
        self.in_shape = tuple(int(v) for v in in_shape)
        self.filt_shape = tuple(int(v) for v in filt_shape)
        self.dtype = dtype
        self.clamp = None if clamp is None else (float(clamp[0]), float(clamp[1]))
        self.snippet = snippet
        h = ctypes.c_void_p()
        if snippet is None:
            C.call("fbcorr_plan_create", ctypes.byref(h), C.I64_3(*self.in_shape),
                   C.I64_4(*self.filt_shape), C.DTYPES[dtype], C.epilogue(self.clamp))
        else:
            lo, hi = snippet_params
            C.call("fbcorr_plan_create_snippet", ctypes.byref(h), C.I64_3(*self.in_shape),
                   C.I64_4(*self.filt_shape), C.DTYPES[dtype], C.Epilogue(C.EPI_SNIPPET, float(lo), float(hi)),
                   snippet.encode())
        self._h = h
        out = C.I64_3()
        C.call("fbcorr_plan_out_shape", h, out)
        self.out_shape = tuple(out)
        fwd, bwd = ctypes.c_size_t(), ctypes.c_size_t()
        C.call("fbcorr_plan_workspace_size", h, ctypes.byref(fwd), ctypes.byref(bwd))
        self.ws_fwd, self.ws_bwd = fwd.value, bwd.value
        self._ws = {}

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            C.load().fbcorr_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    # -- workspace (cached per plan and device; pass ws= for concurrent streams)
    def workspace(self, nbytes: int, device) -> Optional[torch.Tensor]:
        if nbytes == 0:
            return None
        key = (torch.device(device).index, nbytes)
        ws = self._ws.get(key)
        if ws is None:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
            self._ws[key] = ws
        return ws

    # -- calls
    def forward(self, x: torch.Tensor, w: torch.Tensor, y: Optional[torch.Tensor] = None,
                ws: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        _check_tensor(x, "x", self.in_shape)
        _check_tensor(w, "w", self.filt_shape)
        if y is None:
            y = torch.empty(self.out_shape, dtype=torch.float32, device=x.device)
        _check_tensor(y, "y", self.out_shape)
        if ws is None:
            ws = self.workspace(self.ws_fwd, x.device)
        nbytes = ws.numel() * ws.element_size() if ws is not None else 0
        C.call("fbcorr_forward", self._h, _vp(x), _vp(w), _vp(y), _vp(ws), nbytes,
               _stream_handle(stream))
        return y

    def forward_host(self, x: torch.Tensor, w: torch.Tensor, y: Optional[torch.Tensor] = None,
                     bands: int = 0, stream=None) -> torch.Tensor:
        """The forward from host (CPU) tensors with overlapped transfers
        (fbcorr_forward_host).  Page-locked tensors (``pin_memory()``) let the
        copies overlap the compute; the result is complete once ``stream``
        (default: the current stream) reaches this call."""
        for t, name, shape in ((x, "x", self.in_shape), (w, "w", self.filt_shape)):
            _check_host_tensor(t, name, shape)
        if y is None:
            y = torch.empty(self.out_shape, dtype=torch.float32).pin_memory()
        _check_host_tensor(y, "y", self.out_shape)
        C.call("fbcorr_forward_host", self._h, _vp(x), _vp(w), _vp(y), int(bands), _stream_handle(stream))
        return y

    def backward(self, x: torch.Tensor, w: torch.Tensor, g: torch.Tensor,
                 y: Optional[torch.Tensor] = None, need_dx: bool = True, need_dw: bool = True,
                 ws: Optional[torch.Tensor] = None, stream=None):
        _check_tensor(g, "g", self.out_shape)
        if need_dw:
            _check_tensor(x, "x", self.in_shape)
        if need_dx:
            _check_tensor(w, "w", self.filt_shape)
        if y is not None:
            _check_tensor(y, "y", self.out_shape)
        dev = g.device
        dx = torch.empty(self.in_shape, dtype=torch.float32, device=dev) if need_dx else None
        dw = torch.empty(self.filt_shape, dtype=torch.float32, device=dev) if need_dw else None
        if ws is None and need_dw:
            ws = self.workspace(self.ws_bwd, dev)
        nbytes = ws.numel() * ws.element_size() if ws is not None else 0
        C.call("fbcorr_backward", self._h, _vp(x if need_dw else None), _vp(w if need_dx else None),
               _vp(g), _vp(y), _vp(dx), _vp(dw), _vp(ws), nbytes, _stream_handle(stream))
        return dx, dw

    def autotune(self, stream=None) -> None:
        C.call("fbcorr_autotune", self._h, _stream_handle(stream))

    def candidates(self):
        """The forward variants the auto-tuner times for this plan (spec strings)."""
        buf = ctypes.create_string_buffer(1 << 18)
        C.call("fbcorr_plan_candidates", self._h, buf, len(buf))
        return [s for s in buf.value.decode().split("\n") if s]

    def set_variant(self, spec: str) -> None:
        C.call("fbcorr_plan_set_variant", self._h, spec.encode())

    def info(self) -> dict:
        buf = ctypes.create_string_buffer(8192)
        C.call("fbcorr_plan_info", self._h, buf, len(buf))
        return json.loads(buf.value.decode())

    def profile(self, capacity: int) -> None:
        """Record events around the main kernel of the next `capacity` forward calls."""
        C.call("fbcorr_plan_profile", self._h, int(capacity))

    def profile_read(self):
        """Milliseconds of each recorded main-kernel launch (waits for them)."""
        cap = 1 << 16
        buf = (ctypes.c_float * cap)()
        n = ctypes.c_int()
        C.call("fbcorr_plan_profile_read", self._h, buf, cap, ctypes.byref(n))
        return [buf[i] for i in range(n.value)]

    def device_status(self, clear: bool = False) -> int:
        """0, or the FBCORR_ERR_TIMEOUT status once a kernel gave up a bounded wait."""
        return int(C.load().fbcorr_plan_device_status(self._h, 1 if clear else 0))

    @property
    def flops(self) -> int:
        Ho, Wo, N = self.out_shape
        _, fh, fw, D = self.filt_shape
        return 2 * Ho * Wo * N * fh * fw * D


class BatchPlan:
    """Many uneven images in one persistent launch (``fbcorr_batch_plan_create``)."""

    def __init__(self, in_shapes, filt_shapes, dtype: str = "f32", clamp: Clamp = None):
        if len(in_shapes) != len(filt_shapes) or not in_shapes:
            raise ValueError("need matching, non-empty shape lists")
        self.in_shapes = [tuple(int(v) for v in s) for s in in_shapes]
        self.filt_shapes = [tuple(int(v) for v in s) for s in filt_shapes]
        self.out_shapes = [(a[0] - b[1] + 1, a[1] - b[2] + 1, b[0])
                           for a, b in zip(self.in_shapes, self.filt_shapes)]
        n = len(self.in_shapes)
        ins = (ctypes.c_int64 * (3 * n))(*[v for s in self.in_shapes for v in s])
        fls = (ctypes.c_int64 * (4 * n))(*[v for s in self.filt_shapes for v in s])
        h = ctypes.c_void_p()
        C.call("fbcorr_batch_plan_create", ctypes.byref(h), n, ins, fls, C.DTYPES[dtype],
               C.epilogue(clamp))
        self._h = h
        sz = ctypes.c_size_t()
        C.call("fbcorr_batch_plan_workspace_size", h, ctypes.byref(sz))
        self.ws_bytes = sz.value
        self._ws = None
        self.n = n

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            C.load().fbcorr_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        buf = ctypes.create_string_buffer(1 << 16)
        C.call("fbcorr_batch_plan_info", self._h, buf, len(buf))
        return json.loads(buf.value.decode())

    def forward(self, xs, ws_, ys=None, stream=None):
        if len(xs) != self.n or len(ws_) != self.n:
            raise ValueError("one x and one w per image")
        if ys is None:
            ys = [torch.empty(s, dtype=torch.float32, device=xs[0].device) for s in self.out_shapes]
        for k in range(self.n):
            _check_tensor(xs[k], f"x[{k}]", self.in_shapes[k])
            _check_tensor(ws_[k], f"w[{k}]", self.filt_shapes[k])
            _check_tensor(ys[k], f"y[{k}]", self.out_shapes[k])
        arr = ctypes.c_void_p * self.n
        xp = arr(*[t.data_ptr() for t in xs])
        wp = arr(*[t.data_ptr() for t in ws_])
        yp = arr(*[t.data_ptr() for t in ys])
        if self.ws_bytes and self._ws is None:
            self._ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=xs[0].device)
        C.call("fbcorr_forward_batched", self._h, xp, wp, yp, _vp(self._ws), self.ws_bytes,
               _stream_handle(stream))
        return ys

    @property
    def flops(self) -> int:
        return sum(2 * o[0] * o[1] * o[2] * f[1] * f[2] * f[3]
                   for o, f in zip(self.out_shapes, self.filt_shapes))


_plans = {}
_plans_lock = threading.Lock()


class NNPlan:
    """Exact brute-force nearest-neighbour search (fbcorr_nn_*): for each target
    row the index and exact FP32 squared distance of its nearest neighbour row."""

    def __init__(self, n_targets: int, n_neighbors: int, dim: int, dtype: str = "bf16x3"):
        if dtype not in ("bf16x3", "bf16"):
            raise ValueError("dtype must be bf16x3 or bf16")
        self.n_targets, self.n_neighbors, self.dim, self.dtype = int(n_targets), int(n_neighbors), int(dim), dtype
        h = ctypes.c_void_p()
        C.call("fbcorr_nn_plan_create", ctypes.byref(h), self.n_targets, self.n_neighbors, self.dim, C.DTYPES[dtype])
        self._h = h
        n = ctypes.c_size_t()
        C.call("fbcorr_nn_workspace_size", h, ctypes.byref(n))
        self.ws_bytes = n.value
        self._ws = None

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            C.load().fbcorr_nn_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_status(self, clear: bool = False) -> int:
        return int(C.load().fbcorr_nn_plan_device_status(self._h, 1 if clear else 0))

    def last_fallbacks(self) -> int:
        """Targets of the last search whose screening window could not be
        certified and that were searched exhaustively instead (synchronises)."""
        n = ctypes.c_int64()
        C.call("fbcorr_nn_last_fallbacks", self._h, ctypes.byref(n))
        return int(n.value)

    def search(self, targets: torch.Tensor, neighbors: torch.Tensor, stream=None):
        _check_tensor(targets, "targets", (self.n_targets, self.dim))
        _check_tensor(neighbors, "neighbors", (self.n_neighbors, self.dim))
        dev = targets.device
        if self._ws is None or self._ws.device != dev:
            self._ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        idx = torch.empty(self.n_targets, dtype=torch.int64, device=dev)
        dist = torch.empty(self.n_targets, dtype=torch.float32, device=dev)
        C.call("fbcorr_nn_search", self._h, _vp(targets), _vp(neighbors), _vp(idx), _vp(dist), _vp(self._ws),
               self.ws_bytes, _stream_handle(stream))
        return idx, dist

    @property
    def flops(self) -> int:
        """3 FLOPs (difference, multiply, add) per coordinate of every target-neighbour pair."""
        return 3 * self.n_targets * self.n_neighbors * self.dim


def get_plan(in_shape, filt_shape, dtype="f32", clamp: Clamp = None, device=None) -> Plan:
    """A process-wide cache of plans keyed by device, shapes, dtype and epilogue."""
    dev = torch.cuda.current_device() if device is None else torch.device(device).index
    key = (dev, tuple(in_shape), tuple(filt_shape), dtype, None if clamp is None else tuple(clamp))
    with _plans_lock:
        p = _plans.get(key)
        if p is None:
            with torch.cuda.device(dev):
                p = Plan(in_shape, filt_shape, dtype, clamp)
            _plans[key] = p
        return p


class FBCorr(torch.autograd.Function):
    """y = epi(corr(x, w)) with hand-written backward kernels (always FP32)."""

    @staticmethod
    def forward(ctx, x, w, dtype="f32", clamp=None):
        plan = get_plan(x.shape, w.shape, dtype, clamp, x.device)
        y = plan.forward(x.contiguous(), w.contiguous())
        ctx.clamp = clamp
        ctx.save_for_backward(x, w, y)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, w, y = ctx.saved_tensors
        plan = get_plan(x.shape, w.shape, "f32", ctx.clamp, x.device)
        dx, dw = plan.backward(x.contiguous(), w.contiguous(), gy.contiguous(),
                               y if ctx.clamp is not None else None,
                               need_dx=ctx.needs_input_grad[0], need_dw=ctx.needs_input_grad[1])
        return dx, dw, None, None


def fbcorr(x, w, dtype: str = "f32", clamp: Clamp = None):
    """Functional form: differentiable filter-bank correlation."""
    return FBCorr.apply(x, w, dtype, clamp)
