"""A stack of filter-bank layers, each followed by a static non-linearity fused
into the store of its correlation kernel.

This is the structure of the paper's vision models (Sec. 6.2; Fig. 6b): every
layer's bank is "applied across" the output of the previous layer, between
linear filtering and static non-linearities.  The paper gives no parameters for
them, so only the structure is built: each layer is an ordinary plan (FP32
direct or tensor core, tuned per shape), the non-linearity is a snippet
epilogue (fbcorr_plan_create_snippet) and the intermediate outputs stay on the
device.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import torch

from .api import Plan


@dataclass
class Layer:
    filters: int                        # N
    fh: int
    fw: int
    nonlinearity: Optional[str] = None  # snippet expression of y, n, lo, hi (None: linear)
    params: Tuple[float, float] = (0.0, 0.0)


class Cascade:
    def __init__(self, in_shape: Sequence[int], layers: Sequence[Layer], dtype: str = "f32"):
        self.in_shape = tuple(int(v) for v in in_shape)
        self.layers = list(layers)
        self.plans: List[Plan] = []
        shape = self.in_shape
        for L in self.layers:
            filt = (L.filters, L.fh, L.fw, shape[2])
            p = (Plan(shape, filt, dtype, snippet=L.nonlinearity, snippet_params=L.params)
                 if L.nonlinearity else Plan(shape, filt, dtype))
            self.plans.append(p)
            shape = p.out_shape
        self.out_shape = shape

    @property
    def filt_shapes(self):
        return [p.filt_shape for p in self.plans]

    @property
    def flops(self) -> int:
        return sum(p.flops for p in self.plans)

    def autotune(self) -> None:
        for p in self.plans:
            p.autotune()

    def forward(self, x: torch.Tensor, banks: Sequence[torch.Tensor], outs=None, stream=None) -> torch.Tensor:
        """Run every layer on the device; ``outs`` (optional) are the per-layer
        output tensors, reused across calls.  Returns the last layer's output."""
        if len(banks) != len(self.plans):
            raise ValueError(f"need {len(self.plans)} filter banks")
        h = x
        for k, (p, w) in enumerate(zip(self.plans, banks)):
            h = p.forward(h, w, None if outs is None else outs[k], stream=stream)
        return h
