"""Seeded synthetic inputs for filter-bank correlation workloads.

This module holds random-number recipes only -- none of the correlation
arithmetic -- so that both the GPU tests and the CPU oracle can be fed the
same arrays.  Every array is drawn in FP64 with ``numpy.random.default_rng``
and cast to FP32; draw order is x, then w, then g.

Shapes follow the paper's Table "Performance of RTCG auto-tuning on 3D
filter-bank convolutions" (input H x W x D, bank N x fh x fw x D): the
256x256x8 / 64x9x9x8 workload below is that table's first row.  The paper's
inputs came from natural-image model layers that are not available, so
uniform and Gaussian draws of the same shapes stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np


def uniform(rng, shape, lo=0.0, hi=1.0) -> np.ndarray:
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


def normal(rng, shape, var=1.0) -> np.ndarray:
    return (rng.standard_normal(size=shape) * np.sqrt(var)).astype(np.float32)


def zero_mean_unit_norm_bank(rng, N, fh, fw, D) -> np.ndarray:
    """N(0,1) filters, then per filter: subtract the mean and divide by the L2
    norm over (fh, fw, D), in FP64, then cast to FP32."""
    w = rng.standard_normal(size=(N, fh, fw, D))
    w = w - w.mean(axis=(1, 2, 3), keepdims=True)
    w = w / np.sqrt((w * w).sum(axis=(1, 2, 3), keepdims=True))
    return w.astype(np.float32)


def integer_array(rng, shape, lo=-4, hi=4) -> np.ndarray:
    """Integers in [lo, hi] stored as FP32 (exact in FP32 and BF16)."""
    return rng.integers(lo, hi + 1, size=shape).astype(np.float32)


@dataclass
class Workload:
    name: str
    x: np.ndarray                       # [H, W, D] float32
    w: np.ndarray                       # [N, fh, fw, D] float32
    g: Optional[np.ndarray] = None      # [H', W', N] float32 upstream gradient
    clamp: Optional[Tuple[float, float]] = None
    modes: Tuple[str, ...] = ("f32",)

    @property
    def out_shape(self):
        H, W, _ = self.x.shape
        N, fh, fw, _ = self.w.shape
        return (H - fh + 1, W - fw + 1, N)

    @property
    def flops(self) -> int:
        """Algorithmic FLOPs: 2 per multiply-add, 2*H'*W'*N*fh*fw*D."""
        Ho, Wo, N = self.out_shape
        _, fh, fw, D = self.w.shape
        return 2 * Ho * Wo * N * fh * fw * D


def workload_small_f32(seed: int = 1) -> Workload:
    """128x128x8 U[0,1) input, 16 zero-mean unit-norm 9x9x8 filters, no epilogue."""
    rng = np.random.default_rng(seed)
    x = uniform(rng, (128, 128, 8))
    w = zero_mean_unit_norm_bank(rng, 16, 9, 9, 8)
    return Workload("fp32_128x128x8_16x9x9x8", x, w)


def workload_paper_row1_clamp(seed: int = 2) -> Workload:
    """256x256x8 U[0,1) input, 64 zero-mean unit-norm 9x9x8 filters, clamp [0, 1]."""
    rng = np.random.default_rng(seed)
    x = uniform(rng, (256, 256, 8))
    w = zero_mean_unit_norm_bank(rng, 64, 9, 9, 8)
    return Workload("fp32clamp_256x256x8_64x9x9x8", x, w, clamp=(0.0, 1.0))


# The four input / filter-bank shapes of the paper's Table "Performance of RTCG
# auto-tuning on 3D filter-bank convolutions" (Sec. 6.2): (H, W, D), (N, f, f, D).
PAPER_TABLE_SHAPES = (
    ((256, 256, 8), (64, 9, 9, 8)),
    ((512, 512, 4), (32, 13, 13, 4)),
    ((1024, 1024, 8), (16, 5, 5, 8)),
    ((2048, 2048, 4), (4, 8, 8, 4)),
)


def workload_paper_table(row: int, seed: int = 10) -> Workload:
    """Row `row` (0..3) of the paper's table shapes, with the recipe of the
    small workloads: U[0,1) input, zero-mean unit-norm N(0,1) filters."""
    (H, W, D), (N, fh, fw, _) = PAPER_TABLE_SHAPES[row]
    rng = np.random.default_rng(seed + row)
    x = uniform(rng, (H, W, D))
    w = zero_mean_unit_norm_bank(rng, N, fh, fw, D)
    return Workload(f"paper_table_{H}x{W}x{D}_{N}x{fh}x{fw}x{D}", x, w)


def workload_precision(seed: int = 3) -> Workload:
    """512x512x32 U[-1,1) input, 256 filters 5x5x32 drawn N(0, variance 1/800)."""
    rng = np.random.default_rng(seed)
    x = uniform(rng, (512, 512, 32), -1.0, 1.0)
    w = normal(rng, (256, 5, 5, 32), var=1.0 / 800.0)
    return Workload("precision_512x512x32_256x5x5x32", x, w, modes=("f32", "bf16", "bf16x3"))


def workload_differentiation(seed: int = 5) -> Workload:
    """256x256x16 U[0,1) input, 64 filters 7x7x16 N(0, 1/784), upstream g N(0,1)."""
    rng = np.random.default_rng(seed)
    x = uniform(rng, (256, 256, 16))
    w = normal(rng, (64, 7, 7, 16), var=1.0 / 784.0)
    g = normal(rng, (250, 250, 64))
    return Workload("fwdbwd_256x256x16_64x7x7x16", x, w, g=g)


def workload_finite_difference(seed: int = 55) -> Workload:
    """12x12x2 input, 3 filters 3x3x2, g 10x10x3 -- the finite-difference case."""
    rng = np.random.default_rng(seed)
    x = uniform(rng, (12, 12, 2))
    w = normal(rng, (3, 3, 3, 2), var=1.0 / 18.0)
    g = normal(rng, (10, 10, 3))
    return Workload("fd_12x12x2_3x3x3x2", x, w, g=g)


# A three-layer cascade with the paper's first-layer shape: 256x256x8 input, then
# 64 filters 9x9x8 -> 32 filters 5x5x64 -> 16 filters 3x3x32, each bank drawn
# like the small workloads (N(0,1), per-filter zero mean and unit L2 norm).
CASCADE_IN = (256, 256, 8)
CASCADE_BANKS = ((64, 9, 9), (32, 5, 5), (16, 3, 3))


def workload_cascade(seed: int = 6):
    """(x, [w1, w2, w3]): x U[0,1) 256x256x8; bank k of CASCADE_BANKS has the
    depth of the previous layer's output.  Draw order: x, then the banks."""
    rng = np.random.default_rng(seed)
    x = uniform(rng, CASCADE_IN)
    banks = []
    depth = CASCADE_IN[2]
    for (N, fh, fw) in CASCADE_BANKS:
        banks.append(zero_mean_unit_norm_bank(rng, N, fh, fw, depth))
        depth = N
    return x, banks


# Exact nearest-neighbour search (Sec. 6.4): 8x8 patches, 4096 targets and
# 4096 ... 1048576 neighbours (the paper's Table "NN-speedup").  The paper's
# patches come from the van Hateren natural-image database, which is not here;
# synthetic images with the 1/f amplitude spectrum of natural scenes stand in.
NN_TARGETS = 4096
NN_NEIGHBORS = (4096, 16384, 65536, 262144, 1048576)


def synthetic_natural_image(rng, size: int = 512, alpha: float = 1.0) -> np.ndarray:
    """A size x size image with a 1/f^alpha amplitude spectrum and uniform random
    phases, scaled to [0, 1] (FP64)."""
    fy = np.fft.fftfreq(size)[:, None]
    fx = np.fft.rfftfreq(size)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    f[0, 0] = 1.0
    spec = f ** (-alpha) * np.exp(2j * np.pi * rng.uniform(size=f.shape))
    spec[0, 0] = 0.0
    img = np.fft.irfft2(spec, s=(size, size))
    img -= img.min()
    return img / img.max()


def nn_patches(seed: int = 7, n_targets: int = NN_TARGETS, n_neighbors: int = 4096, side: int = 8,
               images: int = 8, size: int = 512):
    """(targets [n_targets, side*side], neighbors [n_neighbors, side*side]) FP32:
    row-major side x side patches at uniform random positions; targets come from
    the first image, neighbours from the other images (``images`` in all)."""
    rng = np.random.default_rng(seed)
    imgs = [synthetic_natural_image(rng, size) for _ in range(images)]
    span = size - side + 1

    def cut(img, count):
        ys = rng.integers(0, span, size=count)
        xs = rng.integers(0, span, size=count)
        win = np.lib.stride_tricks.sliding_window_view(img, (side, side))
        return win[ys, xs].reshape(count, side * side).astype(np.float32)

    targets = cut(imgs[0], n_targets)
    per = [n_neighbors // (images - 1)] * (images - 1)
    per[-1] += n_neighbors - sum(per)
    neighbors = np.concatenate([cut(im, c) for im, c in zip(imgs[1:], per)])
    return targets, neighbors


BATCH_HW = tuple(range(64, 513, 32))
BATCH_D = (4, 8, 16, 32)
BATCH_N = (16, 32, 64, 128)
BATCH_F = (3, 5, 7, 9, 11)


@dataclass
class BatchWorkload:
    name: str
    items: List[Workload] = field(default_factory=list)

    @property
    def flops(self) -> int:
        return sum(it.flops for it in self.items)


def batch_shapes(seed: int = 4, count: int = 64):
    """Shapes only (H, W, D, N, f) of the uneven batch, drawn in the same order
    as ``workload_batch`` so that both agree for the same seed."""
    return [(s[0], s[1], s[2], s[3], s[4]) for s in _batch_draw(seed, count, arrays=False)]


def _batch_draw(seed, count, arrays=True):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        H = int(rng.choice(BATCH_HW))
        W = int(rng.choice(BATCH_HW))
        D = int(rng.choice(BATCH_D))
        N = int(rng.choice(BATCH_N))
        f = int(rng.choice(BATCH_F))
        # the arrays are always drawn so that the shapes of later images do not
        # depend on whether arrays are requested
        x = uniform(rng, (H, W, D))
        w = normal(rng, (N, f, f, D))
        out.append((H, W, D, N, f, x if arrays else None, w if arrays else None))
    return out


def workload_batch(seed: int = 4, count: int = 64) -> BatchWorkload:
    """64 images: H, W uniform over {64, 96, ..., 512}; D over {4, 8, 16, 32};
    N over {16, 32, 64, 128}; f = fh = fw over {3, 5, 7, 9, 11}; each image
    U[0,1) with its own N(0,1) bank."""
    items = []
    for k, (H, W, D, N, f, x, w) in enumerate(_batch_draw(seed, count)):
        items.append(Workload(f"img{k}_{H}x{W}x{D}_{N}x{f}x{f}x{D}", x, w))
    return BatchWorkload("batch64_uneven", items)


def random_case(seed, H, W, D, N, fh, fw, kind="real", with_g=False) -> Workload:
    """A small case for parity tests.  ``kind`` = "real" (U[-1,1) input and
    N(0,1) filters) or "int" (integers in [-4, 4])."""
    rng = np.random.default_rng(seed)
    if kind == "int":
        x = integer_array(rng, (H, W, D))
        w = integer_array(rng, (N, fh, fw, D))
        g = integer_array(rng, (H - fh + 1, W - fw + 1, N)) if with_g else None
    else:
        x = uniform(rng, (H, W, D), -1.0, 1.0)
        w = normal(rng, (N, fh, fw, D))
        g = normal(rng, (H - fh + 1, W - fw + 1, N)) if with_g else None
    return Workload(f"case_{H}x{W}x{D}_{N}x{fh}x{fw}_{kind}_s{seed}", x, w, g=g)
