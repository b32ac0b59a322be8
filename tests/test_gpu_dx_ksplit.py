"""GPU parity of the chunked K-split dL/dx tile: the lanes of a group split
the gradient channels of each chunk, the chunks stream through a cp.async ring,
and a fixed shuffle tree combines the partial blocks.  Checked against the FP64
oracle's dL/dx on ragged shapes (edges, a last chunk and a filter block that are
partly zero fill, accumulator blocks that do not split evenly over the lanes),
bit for bit on integer data, run to run, and on the differentiation workload."""
import numpy as np
import pytest

import oracle
from helpers import dev, host, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5

# every spec fits the shared-memory limit on every shape below (9x9 filters
# included), so the plan runs the forced tile
SPECS = [
    "direct:tr=7,tf=4,wr=2,wf=4,cc=4,pk=1,ks=4,wq=2",          # 14 pairs reduced as 16, 2-stage ring
    "direct:tr=7,tf=4,wr=2,wf=4,cc=8,pk=1,ks=8,wq=2",          # 8 lanes per output
    "direct:tr=8,tf=4,wr=2,wf=4,cc=4,pk=1,pf=1,ks=4,wq=2",     # 3-stage ring
    "direct:tr=4,tf=8,wr=2,wf=2,cc=8,ks=4,wq=1",               # 2 channels per lane, scalar FMAs, 8 filters
]

# (H, W, D, N, fh, fw): dL/dx sums over N gradient channels into D outputs
SHAPES = [
    (40, 52, 16, 24, 7, 7),     # 24 channels: a last 16-channel chunk half zero fill
    (33, 97, 8, 12, 3, 5),      # fh != fw, ragged columns
    (61, 45, 4, 8, 5, 4),       # 4 output channels in a 16-channel filter block
    (9, 9, 4, 4, 9, 9),         # one forward output pixel: dL/dx is all padding halo
]


def _dx(shape, spec, wl, monkeypatch, clamp=None):
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    monkeypatch.setenv("FBCORR_DX_VARIANT", spec)
    H, W, D, N, fh, fw = shape
    p = Plan((H, W, D), (N, fh, fw, D), "f32", clamp)
    dx, _ = p.backward(dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch), need_dw=False)
    torch.cuda.synchronize()
    assert p.info()["dx"]["spec"] == spec
    return host(dx)


@pytest.mark.parametrize("spec", SPECS)
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_chunked_ksplit_dx_matches_oracle(shape, spec, monkeypatch):
    wl = inputs.random_case(1300, *shape, with_g=True)
    dx = _dx(shape, spec, wl, monkeypatch)
    assert normwise_rel(dx, oracle.bwd_input(wl.g, wl.w, wl.x.shape)) <= TOL


@pytest.mark.parametrize("spec", SPECS)
def test_chunked_ksplit_dx_integer_bit_exact_and_deterministic(spec, monkeypatch):
    shape = SHAPES[0]
    wl = inputs.random_case(1400, *shape, kind="int", with_g=True)
    a = _dx(shape, spec, wl, monkeypatch)
    assert np.array_equal(a, oracle.bwd_input(wl.g, wl.w, wl.x.shape))
    wr = inputs.random_case(1401, *shape, with_g=True)
    b1 = _dx(shape, spec, wr, monkeypatch)
    b2 = _dx(shape, spec, wr, monkeypatch)
    assert np.array_equal(b1, b2)


def test_chunked_ksplit_refused_with_a_clamp_mask(monkeypatch):
    """dL/dx of a clamped forward reads the mask with the gradient; the chunked
    tile copies the gradient as it is, so a plan with a clamp refuses it."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    from paper_0911_3456_gb300._capi import FbcorrError
    monkeypatch.setenv("FBCORR_DX_VARIANT", SPECS[0])
    shape = SHAPES[0]
    wl = inputs.random_case(1500, *shape, with_g=True)
    H, W, D, N, fh, fw = shape
    p = Plan((H, W, D), (N, fh, fw, D), "f32", (-0.5, 0.5))
    x, w, g = dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch)
    y = p.forward(x, w)
    with pytest.raises(FbcorrError, match="UNSUPPORTED"):
        p.backward(x, w, g, y, need_dw=False)


@pytest.mark.parametrize("spec", SPECS[:3])
def test_chunked_ksplit_dx_differentiation_workload(spec, monkeypatch):
    """256x256x16 input, 64 filters 7x7x16, g 250x250x64: every element of
    dL/dx against the oracle."""
    wl = inputs.workload_differentiation()
    dx = _dx(wl.x.shape + wl.w.shape[:3], spec, wl, monkeypatch)
    assert normwise_rel(dx, oracle.bwd_input(wl.g, wl.w, wl.x.shape)) <= TOL
