"""fbcorr_forward_host: the forward from host buffers with banded, overlapped
transfers, against the FP64 oracle and against the device-resident forward,
through the C ABI."""
import numpy as np
import pytest

import oracle
from helpers import dev, host, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16x3": 1e-5, "bf16": 1e-2}


def _host_tensors(torch, wl, pinned):
    x = torch.from_numpy(np.ascontiguousarray(wl.x))
    w = torch.from_numpy(np.ascontiguousarray(wl.w))
    if pinned:
        x, w = x.pin_memory(), w.pin_memory()
    return x, w


@pytest.mark.parametrize("mode", ["f32", "bf16x3", "bf16"])
@pytest.mark.parametrize("bands", [0, 1, 3, 50])
def test_forward_host_matches_oracle_and_device(mode, bands):
    """Every band count (automatic, one band, uneven bands, more bands than
    4-row groups) gives the oracle's result within the mode's tolerance and
    the device-resident forward's result."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(2100, 61, 70, 16, 24, 5, 4, kind="real")
    p = Plan(wl.x.shape, wl.w.shape, mode)
    x, w = _host_tensors(torch, wl, pinned=True)
    y = p.forward_host(x, w, bands=bands)
    torch.cuda.synchronize()
    ref = oracle.fwd(wl.x, wl.w)
    got = y.numpy().astype(np.float64)
    assert normwise_rel(got, ref) <= TOL[mode]
    yd = host(p.forward(dev(wl.x, torch), dev(wl.w, torch)))
    assert np.abs(got - yd).max() <= 1e-6 * np.abs(ref).max()


def test_forward_host_pageable_clamp_and_stream():
    """Pageable (not page-locked) host memory, a clamp epilogue and a
    non-default stream; a second call with another band count re-plans."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(2200, 45, 33, 8, 10, 3, 3, kind="real")
    p = Plan(wl.x.shape, wl.w.shape, "f32", (-0.5, 0.5))
    x, w = _host_tensors(torch, wl, pinned=False)
    s = torch.cuda.Stream()
    ref = oracle.fwd(wl.x, wl.w, epilogue=(-0.5, 0.5))
    scale = np.abs(oracle.fwd(wl.x, wl.w)).max()
    for bands in (2, 5):
        y = torch.empty(p.out_shape, dtype=torch.float32)
        p.forward_host(x, w, y, bands=bands, stream=s)
        s.synchronize()
        assert np.abs(y.numpy() - ref).max() <= 1e-5 * scale
    assert p.device_status() == 0


def test_forward_host_integer_bit_exact():
    """Integer inputs: the banded host path is exact in every mode."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(2300, 40, 52, 8, 20, 3, 5, kind="int")
    ref = oracle.fwd(wl.x, wl.w)
    x, w = _host_tensors(torch, wl, pinned=True)
    for mode in ("f32", "bf16", "bf16x3"):
        p = Plan(wl.x.shape, wl.w.shape, mode)
        y = p.forward_host(x, w, bands=4)
        torch.cuda.synchronize()
        assert np.array_equal(y.numpy().astype(np.float64), ref), mode


def test_forward_host_rejects_device_tensors():
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(2400, 20, 20, 4, 3, 3, 3)
    p = Plan(wl.x.shape, wl.w.shape, "f32")
    with pytest.raises(ValueError):
        p.forward_host(dev(wl.x, torch), dev(wl.w, torch))


@pytest.mark.parametrize("shape", [(5, 40, 4, 3, 5, 3), (3, 17, 8, 2, 3, 3), (64, 20, 8, 5, 1, 1)],
                         ids=lambda s: "x".join(map(str, s)))
def test_forward_host_small_outputs(shape):
    """Outputs of 1, 1 and 64 rows: automatic banding never makes a band of no
    rows, and a single output row still goes through the band plans."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(2450, *shape)
    p = Plan(wl.x.shape, wl.w.shape, "f32")
    x, w = _host_tensors(torch, wl, pinned=True)
    for bands in (0, 1, 7):
        y = p.forward_host(x, w, bands=bands)
        torch.cuda.synchronize()
        assert normwise_rel(y.numpy(), oracle.fwd(wl.x, wl.w)) <= 1e-5
