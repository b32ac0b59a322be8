"""GPU parity of the hand-written backward kernels (dL/dx, dL/dw) against the
FP64 oracle's gradients, and of the autograd wrapper against finite
differences."""
import numpy as np
import pytest

import oracle
from helpers import dev, host, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = [
    (12, 12, 2, 3, 3, 3),
    (37, 45, 3, 5, 4, 2),
    (40, 52, 16, 24, 7, 7),
    (33, 97, 8, 12, 3, 5),
    (9, 9, 4, 3, 9, 9),
    (30, 30, 5, 6, 1, 1),
]


def _plan(shape, clamp=None):
    from paper_0911_3456_gb300.api import Plan
    H, W, D, N, fh, fw = shape
    return Plan((H, W, D), (N, fh, fw, D), "f32", clamp)


@pytest.mark.parametrize("shape", CASES, ids=lambda s: "x".join(map(str, s)))
def test_backward_matches_oracle(shape):
    torch = torch_cuda()
    wl = inputs.random_case(800, *shape, with_g=True)
    p = _plan(shape)
    dx, dw = p.backward(dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch))
    torch.cuda.synchronize()
    assert normwise_rel(host(dx), oracle.bwd_input(wl.g, wl.w, wl.x.shape)) <= TOL
    assert normwise_rel(host(dw), oracle.bwd_filt(wl.x, wl.g, wl.w.shape)) <= TOL


@pytest.mark.parametrize("shape", CASES[:4], ids=lambda s: "x".join(map(str, s)))
def test_backward_integer_bit_exact(shape):
    torch = torch_cuda()
    wl = inputs.random_case(900, *shape, kind="int", with_g=True)
    p = _plan(shape)
    dx, dw = p.backward(dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch))
    torch.cuda.synchronize()
    assert np.array_equal(host(dx), oracle.bwd_input(wl.g, wl.w, wl.x.shape))
    assert np.array_equal(host(dw), oracle.bwd_filt(wl.x, wl.g, wl.w.shape))


def test_backward_with_clamp_mask():
    torch = torch_cuda()
    shape = (30, 41, 4, 8, 3, 4)
    wl = inputs.random_case(1000, *shape, with_g=True)
    clamp = (-0.5, 0.5)
    p = _plan(shape, clamp)
    x, w, g = dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch)
    y = p.forward(x, w)
    dx, dw = p.backward(x, w, g, y)
    torch.cuda.synchronize()
    yh = host(y)
    # mask decisions are taken on the GPU's FP32 y, by both sides
    assert normwise_rel(host(dx), oracle.bwd_input(wl.g, wl.w, wl.x.shape, y=yh, epilogue=clamp)) <= TOL
    assert normwise_rel(host(dw), oracle.bwd_filt(wl.x, wl.g, wl.w.shape, y=yh, epilogue=clamp)) <= TOL


def test_backward_only_dx_or_only_dw():
    torch = torch_cuda()
    shape = (20, 24, 3, 4, 3, 3)
    wl = inputs.random_case(1100, *shape, with_g=True)
    p = _plan(shape)
    dx, dw = p.backward(dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch), need_dw=False)
    assert dw is None and normwise_rel(host(dx), oracle.bwd_input(wl.g, wl.w, wl.x.shape)) <= TOL
    dx, dw = p.backward(dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch), need_dx=False)
    assert dx is None and normwise_rel(host(dw), oracle.bwd_filt(wl.x, wl.g, wl.w.shape)) <= TOL


def test_concurrent_gradients_match_single_and_capture_in_a_graph():
    """With both gradients the library runs dL/dw on the plan's side stream,
    forked from and joined back to the caller's stream: each gradient is
    bit-identical to the one computed alone, the call (with its fork and join)
    is captured into a CUDA graph, and replaying the graph gives the same bits."""
    torch = torch_cuda()
    shape = (70, 66, 8, 24, 5, 3)
    wl = inputs.random_case(1150, *shape, with_g=True)
    p = _plan(shape)
    x, w, g = dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch)
    dx_only, _ = p.backward(x, w, g, need_dw=False)
    _, dw_only = p.backward(x, w, g, need_dx=False)
    dx, dw = p.backward(x, w, g)
    torch.cuda.synchronize()
    assert torch.equal(dx, dx_only) and torch.equal(dw, dw_only)
    assert normwise_rel(host(dw), oracle.bwd_filt(wl.x, wl.g, wl.w.shape)) <= TOL
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        p.backward(x, w, g)          # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gx, gw = p.backward(x, w, g)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(gx, dx) and torch.equal(gw, dw)


def test_dw_deterministic():
    torch = torch_cuda()
    shape = (64, 64, 8, 16, 5, 5)
    wl = inputs.random_case(1200, *shape, with_g=True)
    p = _plan(shape)
    x, w, g = dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch)
    _, a = p.backward(x, w, g)
    a = a.clone()
    _, b = p.backward(x, w, g)
    assert torch.equal(a, b)


def test_autograd_function_against_finite_differences():
    """The 12x12x2 / 3 filters 3x3x2 case: GPU gradients through
    torch.autograd against central differences of L = <y, g> computed with the
    FP64 oracle (exact up to rounding: L is bilinear)."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import fbcorr
    wl = inputs.workload_finite_difference()
    x = dev(wl.x, torch).requires_grad_(True)
    w = dev(wl.w, torch).requires_grad_(True)
    y = fbcorr(x, w)
    (y * dev(wl.g, torch)).sum().backward()
    h = 1e-3
    x64, w64, g64 = (np.asarray(a, np.float64) for a in (wl.x, wl.w, wl.g))

    def L(xx, ww):
        return float((oracle.fwd(xx, ww) * g64).sum())

    fdx = np.empty_like(x64)
    for idx in np.ndindex(*x64.shape):
        a = x64.copy(); a[idx] += h
        b = x64.copy(); b[idx] -= h
        fdx[idx] = (L(a, w64) - L(b, w64)) / (2 * h)
    fdw = np.empty_like(w64)
    for idx in np.ndindex(*w64.shape):
        a = w64.copy(); a[idx] += h
        b = w64.copy(); b[idx] -= h
        fdw[idx] = (L(x64, a) - L(x64, b)) / (2 * h)
    assert normwise_rel(host(x.grad), fdx) <= TOL
    assert normwise_rel(host(w.grad), fdw) <= TOL


def test_differentiation_config_full():
    """256x256x16 input, 64 filters 7x7x16 N(0, 1/784), g N(0,1) 250x250x64:
    forward, dL/dx and dL/dw against the oracle on every element."""
    torch = torch_cuda()
    wl = inputs.workload_differentiation()
    from paper_0911_3456_gb300.api import Plan
    p = Plan(wl.x.shape, wl.w.shape)
    x, w, g = dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch)
    y = p.forward(x, w)
    dx, dw = p.backward(x, w, g)
    torch.cuda.synchronize()
    assert normwise_rel(host(y), oracle.fwd(wl.x, wl.w)) <= TOL
    assert normwise_rel(host(dx), oracle.bwd_input(wl.g, wl.w, wl.x.shape)) <= TOL
    assert normwise_rel(host(dw), oracle.bwd_filt(wl.x, wl.g, wl.w.shape)) <= TOL


@pytest.mark.parametrize("dx_spec", ["direct:tr=4,tf=4,wr=4,wf=2,cc=8,pk=1",
                                     "direct:tr=2,tf=4,wr=2,wf=4,cc=8,pk=1"])
def test_dx_register_prefetch_is_bit_identical(dx_spec, monkeypatch):
    """The dL/dx kernel (flipped bank, 24 gradient channels in 8-channel
    chunks) with the register prefetch of the next chunk gives the plain
    kernel's bits, with and without the clamp mask, and the oracle's gradient."""
    torch = torch_cuda()
    shape = (40, 52, 16, 24, 7, 7)
    wl = inputs.random_case(1100, *shape, with_g=True)
    for clamp in (None, (-0.5, 0.5)):
        outs = []
        for pf in ("", ",pf=1"):
            monkeypatch.setenv("FBCORR_DX_VARIANT", dx_spec + pf)
            p = _plan(shape, clamp)
            x, w, g = dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch)
            y = p.forward(x, w) if clamp else None
            dx, _ = p.backward(x, w, g, y, need_dw=False)
            torch.cuda.synchronize()
            assert p.info()["dx"]["spec"] == dx_spec + pf
            outs.append(host(dx))
        assert np.array_equal(outs[0], outs[1])
        if clamp is None:
            assert normwise_rel(outs[1], oracle.bwd_input(wl.g, wl.w, wl.x.shape)) <= TOL


@pytest.mark.parametrize("shape", [(40, 52, 16, 24, 7, 7), (33, 97, 8, 12, 3, 5), (70, 130, 32, 40, 5, 5)],
                         ids=lambda s: "x".join(map(str, s)))
def test_dw_packed_pairs_bit_identical(shape, monkeypatch):
    """dL/dw with packed-pair FMAs, chunk totals in registers (FBCORR_DW_PK=1)
    or in shared memory (FBCORR_DW_PK=2), gives the scalar kernel's bits (the
    same per-lane multiply-adds and the same additions in the same order) and
    the oracle's gradient."""
    torch = torch_cuda()
    wl = inputs.random_case(1200, *shape, with_g=True)
    outs = []
    for pk in ("0", "1", "2"):
        monkeypatch.setenv("FBCORR_DW_PK", pk)
        p = _plan(shape)
        _, dw = p.backward(dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch), need_dx=False)
        torch.cuda.synchronize()
        assert p.info()["dw"]["packed_pairs"] == int(pk)
        outs.append(host(dw))
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])
    assert normwise_rel(outs[2], oracle.bwd_filt(wl.x, wl.g, wl.w.shape)) <= TOL
