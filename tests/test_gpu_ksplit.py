"""GPU parity of the K-split forward tile (ks lanes per output split the depth
and combine their partial sums by warp shuffles) against the FP64 oracle,
through the C ABI: random data within the FP32 tolerance, integer data bit for
bit, the fused clamp and snippet epilogues, packed-pair FMAs bit-identical to
scalar ones, run-to-run determinism, and the tuner offering the tile."""
import numpy as np
import pytest

import oracle
from helpers import dev, host, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5

# (shape H, W, D, N, fh, fw), spec: several CTA tiles with ragged tails in
# every dimension, depths that need zero padding channels, all four ks values
CASES = [
    ((128, 128, 8, 16, 9, 9), "direct:tr=4,tf=8,wr=2,wf=1,cc=0,ks=8,wq=4"),
    ((70, 66, 8, 16, 9, 9), "direct:tr=2,tf=8,wr=4,wf=2,cc=0,ks=8,wq=2"),
    ((37, 45, 3, 5, 4, 2), "direct:tr=4,tf=4,wr=1,wf=2,cc=0,ks=4,wq=8"),
    ((33, 97, 16, 12, 3, 5), "direct:tr=4,tf=8,wr=2,wf=2,cc=0,ks=16,wq=4"),
    ((50, 70, 4, 20, 8, 8), "direct:tr=8,tf=4,wr=1,wf=1,cc=0,ks=4,wq=4"),
    ((9, 9, 8, 3, 9, 9), "direct:tr=8,tf=8,wr=1,wf=1,cc=0,ks=32,wq=2"),     # output 1 x 1
    ((41, 53, 6, 27, 5, 3), "direct:tr=4,tf=8,wr=2,wf=4,cc=0,ks=8,wq=2"),  # depth 6 padded to 8
    ((30, 61, 24, 9, 3, 3), "direct:tr=2,tf=16,wr=4,wf=1,cc=0,ks=8,wq=4"),  # three channels per lane
    # the depth share in the high lane bits (sh=1), a 16-row register block
    ((128, 128, 8, 16, 9, 9), "direct:tr=16,tf=4,wr=1,wf=4,cc=0,ks=8,wq=2,sh=1"),
    ((37, 45, 3, 5, 4, 2), "direct:tr=8,tf=4,wr=2,wf=2,cc=0,ks=4,wq=2,sh=1"),
    ((33, 97, 16, 12, 3, 5), "direct:tr=8,tf=8,wr=1,wf=2,cc=0,ks=16,wq=4,sh=1"),
]


def _ids(c):
    return "x".join(map(str, c[0])) + "_t" + c[1].split("tr=")[1].split(",")[0] + "_" + \
        c[1].split("ks=")[1].replace(",", "_")


def _run(torch, x, w, spec, clamp=None):
    from paper_0911_3456_gb300.api import Plan
    p = Plan(x.shape, w.shape, "f32", clamp)
    p.set_variant(spec)
    assert p.info()["fwd"]["spec"] == spec
    y = p.forward(dev(x, torch), dev(w, torch))
    torch.cuda.synchronize()
    return host(y), p


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_ksplit_matches_oracle(case):
    torch = torch_cuda()
    shape, spec = case
    wl = inputs.random_case(4100, *shape)
    ref = oracle.fwd(wl.x, wl.w)
    for pk in ("", ",pk=1"):
        s = spec.replace(",ks=", pk + ",ks=")
        y, _ = _run(torch, wl.x, wl.w, s)
        assert y.shape == ref.shape
        assert normwise_rel(y, ref) <= TOL_F32, s


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_ksplit_integer_bit_exact_and_pairs_identical(case):
    """Integers in [-4, 4]: every partial sum and every shuffle-combined sum is
    an exact FP32 integer, so the output equals the oracle bit for bit; with
    real data the packed-pair form gives the scalar form's bits."""
    torch = torch_cuda()
    shape, spec = case
    wl = inputs.random_case(4200, *shape, kind="int")
    y, _ = _run(torch, wl.x, wl.w, spec.replace(",ks=", ",pk=1,ks="))
    assert np.array_equal(y, oracle.fwd(wl.x, wl.w))
    wr = inputs.random_case(4300, *shape)
    y0, _ = _run(torch, wr.x, wr.w, spec)
    y1, p1 = _run(torch, wr.x, wr.w, spec.replace(",ks=", ",pk=1,ks="))
    assert "_pk1_ks" in p1.info()["fwd"]["kernel"]
    assert np.array_equal(y0, y1)


@pytest.mark.parametrize("case", CASES[:4], ids=_ids)
def test_ksplit_clamp(case):
    torch = torch_cuda()
    shape, spec = case
    wl = inputs.random_case(4400, *shape)
    y, _ = _run(torch, wl.x, wl.w, spec, clamp=(-0.5, 0.75))
    scale = np.abs(oracle.fwd(wl.x, wl.w)).max()
    assert np.abs(y - oracle.fwd(wl.x, wl.w, epilogue=(-0.5, 0.75))).max() <= TOL_F32 * scale
    assert y.min() >= -0.5 and y.max() <= 0.75


def test_ksplit_snippet_epilogue():
    """A user expression fused into the K-split store (leaky ReLU with a
    per-filter term), against the oracle followed by the same expression."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    shape, spec = CASES[1]
    wl = inputs.random_case(4500, *shape)
    p = Plan(wl.x.shape, wl.w.shape, "f32", snippet="y > 0.f ? y : 0.1f * y + 0.001f * n")
    p.set_variant(spec)
    y = host(p.forward(dev(wl.x, torch), dev(wl.w, torch)))
    ref = oracle.fwd(wl.x, wl.w)
    n = np.arange(ref.shape[2], dtype=np.float64)
    ref = np.where(ref > 0, ref, 0.1 * ref + 0.001 * n)
    assert np.abs(y - ref).max() <= 2 * TOL_F32 * np.abs(oracle.fwd(wl.x, wl.w)).max()


def test_ksplit_deterministic_and_guard_bands():
    """The shuffle tree is fixed: two runs give the same bits.  The output
    written through a view leaves the bytes around it untouched."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    shape, spec = CASES[6]
    wl = inputs.random_case(4600, *shape)
    p = Plan(wl.x.shape, wl.w.shape)
    p.set_variant(spec)
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    n = int(np.prod(p.out_shape))
    buf = torch.full((n + 2048,), 123.0, device="cuda")
    y = buf[1024:1024 + n].view(p.out_shape)
    p.forward(x, w, y=y)
    a = y.clone()
    p.forward(x, w, y=y)
    torch.cuda.synchronize()
    assert torch.equal(a, y)
    assert torch.all(buf[:1024] == 123.0) and torch.all(buf[1024 + n:] == 123.0)
    assert normwise_rel(host(y), oracle.fwd(wl.x, wl.w)) <= TOL_F32


def test_ksplit_refused_for_backward_and_offered_by_tuner():
    """The tuner times K-split tiles beside the lane-per-column tiles on the
    first configuration's shape; whatever it picks matches the oracle, and the
    backward of a plan never runs the forward K-split tile."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.workload_small_f32()
    p = Plan(wl.x.shape, wl.w.shape)
    assert any(",ks=" in s for s in p.candidates())
    p.autotune()
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    y = host(p.forward(x, w))
    assert normwise_rel(y, oracle.fwd(wl.x, wl.w)) <= TOL_F32
    # the backward never runs the forward K-split tile (the whole depth in one
    # stage, cc=0); the chunked dL/dx tile (cc > 0) is its own family
    dx_spec = p.info().get("dx", {}).get("spec", "")
    assert ",ks=" not in dx_spec or ",cc=0," not in dx_spec
