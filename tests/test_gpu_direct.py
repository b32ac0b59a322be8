"""GPU parity of the FP32 direct path (forward + fused clamp) against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from helpers import dev, host, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5

SMALL = [
    # H, W, D, N, fh, fw  -- several tiles plus ragged tails in every dimension
    (37, 45, 3, 5, 4, 2),
    (70, 66, 8, 16, 9, 9),
    (33, 97, 16, 12, 3, 5),
    (20, 20, 1, 1, 1, 1),
    (9, 9, 4, 3, 9, 9),        # output 1 x 1
    (64, 40, 32, 40, 5, 5),
    (50, 70, 4, 20, 8, 8),     # even filter size
    (16, 300, 2, 7, 2, 13),
]


def _run(torch, x, w, clamp=None, spec=None):
    from paper_0911_3456_gb300.api import Plan
    p = Plan(x.shape, w.shape, "f32", clamp)
    if spec:
        p.set_variant(spec)
    y = p.forward(dev(x, torch), dev(w, torch))
    torch.cuda.synchronize()
    return host(y), p


@pytest.mark.parametrize("shape", SMALL, ids=lambda s: "x".join(map(str, s)))
def test_forward_matches_oracle(shape):
    torch = torch_cuda()
    wl = inputs.random_case(100, *shape)
    y, _ = _run(torch, wl.x, wl.w)
    ref = oracle.fwd(wl.x, wl.w)
    assert y.shape == ref.shape
    assert normwise_rel(y, ref) <= TOL_F32


@pytest.mark.parametrize("shape", SMALL[:5], ids=lambda s: "x".join(map(str, s)))
def test_forward_clamp_matches_oracle(shape):
    torch = torch_cuda()
    wl = inputs.random_case(200, *shape)
    y, _ = _run(torch, wl.x, wl.w, clamp=(-0.5, 0.75))
    ref = oracle.fwd(wl.x, wl.w, epilogue=(-0.5, 0.75))
    # the clamp is 1-Lipschitz, so the arithmetic error is judged against the
    # magnitude of the unclamped accumulator
    scale = np.abs(oracle.fwd(wl.x, wl.w)).max()
    assert np.abs(y - ref).max() <= TOL_F32 * scale
    assert y.min() >= -0.5 and y.max() <= 0.75


@pytest.mark.parametrize("shape", SMALL, ids=lambda s: "x".join(map(str, s)))
def test_integer_inputs_bit_exact(shape):
    """Integers in [-4, 4]: every partial sum is an exact FP32 integer, so any
    summation order must reproduce the oracle bit for bit."""
    torch = torch_cuda()
    wl = inputs.random_case(300, *shape, kind="int")
    y, _ = _run(torch, wl.x, wl.w)
    assert np.array_equal(y, oracle.fwd(wl.x, wl.w))


def test_delta_filters_copy_input_windows():
    torch = torch_cuda()
    rng = np.random.default_rng(3)
    H, W, D, fh, fw = 40, 70, 3, 4, 5
    x = rng.uniform(-1, 1, (H, W, D)).astype(np.float32)
    taps = [(i, j, d) for i in range(fh) for j in range(fw) for d in range(D)]
    w = np.zeros((len(taps), fh, fw, D), np.float32)
    for n, (i, j, d) in enumerate(taps):
        w[n, i, j, d] = 1.0
    y, _ = _run(torch, x, w)
    Ho, Wo = H - fh + 1, W - fw + 1
    for n, (i, j, d) in enumerate(taps):
        assert np.array_equal(y[:, :, n], x[i:i + Ho, j:j + Wo, d].astype(np.float64))


def test_default_variant_matches_oracle():
    torch = torch_cuda()
    wl = inputs.random_case(400, 45, 61, 8, 10, 5, 3)
    y, p = _run(torch, wl.x, wl.w, clamp=(-1.0, 1.0), spec="default")
    assert p.info()["fwd"]["kind"] == "default"
    scale = np.abs(oracle.fwd(wl.x, wl.w)).max()
    assert np.abs(y - oracle.fwd(wl.x, wl.w, epilogue=(-1.0, 1.0))).max() <= TOL_F32 * scale


@pytest.mark.parametrize("spec", ["direct:tr=8,tf=8,wr=1,wf=2,cc=0", "direct:tr=2,tf=4,wr=4,wf=1,cc=0",
                                  "direct:tr=4,tf=8,wr=2,wf=4,cc=4", "direct:tr=8,tf=4,wr=2,wf=1,cc=0",
                                  "direct:tr=4,tf=4,wr=2,wf=4,cc=4", "direct:tr=2,tf=8,wr=8,wf=1,cc=0"])
def test_every_tile_shape_matches_oracle(spec):
    torch = torch_cuda()
    wl = inputs.random_case(500, 51, 77, 8, 27, 5, 4)
    y, p = _run(torch, wl.x, wl.w, spec=spec)
    assert p.info()["fwd"]["spec"] == spec
    assert normwise_rel(y, oracle.fwd(wl.x, wl.w)) <= TOL_F32


@pytest.mark.parametrize("spec,clamp", [("direct:tr=8,tf=8,wr=2,wf=2,cc=4", None),
                                        ("direct:tr=2,tf=4,wr=4,wf=1,cc=0", (-1.0, 1.0)),
                                        ("direct:tr=4,tf=8,wr=2,wf=4,cc=4", (-0.5, 0.5)),
                                        ("direct:tr=8,tf=4,wr=3,wf=1,cc=0", None)])
def test_packed_pair_fma_is_bit_identical(spec, clamp):
    """pk=1 issues the same multiply-adds as fma.rn.f32x2 pairs over adjacent
    filters; each lane rounds like fmaf in the same order, so the output must
    equal the scalar variant's bit for bit (27 filters: a ragged filter tile)."""
    torch = torch_cuda()
    wl = inputs.random_case(510, 51, 77, 8, 27, 5, 4)
    y0, _ = _run(torch, wl.x, wl.w, clamp=clamp, spec=spec)
    y1, p1 = _run(torch, wl.x, wl.w, clamp=clamp, spec=spec + ",pk=1")
    assert p1.info()["fwd"]["spec"] == spec + ",pk=1"
    assert p1.info()["fwd"]["kernel"].endswith("_pk1")
    assert np.array_equal(y0, y1)
    ref = oracle.fwd(wl.x, wl.w, epilogue=clamp) if clamp else oracle.fwd(wl.x, wl.w)
    assert np.abs(y1 - ref).max() <= TOL_F32 * np.abs(oracle.fwd(wl.x, wl.w)).max()


def test_run_to_run_bitwise_determinism():
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(600, 80, 90, 8, 32, 7, 7)
    p = Plan(wl.x.shape, wl.w.shape)
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    a = p.forward(x, w).clone()
    b = p.forward(x, w)
    assert torch.equal(a, b)


def test_guard_bands_untouched():
    """Output written through a view into a larger buffer: the bytes before and
    after the output stay as they were (no out-of-bounds stores)."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(700, 33, 47, 4, 9, 3, 3)
    p = Plan(wl.x.shape, wl.w.shape)
    n = int(np.prod(p.out_shape))
    buf = torch.full((n + 2048,), 123.0, device="cuda")
    y = buf[1024:1024 + n].view(p.out_shape)
    p.forward(dev(wl.x, torch), dev(wl.w, torch), y=y)
    torch.cuda.synchronize()
    assert torch.all(buf[:1024] == 123.0) and torch.all(buf[1024 + n:] == 123.0)
    assert normwise_rel(host(y), oracle.fwd(wl.x, wl.w)) <= TOL_F32


def test_small_config_full_parity():
    """128x128x8 input, 16 zero-mean unit-norm 9x9x8 filters, no epilogue."""
    torch = torch_cuda()
    wl = inputs.workload_small_f32()
    y, _ = _run(torch, wl.x, wl.w)
    assert normwise_rel(y, oracle.fwd(wl.x, wl.w)) <= TOL_F32


def test_paper_row1_clamp_full_parity():
    """256x256x8 input, 64 filters 9x9x8, clamp [0, 1] fused (the paper's table row 1)."""
    torch = torch_cuda()
    wl = inputs.workload_paper_row1_clamp()
    y, _ = _run(torch, wl.x, wl.w, clamp=wl.clamp)
    scale = np.abs(oracle.fwd(wl.x, wl.w)).max()
    assert np.abs(y - oracle.fwd(wl.x, wl.w, epilogue=wl.clamp)).max() <= TOL_F32 * scale


def test_precision_config_direct_sampled():
    """512x512x32 with 256 filters 5x5x32 on the FP32 direct kernel: sampled
    outputs (edges and random interior points) against the oracle."""
    torch = torch_cuda()
    wl = inputs.workload_precision()
    y, _ = _run(torch, wl.x, wl.w)
    Ho, Wo, N = y.shape
    rng = np.random.default_rng(11)
    idx = np.stack([rng.integers(0, Ho, 3000), rng.integers(0, Wo, 3000), rng.integers(0, N, 3000)], 1)
    edges = np.array([[0, 0, 0], [Ho - 1, Wo - 1, N - 1], [0, Wo - 1, 17], [Ho - 1, 0, 200]])
    idx = np.concatenate([idx, edges])
    ref = oracle.fwd_points(wl.x, wl.w, idx)
    got = y[tuple(idx.T)]
    assert np.abs(got - ref).max() / np.abs(ref).max() <= TOL_F32


def test_bad_pointer_alignment_rejected():
    torch = torch_cuda()
    from paper_0911_3456_gb300 import _capi as C
    from paper_0911_3456_gb300.api import Plan
    p = Plan((16, 16, 4), (2, 3, 3, 4))
    x = torch.zeros(16 * 16 * 4 + 1, device="cuda")[1:]
    w = torch.zeros((2, 3, 3, 4), device="cuda")
    y = torch.zeros(p.out_shape, device="cuda")
    import ctypes
    st = C.load().fbcorr_forward(p.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                 ctypes.c_void_p(y.data_ptr()), None, 0, None)
    assert st == 4


@pytest.mark.parametrize("D,cc", [(6, 4), (12, 8), (10, 4), (3, 4)])
def test_ragged_channel_chunks(D, cc):
    """Depth not a multiple of the channel chunk: the last chunk is zero-padded."""
    torch = torch_cuda()
    wl = inputs.random_case(510 + D, 41, 70, D, 12, 3, 5)
    y, p = _run(torch, wl.x, wl.w, spec=f"direct:tr=4,tf=4,wr=2,wf=2,cc={cc}")
    assert normwise_rel(y, oracle.fwd(wl.x, wl.w)) <= TOL_F32


@pytest.mark.parametrize("row", [1, 2, 3])
def test_paper_table_shapes_sampled(row):
    """The paper's other table shapes (512x512x4 / 32x13x13x4, 1024x1024x8 /
    16x5x5x8, 2048x2048x4 / 4x8x8x4): first, middle and last output rows and
    random points against the oracle, with the default and the heuristic tile."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.workload_paper_table(row)
    p = Plan(wl.x.shape, wl.w.shape)
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    Ho, Wo, N = p.out_shape
    fh = wl.w.shape[1]
    rng = np.random.default_rng(row)
    idx = np.stack([rng.integers(0, Ho, 2000), rng.integers(0, Wo, 2000), rng.integers(0, N, 2000)], 1)
    ref_pts = oracle.fwd_points(wl.x, wl.w, idx)
    for spec in (None, "default"):
        if spec:
            p.set_variant(spec)
        y = host(p.forward(x, w))
        for r in (0, Ho // 2, Ho - 1):
            ref = oracle.fwd(wl.x[r:r + fh], wl.w)[0]
            assert np.abs(y[r] - ref).max() <= TOL_F32 * np.abs(ref).max(), (spec, r)
        assert np.abs(y[tuple(idx.T)] - ref_pts).max() <= TOL_F32 * np.abs(ref_pts).max(), spec


@pytest.mark.parametrize("shape,spec", [
    ((51, 77, 8, 27, 5, 4), "direct:tr=4,tf=8,wr=2,wf=2,cc=4,pk=1"),      # two 4-channel chunks
    ((41, 70, 10, 12, 3, 5), "direct:tr=8,tf=4,wr=3,wf=1,cc=4,pk=1"),     # depth 10: scalar staging, ragged chunk
    ((64, 40, 32, 40, 5, 5), "direct:tr=2,tf=4,wr=4,wf=2,cc=8,pk=1"),     # four 8-channel chunks
], ids=["c8cc4", "c10cc4", "c32cc8"])
def test_register_prefetch_is_bit_identical(shape, spec):
    """pf=1 loads the next channel chunk into registers while the current one is
    summed and stores it afterwards: the same sums in the same order, so the
    output equals the plain tile's bit for bit (with and without the clamp)."""
    torch = torch_cuda()
    wl = inputs.random_case(520, *shape)
    for clamp in (None, (-0.5, 0.5)):
        y0, _ = _run(torch, wl.x, wl.w, clamp=clamp, spec=spec)
        y1, p1 = _run(torch, wl.x, wl.w, clamp=clamp, spec=spec + ",pf=1")
        assert p1.info()["fwd"]["kernel"].endswith("_pf1")
        assert np.array_equal(y0, y1)
        ref = oracle.fwd(wl.x, wl.w, epilogue=clamp)
        assert np.abs(y1 - ref).max() <= TOL_F32 * np.abs(oracle.fwd(wl.x, wl.w)).max()


@pytest.mark.parametrize("shape,spec", [
    ((40, 70, 32, 24, 5, 5), "direct:tr=8,tf=8,wr=2,wf=2,cc=8,pk=1"),
    ((33, 50, 16, 20, 7, 3), "direct:tr=7,tf=4,wr=2,wf=4,cc=8,pk=1,pf=1"),
    ((30, 45, 8, 16, 9, 9), "direct:tr=8,tf=4,wr=3,wf=2,cc=0,pk=1,ks=8,wq=2,sh=1"),
])
@pytest.mark.parametrize("mb", [2, 3])
def test_occupancy_bound_is_bit_identical(shape, spec, mb):
    """mb=M compiles the same tile with __launch_bounds__(threads, M): only the
    register allocation changes, so the output equals the unbounded tile's bit for
    bit."""
    torch = torch_cuda()
    wl = inputs.random_case(530, *shape)
    y0, _ = _run(torch, wl.x, wl.w, spec=spec)
    y1, p1 = _run(torch, wl.x, wl.w, spec=spec + f",mb={mb}")
    assert p1.info()["fwd"]["kernel"].endswith(f"_mb{mb}")
    assert np.array_equal(y0, y1)
