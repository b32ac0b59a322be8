"""GPU parity of the tcgen05 tensor-core path (BF16 and split-BF16) against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from helpers import dev, host, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"bf16": 1e-2, "bf16x3": 1e-5}


def gamma(mode, K):
    """Elementwise bound factor: |y - y_exact| <= gamma * sum_k |x_k w_k|.
    BF16: each operand rounded (unit roundoff 2^-8) -> 2*2^-8 + 2^-16 per product.
    Split BF16: v = hi + lo + e with |e| <= 2^-16 |v|; the dropped lo*lo term is
    <= 2^-16 |xw| -> about 3.05 * 2^-16 per product.  Plus FP32 accumulation:
    one rounding of at most 2 ulp (2^-22) per MMA into the accumulator, K/16
    (BF16) or 3K/16 (split) MMAs."""
    n_mma = (K + 15) // 16 * (3 if mode == "bf16x3" else 1)
    per_term = (2 * 2.0 ** -8 + 2.0 ** -16) if mode == "bf16" else 3.05 * 2.0 ** -16
    return per_term + n_mma * 2.0 ** -22


def assert_within_bound(y, x, w, mode, clamp=None):
    ref = oracle.fwd(x, w, epilogue=clamp)
    absref = oracle.fwd(np.abs(x), np.abs(w))
    K = w.shape[1] * w.shape[2] * w.shape[3]
    bound = gamma(mode, K) * absref
    excess = np.abs(y - ref) - bound
    assert excess.max() <= 0, (mode, float(excess.max()), float(normwise_rel(y, ref)))

SHAPES = [
    # H, W, D, N, fh, fw: ragged tiles, N not a multiple of 16, N > 256 (two
    # filter tiles), D below / above 16, fh != fw, 1x1 filters
    (20, 150, 16, 16, 3, 3),
    (37, 45, 3, 5, 4, 2),
    (40, 200, 32, 64, 5, 5),
    (33, 97, 8, 20, 3, 5),
    (25, 140, 16, 300, 2, 3),
    (18, 260, 48, 40, 7, 7),
    (30, 131, 64, 256, 1, 1),
    (9, 9, 4, 3, 9, 9),
]


def _plan(torch, mode, x, w, clamp=None):
    from paper_0911_3456_gb300.api import Plan
    return Plan(x.shape, w.shape, mode, clamp)


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_tc_matches_oracle(mode, shape):
    torch = torch_cuda()
    wl = inputs.random_case(1300, *shape)
    p = _plan(torch, mode, wl.x, wl.w)
    y = host(p.forward(dev(wl.x, torch), dev(wl.w, torch)))
    torch.cuda.synchronize()
    assert p.device_status() == 0
    assert_within_bound(y, wl.x, wl.w, mode)
    if mode == "bf16":
        assert normwise_rel(y, oracle.fwd(wl.x, wl.w)) <= TOL[mode]


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
@pytest.mark.parametrize("shape", SHAPES[:6], ids=lambda s: "x".join(map(str, s)))
def test_tc_integer_bit_exact(mode, shape):
    """Integers in [-4, 4] are exact in BF16 and every partial sum is an exact
    FP32 integer: both modes must reproduce the oracle bit for bit."""
    torch = torch_cuda()
    wl = inputs.random_case(1400, *shape, kind="int")
    p = _plan(torch, mode, wl.x, wl.w)
    y = host(p.forward(dev(wl.x, torch), dev(wl.w, torch)))
    assert np.array_equal(y, oracle.fwd(wl.x, wl.w))


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_tc_clamp(mode):
    torch = torch_cuda()
    wl = inputs.random_case(1500, 40, 133, 16, 48, 3, 3)
    clamp = (-0.5, 0.5)
    p = _plan(torch, mode, wl.x, wl.w, clamp)
    y = host(p.forward(dev(wl.x, torch), dev(wl.w, torch)))
    assert_within_bound(y, wl.x, wl.w, mode, clamp)   # the clamp is 1-Lipschitz
    assert y.min() >= -0.5 and y.max() <= 0.5


def test_tc_delta_filters_bit_exact():
    """Unit-impulse filters copy shifted input windows; with BF16-representable
    inputs both modes are exact."""
    torch = torch_cuda()
    rng = np.random.default_rng(4)
    H, W, D, fh, fw = 20, 150, 16, 3, 4
    x = rng.integers(-64, 64, (H, W, D)).astype(np.float32) / 8.0
    taps = [(i, j, d) for i in range(fh) for j in range(fw) for d in (0, 5, 15)]
    w = np.zeros((len(taps), fh, fw, D), np.float32)
    for n, (i, j, d) in enumerate(taps):
        w[n, i, j, d] = 1.0
    Ho, Wo = H - fh + 1, W - fw + 1
    for mode in ("bf16", "bf16x3"):
        y = host(_plan(torch, mode, x, w).forward(dev(x, torch), dev(w, torch)))
        for n, (i, j, d) in enumerate(taps):
            assert np.array_equal(y[:, :, n], x[i:i + Ho, j:j + Wo, d].astype(np.float64)), (mode, i, j, d)


def test_tc_deterministic_and_guard_bands():
    torch = torch_cuda()
    wl = inputs.random_case(1600, 30, 170, 32, 96, 5, 5)
    p = _plan(torch, "bf16x3", wl.x, wl.w)
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    n = int(np.prod(p.out_shape))
    buf = torch.full((n + 4096,), 7.0, device="cuda")
    y = buf[2048:2048 + n].view(p.out_shape)
    p.forward(x, w, y=y)
    a = y.clone()
    p.forward(x, w, y=y)
    torch.cuda.synchronize()
    assert torch.equal(a, y)
    assert torch.all(buf[:2048] == 7.0) and torch.all(buf[2048 + n:] == 7.0)


def test_precision_config_full_size():
    """512x512x32 U[-1,1) input, 256 filters 5x5x32 N(0, 1/800): split-BF16 at
    <= 1e-5 and BF16 at <= 1e-2 (normwise) on output rows spanning the image
    (first, last, and a band in the middle), plus random points."""
    torch = torch_cuda()
    wl = inputs.workload_precision()
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    rows = [0, 1, 250, 251, 252, 506, 507]
    Ho, Wo, N = wl.out_shape
    rng = np.random.default_rng(12)
    idx = np.stack([rng.integers(0, Ho, 4000), rng.integers(0, Wo, 4000), rng.integers(0, N, 4000)], 1)
    ref_pts = oracle.fwd_points(wl.x, wl.w, idx)
    errs = {}
    for mode in ("bf16", "bf16x3"):
        p = _plan(torch, mode, wl.x, wl.w)
        y = host(p.forward(x, w))
        assert p.device_status() == 0
        e = 0.0
        for r in rows:
            ref = oracle.fwd(wl.x[r:r + 5], wl.w)[0]
            e = max(e, np.abs(y[r] - ref).max() / np.abs(ref).max())
        e = max(e, np.abs(y[tuple(idx.T)] - ref_pts).max() / np.abs(ref_pts).max())
        errs[mode] = e
        assert e <= TOL[mode], (mode, e)
    print("precision config errors:", errs)


def test_split_beats_bf16_and_approaches_fp32():
    """On zero-mean, unit-norm filters (the paper's first table row, 256x256x8
    with 64 filters 9x9x8) split-BF16 stays within 1e-5 normwise while plain
    BF16 does not reach it."""
    torch = torch_cuda()
    wl = inputs.workload_paper_row1_clamp()
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    ref = oracle.fwd(wl.x, wl.w)
    e = {}
    for mode in ("bf16", "bf16x3"):
        e[mode] = normwise_rel(host(_plan(torch, mode, wl.x, wl.w).forward(x, w)), ref)
    assert e["bf16x3"] <= 1e-5 < e["bf16"] <= 1e-2, e


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_every_tensor_core_configuration_matches(mode):
    """Every configuration the auto-tuner may pick (ring depths, filter-tile
    width, taps per B stage -- including a last stage with fewer taps --,
    epilogue warps, conversion of x by the pre-pass, by converter warps from
    global memory or from a ring of raw rows) gives the same result on integer
    inputs, bit for bit."""
    torch = torch_cuda()
    from paper_0911_3456_gb300 import _capi as C
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(1700, 21, 140, 32, 272, 3, 5, kind="int")
    ref = oracle.fwd(wl.x, wl.w)
    p = Plan(wl.x.shape, wl.w.shape, mode)
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    # every generated kernel (taps per stage x epilogue warps x conversion of x),
    # each with one of four ring / filter-tile shapes, plus ring-depth variations
    # of one kernel
    rings = [(2, 2, 256), (3, 4, 128), (2, 3, 128), (3, 2, 256)]
    specs = set()
    k = 0
    for bt in (1, 2, 3, 5):
        for ew in (4, 8):
            for fz, nr in ((0, 0), (1, 0), (2, 2), (2, 3)):
                na, nb, nt = rings[k % len(rings)]
                cw = 0 if fz == 0 else (4, 8)[k % 2]
                k += 1
                specs.add(f"tcgen05:na={na},nb={nb},nt={nt},bt={bt},ew={ew},fz={fz},nr={nr},cw={cw}")
    for na, nb, nt in [(2, 4, 256), (3, 3, 256), (2, 2, 128), (3, 4, 256)]:
        specs.add(f"tcgen05:na={na},nb={nb},nt={nt},bt=2,ew=8,fz=2,nr=2,cw=8")
    ran = 0
    for sp in sorted(specs):
        try:
            p.set_variant(sp)
        except C.FbcorrError:
            continue              # does not fit this shape's shared memory
        assert p.info()["fwd"]["spec"] == sp
        y = host(p.forward(x, w))
        assert np.array_equal(y, ref), sp
        ran += 1
    assert ran >= 24


@pytest.mark.parametrize("mode", ["f32", "bf16", "bf16x3"])
def test_forward_captures_into_a_cuda_graph(mode):
    """The forward is CUDA-graph capturable in every mode -- for the tensor-core
    modes that includes the operand split and the correlation kernel launched as
    its programmatic dependent -- and replaying the graph gives the eager bits."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(1770, 37, 96, 16, 40, 3, 3)
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    p = Plan(wl.x.shape, wl.w.shape, mode)
    y_eager = p.forward(x, w).clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        p.forward(x, w)                 # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    y = torch.empty(p.out_shape, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        p.forward(x, w, y)
    for _ in range(2):
        y.zero_()
        graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, y_eager)
    assert p.device_status() == 0


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_tail_halves_bit_exact(mode, monkeypatch):
    """With SM count + 8 tiles of one 256-wide filter tile, the last partial
    round (8 tiles) runs as 16 half items of 128 filters each, with their B
    operand from the half-width planes; every store path gives the oracle's bits
    on integer inputs, and the same bits with the halves switched off."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    W, fh, fw = 128, 3, 3
    H = sms + 8 + fh - 1                      # H' * W / 128 = sms + 8 tiles
    wl = inputs.random_case(1760, H, W, 16, 256, fh, fw, kind="int")
    ref = oracle.fwd(wl.x, wl.w)
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    base = "tcgen05:na=2,nb=3,nt=256,bt=3,ew=8,fz=1,nr=0,cw=8"
    for suffix in ("", ",ts=1,sb=1", ",ts=32,sb=1"):
        p = Plan(wl.x.shape, wl.w.shape, mode)
        p.set_variant(base + suffix)
        assert p.info()["fwd"]["detail"]["tail_half_tiles"] == 8
        assert np.array_equal(host(p.forward(x, w)), ref), suffix
    monkeypatch.setenv("FBCORR_TAIL_HALVES", "0")
    p = Plan(wl.x.shape, wl.w.shape, mode)
    p.set_variant(base)
    assert p.info()["fwd"]["detail"]["tail_half_tiles"] == 0
    assert np.array_equal(host(p.forward(x, w)), ref)


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
@pytest.mark.parametrize("shape", [(37, 96, 16, 96, 3, 3), (37, 128, 32, 320, 5, 5), (21, 140, 32, 40, 3, 5)],
                         ids=lambda s: "x".join(map(str, s)))
def test_store_modes_bit_exact(mode, shape):
    """Direct stores, the staged transpose (ts=1), tiled bulk stores through a
    tensor map (ts=32: needs W % 32 == 0, N % 4 == 0 and a filter tile that is a
    multiple of 32, else refused) give the oracle's bits on integer inputs,
    with and without the clamp;
    an output that is not 16-byte aligned is refused before any launch."""
    torch = torch_cuda()
    from paper_0911_3456_gb300 import _capi as C
    from paper_0911_3456_gb300.api import Plan
    H, W, D, N, fh, fw = shape
    wl = inputs.random_case(1750, *shape, kind="int")
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    tiled_ok = W % 32 == 0 and N % 4 == 0
    base = "tcgen05:na=2,nb=2,nt=256,bt=1,ew=8,fz=1,nr=0,cw=8"
    suffixes = ("", ",ts=1,sb=1", ",ts=32,sb=1", ",ts=32,sb=2")
    for clamp in (None, (-40.0, 40.0)):
        ref = oracle.fwd(wl.x, wl.w, epilogue=clamp)
        p = Plan(wl.x.shape, wl.w.shape, mode, clamp)
        ran = 0
        for suffix in suffixes:
            try:
                p.set_variant(base + suffix)
            except C.FbcorrError as e:
                assert "ts=32" in suffix and not tiled_ok, (suffix, str(e))
                continue
            assert np.array_equal(host(p.forward(x, w)), ref), suffix
            if "ts=32" in suffix:
                buf = torch.empty(ref.size + 1, device="cuda")
                with pytest.raises(C.FbcorrError) as e:
                    p.forward(x, w, buf[1:].view(ref.shape))   # 4 bytes past a 16-byte boundary
                assert e.value.status_name == "FBCORR_ERR_ALIGNMENT"
            ran += 1
        assert ran == (4 if tiled_ok else 2)


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
@pytest.mark.parametrize("shape", [(20, 150, 16, 16, 3, 3), (37, 45, 4, 20, 4, 2), (18, 260, 28, 40, 7, 7),
                                   (9, 9, 12, 3, 9, 9)], ids=lambda s: "x".join(map(str, s)))
def test_fused_conversion_matches_prepass(mode, shape):
    """x converted inside the kernel (fz=1 from global memory, fz=2 from a ring of
    raw rows) and by the pre-pass (fz=0) give the same bits, including the
    zero-filled tail past the end of the image."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(1800, *shape)
    p = Plan(wl.x.shape, wl.w.shape, mode)
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    outs = {}
    for fz, nr, cw in ((0, 0, 0), (1, 0, 8), (2, 2, 4)):
        p.set_variant(f"tcgen05:na=2,nb=2,nt=256,bt=1,ew=4,fz={fz},nr={nr},cw={cw}")
        outs[fz] = host(p.forward(x, w))
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])
    assert_within_bound(outs[1], wl.x, wl.w, mode)


def test_fused_conversion_limits():
    """Conversion inside the kernel needs D % 4 == 0 (x is read in 16-byte units);
    from registers (fz=1) also at most 32 channels.  Other depths take the
    pre-pass, and a spec that does not fit is refused."""
    torch_cuda()
    from paper_0911_3456_gb300 import _capi as C
    from paper_0911_3456_gb300.api import Plan
    p = Plan((16, 40, 6), (8, 3, 3, 6), "bf16")
    assert ",fz=0," in p.info()["fwd"]["spec"]
    for fz, nr in ((1, 0), (2, 2)):
        with pytest.raises(C.FbcorrError):
            p.set_variant(f"tcgen05:na=2,nb=2,nt=256,bt=1,ew=4,fz={fz},nr={nr},cw=8")
    p = Plan((16, 40, 48), (8, 3, 3, 48), "bf16")
    assert ",fz=2," in p.info()["fwd"]["spec"]
    with pytest.raises(C.FbcorrError):
        p.set_variant("tcgen05:na=2,nb=2,nt=256,bt=1,ew=4,fz=1,nr=0,cw=8")


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
@pytest.mark.parametrize("shape", [(37, 96, 16, 160, 3, 3), (21, 140, 32, 40, 3, 5), (40, 64, 32, 256, 5, 5),
                                   (9, 9, 12, 3, 9, 9)], ids=lambda s: "x".join(map(str, s)))
def test_resident_bank_bit_exact(mode, shape):
    """rs=1 loads the B ring once with every tap of the CTA's filter tile and
    walks pixel tiles under it (two filter tiles: the CTAs split into two
    groups): the same MMAs in the same order as the streamed ring, so the same
    bits; on integer inputs the oracle's.  Shapes whose filter tile does not
    fit in shared memory are refused."""
    torch = torch_cuda()
    from paper_0911_3456_gb300 import _capi as C
    from paper_0911_3456_gb300.api import Plan
    H, W, D, N, fh, fw = shape
    p = Plan((H, W, D), (N, fh, fw, D), mode)
    res = [s for s in p.candidates() if s.endswith(",rs=1")]
    ran = 0
    for nt in (256, 128):
        specs = [s for s in res if f",nt={nt}," in s]
        if not specs:
            continue
        spec = specs[0]
        streamed = spec.split(",nb=")[0] + ",nb=2," + spec.split(",nb=")[1].split(",", 1)[1]
        streamed = streamed.replace(",rs=1", "")
        for kind in ("int", "real"):
            wl = inputs.random_case(1900, *shape, kind=kind)
            x, w = dev(wl.x, torch), dev(wl.w, torch)
            p.set_variant(spec)
            y_res = host(p.forward(x, w))
            assert p.device_status() == 0
            try:
                p.set_variant(streamed)
            except C.FbcorrError:
                continue
            y_str = host(p.forward(x, w))
            assert np.array_equal(y_res, y_str), (spec, streamed)
            if kind == "int":
                assert np.array_equal(y_res, oracle.fwd(wl.x, wl.w)), spec
        ran += 1
    if mode == "bf16" and shape[2] <= 32 and shape[3] <= 256:
        assert ran >= 1


PAIR_SHAPES = [
    # one 256-wide filter tile: an odd pixel-tile count (the odd CTA of the last
    # pair holds a tile past the image), W not a multiple of 32, six and eight
    # chunk planes, 1x1 filters, N padded to 256
    (41, 64, 32, 256, 5, 5),
    (40, 200, 32, 256, 5, 5),
    (18, 128, 48, 256, 7, 7),
    (30, 131, 64, 256, 1, 1),
    (12, 96, 8, 250, 3, 3),
]


def _single_cta(spec, p, C):
    """A single-CTA kernel: the same configuration (with a two-stage ring when
    the pair's ring does not fit), else the first single-CTA candidate -- every
    tensor-core variant sums the same products in the same order."""
    base = spec.replace(",cg=2", "")
    cands = [base, base.split(",nb=")[0] + ",nb=2," + base.split(",nb=")[1].split(",", 1)[1]]
    cands += [s for s in p.candidates() if ",cg=2" not in s][:1]
    for cand in cands:
        try:
            p.set_variant(cand)
            return cand
        except C.FbcorrError:
            continue
    return None


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
@pytest.mark.parametrize("shape", PAIR_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_cta_pair_bit_exact(mode, shape):
    """cg=2 runs each pair of 128-pixel tiles as one M = 256 tile on two SMs
    (cta_group::2 MMAs, half of the bank staged in each CTA): the same products
    summed in the same order as the single-CTA kernel, so the same bits, with
    every conversion path (pre-pass, converters, raw-row ring) and store path;
    on integer inputs the oracle's."""
    torch = torch_cuda()
    from paper_0911_3456_gb300 import _capi as C
    from paper_0911_3456_gb300.api import Plan
    H, W, D, N, fh, fw = shape
    clamp = (-0.5, 0.75) if shape[0] == 12 else None
    p = Plan((H, W, D), (N, fh, fw, D), mode, clamp)
    pairs = [s for s in p.candidates() if s.endswith(",cg=2")]
    assert pairs, "a single 256-wide filter tile offers CTA pairs"
    # one configuration per (conversion, store path)
    picked = {}
    for s in pairs:
        key = (s.split(",fz=")[1][0], s.split(",ts=")[1].split(",")[0] if ",ts=" in s else "0")
        picked.setdefault(key, s)
    for spec in picked.values():
        for kind in ("int", "real"):
            wl = inputs.random_case(2200, *shape, kind=kind)
            x, w = dev(wl.x, torch), dev(wl.w, torch)
            p.set_variant(spec)
            assert p.info()["fwd"]["detail"]["mma"].startswith("256x256x16")
            y_pair = host(p.forward(x, w))
            assert p.device_status() == 0, spec
            single = _single_cta(spec, p, C)
            assert single is not None, spec
            y_one = host(p.forward(x, w))
            assert np.array_equal(y_pair, y_one), (spec, single)
            if kind == "int":
                assert np.array_equal(y_pair, oracle.fwd(wl.x, wl.w, epilogue=clamp)), spec


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
@pytest.mark.parametrize("shape", [(196, 128, 32, 256, 5, 5), (195, 128, 16, 250, 3, 3)],
                         ids=lambda s: "x".join(map(str, s)))
def test_cta_pair_tail_halves_bit_exact(mode, shape, monkeypatch):
    """96 pairs of tiles on 76 pairs of SMs: the last 20 pairs run as two
    M = 256, N = 128 work items each, every CTA staging a quarter of the bank
    from the quarter-width planes.  Per output the same products in the same
    order: the bits of the pair kernel without tail halves and of the
    single-CTA kernel, and on integer inputs the oracle's.  The second shape
    has an odd tile count, so the odd CTA of the last (split) pair holds a
    tile past the image."""
    torch = torch_cuda()
    from paper_0911_3456_gb300 import _capi as C
    from paper_0911_3456_gb300.api import Plan
    H, W, D, N, fh, fw = shape
    p = Plan((H, W, D), (N, fh, fw, D), mode)
    pairs = [s for s in p.candidates() if s.endswith(",cg=2")]
    assert pairs
    spec = pairs[0]
    for kind in ("int", "real"):
        wl = inputs.random_case(2400, *shape, kind=kind)
        x, w = dev(wl.x, torch), dev(wl.w, torch)
        monkeypatch.setenv("FBCORR_TAIL_HALVES", "1")
        p.set_variant(spec)
        det = p.info()["fwd"]["detail"]
        sms = p.info().get("sm_count", 152)
        npairs = (det["tiles"] + 1) // 2
        rem = npairs % (sms // 2)
        expect_tail = npairs > sms // 2 and 0 < rem and 2 * rem <= sms // 2
        assert det["tail_half_tiles"] == (2 * rem if expect_tail else 0), det
        y_tail = host(p.forward(x, w))
        assert p.device_status() == 0, spec
        monkeypatch.setenv("FBCORR_TAIL_HALVES", "0")
        p.set_variant(spec)
        assert p.info()["fwd"]["detail"]["tail_half_tiles"] == 0
        y_whole = host(p.forward(x, w))
        assert np.array_equal(y_tail, y_whole), spec
        single = _single_cta(spec, p, C)
        assert single is not None, spec
        y_one = host(p.forward(x, w))
        assert np.array_equal(y_tail, y_one), (spec, single)
        if kind == "int":
            assert np.array_equal(y_tail, oracle.fwd(wl.x, wl.w)), spec
