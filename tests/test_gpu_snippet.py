"""Snippet epilogues (fbcorr_plan_create_snippet): a user C expression compiled
into the store path of the generated forward kernels, against the FP64 oracle
followed by the same function in numpy, through the C ABI."""
import numpy as np
import pytest

import oracle
from helpers import dev, host, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16x3": 1e-5, "bf16": 1e-2}
SHAPE = (37, 70, 16, 24, 5, 3)   # several tiles, ragged tails, fh != fw

# (expression, numpy equivalent on the FP64 accumulator z, filter index n, params)
SNIPPETS = {
    "leaky_relu": ("y > 0.f ? y : lo * y", lambda z, n, lo, hi: np.where(z > 0, z, lo * z), (0.1, 0.0)),
    "tanh_scaled": ("hi * tanhf(y)", lambda z, n, lo, hi: hi * np.tanh(z), (0.0, 2.0)),
    "per_filter_bias": ("y + lo * (float)n", lambda z, n, lo, hi: z + lo * n, (0.25, 0.0)),
}


def _plan(mode, wl, expr, params):
    from paper_0911_3456_gb300.api import Plan
    return Plan(wl.x.shape, wl.w.shape, mode, snippet=expr, snippet_params=params)


@pytest.mark.parametrize("mode", ["f32", "bf16x3", "bf16"])
@pytest.mark.parametrize("name", sorted(SNIPPETS))
def test_snippet_matches_oracle(mode, name):
    """Each snippet is 1-Lipschitz in y up to its scale, so the arithmetic error
    of the correlation carries over (scaled) to the output."""
    torch = torch_cuda()
    expr, fn, params = SNIPPETS[name]
    wl = inputs.random_case(2500, *SHAPE)
    p = _plan(mode, wl, expr, params)
    y = host(p.forward(dev(wl.x, torch), dev(wl.w, torch)))
    z = oracle.fwd(wl.x, wl.w)
    n = np.arange(wl.w.shape[0])[None, None, :]
    ref = fn(z, n, *params)
    lip = max(1.0, abs(params[1]))
    tol = TOL[mode] * lip * np.abs(z).max() + 8 * np.finfo(np.float32).eps * np.abs(ref).max()
    assert np.abs(y - ref).max() <= tol, name


@pytest.mark.parametrize("mode", ["f32", "bf16x3"])
def test_clamp_snippet_equals_builtin_clamp(mode):
    """The clamp written as a snippet gives the built-in clamp epilogue's bits."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(2600, *SHAPE)
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    a = host(Plan(wl.x.shape, wl.w.shape, mode, (-0.5, 0.5)).forward(x, w))
    b = host(_plan(mode, wl, "fminf(fmaxf(y, lo), hi)", (-0.5, 0.5)).forward(x, w))
    assert np.array_equal(a, b)


def test_snippet_plan_autotunes_without_the_prebuilt_default():
    """FP32 tuning of a snippet plan times only generated tiles and keeps the
    snippet; the result still matches the oracle."""
    torch = torch_cuda()
    wl = inputs.random_case(2700, *SHAPE)
    p = _plan("f32", wl, "y > 0.f ? y : 0.f", (0.0, 0.0))
    p.autotune()
    assert p.info()["fwd"]["spec"] != "default"
    y = host(p.forward(dev(wl.x, torch), dev(wl.w, torch)))
    ref = np.maximum(oracle.fwd(wl.x, wl.w), 0.0)
    assert normwise_rel(y, ref) <= 1e-5


def test_snippet_plan_is_forward_only_and_reports_compile_errors():
    torch = torch_cuda()
    from paper_0911_3456_gb300 import _capi as C
    wl = inputs.random_case(2800, 20, 20, 4, 3, 3, 3, with_g=True)
    p = _plan("f32", wl, "2.f * y", (0.0, 0.0))
    with pytest.raises(C.FbcorrError) as e:
        p.backward(dev(wl.x, torch), dev(wl.w, torch), dev(wl.g, torch))
    assert e.value.status_name == "FBCORR_ERR_UNSUPPORTED"
    with pytest.raises(C.FbcorrError) as e:
        _plan("f32", wl, "y + undefined_symbol", (0.0, 0.0))
    assert e.value.status_name == "FBCORR_ERR_NVRTC"


def test_snippet_plan_autotunes_on_the_tensor_cores():
    """Tuning a split-BF16 snippet plan times generated tcgen05 variants that all
    carry the snippet; the tuned plan still matches the oracle."""
    torch = torch_cuda()
    wl = inputs.random_case(2900, *SHAPE)
    p = _plan("bf16x3", wl, "y > 0.f ? y : lo * y", (0.2, 0.0))
    p.autotune()
    assert p.info()["fwd"]["detail"]["kernel"].split("_u")[-1] != p.info()["fwd"]["detail"]["kernel"]
    y = host(p.forward(dev(wl.x, torch), dev(wl.w, torch)))
    z = oracle.fwd(wl.x, wl.w)
    ref = np.where(z > 0, z, 0.2 * z)
    assert np.abs(y - ref).max() <= 1e-5 * np.abs(z).max()


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_snippet_through_every_tensor_core_store_path(mode):
    """The snippet is applied before the store in every epilogue path of the
    tensor-core kernel -- direct stores, the staged transpose, tiled bulk stores
    -- and in the tail halves (SM count + 8 tiles of a 256-wide filter tile):
    all give the same bits on integer inputs, and the oracle's."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    wl = inputs.random_case(3000, sms + 8 + 2, 128, 16, 256, 3, 3, kind="int")
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    expr, params = "y > 0.f ? y : lo * y", (0.25, 0.0)     # exact on integers: y * 1/4
    z = oracle.fwd(wl.x, wl.w)
    ref = np.where(z > 0, z, 0.25 * z)
    base = "tcgen05:na=2,nb=3,nt=256,bt=3,ew=8,fz=1,nr=0,cw=8"
    for suffix in ("", ",ts=1,sb=1", ",ts=32,sb=1"):
        p = _plan(mode, wl, expr, params)
        p.set_variant(base + suffix)
        assert p.info()["fwd"]["detail"]["tail_half_tiles"] == 8
        assert np.array_equal(host(p.forward(x, w)), ref), suffix
