"""The forward entry point that allocates nothing (fbcorr_forward_noalloc).

It exists for callers that cannot allocate device memory when they run the
correlation; it must give the same output as fbcorr_forward with a workspace.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import dev, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import _capi as C
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(lib, p, x, w, y, stream):
    st = lib.fbcorr_forward_noalloc(p.handle, _vp(x), _vp(w), _vp(y), ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, C.last_error()


@pytest.mark.parametrize("spec", [None, "tcgen05:na=2,nb=2,nt=256,bt=1,ew=4,fz=0,nr=0,cw=0"],
                         ids=["default", "prepass"])
def test_noalloc_forward_matches_workspace_forward_twice(spec):
    """Two calls in a row on one split-BF16 plan, each with new inputs, and
    between them a call of another plan (larger in every dimension, large
    non-zero values, the pre-pass variant, so that it writes x and w planes
    over the whole region the first plan uses, padding included).  The
    built-in scratch keeps whatever the previous call wrote, so each check
    shows that nothing stale is read: the output equals the workspace path bit
    for bit, and the oracle within the split-BF16 gate (integer data: exactly)."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    lib = C.load()
    shape = (40, 150, 32, 64, 5, 5)
    p = Plan(shape[:3], (shape[3], shape[4], shape[5], shape[2]), "bf16x3")
    if spec:
        p.set_variant(spec)
    assert 0 < p.ws_fwd <= 48 << 20
    other_shape = (64, 200, 48, 96, 7, 7)
    other = Plan(other_shape[:3], (other_shape[3], other_shape[4], other_shape[5], other_shape[2]), "bf16x3")
    other.set_variant("tcgen05:na=2,nb=2,nt=256,bt=1,ew=4,fz=0,nr=0,cw=0")
    assert p.ws_fwd < other.ws_fwd <= 48 << 20
    stream = torch.cuda.current_stream()
    for seed, kind in ((71, "int"), (72, "real")):
        wl = inputs.random_case(seed, *shape, kind=kind)
        x, w = dev(wl.x, torch), dev(wl.w, torch)
        y_ref = p.forward(x, w)                       # existing entry, caller workspace
        y = torch.full_like(y_ref, float("nan"))
        _noalloc(lib, p, x, w, y, stream)
        torch.cuda.synchronize()
        a = y.cpu().numpy()
        assert np.isfinite(a).all()
        assert np.array_equal(a, y_ref.cpu().numpy())   # same kernels, same order
        ref = oracle.fwd(wl.x, wl.w)
        if kind == "int":
            assert np.array_equal(a.astype(np.float64), ref)
        else:
            assert normwise_rel(a, ref) <= 2e-5
        # the other plan fills the shared scratch with large non-zero planes
        ow = inputs.random_case(seed + 100, *other_shape)
        ox, oww = dev(1e3 * ow.x + 5e2, torch), dev(1e3 * ow.w + 5e2, torch)
        oy = torch.empty(other.out_shape, device="cuda")
        _noalloc(lib, other, ox, oww, oy, stream)
        torch.cuda.synchronize()
        assert np.isfinite(oy.cpu().numpy()).all()


def test_noalloc_rejects_plans_beyond_the_scratch_size():
    torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    lib = C.load()
    p = Plan((1024, 1024, 64), (16, 3, 3, 64), "bf16x3")   # needs far more than 48 MiB
    assert p.ws_fwd > 48 << 20
    st = lib.fbcorr_forward_noalloc(p.handle, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                    ctypes.c_void_p(16), None)
    assert st == 5 and "scratch" in C.last_error()
