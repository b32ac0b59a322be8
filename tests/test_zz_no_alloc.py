"""The forward entry point that allocates nothing (fbcorr_forward_noalloc).

It exists for callers that cannot allocate device memory when they run the
correlation; it must give the same output as fbcorr_forward with a workspace.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

from helpers import dev, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import _capi as C
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_forward_matches_workspace_forward_twice():
    """Two calls in a row on one split-BF16 plan, each with new inputs: the
    built-in scratch keeps the previous call's contents, so the second call
    shows that nothing stale is read."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    lib = C.load()
    shape = (40, 150, 32, 64, 5, 5)
    p = Plan(shape[:3], (shape[3], shape[4], shape[5], shape[2]), "bf16x3")
    assert 0 < p.ws_fwd <= 48 << 20
    stream = torch.cuda.current_stream()
    for seed in (71, 72):
        wl = inputs.random_case(seed, *shape)
        x, w = dev(wl.x, torch), dev(wl.w, torch)
        y_ref = p.forward(x, w)                       # existing entry, caller workspace
        y = torch.full_like(y_ref, float("nan"))
        st = lib.fbcorr_forward_noalloc(p.handle, _vp(x), _vp(w), _vp(y),
                                        ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, C.last_error()
        torch.cuda.synchronize()
        a = y.cpu().numpy()
        b = y_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert normwise_rel(a, b) <= 1e-5
        assert np.array_equal(a, b)                   # same kernels, same order


def test_noalloc_rejects_plans_beyond_the_scratch_size():
    torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    lib = C.load()
    p = Plan((1024, 1024, 64), (16, 3, 3, 64), "bf16x3")   # needs far more than 48 MiB
    assert p.ws_fwd > 48 << 20
    st = lib.fbcorr_forward_noalloc(p.handle, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                    ctypes.c_void_p(16), None)
    assert st == 5 and "scratch" in C.last_error()
