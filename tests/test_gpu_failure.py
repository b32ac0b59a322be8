"""Failure detection on the GPU without faulting it: bounded waits that run
out report a status the host reads, code-generation failure falls back to the
prebuilt kernel, and a corrupt tuning cache is ignored."""
import os

import numpy as np
import pytest

import oracle
from helpers import dev, host, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu


class _env:
    def __init__(self, **kv):
        self.kv = kv
        self.old = {}

    def __enter__(self):
        for k, v in self.kv.items():
            self.old[k] = os.environ.get(k)
            os.environ[k] = v

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("spec,N", [(None, 32), ("tcgen05:na=2,nb=3,nt=256,bt=1,ew=8,fz=1,nr=0,cw=8,ts=1,sb=1", 32),
                                    ("tcgen05:na=2,nb=4,nt=256,bt=1,ew=4,fz=1,nr=0,cw=8,cg=2", 256)],
                         ids=["default", "staged_stores", "cta_pair"])
def test_dropped_copy_times_out_and_context_survives(spec, N):
    """FBCORR_FAULT=tcdrop makes the producer skip one copy that the MMA warp
    waits for -- an arrival that never comes.  Every wait is bounded (here
    50 ms): the kernel records FBCORR_ERR_TIMEOUT in host-mapped memory, drains
    its own copies and MMAs, frees TMEM and returns; the next plan on the same
    context computes correct results, with the default variant, with the
    staged-store epilogue, and with CTA pairs (both CTAs of a pair give up on
    their own bounded waits and meet at the closing cluster barrier)."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(3000, 20, 150, 16, N, 3, 3)
    x, w = dev(wl.x, torch), dev(wl.w, torch)
    with _env(FBCORR_FAULT="tcdrop", FBCORR_WAIT_MS="50"):
        bad = Plan(wl.x.shape, wl.w.shape, "bf16x3")
    if spec:
        bad.set_variant(spec)
    bad.forward(x, w)
    torch.cuda.synchronize()                    # the launch itself succeeds
    assert bad.device_status() == 9             # FBCORR_ERR_TIMEOUT
    assert bad.device_status(clear=True) == 9
    assert bad.device_status() == 0
    good = Plan(wl.x.shape, wl.w.shape, "bf16x3")
    y = host(good.forward(x, w))
    torch.cuda.synchronize()
    assert good.device_status() == 0
    assert normwise_rel(y, oracle.fwd(wl.x, wl.w)) <= 2e-5


def test_nvrtc_failure_falls_back_to_prebuilt_kernel(tmp_path):
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    wl = inputs.random_case(3100, 30, 41, 4, 6, 3, 3)
    with _env(FBCORR_FAULT="nvrtc,nocache", FBCORR_CACHE_DIR=str(tmp_path)):
        p = Plan(wl.x.shape, wl.w.shape, "f32")
        assert p.info()["fwd"]["kind"] == "default"
        y = host(p.forward(dev(wl.x, torch), dev(wl.w, torch)))
    assert normwise_rel(y, oracle.fwd(wl.x, wl.w)) <= 1e-5


def test_corrupt_tune_cache_is_ignored(tmp_path):
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import Plan
    (tmp_path / "tune.tsv").write_bytes(b"\x00\xffgarbage\nno-tab-line\n\tempty-key\nkey-only\t\n")
    wl = inputs.random_case(3200, 30, 41, 4, 6, 3, 3)
    with _env(FBCORR_CACHE_DIR=str(tmp_path)):
        p = Plan(wl.x.shape, wl.w.shape, "f32")
        assert p.info()["fwd"]["source"] == "heuristic"
        p.autotune()                               # rewrites the cache atomically
        assert p.info()["fwd"]["source"] == "tuned"
        q = Plan(wl.x.shape, wl.w.shape, "f32")
        assert q.info()["fwd"]["source"] == "cache"
        y = host(q.forward(dev(wl.x, torch), dev(wl.w, torch)))
    assert normwise_rel(y, oracle.fwd(wl.x, wl.w)) <= 1e-5
    text = (tmp_path / "tune.tsv").read_text(errors="replace")
    assert "direct:" in text or "default" in text
