"""GPU parity of the batched persistent forward (one launch, many uneven
images, each with its own bank) against the FP64 oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import dev, host, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu


def _batch(seed, shapes, kind="real"):
    items = []
    for k, (H, W, D, N, fh, fw) in enumerate(shapes):
        items.append(inputs.random_case(seed + k, H, W, D, N, fh, fw, kind=kind))
    return items


SHAPES = [(40, 70, 8, 16, 3, 3), (33, 45, 4, 32, 5, 5), (64, 64, 16, 20, 7, 7), (20, 150, 32, 64, 11, 11),
          (17, 19, 3, 5, 2, 4), (50, 33, 16, 128, 9, 9), (12, 12, 8, 16, 3, 3)]


def test_batched_matches_oracle_and_single_plans():
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import BatchPlan
    items = _batch(2000, SHAPES)
    bp = BatchPlan([it.x.shape for it in items], [it.w.shape for it in items])
    info = bp.info()
    assert info["launches"] == 1 and info["images"] == len(items)
    xs = [dev(it.x, torch) for it in items]
    ws = [dev(it.w, torch) for it in items]
    ys = bp.forward(xs, ws)
    torch.cuda.synchronize()
    for it, y in zip(items, ys):
        assert normwise_rel(host(y), oracle.fwd(it.x, it.w)) <= 1e-5, it.name


def test_batched_integer_bit_exact_and_repeatable():
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import BatchPlan
    items = _batch(2100, SHAPES, kind="int")
    bp = BatchPlan([it.x.shape for it in items], [it.w.shape for it in items])
    xs = [dev(it.x, torch) for it in items]
    ws = [dev(it.w, torch) for it in items]
    ys = bp.forward(xs, ws)
    first = [y.clone() for y in ys]
    ys2 = bp.forward(xs, ws, ys)          # graph replay with the same pointers
    torch.cuda.synchronize()
    for it, a, b in zip(items, first, ys2):
        assert np.array_equal(host(a), oracle.fwd(it.x, it.w))
        assert torch.equal(a, b)


def test_batched_new_pointers_update_the_graph():
    """A second call with different tensors (new pointers) must use them."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import BatchPlan
    items = _batch(2200, SHAPES[:4])
    bp = BatchPlan([it.x.shape for it in items], [it.w.shape for it in items])
    bp.forward([dev(it.x, torch) for it in items], [dev(it.w, torch) for it in items])
    items2 = _batch(2300, SHAPES[:4])
    ys = bp.forward([dev(it.x, torch) for it in items2], [dev(it.w, torch) for it in items2])
    torch.cuda.synchronize()
    for it, y in zip(items2, ys):
        assert normwise_rel(host(y), oracle.fwd(it.x, it.w)) <= 1e-5


def test_batched_clamp():
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import BatchPlan
    items = _batch(2400, SHAPES[:3])
    bp = BatchPlan([it.x.shape for it in items], [it.w.shape for it in items], clamp=(-0.5, 0.5))
    ys = bp.forward([dev(it.x, torch) for it in items], [dev(it.w, torch) for it in items])
    torch.cuda.synchronize()
    for it, y in zip(items, ys):
        scale = np.abs(oracle.fwd(it.x, it.w)).max()
        assert np.abs(host(y) - oracle.fwd(it.x, it.w, epilogue=(-0.5, 0.5))).max() <= 1e-5 * scale


def test_batch_workload_64_images_sampled():
    """The 64-image uneven batch (H, W in 64..512, D in {4..32}, N in {16..128},
    f in {3..11}): every image checked on two output rows (first and last)
    plus random points against the oracle."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import BatchPlan
    bw = inputs.workload_batch()
    bp = BatchPlan([it.x.shape for it in bw.items], [it.w.shape for it in bw.items])
    assert bp.flops == bw.flops
    ys = bp.forward([dev(it.x, torch) for it in bw.items], [dev(it.w, torch) for it in bw.items])
    torch.cuda.synchronize()
    rng = np.random.default_rng(44)
    for it, y in zip(bw.items, ys):
        yh = host(y)
        Ho, Wo, N = it.out_shape
        fh = it.w.shape[1]
        for r in (0, Ho - 1):
            ref = oracle.fwd(it.x[r:r + fh], it.w)[0]
            assert np.abs(yh[r] - ref).max() <= 1e-5 * np.abs(ref).max(), (it.name, r)
        idx = np.stack([rng.integers(0, Ho, 200), rng.integers(0, Wo, 200), rng.integers(0, N, 200)], 1)
        ref = oracle.fwd_points(it.x, it.w, idx)
        assert np.abs(yh[tuple(idx.T)] - ref).max() <= 1e-5 * np.abs(ref).max(), it.name


def test_batched_bad_arguments():
    torch_cuda()
    from paper_0911_3456_gb300 import _capi as C
    lib = C.load()
    h = ctypes.c_void_p()
    ins = (ctypes.c_int64 * 3)(8, 8, 2)
    fls = (ctypes.c_int64 * 4)(1, 9, 3, 2)       # fh > H
    assert lib.fbcorr_batch_plan_create(ctypes.byref(h), 1, ins, fls, 0, C.epilogue()) == 2
    fls = (ctypes.c_int64 * 4)(1, 3, 3, 2)
    assert lib.fbcorr_batch_plan_create(ctypes.byref(h), 0, ins, fls, 0, C.epilogue()) == 1
    assert lib.fbcorr_batch_plan_create(ctypes.byref(h), 1, ins, fls, 1, C.epilogue()) == 3  # BF16


@pytest.mark.parametrize("clamp", [None, (0.0, 1.5)])
def test_batched_ksplit_variants(clamp, monkeypatch):
    """Batch variants may run the K-split tile (lanes of a group split the
    depth of a short reduction and combine their sums by warp shuffles) inside
    the persistent kernel; FBCORR_BATCH_KS=1 gives every variant that takes one
    its first K-split tile.  Every image against the oracle (integer data:
    exactly), including 4- and 3-channel images, ragged columns and the clamp."""
    torch = torch_cuda()
    from paper_0911_3456_gb300.api import BatchPlan
    monkeypatch.setenv("FBCORR_BATCH_KS", "1")
    shapes = [(40, 70, 8, 16, 3, 3), (33, 45, 4, 32, 5, 5), (64, 64, 16, 20, 7, 7), (12, 12, 8, 16, 3, 3),
              (37, 29, 4, 16, 9, 9), (17, 19, 3, 5, 2, 4), (70, 90, 8, 64, 5, 5)]
    for kind in ("int", "real"):
        items = _batch(2500, shapes, kind=kind)
        bp = BatchPlan([it.x.shape for it in items], [it.w.shape for it in items], clamp=clamp)
        specs = [v["spec"] for v in bp.info()["variants"]]
        assert sum(",ks=" in s for s in specs) >= 3, specs
        xs = [dev(it.x, torch) for it in items]
        ws = [dev(it.w, torch) for it in items]
        ys = bp.forward(xs, ws)
        torch.cuda.synchronize()
        for it, y in zip(items, ys):
            ref = oracle.fwd(it.x, it.w, epilogue=clamp)
            if kind == "int":
                assert np.array_equal(host(y), ref), it.name
            else:
                assert normwise_rel(host(y), ref) <= 1e-5, it.name
