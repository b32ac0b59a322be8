"""The three-layer cascade (filter bank -> static non-linearity -> next bank
across the previous layer's output), against the FP64 oracle run layer by layer
with the same non-linearities in numpy (intermediates rounded to FP32 like the
device's)."""
import numpy as np
import pytest

import oracle
from helpers import dev, host, normwise_rel, torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu

LAYERS = [(8, 5, 5, "y > 0.f ? y : 0.f", lambda z: np.maximum(z, 0.0)),
          (6, 3, 4, "fminf(fmaxf(y, lo), hi)", lambda z: np.clip(z, -1.0, 1.0)),
          (4, 3, 3, None, lambda z: z)]


@pytest.mark.parametrize("mode", ["f32", "bf16x3"])
def test_cascade_matches_layerwise_oracle(mode):
    torch = torch_cuda()
    from paper_0911_3456_gb300.cascade import Cascade, Layer
    rng = np.random.default_rng(2900)
    x = inputs.uniform(rng, (40, 44, 4))
    banks, depth = [], 4
    for (N, fh, fw, _, _) in LAYERS:
        banks.append(inputs.normal(rng, (N, fh, fw, depth), 1.0 / (fh * fw * depth)))
        depth = N
    cas = Cascade(x.shape, [Layer(N, fh, fw, expr, (-1.0, 1.0)) for (N, fh, fw, expr, _) in LAYERS], mode)
    y = host(cas.forward(dev(x, torch), [dev(w, torch) for w in banks]))
    h = x
    for (_, _, _, _, fn), w in zip(LAYERS, banks):
        h = fn(oracle.fwd(h, w)).astype(np.float32)
    assert y.shape == h.shape == cas.out_shape
    assert normwise_rel(y, h) <= 5e-5


def test_cascade_workload_shapes():
    """The bench's cascade: 256x256x8 -> 64x9x9 -> 32x5x5 -> 16x3x3."""
    torch_cuda()
    from paper_0911_3456_gb300.cascade import Cascade, Layer
    x, banks = inputs.workload_cascade()
    cas = Cascade(x.shape, [Layer(w.shape[0], w.shape[1], w.shape[2], "y > 0.f ? y : 0.f") for w in banks])
    assert cas.filt_shapes == [w.shape for w in banks]
    assert cas.out_shape == (242, 242, 16)
    assert cas.flops == sum(2 * (a - f + 1) * (b - g + 1) * n * f * g * d
                            for (a, b, d), (n, f, g, _) in zip([(256, 256, 8), (248, 248, 64), (244, 244, 32)],
                                                               [w.shape for w in banks]))
