"""Checks that pin the FP64 oracle to facts other than its own formula.

Each function takes an oracle module (``orc``) and raises AssertionError when
the oracle disagrees with:
  * hand-worked examples (tests/golden), derived with pencil and paper;
  * a library special case (scipy.signal.correlate2d / convolve2d, torch conv2d
    in float64), which computes the same 'valid' cross-correlation;
  * closed forms (delta filters, constant and affine inputs);
  * invariants (linearity, the adjoint identity, finite differences).
The same functions are run against deliberately broken copies of the oracle
(test_oracle.py) to show that each plausible mistake is caught.
"""
import numpy as np
from scipy import signal

from conftest import read_golden


def _arr(vals, shape):
    return np.array(vals, dtype=np.float64).reshape(shape)


def pin_golden_hand(orc):
    G = read_golden("hand_case_3x3.txt")
    x = _arr(G["x"], [int(v) for v in G["x_shape"]])
    w = _arr(G["w"], [int(v) for v in G["w_shape"]])
    g = _arr(G["g"], (2, 2, 1))
    assert np.array_equal(orc.fwd(x, w).ravel(), np.array(G["y"]))
    assert np.array_equal(orc.bwd_input(g, w, x.shape).ravel(), np.array(G["dx"]))
    assert np.array_equal(orc.bwd_filt(x, g, w.shape).ravel(), np.array(G["dw"]))
    lo, hi = G["clamp"]
    yc = orc.fwd(x, w, epilogue=(lo, hi))
    assert np.array_equal(yc.ravel(), np.array(G["y_clamp"]))
    assert np.array_equal(orc.bwd_input(g, w, x.shape, y=yc, epilogue=(lo, hi)).ravel(),
                          np.array(G["dx_clamp"]))
    assert np.array_equal(orc.bwd_filt(x, g, w.shape, y=yc, epilogue=(lo, hi)).ravel(),
                          np.array(G["dw_clamp"]))
    G2 = read_golden("hand_case_two_channel.txt")
    x2 = _arr(G2["x"], [int(v) for v in G2["x_shape"]])
    w2 = _arr(G2["w"], [int(v) for v in G2["w_shape"]])
    assert np.array_equal(orc.fwd(x2, w2).ravel(), np.array(G2["y"]))


def _rand(seed, H, W, D, N, fh, fw):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (H, W, D))
    w = rng.standard_normal((N, fh, fw, D))
    g = rng.standard_normal((H - fh + 1, W - fw + 1, N))
    return x, w, g


# (H, W, D, N, fh, fw); the last has the even square 8x8 filters and depth 4 of
# the fourth row of the paper's filter-bank table (2048x2048x4 input, 4x8x8x4 bank)
SHAPES = [(7, 9, 3, 4, 3, 2), (6, 5, 2, 3, 1, 4), (10, 8, 5, 2, 4, 3), (5, 5, 1, 1, 5, 5),
          (12, 11, 4, 4, 8, 8)]


def pin_scipy_forward(orc):
    """Per output channel: sum over d of scipy's 2D 'valid' correlation."""
    for k, (H, W, D, N, fh, fw) in enumerate(SHAPES):
        x, w, _ = _rand(10 + k, H, W, D, N, fh, fw)
        y = orc.fwd(x, w)
        for n in range(N):
            ref = sum(signal.correlate2d(x[:, :, d], w[n, :, :, d], mode="valid") for d in range(D))
            np.testing.assert_allclose(y[:, :, n], ref, rtol=1e-12, atol=1e-12)


def pin_scipy_backward(orc):
    """dx = sum_n full 2D convolution of g with w; dw = 'valid' correlation of x with g."""
    for k, (H, W, D, N, fh, fw) in enumerate(SHAPES):
        x, w, g = _rand(20 + k, H, W, D, N, fh, fw)
        dx = orc.bwd_input(g, w, x.shape)
        dw = orc.bwd_filt(x, g, w.shape)
        for d in range(D):
            ref = sum(signal.convolve2d(g[:, :, n], w[n, :, :, d], mode="full") for n in range(N))
            np.testing.assert_allclose(dx[:, :, d], ref, rtol=1e-12, atol=1e-12)
        for n in range(N):
            for d in range(D):
                ref = signal.correlate2d(x[:, :, d], g[:, :, n], mode="valid")
                np.testing.assert_allclose(dw[n, :, :, d], ref, rtol=1e-12, atol=1e-11)


def pin_torch_conv2d(orc):
    """torch.nn.functional.conv2d is a cross-correlation without padding."""
    import torch
    for k, (H, W, D, N, fh, fw) in enumerate(SHAPES):
        x, w, _ = _rand(30 + k, H, W, D, N, fh, fw)
        ref = torch.nn.functional.conv2d(torch.from_numpy(x).permute(2, 0, 1)[None],
                                         torch.from_numpy(w).permute(0, 3, 1, 2))
        ref = ref[0].permute(1, 2, 0).numpy()
        np.testing.assert_allclose(orc.fwd(x, w), ref, rtol=1e-12, atol=1e-12)


def pin_delta_filters(orc):
    """w[n] = unit impulse at (i0, j0, d0) copies a shifted window of channel d0."""
    rng = np.random.default_rng(5)
    H, W, D, fh, fw = 9, 11, 3, 4, 3
    x = rng.uniform(-1, 1, (H, W, D))
    taps = [(i, j, d) for i in range(fh) for j in range(fw) for d in range(D)]
    w = np.zeros((len(taps), fh, fw, D))
    for n, (i, j, d) in enumerate(taps):
        w[n, i, j, d] = 1.0
    y = orc.fwd(x, w)
    Ho, Wo = H - fh + 1, W - fw + 1
    for n, (i, j, d) in enumerate(taps):
        assert np.array_equal(y[:, :, n], x[i:i + Ho, j:j + Wo, d]), (i, j, d)


def pin_constant_and_affine(orc):
    """Constant input c gives c * sum(w); affine input a*p + b*q + c*d + e gives
    (a*p + b*q + e) * S_n + sum_{i,j,d} w[n,i,j,d] (a*i + b*j + c*d), S_n = sum of filter n."""
    rng = np.random.default_rng(6)
    H, W, D, N, fh, fw = 8, 10, 3, 4, 3, 2
    w = rng.standard_normal((N, fh, fw, D))
    y = orc.fwd(np.full((H, W, D), 2.5), w)
    S = w.sum(axis=(1, 2, 3))
    np.testing.assert_allclose(y, np.broadcast_to(2.5 * S, y.shape), rtol=1e-12, atol=1e-12)
    a, b, c, e = 3.0, -7.0, 0.25, 1.5
    P, Q, Dd = np.meshgrid(np.arange(H), np.arange(W), np.arange(D), indexing="ij")
    x = a * P + b * Q + c * Dd + e
    y = orc.fwd(x, w)
    I, J, DD = np.meshgrid(np.arange(fh), np.arange(fw), np.arange(D), indexing="ij")
    T = (w * (a * I + b * J + c * DD)[None]).sum(axis=(1, 2, 3))
    Ho, Wo = H - fh + 1, W - fw + 1
    p = np.arange(Ho)[:, None, None]
    q = np.arange(Wo)[None, :, None]
    ref = (a * p + b * q + e) * S[None, None, :] + T[None, None, :]
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-10)


def pin_linearity(orc):
    x1, w1, _ = _rand(40, 9, 8, 3, 2, 3, 2)
    x2, w2, _ = _rand(41, 9, 8, 3, 2, 3, 2)
    a, b = 0.75, -1.25
    np.testing.assert_allclose(orc.fwd(a * x1 + b * x2, w1),
                               a * orc.fwd(x1, w1) + b * orc.fwd(x2, w1), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(orc.fwd(x1, a * w1 + b * w2),
                               a * orc.fwd(x1, w1) + b * orc.fwd(x1, w2), rtol=1e-12, atol=1e-12)


def pin_adjoint(orc):
    """<corr(x, w), g> = <x, dL/dx> = <w, dL/dw> for L = <corr(x, w), g>."""
    for k, (H, W, D, N, fh, fw) in enumerate(SHAPES):
        x, w, g = _rand(50 + k, H, W, D, N, fh, fw)
        lhs = float((orc.fwd(x, w) * g).sum())
        r1 = float((x * orc.bwd_input(g, w, x.shape)).sum())
        r2 = float((w * orc.bwd_filt(x, g, w.shape)).sum())
        assert abs(lhs - r1) <= 1e-12 * max(1.0, abs(lhs)), (lhs, r1)
        assert abs(lhs - r2) <= 1e-12 * max(1.0, abs(lhs)), (lhs, r2)


def pin_finite_differences(orc, x=None, w=None, g=None, h=1e-3):
    """L(x, w) = <corr(x, w), g> is bilinear, so central differences are exact up
    to rounding for any step h; compare every input and filter coordinate."""
    if x is None:
        x, w, g = _rand(55, 6, 7, 2, 2, 3, 2)
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    g = np.asarray(g, np.float64)

    def L(xx, ww):
        return float((orc.fwd(xx, ww) * g).sum())

    dx = orc.bwd_input(g, w, x.shape)
    dw = orc.bwd_filt(x, g, w.shape)
    fdx = np.empty_like(x)
    for idx in np.ndindex(*x.shape):
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        fdx[idx] = (L(xp, w) - L(xm, w)) / (2 * h)
    fdw = np.empty_like(w)
    for idx in np.ndindex(*w.shape):
        wp = w.copy(); wp[idx] += h
        wm = w.copy(); wm[idx] -= h
        fdw[idx] = (L(x, wp) - L(x, wm)) / (2 * h)
    assert np.abs(fdx - dx).max() <= 1e-9 * max(1.0, np.abs(dx).max())
    assert np.abs(fdw - dw).max() <= 1e-9 * max(1.0, np.abs(dw).max())


def pin_clamp(orc):
    """The clamp is the elementwise min/max of the plain output; its gradient
    passes g only where lo < y < hi strictly (a kink-free FD check away from
    the bounds)."""
    x, w, g = _rand(60, 8, 9, 2, 3, 3, 3)
    lo, hi = -0.5, 0.75
    y = orc.fwd(x, w)
    yc = orc.fwd(x, w, epilogue=(lo, hi))
    assert np.array_equal(yc, np.minimum(np.maximum(y, lo), hi))
    inside = (y > lo) & (y < hi)
    assert inside.any() and (~inside).any()
    dx = orc.bwd_input(g, w, x.shape, y=yc, epilogue=(lo, hi))
    dw = orc.bwd_filt(x, g, w.shape, y=yc, epilogue=(lo, hi))
    # directional finite difference: with a step small enough that no output
    # crosses a bound, L(x) = <clamp(corr(x, w)), g> is linear along it
    rng = np.random.default_rng(61)
    margin = np.minimum(np.abs(y - lo), np.abs(y - hi)).min()
    assert margin > 1e-6
    vx = rng.standard_normal(x.shape)
    vw = rng.standard_normal(w.shape)
    h = 1e-3 * margin / max(np.abs(vx).sum(), np.abs(vw).sum())

    def L(xx, ww):
        return float((orc.fwd(xx, ww, epilogue=(lo, hi)) * g).sum())

    fd_x = (L(x + h * vx, w) - L(x - h * vx, w)) / (2 * h)
    fd_w = (L(x, w + h * vw) - L(x, w - h * vw)) / (2 * h)
    assert abs(fd_x - float((dx * vx).sum())) <= 1e-6 * max(1.0, abs(fd_x))
    assert abs(fd_w - float((dw * vw).sum())) <= 1e-6 * max(1.0, abs(fd_w))


def pin_points(orc):
    """The pointwise entry points agree with the full ones."""
    x, w, g = _rand(70, 9, 10, 3, 4, 3, 4)
    y = orc.fwd(x, w, epilogue=(-1.0, 1.0))
    rng = np.random.default_rng(71)
    idx = np.stack([rng.integers(0, s, 50) for s in y.shape], axis=1)
    assert np.array_equal(orc.fwd_points(x, w, idx, epilogue=(-1.0, 1.0)), y[tuple(idx.T)])
    dx = orc.bwd_input(g, w, x.shape)
    idx = np.stack([rng.integers(0, s, 50) for s in x.shape], axis=1)
    assert np.array_equal(orc.bwd_input_points(g, w, x.shape, idx), dx[tuple(idx.T)])
    # with the clamp the gradient passes only where -1 < y < 1 (both occur here)
    inside = (y > -1.0) & (y < 1.0)
    assert inside.any() and (~inside).any()
    dxc = orc.bwd_input(g, w, x.shape, y=y, epilogue=(-1.0, 1.0))
    assert not np.array_equal(dxc, dx)
    assert np.array_equal(orc.bwd_input_points(g, w, x.shape, idx, y=y, epilogue=(-1.0, 1.0)),
                          dxc[tuple(idx.T)])


# --- exact nearest-neighbour search (Sec. 6.4) ---------------------------------

def pin_nn_golden_hand(orc):
    G = read_golden("nn_hand_case.txt")
    dim = int(G["dim"][0])
    t = _arr(G["targets"], (-1, dim))
    n = _arr(G["neighbors"], (-1, dim))
    idx, d, d2 = orc.nn(t, n)
    assert idx.tolist() == [int(v) for v in G["idx"]]
    assert d.tolist() == G["dist"] and d2.tolist() == G["dist2"]


def pin_nn_scipy(orc):
    """scipy's pairwise squared distances + argmin (first minimum) on random data."""
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(60)
    t = rng.standard_normal((40, 16))
    n = rng.standard_normal((700, 16))
    idx, d, d2 = orc.nn(t, n)
    D = cdist(t, n, "sqeuclidean")
    assert np.array_equal(idx, D.argmin(axis=1))
    assert np.allclose(d, D.min(axis=1), rtol=1e-12, atol=0)
    D[np.arange(len(t)), idx] = np.inf
    assert np.allclose(d2, D.min(axis=1), rtol=1e-12, atol=0)


def pin_nn_invariants(orc):
    """Exact cases on integer data: a target that is also a neighbour is at
    distance 0; duplicates resolve to the lower index with a zero gap; a
    permutation of the neighbours permutes the answer; a common translation
    changes nothing."""
    rng = np.random.default_rng(61)
    n = rng.integers(-20, 21, size=(300, 8)).astype(np.float64)
    t = rng.integers(-20, 21, size=(25, 8)).astype(np.float64)
    t[3] = n[123]
    n[250] = n[40]
    t[7] = n[40] + np.array([1, 0, 0, 0, 0, 0, 0, 0])
    idx, d, d2 = orc.nn(t, n)
    assert idx[3] == 123 and d[3] == 0.0
    assert idx[7] == 40 and d[7] == 1.0 and d2[7] == 1.0
    perm = rng.permutation(len(n))
    idx_p, d_p, _ = orc.nn(t, n[perm])
    assert np.array_equal(d_p, d)
    gap = d2 > d                      # unique nearest neighbour: the index is well defined
    assert np.array_equal(perm[idx_p][gap], idx[gap])
    c = rng.integers(-50, 51, size=8).astype(np.float64)
    idx_c, d_c, d2_c = orc.nn(t + c, n + c)
    assert np.array_equal(idx_c, idx) and np.array_equal(d_c, d) and np.array_equal(d2_c, d2)


ALL_PINS = [pin_nn_golden_hand, pin_nn_scipy, pin_nn_invariants,
            pin_golden_hand, pin_scipy_forward, pin_scipy_backward, pin_torch_conv2d,
            pin_delta_filters, pin_constant_and_affine, pin_linearity, pin_adjoint,
            pin_finite_differences, pin_clamp, pin_points]
