"""Exact nearest-neighbour search (fbcorr_nn_*) against the FP64 oracle, through
the C ABI.  The nearest neighbour is unique only up to the arithmetic: where
the oracle's best and runner-up distances are further apart than the search's
error, the index must match exactly; elsewhere the returned neighbour must be
within that error of the best.  Distances are compared with the FP32 bound of
the exact re-ranking."""
import numpy as np
import pytest

import oracle
from helpers import torch_cuda
from paper_0911_3456_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(torch, t, n, dtype="bf16x3", fallbacks=False):
    from paper_0911_3456_gb300.api import NNPlan
    p = NNPlan(t.shape[0], n.shape[0], t.shape[1], dtype)
    idx, dist = p.search(torch.from_numpy(t).cuda(), torch.from_numpy(n).cuda())
    torch.cuda.synchronize()
    assert p.device_status() == 0
    out = idx.cpu().numpy(), dist.cpu().numpy().astype(np.float64)
    return out + (p.last_fallbacks(),) if fallbacks else out


def _fp32_separated(ref_d, ref_d2, dim):
    """Targets whose nearest neighbour is unique by more than the FP32 rounding
    of the exact distances ((dim + 3) * 2^-24 relative, twice, with margin)."""
    return (ref_d2 - ref_d) > 4 * (dim + 3) * 2.0 ** -24 * ref_d2 + 1e-30


def _check(t, n, idx, dist, tol_rel_pair, min_sep=0.5):
    """tol_rel_pair: the screening error bound as a fraction of sum_k |t_k||n_k|."""
    ref_idx, ref_d, ref_d2 = oracle.nn(t, n)
    t64, n64 = t.astype(np.float64), n.astype(np.float64)
    chosen = ((t64 - n64[idx]) ** 2).sum(axis=1)                 # FP64 distance of our answer
    scale = np.abs(t64).sum(axis=1) * np.abs(n64).max() * 4.0    # >= 2 sum_k |t_k||n_k| for any n
    eps = tol_rel_pair * scale + 1e-6 * ref_d
    # the returned neighbour is (within the error) a nearest one ...
    assert np.all(chosen <= ref_d + 2 * eps)
    # ... and exactly the oracle's wherever the oracle's nearest is unique by a margin
    sep = (ref_d2 - ref_d) > 4 * eps
    assert np.array_equal(idx[sep], ref_idx[sep])
    assert sep.mean() >= min_sep
    # the distance is the exact FP32 one for the returned neighbour
    assert np.allclose(dist, chosen, rtol=64 * 2.0 ** -23, atol=1e-7)
    # the search returns the argmin of the exact FP32 distance over all
    # neighbours, so wherever the oracle's nearest is unique beyond FP32
    # rounding the index is the oracle's
    fs = _fp32_separated(ref_d, ref_d2, t.shape[1])
    assert np.array_equal(idx[fs], ref_idx[fs])


@pytest.mark.parametrize("nt,nn,dim", [(300, 5000, 64), (129, 257, 3), (128, 256, 16), (1, 3000, 33)])
def test_random_sets_match_oracle(nt, nn, dim):
    torch = torch_cuda()
    rng = np.random.default_rng(3000 + nt + nn + dim)
    t = rng.standard_normal((nt, dim)).astype(np.float32)
    n = rng.standard_normal((nn, dim)).astype(np.float32)
    idx, dist = _run(torch, t, n)
    _check(t, n, idx, dist, 4 * 2.0 ** -16)


def test_integer_sets_exact_with_ties():
    """Integer coordinates: every distance is exact in FP32; duplicated
    neighbours and targets equal to neighbours resolve to the lowest index."""
    torch = torch_cuda()
    rng = np.random.default_rng(3100)
    n = rng.integers(-8, 9, size=(3000, 24)).astype(np.float32)
    t = rng.integers(-8, 9, size=(400, 24)).astype(np.float32)
    n[2500] = n[17]
    t[5] = n[17]
    t[6] = n[2999]
    idx, dist = _run(torch, t, n)
    ref_idx, ref_d, ref_d2 = oracle.nn(t, n)
    assert idx[5] == 17 and dist[5] == 0.0 and idx[6] == 2999
    sep = ref_d2 > ref_d
    assert np.array_equal(idx[sep], ref_idx[sep])
    assert np.array_equal(dist, ref_d)


def test_natural_patches_against_oracle():
    """The paper's setting at a size the oracle finishes quickly: 4096 8x8
    patches against 65536 (synthetic 1/f images stand in for natural images)."""
    torch = torch_cuda()
    t, n = inputs.nn_patches(n_neighbors=65536)
    idx, dist = _run(torch, t, n)
    _check(t, n, idx, dist, 4 * 2.0 ** -16, min_sep=0.0)
    # every target whose nearest neighbour is unique beyond FP32 rounding gets
    # exactly the oracle's
    ref_idx, ref_d, ref_d2 = oracle.nn(t, n)
    fs = _fp32_separated(ref_d, ref_d2, t.shape[1])
    assert fs.mean() >= 0.95
    assert np.array_equal(idx[fs], ref_idx[fs])


def test_plain_bf16_screening_is_reranked_exactly():
    """Plain BF16 screens coarsely; on well-separated clusters the exact
    re-ranking still returns the oracle's answers and exact distances."""
    torch = torch_cuda()
    rng = np.random.default_rng(3200)
    centers = rng.standard_normal((2000, 32)).astype(np.float32) * 10
    n = centers + 0.01 * rng.standard_normal(centers.shape).astype(np.float32)
    t = centers[rng.integers(0, 2000, size=300)] + 0.01 * rng.standard_normal((300, 32)).astype(np.float32)
    idx, dist = _run(torch, t, n, "bf16")
    ref_idx, ref_d, _ = oracle.nn(t, n)
    assert np.array_equal(idx, ref_idx)
    assert np.allclose(dist, ref_d, rtol=1e-5, atol=1e-7)


def _planted(spread, seed=3400, nn=5120):
    """Target 0 is the all-ones vector of 64 coordinates.  Twelve neighbours lie
    around it: the true nearest n* = 1 + a (every coordinate) and eleven at
    1 - b_k with b_k slightly larger than a.  Plain BF16 rounds every one of them
    to the all-ones vector, so the screened key of n* is the largest of the
    twelve by 128 (a + b) while its exact distance, 64 a^2, is the smallest: the
    true nearest is not among the first four screened, and all twelve lie within
    the screening error of the best.  The other neighbours are far away, so the
    window of the one target holds exactly the twelve.
    spread=True puts the twelve in twelve different neighbour tiles (one per
    screening part: the window holds them all and is certified without the
    fallback); spread=False puts them in the first 32 columns of one tile (one
    part keeps only two of them, so the target is searched exhaustively).
    nn=16384 (64 neighbour tiles) makes the plan screen the first four tiles
    first for the key thresholds: spread, that sample holds four of the twelve."""
    rng = np.random.default_rng(seed)
    dim = 64
    n = (1.0 + 3.0 * rng.standard_normal((nn, dim))).astype(np.float32)
    t = np.ones((1, dim), np.float32)
    a = 1e-3
    slots = [256 * k + 7 for k in range(12)] if spread else [256 * 9 + k for k in range(12)]
    star = slots[5]
    for k, j in enumerate(slots):
        n[j] = (1.0 + a) if j == star else (1.0 - a * (1.02 + 0.01 * k))
    return t, n, star


@pytest.mark.parametrize("nn", [5120, 16384], ids=["no_threshold", "sampled_threshold"])
@pytest.mark.parametrize("spread", [True, False], ids=["window_certified", "exhaustive_fallback"])
@pytest.mark.parametrize("dtype", ["bf16", "bf16x3"])
def test_nearest_beyond_the_first_four_screened(spread, dtype, nn):
    """Twelve neighbours within the screening error of the true nearest, which
    screens last of them (plain BF16): the index must be the oracle's.  Either
    every candidate of the certified window is re-ranked exactly, or the target
    whose window a part may have truncated is searched exhaustively -- also when
    the key threshold comes from a sample that holds some of the twelve."""
    torch = torch_cuda()
    t, n, star = _planted(spread, nn=nn)
    ref_idx, ref_d, ref_d2 = oracle.nn(t, n)
    assert ref_idx[0] == star
    if dtype == "bf16":
        # the construction: in plain BF16 every planted neighbour rounds to the
        # target itself, so n* has the largest screened key of the twelve
        n_bf = n.view(np.uint32)
        assert np.all(((n_bf[star] + 0x8000) & 0xFFFF0000) == np.float32(1.0).view(np.uint32))
    idx, dist, fb = _run(torch, t, n, dtype, fallbacks=True)
    assert idx[0] == star
    assert dist[0] == np.float32(dist[0]) and abs(dist[0] - ref_d[0]) <= 1e-3 * ref_d[0]
    if dtype == "bf16":
        assert fb == (0 if spread else 1)


def test_exhaustive_fallback_many_targets():
    """Many targets with truncated windows at once (duplicated neighbours: every
    target has a whole tile of near-ties in plain BF16): the fallback handles
    them all, and every answer is the argmin of the exact distance."""
    torch = torch_cuda()
    rng = np.random.default_rng(3500)
    dim = 32
    base = (rng.standard_normal((300, dim)) * 4).astype(np.float32)
    n = np.repeat(base, 8, axis=0) + (1e-4 * rng.standard_normal((2400, dim))).astype(np.float32)
    t = base[rng.integers(0, 300, size=500)] + (1e-4 * rng.standard_normal((500, dim))).astype(np.float32)
    idx, dist, fb = _run(torch, t, n, "bf16", fallbacks=True)
    assert fb > 0
    ref_idx, ref_d, ref_d2 = oracle.nn(t, n)
    fs = _fp32_separated(ref_d, ref_d2, dim)
    assert fs.mean() >= 0.9
    assert np.array_equal(idx[fs], ref_idx[fs])
    chosen = ((t.astype(np.float64) - n.astype(np.float64)[idx]) ** 2).sum(axis=1)
    assert np.allclose(dist, chosen, rtol=64 * 2.0 ** -23, atol=1e-9)


@pytest.mark.parametrize("nt,nn,dim", [(1, 1, 1), (5, 2, 64), (200, 700, 8), (130, 1000, 48)])
def test_edge_sizes(nt, nn, dim):
    """One neighbour, two neighbours, dimensions that are not a multiple of 16,
    partial target and neighbour tiles."""
    torch = torch_cuda()
    rng = np.random.default_rng(3300 + nt + nn + dim)
    t = rng.standard_normal((nt, dim)).astype(np.float32)
    n = rng.standard_normal((nn, dim)).astype(np.float32)
    idx, dist = _run(torch, t, n)
    ref_idx, ref_d, ref_d2 = oracle.nn(t, n)
    sep = ref_d2 > ref_d * (1 + 1e-3) + 1e-6
    assert np.array_equal(idx[sep], ref_idx[sep])
    assert np.all((idx >= 0) & (idx < nn))
    chosen = ((t.astype(np.float64) - n.astype(np.float64)[idx]) ** 2).sum(axis=1)
    assert np.allclose(dist, chosen, rtol=64 * 2.0 ** -23, atol=1e-6)


def test_plan_refusals():
    torch_cuda()
    from paper_0911_3456_gb300 import _capi as C
    from paper_0911_3456_gb300.api import NNPlan
    with pytest.raises(C.FbcorrError):
        NNPlan(10, 10, 65)              # more than 64 dimensions
    with pytest.raises(ValueError):
        NNPlan(10, 10, 8, "f32")        # screening runs on the tensor cores


@pytest.mark.parametrize("dtype", ["bf16", "bf16x3"])
def test_sampled_key_threshold_changes_no_answer(dtype):
    """The key threshold from the sample screening (FBCORR_NN_PRESCREEN, on by
    default from 32 neighbour tiles) only drops keys that cannot enter a window:
    indices and distances are bit-identical with and without it."""
    import os
    torch = torch_cuda()
    t, n = inputs.nn_patches(n_neighbors=65536)
    t = t[:1024]
    with_thr = _run(torch, t, n, dtype, fallbacks=True)
    old = os.environ.get("FBCORR_NN_PRESCREEN")
    os.environ["FBCORR_NN_PRESCREEN"] = "0"
    try:
        without = _run(torch, t, n, dtype, fallbacks=True)
    finally:
        if old is None:
            os.environ.pop("FBCORR_NN_PRESCREEN")
        else:
            os.environ["FBCORR_NN_PRESCREEN"] = old
    assert np.array_equal(with_thr[0], without[0])
    assert np.array_equal(with_thr[1], without[1])
