"""Host-side pieces of bench.py that need no GPU: the CPU-baseline leg, which
times the FP64 oracle on a sample of consecutive output rows sized for a time
target (at most the whole output)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_0911_3456_gb300 import inputs  # noqa: E402


def test_cpu_baseline_covers_the_whole_output_when_it_fits():
    """The small FP32 workload (128x128x8, 16 filters 9x9x8) takes far less
    than the target, so the sample is every output row and matches the oracle
    on the full input."""
    oracle.build()
    wl = inputs.workload_small_f32()
    res, (r0, y) = bench.cpu_baseline(wl, target_s=30.0)
    Ho = wl.out_shape[0]
    assert r0 == 0 and y.shape == tuple(wl.out_shape)
    assert res["sample"].startswith(f"{Ho} consecutive output rows")
    assert res["kind"] == "oracle" and res["cores"] == oracle.max_threads()
    assert res["value"] > 0 and res["seconds"] > 0
    assert np.array_equal(y, oracle.fwd(wl.x, wl.w))


def test_cpu_baseline_partial_sample_is_a_centred_slab():
    """A short target gives a centred slab of consecutive rows (the calibration
    runs on two rows per oracle thread), and the slab is the oracle on the
    matching input rows."""
    oracle.build()
    wl = inputs.workload_paper_row1_clamp()        # 248 output rows of 248 x 64
    Ho = wl.out_shape[0]
    k = max(1, min(Ho, 2 * oracle.max_threads()))
    _, _, dtk, _ = bench.oracle_rows_sample(wl, k)
    target = 3.0 * dtk
    _, (r0, y) = bench.cpu_baseline(wl, target_s=target)
    rows = y.shape[0]
    assert 1 <= rows <= Ho
    assert r0 == (Ho - rows) // 2
    # the slab is the oracle on the matching input rows
    fh = wl.w.shape[1]
    ref = oracle.fwd(wl.x[r0:r0 + rows + fh - 1], wl.w)
    assert np.array_equal(y, ref)


def test_cpu_baseline_reports_an_extrapolated_single_core_figure():
    oracle.build()
    wl = inputs.workload_small_f32()
    before = oracle.max_threads()
    res, _ = bench.cpu_baseline(wl, target_s=0.4)
    one = res["single_core"]
    assert one["cores"] == 1 and 1 <= one["rows"] <= wl.out_shape[0]
    assert one["value"] > 0 and "extrapolated" in one["note"]
    assert abs(one["whole_output_seconds_extrapolated"] - one["seconds"] / one["rows"] * wl.out_shape[0]) < 1e-9
    assert oracle.max_threads() == before          # the oracle's thread count is restored
