"""CPU tests of the FP64 oracle against its pins (see oracle_pins.py)."""
import os
import shutil
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
import oracle_pins
from paper_0911_3456_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin(oracle)


def test_finite_differences_fd_case():
    """The 12x12x2 input / 3 filters 3x3x2 case: every coordinate of dL/dx and
    dL/dw against central differences in FP64 (h = 1e-3)."""
    wl = inputs.workload_finite_difference()
    oracle_pins.pin_finite_differences(oracle, wl.x, wl.w, wl.g)


def test_integer_exactness_against_scipy():
    """Integer inputs in [-4, 4]: every partial sum is an exact integer, so the
    oracle must equal scipy's integer correlation exactly."""
    from scipy import signal
    wl = inputs.random_case(7, 20, 23, 5, 3, 4, 6, kind="int")
    y = oracle.fwd(wl.x, wl.w)
    xi = wl.x.astype(np.int64)
    wi = wl.w.astype(np.int64)
    for n in range(wl.w.shape[0]):
        ref = sum(signal.correlate2d(xi[:, :, d], wi[n, :, :, d], mode="valid")
                  for d in range(wl.x.shape[2]))
        assert np.array_equal(y[:, :, n], ref.astype(np.float64))


def test_thread_count_does_not_change_results():
    wl = inputs.random_case(8, 17, 19, 3, 5, 3, 3, with_g=True)
    oracle.set_threads(1)
    try:
        a = (oracle.fwd(wl.x, wl.w), oracle.bwd_input(wl.g, wl.w, wl.x.shape),
             oracle.bwd_filt(wl.x, wl.g, wl.w.shape))
    finally:
        oracle.set_threads(0)
    b = (oracle.fwd(wl.x, wl.w), oracle.bwd_input(wl.g, wl.w, wl.x.shape),
         oracle.bwd_filt(wl.x, wl.g, wl.w.shape))
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_bad_shapes_rejected():
    x = np.zeros((4, 4, 2))
    with pytest.raises(ValueError):
        oracle.fwd(x, np.zeros((1, 5, 2, 2)))       # fh > H
    with pytest.raises(ValueError):
        oracle.fwd(x, np.zeros((1, 2, 2, 3)))       # depth mismatch
    with pytest.raises(ValueError):
        oracle.fwd_points(x, np.zeros((1, 2, 2, 2)), [[3, 0, 0]])  # p >= H'


def test_paper_table_boost_column():
    """The paper's Boost column equals tuned/default - 1 on every row (the
    reading used for the default-vs-tuned report)."""
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "paper_fbconv3_table.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 19
    for r in rows:
        default, tuned, boost = float(r[4]), float(r[6]), float(r[8])
        assert abs(100.0 * (tuned / default - 1.0) - boost) < 0.06, r


# --- mutation tests: each plausible mistake in the oracle fails some pin -------

MUTANTS = {
    "filter_flip": ("w[((n * fh + i) * fw + j) * D + d];\n    return s;",
                    "w[((n * fh + (fh - 1 - i)) * fw + (fw - 1 - j)) * D + d];\n    return s;"),
    "dropped_channel": ("for (int64_t d = 0; d < D; ++d)\n                s += x[",
                        "for (int64_t d = 1; d < D; ++d)\n                s += x["),
    "dropped_last_column_tap": ("for (int64_t j = 0; j < fw; ++j)\n            for (int64_t d = 0; d < D; ++d)\n                s += x[",
                                "for (int64_t j = 0; j < fw - 1; ++j)\n            for (int64_t d = 0; d < D; ++d)\n                s += x["),
    "float_accumulator": ("    double s = 0.0;\n    for (int64_t i = 0; i < fh; ++i)",
                          "    float s = 0.0f;\n    for (int64_t i = 0; i < fh; ++i)"),
    "clamp_wrong_bound": ("if (v < lo) v = lo;", "if (v < lo) v = hi;"),
    "clamp_mask_not_strict": ("if (!(v > lo && v < hi)) return 0.0;",
                              "if (!(v >= lo && v <= hi)) return 0.0;"),
    "dx_flipped_filter": ("s += g_eff(g, y, (po * Wo + qo) * N + n, epi_kind, lo, hi) *\n                                 w[((n * fh + i) * fw + j) * D + d];",
                          "s += g_eff(g, y, (po * Wo + qo) * N + n, epi_kind, lo, hi) *\n                                 w[((n * fh + (fh - 1 - i)) * fw + (fw - 1 - j)) * D + d];"),
    "dx_wrong_shift_sign": ("const int64_t po = p - i;\n                        if (po < 0 || po >= Ho) continue;\n                        for (int64_t j = 0; j < fw; ++j) {\n                            const int64_t qo = q - j;",
                            "const int64_t po = p - i;\n                        if (po < 0 || po >= Ho) continue;\n                        for (int64_t j = 0; j < fw; ++j) {\n                            const int64_t qo = q + j - (fw - 1);"),
    "dw_dropped_last_row": ("for (int64_t p = 0; p < Ho; ++p)\n            for (int64_t q = 0; q < Wo; ++q)\n                s += g_eff",
                            "for (int64_t p = 0; p < Ho - 1; ++p)\n            for (int64_t q = 0; q < Wo; ++q)\n                s += g_eff"),
    "dw_swapped_ij_decode": ("const int64_t j = (e / D) % fw;\n        const int64_t i = (e / (D * fw)) % fh;",
                             "const int64_t i = (e / D) % fh;\n        const int64_t j = (e / (D * fh)) % fw;"),
    "dx_last_output_row_dropped": ("                        if (po < 0 || po >= Ho) continue;",
                                   "                        if (po < 0 || po >= Ho - 1) continue;"),
    "dw_clamp_mask_ignored": ("                s += g_eff(g, y, (p * Wo + q) * N + n, epi_kind, lo, hi) *",
                              "                s += g[(p * Wo + q) * N + n] *"),
    "dx_points_clamp_mask_ignored": ("qo >= Wo) continue;\n                    s += g_eff(g, y, (po * Wo + qo) * N + n, epi_kind, lo, hi) *",
                                     "qo >= Wo) continue;\n                    s += g[(po * Wo + qo) * N + n] *"),
    "fwd_points_clamp_dropped": ("        if (epi_kind == ORACLE_EPI_CLAMP) s = clamp_d(s, lo, hi);\n        out[k] = s;",
                                 "        out[k] = s;"),
}

# planted mistakes in the nearest-neighbour oracle (nn_oracle.c)
NN_MUTANTS = {
    "nn_ties_to_highest_index": ("            if (d < best) {", "            if (d <= best) {"),
    "nn_absolute_not_squared": ("                d += e * e;", "                d += fabs(e);"),
    "nn_dropped_last_dimension": ("for (int64_t k = 0; k < dim; ++k) {", "for (int64_t k = 0; k < dim - 1; ++k) {"),
    "nn_runner_up_misses_later": ("            } else if (d < second) {\n                second = d;\n            }",
                                  "            }"),
    "nn_old_best_not_demoted": ("                second = best;\n                best = d;", "                best = d;"),
    "nn_skips_last_neighbour": ("for (int64_t j = 0; j < nn; ++j) {", "for (int64_t j = 0; j < nn - 1; ++j) {"),
    "nn_neighbour_row_stride": ("const double* nj = n + j * dim;", "const double* nj = n + j;"),
}

_RUNNER = textwrap.dedent("""
    import importlib.util, sys, json
    sys.path.insert(0, {tests!r})
    spec = importlib.util.spec_from_file_location("oracle_mutant", {init!r})
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(force=True)
    import oracle_pins
    failed = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(mod)
        except Exception as e:
            failed.append(pin.__name__)
    print(json.dumps(failed))
""")


@pytest.mark.parametrize("name", sorted(MUTANTS) + sorted(NN_MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    """A copy of the oracle with one planted mistake must fail at least one pin."""
    src_dir = os.path.join(ROOT, "oracle")
    dst = tmp_path / "oracle_mutant"
    dst.mkdir()
    for f in ("__init__.py", "fbcorr_oracle.c", "nn_oracle.c"):
        shutil.copy(os.path.join(src_dir, f), dst / f)
    target = "fbcorr_oracle.c" if name in MUTANTS else "nn_oracle.c"
    with open(os.path.join(src_dir, target)) as f:
        src = f.read()
    old, new = MUTANTS[name] if name in MUTANTS else NN_MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/found"
    (dst / target).write_text(src.replace(old, new))
    script = _RUNNER.format(tests=os.path.join(ROOT, "tests"), init=str(dst / "__init__.py"))
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=600,
                       cwd=str(tmp_path))
    # a crash of the mutant counts as detected as well
    if r.returncode == 0:
        import json
        failed = json.loads(r.stdout.strip().splitlines()[-1])
        assert failed, f"mutant {name} passed every pin"
