"""GPU: the predictor's launch shapes and the autotuner that chooses among them.

Every shape computes the same outputs.  The block-per-cell kernel at either
block width (FP64, and mixed precision with an FP64 sweep) and the mixed
warp-per-cell shapes with 2 or 4 cells per block are bit for bit equal, so
the default autotuning among them never changes a result.  The block-per-cell mixed kernel and the
tensor-pipe contractions (TF32 split into high and low parts, three products
per tile) round differently in FP32 and agree with the default within FP32
rounding of the space-time correction."""
import numpy as np
import pytest

from paper_1406_7416_gb300 import adg, build_lib, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


def _run(w, prec, shape, steps, dt=None):
    s = adg.Solver.from_workload(w, prec)
    s.set_option(adg.OPT_PREDICTOR, shape)
    s.init_problem(w["problem"])
    if dt is None:
        for _ in range(steps):
            s.step_cfl(0.5 * w["cfl"])
    else:
        for _ in range(steps):
            s.step(dt)
    out = s.read_full()
    troubled = s.troubled_count()
    assert s.status() == adg.OK
    assert s.info()["predictor"] == shape
    s.close()
    return out, troubled


FP64_CASES = {
    "explosion2d_N3_12": lambda: inputs.explosion_2d(n=12, N=3),
    "quadvortex_N5_8": lambda: inputs.quadrants_vortex_2d(n=8, N=5, steps=None),
    "quadrants_N9_5": lambda: inputs.quadrants_2d(n=5, N=9),
    "explosion3d_N2_5": lambda: inputs.explosion_3d(n=5, N=2),
}


@pytest.mark.parametrize("name", sorted(FP64_CASES))
def test_fp64_shapes_are_bitwise_equal(name):
    """4 limited CFL steps with each FP64 shape: DOFs, flags and subcell data
    bit for bit equal."""
    w = FP64_CASES[name]()
    ref, troubled = _run(w, adg.PREC_FP64, adg.PRED_BLOCK, 4)
    got, _ = _run(w, adg.PREC_FP64, adg.PRED_BLOCK_ALT, 4)
    assert troubled > 0
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)


def test_block_widths_are_bitwise_equal_with_an_fp64_sweep():
    """Mixed precision at N = 7 (one FP64 Picard sweep, block-per-cell kernel):
    both block widths bit for bit equal over 4 limited steps."""
    w = inputs.quadrants_2d(n=6, N=7)
    ref, troubled = _run(w, adg.PREC_MIXED_FP32, adg.PRED_BLOCK, 4)
    got, _ = _run(w, adg.PREC_MIXED_FP32, adg.PRED_BLOCK_ALT, 4)
    assert troubled > 0
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)


MIXED_CASES = {
    "explosion2d_N2_10": lambda: inputs.explosion_2d(n=10, N=2),
    "quadvortex_N5_16": lambda: inputs.quadrants_vortex_2d(n=16, N=5, steps=None),
    "explosion3d_N1_5": lambda: inputs.explosion_3d(n=5, N=1),
    "explosion3d_N3_6": lambda: inputs.explosion_3d(n=6, N=3),
}


def _max_dt(w):
    s = adg.Solver.from_workload(w, adg.PREC_FP64)
    s.init_problem(w["problem"])
    dt = s.max_dt(0.5 * w["cfl"])
    s.close()
    return dt


@pytest.mark.parametrize("name", sorted(MIXED_CASES))
def test_mixed_shapes_agree(name):
    """4 fixed steps in mixed precision with each shape: the warp-per-cell
    shapes with 1, 2 and 4 cells per block are bit for bit equal; the
    block-per-cell kernel and the tensor-pipe contractions stay within 2e-7
    of them in relative L1 per variable (FP32 rounding of the space-time
    correction, measured against variables that start at zero, like the 3D
    explosion's momenta), with the same flags."""
    w = MIXED_CASES[name]()
    dt = _max_dt(w)
    ref, troubled = _run(w, adg.PREC_MIXED_FP32, adg.PRED_WARP4, 4, dt)
    assert troubled > 0
    for shape in (adg.PRED_WARP1, adg.PRED_WARP2):
        got, _ = _run(w, adg.PREC_MIXED_FP32, shape, 4, dt)
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)
    for shape in (adg.PRED_BLOCK, adg.PRED_WARP4_TC):
        got, _ = _run(w, adg.PREC_MIXED_FP32, shape, 4, dt)
        np.testing.assert_array_equal(got[1], ref[1])
        d = np.abs(got[0] - ref[0]).sum(axis=(0, 2)) / np.abs(ref[0]).sum(axis=(0, 2))
        assert np.all(d <= 2e-7), (shape, d)


def test_autotune_times_the_candidates_and_keeps_the_fastest():
    w = inputs.quadrants_vortex_2d(n=32, N=5, steps=None)
    s = adg.Solver.from_workload(w, adg.PREC_MIXED_FP32)
    s.init_problem(w["problem"])
    s.step_cfl(w["cfl"])                    # the first step tunes (default mode)
    assert s.info()["predictor"] in (adg.PRED_WARP1, adg.PRED_WARP2, adg.PRED_WARP4)
    ms = s.autotune(2)
    timed = {k for k, v in ms.items() if np.isfinite(v)}
    assert timed == {"warp1", "warp2", "warp4"}
    best = min(timed, key=lambda k: ms[k])
    assert adg.PRED_NAMES[s.info()["predictor"]] == best
    s.set_option(adg.OPT_PREDICTOR, -2)      # every shape, the contraction path included
    ms = s.autotune(2)
    timed = {k for k, v in ms.items() if np.isfinite(v)}
    assert timed == {"block", "block_alt", "warp1", "warp2", "warp4", "warp4_tc"}
    best = min(timed, key=lambda k: ms[k])
    assert adg.PRED_NAMES[s.info()["predictor"]] == best
    s.step_cfl(w["cfl"])
    assert s.status() == adg.OK
    s.close()
    f = adg.Solver.from_workload(w, adg.PREC_FP64)
    f.init_problem(w["problem"])
    f.step_cfl(w["cfl"])
    ms = f.autotune(2)
    assert {k for k, v in ms.items() if np.isfinite(v)} == {"block", "block_alt"}
    f.close()
