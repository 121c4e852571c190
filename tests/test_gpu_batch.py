"""GPU: batched stepping (adg_batch_*, adg_step_batch) against stepping each
state alone.  Per-state work is the same arithmetic in both cases, so in FP64
(and in mixed precision) every state's DOFs, flags and subcell data after the
steps are bitwise equal alone and in the mix."""
import time

import numpy as np
import pytest

from paper_1406_7416_gb300 import adg, build_lib, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


def _workloads():
    ws = [inputs.explosion_2d(n=16, N=3),
          inputs.quadrants_2d(n=12, N=5),
          inputs.quadrants_vortex_2d(n=10, N=3),
          inputs.explosion_2d(n=9, N=2),
          inputs.explosion_3d(n=5, N=1)]
    ws[1]["ncell"] = (12, 10)
    ws[1]["dx"] = (1.0 / 12, 1.0 / 10)
    ws[4]["problem"]["cell_rho_factor"] = None
    return ws


def _make(w, prec, t_end=0.0):
    s = adg.Solver.from_workload(w, prec)
    if t_end:
        s.set_option(adg.OPT_END_TIME, t_end)
    s.init_problem(w["problem"])
    return s


def _state(s):
    d, b, sub = s.read_full()
    return d, b, sub


def _assert_same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(np.isnan(x) if x.dtype.kind == "f" else x,
                                      np.isnan(y) if y.dtype.kind == "f" else y)
        if x.dtype.kind == "f":
            np.testing.assert_array_equal(np.nan_to_num(x), np.nan_to_num(y))


@pytest.mark.parametrize("prec", [adg.PREC_FP64, adg.PREC_MIXED_FP32])
def test_fixed_steps_alone_equal_in_batch(prec):
    ws = _workloads()
    alone = [_make(w, prec) for w in ws]
    mixed = [_make(w, prec) for w in ws]
    dts = np.array([0.5 * s.max_dt(w["cfl"]) for s, w in zip(alone, ws)])
    for _ in range(3):
        for s, dt in zip(alone, dts):
            s.step(dt)
    batch = adg.Batch(mixed)
    for _ in range(2):
        batch.step(dts)
    batch.close()
    adg.step_batch(mixed, dts)                    # one-shot batch of the same states
    for a, m in zip(alone, mixed):
        _assert_same(_state(a), _state(m))
        assert a.status() == adg.OK and m.status() == adg.OK
    for s in alone + mixed:
        s.close()


def test_cfl_steps_with_graph_replay_equal_alone():
    ws = _workloads()
    alone = [_make(w, adg.PREC_FP64) for w in ws]
    mixed = [_make(w, adg.PREC_FP64) for w in ws]
    cfl = 0.05
    for s in alone:
        for _ in range(4):
            s.step_cfl(cfl)
    batch = adg.Batch(mixed)
    for _ in range(4):                            # step 1 captured, 2-4 replays
        batch.step(cfl=cfl)
    batch.close()
    for a, m in zip(alone, mixed):
        _assert_same(_state(a), _state(m))
        assert a.time() == m.time()
    for s in alone + mixed:
        s.close()


def test_end_times_stop_each_state():
    ws = _workloads()[:3]
    t_ends = [0.004, 0.010, 0.002]
    ss = [_make(w, adg.PREC_FP64, t) for w, t in zip(ws, t_ends)]
    batch = adg.Batch(ss)
    frozen = None
    for it in range(400):
        batch.step(cfl=0.05)
        if it == 300:
            frozen = [s.read() for s in ss]
    batch.close()
    for s, t in zip(ss, t_ends):
        np.testing.assert_allclose(s.time()[0], t, rtol=1e-14)
    for s, f in zip(ss, frozen):                  # idle after reaching the end time
        np.testing.assert_array_equal(s.read(), f)
        s.close()


@pytest.mark.parametrize("prec", [adg.PREC_FP64, adg.PREC_MIXED_FP32])
def test_host_sized_passes_equal_device_sized_passes(prec):
    """adg_step with ADG_OPT_HOST_PASSES = 1 (the host reads the troubled count
    after the DG phase and launches the passes it needs) leaves the same
    state, bit for bit, as the default graph step whose conditional loop sizes
    the passes on the device; a small scratch budget forces several passes,
    and both run the same number of passes (the graph adds its loop kernels:
    one per step and one per pass)."""
    w = inputs.quadrants_2d(n=24, N=3)
    out = []
    for host in (1, 0):
        s = adg.Solver.from_workload(w, prec)
        s.set_option(adg.OPT_SCRATCH_BYTES, 4 * 2 ** 20)       # ~36 troubled cells per pass
        s.set_option(adg.OPT_HOST_PASSES, host)
        s.init_problem(w["problem"])
        info = s.info()
        assert info["chunk"] < 64
        l0 = info["launches"]
        for _ in range(6):
            s.step_cfl(w["cfl"])
        launched = s.info()["launches"] - l0
        assert s.troubled_count() > 2 * info["chunk"]
        out.append((_state(s), s.time(), launched))
        assert s.status() == adg.OK
        s.close()
    _assert_same(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    D, steps = 2, 6
    fixed = 2 + (D + 2) + 4 + 2 + 1                 # speed max + begin, DG, first-order layer, fix, end
    passes, rem = divmod(out[0][2] - steps * fixed, 2 * D + 4)
    assert rem == 0 and passes > 2 * steps
    assert out[1][2] == steps * (fixed + 1) + passes * (2 * D + 5)


@pytest.mark.parametrize("prec", [adg.PREC_FP64, adg.PREC_MIXED_FP32])
def test_batch_graph_loops_several_passes(prec):
    """Batched CFL steps (one graph, a device-sized pass loop per group) with a
    scratch budget small enough for several passes per step: every state
    bitwise equal to stepping it alone with host-sized passes."""
    ws = [inputs.quadrants_2d(n=24, N=3), inputs.quadrants_vortex_2d(n=18, N=3),
          inputs.explosion_2d(n=16, N=2)]
    states = []
    for host in (1, 0):
        row = []
        for w in ws:
            s = adg.Solver.from_workload(w, prec)
            s.set_option(adg.OPT_SCRATCH_BYTES, 4 * 2 ** 20)
            s.set_option(adg.OPT_HOST_PASSES, host)
            s.init_problem(w["problem"])
            row.append(s)
        states.append(row)
    cfl = 0.05
    for s in states[0]:
        for _ in range(5):
            s.step_cfl(cfl)
    batch = adg.Batch(states[1])
    for _ in range(5):                            # step 1 captured, 2-5 replays
        batch.step(cfl=cfl)
    batch.close()
    assert max(s.troubled_count() for s in states[0]) > 2 * states[0][0].info()["chunk"]
    for a, m in zip(*states):
        _assert_same(_state(a), _state(m))
        assert a.time() == m.time()
        assert a.status() == adg.OK and m.status() == adg.OK
    for s in states[0] + states[1]:
        s.close()


@pytest.mark.parametrize("host", [0, 1])
def test_profiled_steps_time_every_phase(host):
    """ADG_OPT_PROFILE on graph steps (event nodes inside the step graph, a
    ring of event sets so that the host may run ahead) and on host-sized
    steps (plain event records): every step timed, every phase positive, the
    phases together within the wall time of the steps; profiling changes no
    result."""
    w = inputs.quadrants_2d(n=32, N=3)
    res = []
    for prof in (0, 1):
        s = adg.Solver.from_workload(w, adg.PREC_FP64)
        s.set_option(adg.OPT_HOST_PASSES, host)
        s.init_problem(w["problem"])
        s.set_option(adg.OPT_PROFILE, prof)
        t0 = time.perf_counter()
        for _ in range(7):
            s.step_cfl(w["cfl"])
        res.append(_state(s))
        wall_ms = (time.perf_counter() - t0) * 1e3
        if prof:
            ph, n = s.phase_times()
            assert n == 7
            assert all(v > 0.0 for v in ph.values()), ph
            assert sum(ph.values()) <= wall_ms
        assert s.status() == adg.OK
        s.close()
    _assert_same(res[0], res[1])
