"""GPU: batched stepping (adg_batch_*, adg_step_batch) against stepping each
state alone.  Per-state work is the same arithmetic in both cases, so in FP64
(and in mixed precision) every state's DOFs, flags and subcell data after the
steps are bitwise equal alone and in the mix."""
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
    for _ in range(4):                            # step 1 plain, step 2 captured, 3-4 replays
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
def test_host_sized_passes_equal_async_passes(prec):
    """adg_step with ADG_OPT_HOST_PASSES (the host reads the troubled count
    after the DG phase and launches only the passes it needs) leaves the same
    state, bit for bit, as the fully asynchronous step that launches every
    pass the capacity allows; a small scratch budget forces several passes."""
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
        out.append((_state(s), s.time(), launched, info["launches_per_step"]))
        assert s.status() == adg.OK
        s.close()
    _assert_same(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    assert out[1][2] == 6 * out[1][3]                # asynchronous: every pass launched
    assert out[0][2] < out[1][2]
