"""GPU: the continuous-batching server.  Runs that arrive while others are on
the GPU are admitted as memory allows, stepped together, and finish with the
same result as when each runs alone (bitwise: per-run work and time steps do
not depend on the other runs)."""
import numpy as np
import pytest

from paper_1406_7416_gb300 import adg, build_lib, inputs
from paper_1406_7416_gb300.serving import RunSpec, Server, poisson_arrivals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


def _runs(count=6, t_end=0.01):
    specs = inputs.serving_runs(count=count, sizes=(16, 24, 32), orders=(2, 3), t_end=t_end)
    arrivals = poisson_arrivals(count, rate=200.0, seed=11)
    return [RunSpec(w, t_end, a, i) for i, (w, a) in enumerate(zip(specs, arrivals))]


def _alone(r, prec):
    w = r.w
    s = adg.Solver.from_workload(w, prec)
    s.set_option(adg.OPT_END_TIME, r.t_end)
    s.init_problem(w["problem"])
    while s.time()[0] < r.t_end * (1.0 - 1e-12):
        s.step_cfl(w["cfl"])
    out = s.read_full()
    s.close()
    return out


@pytest.mark.parametrize("prec", [adg.PREC_FP64, adg.PREC_MIXED_FP32])
def test_runs_in_the_mix_equal_runs_alone(prec):
    runs = _runs()
    stats = Server(hbm_budget=1 << 40, prec=prec, steps_per_poll=4, keep_results=True).serve(runs)
    assert stats["runs"] == len(runs) and stats["steps"] > 0
    for r in runs:
        ref = _alone(r, prec)
        for a, b in zip(r.result, ref):
            if a.dtype.kind == "f":
                np.testing.assert_array_equal(np.nan_to_num(a), np.nan_to_num(b))
            else:
                np.testing.assert_array_equal(a, b)


def test_hbm_budget_limits_resident_runs():
    runs = _runs(count=5)
    for r in runs:
        r.arrival = 0.0
    srv = Server(hbm_budget=1, prec=adg.PREC_FP64, steps_per_poll=2)
    stats = srv.serve(runs)
    # a budget of one byte admits one run at a time: completions are ordered
    # and no run was admitted before the previous one finished
    order = sorted(runs, key=lambda r: r.admitted)
    for a, b in zip(order, order[1:]):
        assert b.admitted >= a.finished
    assert stats["latency_max_s"] >= stats["latency_p50_s"]
