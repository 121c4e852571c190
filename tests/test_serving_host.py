"""Host logic of the continuous-batching server (serving.py), on the CPU:
the device calls are replaced by a fake library whose states advance their
simulated time by a fixed step per batched step, cut at their end time as
the device step is, and the clock is simulated.  Checks admission by the
memory budget, batch rebuilds on membership changes, retirement at the end
time, retirement of stalled runs as failed, their retry at a smaller CFL number,
the no-admission wall limit and the statistics."""
import types

import numpy as np
import pytest

from paper_1406_7416_gb300 import serving

pytestmark = pytest.mark.timeout(60)     # a broken retirement rule would loop forever


class FakeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


class FakeSolver:
    def __init__(self, w, prec):
        self.w = w
        self.prec = prec
        self.t = 0.0
        self.n = 0
        self.t_end = 0.0
        self._dt = w["fake_dt"]
        self.cfl = None
        self.closed = False

    @property
    def dt(self):
        # a state whose CFL number is at least w["fake_fail_cfl"] loses
        # admissibility after three steps (only in precision w["fake_fail_prec"]
        # when that is given)
        fails_here = self.w.get("fake_fail_prec") in (None, self.prec)
        if (fails_here and self.cfl is not None and self.cfl >= self.w.get("fake_fail_cfl", np.inf)
                and self.n >= 3):
            return 0.0
        return self._dt

    @classmethod
    def from_workload(cls, w, prec):
        return cls(w, prec)

    def set_stream(self, s):
        pass

    def set_option(self, opt, value):
        if opt == FAKE.OPT_END_TIME:
            self.t_end = value
        if opt == FAKE.OPT_CFL:
            self.cfl = value

    def init_problem(self, problem):
        pass

    def bytes_held(self):
        return self.w["fake_bytes"]

    def time(self):
        return self.t, self.n

    def status(self):
        # a state that stopped stepping has no admissible wave speed: the real
        # library's status call raises then
        if self.dt == 0.0:
            raise FakeError(-6, "no admissible wave speed")
        return 0

    def read_full(self):
        return (np.array([self.t]),)

    def close(self):
        self.closed = True


class FakeBatch:
    built = []

    def __init__(self, solvers, stream=0):
        self.solvers = list(solvers)
        FakeBatch.built.append([id(s) for s in solvers])

    def step(self, cfl=0.0):
        for s in self.solvers:
            assert not s.closed
            if serving.reached_end(s.t, s.t_end) or not s.dt > 0.0:
                continue                      # idle past the end, or no admissible dt
            s.t = min(s.t + s.dt, s.t_end) if s.t + s.dt < s.t_end else s.t_end
            s.n += 1

    def close(self):
        pass


FAKE = types.SimpleNamespace(Solver=FakeSolver, Batch=FakeBatch, OPT_CFL=9, OPT_END_TIME=8,
                             PREC_FP64=0, PREC_MIXED_FP32=1, AdgError=FakeError)


class Clock:
    """Simulated seconds: every call advances 1 ms."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t


@pytest.fixture
def fake_lib(monkeypatch):
    monkeypatch.setattr(serving, "adg", FAKE)
    monkeypatch.setattr(serving.time, "sleep", lambda s: None)
    FakeBatch.built = []


def _run(i, dt=0.01, nbytes=100, t_end=0.1, arrival=0.0, shape=None, fail_cfl=np.inf,
         fail_prec=None):
    w = {"dim": 2, "N": 3, "ncell": shape or (8 + i, 8), "cfl": 0.1, "problem": None,
         "fake_dt": dt, "fake_bytes": nbytes, "fake_fail_cfl": fail_cfl, "fake_fail_prec": fail_prec}
    return serving.RunSpec(w, t_end, arrival, i)


class Tracking(serving.Server):
    """Records the resident memory at each admission."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.peak = 0
        self.resident = []

    def _admit(self, r):
        super()._admit(r)
        self.resident = [x for x in self.resident if x.finished is None] + [r]
        self.peak = max(self.peak, sum(x.bytes for x in self.resident))


def test_budget_limits_resident_runs_of_one_shape(fake_lib):
    """Once a run of a shape was admitted its size is known: at most two runs
    of 100 bytes are resident under a 250-byte budget."""
    runs = [_run(i, nbytes=100, shape=(16, 16)) for i in range(7)]
    srv = Tracking(250, steps_per_poll=4)
    st = srv.serve(runs, clock=Clock())
    assert st["runs"] == 7 and st["failed"] == 0
    assert srv.peak == 200


def test_budget_limits_resident_runs_and_every_run_finishes(fake_lib):
    """Shapes never seen before are admitted while the resident bytes are
    within the budget, so the budget is exceeded by one run at most."""
    runs = [_run(i, nbytes=100) for i in range(7)]
    srv = Tracking(250, steps_per_poll=4)
    st = srv.serve(runs, clock=Clock())
    assert st["runs"] == 7 and st["failed"] == 0 and st["unserved"] == 0
    assert 250 < srv.peak <= 250 + 100
    for r in runs:
        assert r.finished is not None and r.finished >= r.admitted >= r.arrival
        assert r.steps == 10                      # t_end / dt steps, the last one cut
        assert serving.reached_end(r.solver.t if r.solver else r.t_end, r.t_end)
    assert st["steps"] == 70
    assert st["stdof_updates"] == sum(r.stdofs_per_step * 10 for r in runs)


def test_batch_rebuilt_only_when_membership_changes(fake_lib):
    runs = [_run(0, dt=0.05), _run(1, dt=0.01)]
    serving.Server(10 ** 9, steps_per_poll=1).serve(runs, clock=Clock())
    # both admitted at t = 0 (one batch); run 0 ends after 2 steps (one rebuild to run 1 alone)
    assert len(FakeBatch.built) == 2
    assert len(FakeBatch.built[0]) == 2 and len(FakeBatch.built[1]) == 1


def test_stalled_run_is_retired_as_failed(fake_lib):
    runs = [_run(0), _run(1, dt=0.0), _run(2)]
    st = serving.Server(10 ** 9, steps_per_poll=2).serve(runs, clock=Clock())
    assert st["failed"] == 1 and st["failed_ids"] == [1] and st["runs"] == 2
    assert runs[1].failed and runs[1].steps == 0 and runs[1].status == -6
    assert not runs[0].failed and not runs[2].failed


def test_no_admission_after_the_wall_limit(fake_lib):
    runs = [_run(0, arrival=0.0), _run(1, arrival=50.0)]
    st = serving.Server(10 ** 9, steps_per_poll=1).serve(runs, clock=Clock(), max_wall=0.5)
    assert st["runs"] == 1 and st["unserved"] == 1 and runs[1].finished is None


def test_latency_statistics_and_end_test():
    assert serving.reached_end(1.0, 1.0)
    assert serving.reached_end(1.0 - 1e-13, 1.0)
    assert not serving.reached_end(1.0 - 1e-9, 1.0)
    a = serving.poisson_arrivals(20000, 4.0, seed=3)
    assert np.all(np.diff(a) > 0)
    assert abs(np.mean(np.diff(a)) - 0.25) < 0.01
    np.testing.assert_array_equal(a, serving.poisson_arrivals(20000, 4.0, seed=3))


def test_results_kept_on_request(fake_lib):
    runs = [_run(0, t_end=0.05)]
    serving.Server(10 ** 9, keep_results=True).serve(runs, clock=Clock())
    assert runs[0].result[0][0] == pytest.approx(0.05)


def test_failed_run_is_retried_at_a_smaller_cfl(fake_lib):
    """Run 1 loses admissibility after three steps at the workload's CFL
    number: with one retry it starts again from its initial data at half the
    CFL number and finishes; its failed attempt's steps are not counted as
    work, and its latency runs from its arrival."""
    runs = [_run(0), _run(1, fail_cfl=0.1), _run(2)]
    st = serving.Server(10 ** 9, steps_per_poll=2, retries=1, retry_prec=None,
                        retry_cfl_factor=0.5).serve(runs, clock=Clock())
    assert st["runs"] == 3 and st["failed"] == 0
    assert st["retried"] == 1 and st["retried_served"] == 1 and st["retried_ids"] == [1]
    r = runs[1]
    assert r.attempts == 1 and r.cfl_scale == 0.5 and r.prec is None
    assert not r.failed and r.status == 0
    assert r.wasted_steps == 3 and r.steps == 10 and st["wasted_steps"] == 3
    assert st["steps"] == 30
    assert st["stdof_updates"] == sum(x.stdofs_per_step * 10 for x in runs)
    assert r.finished > r.admitted > r.arrival


def test_run_failing_every_attempt_is_retired_as_failed(fake_lib):
    """A run that fails at every CFL number is retired as failed once its
    retries are spent; without retries it is retired at the first failure."""
    runs = [_run(0, fail_cfl=0.0), _run(1)]
    st = serving.Server(10 ** 9, steps_per_poll=2, retries=2,
                        retry_cfl_factor=0.5).serve(runs, clock=Clock())
    assert st["failed"] == 1 and st["runs"] == 1 and st["failed_ids"] == [0]
    assert runs[0].attempts == 2 and runs[0].cfl_scale == 0.25 and runs[0].status == -6
    assert st["wasted_steps"] == 9 and runs[0].steps == 3
    runs = [_run(0, fail_cfl=0.0)]
    st = serving.Server(10 ** 9, steps_per_poll=2).serve(runs, clock=Clock())
    assert st["failed"] == 1 and runs[0].attempts == 0 and st["retried"] == 0


def test_default_retry_restarts_in_fp64_at_the_same_cfl(fake_lib):
    """Run 1 loses admissibility in mixed precision only: the default retry
    restarts it in FP64 at its own CFL number, and it finishes."""
    runs = [_run(0), _run(1, fail_cfl=0.1, fail_prec=1), _run(2)]
    st = serving.Server(10 ** 9, steps_per_poll=2, retries=1).serve(runs, clock=Clock())
    assert st["runs"] == 3 and st["failed"] == 0 and st["retried_served"] == 1
    r = runs[1]
    assert r.attempts == 1 and r.prec == 0 and r.cfl_scale == 1.0 and r.steps == 10
    assert all(x.prec is None for x in (runs[0], runs[2]))
