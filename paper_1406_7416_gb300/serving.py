"""Continuous-batching server for independent simulation runs.

Runs (one 2D/3D Euler problem each, with its own grid, degree and end time)
arrive over time.  The server admits a run when its device memory fits the
HBM budget, keeps every admitted run's state resident on the device, and
advances all of them together: each poll interval issues a few batched CFL
steps (adg_batch_step, one CUDA graph per membership), then reads each run's
simulated time; finished runs are retired, which frees memory for waiting
runs, and the batch is rebuilt whenever its membership changes.  A run that
takes no step over a whole poll before its end time (no finite positive CFL
time step, e.g. after a loss of positivity) has failed: with retries left it is
started again from its initial data in the retry precision (FP64 by default)
and at retry_cfl_factor times its CFL number (the time step of Eq. (cfl) is
an upper bound; any smaller step is admissible), else it is retired as
failed.  Reports the latency of every run (arrival to completion,
retries included) and the aggregate space-time DOF update rate (the steps of
failed attempts are not counted as work done).
"""
import collections
import time

import numpy as np

from . import adg


class RunSpec:
    """One request: a workload dict (see inputs.py) with an end time."""

    def __init__(self, workload, t_end, arrival=0.0, rid=0):
        self.w = workload
        self.t_end = float(t_end)
        self.arrival = float(arrival)
        self.rid = rid
        self.solver = None
        self.admitted = None
        self.finished = None
        self.steps = 0
        self.bytes = 0
        self.result = None
        self.status = 0
        self.failed = False
        self.attempts = 0          # retries taken
        self.cfl_scale = 1.0       # factor on the workload's CFL number
        self.prec = None           # precision override of a retried run (None: the server's)
        self.wasted_steps = 0      # steps of failed attempts

    @property
    def stdofs_per_step(self):
        w = self.w
        return int(np.prod(w["ncell"])) * (w["N"] + 1) ** (w["dim"] + 1)


class Server:
    """hbm_budget: bytes of device memory the resident runs may hold."""

    def __init__(self, hbm_budget, prec=adg.PREC_MIXED_FP32, steps_per_poll=8, keep_results=False,
                 stream=0, retries=0, retry_prec=adg.PREC_FP64, retry_cfl_factor=1.0):
        self.budget = int(hbm_budget)
        self.retries = int(retries)
        self.retry_prec = retry_prec          # None: keep the server's precision
        self.retry_cfl_factor = float(retry_cfl_factor)
        self.prec = prec
        self.steps_per_poll = steps_per_poll
        self.keep = keep_results
        self.stream = stream
        self.bytes_cache = {}

    def _key(self, w, prec):
        return (w["dim"], w["N"], tuple(w["ncell"]), prec)

    def _admit(self, r):
        w = r.w
        s = adg.Solver.from_workload(w, self.prec if r.prec is None else r.prec)
        if self.stream:
            s.set_stream(self.stream)
        s.set_option(adg.OPT_CFL, w["cfl"] * r.cfl_scale)
        s.set_option(adg.OPT_END_TIME, r.t_end)
        s.init_problem(w["problem"])
        r.solver = s
        r.bytes = s.bytes_held()
        self.bytes_cache[self._key(w, r.prec)] = r.bytes

    def serve(self, runs, clock=time.perf_counter, max_wall=None):
        """Serve `runs` (RunSpec, arrival times in seconds from the start);
        returns a dict of statistics.  Runs finish in place (r.finished).
        With max_wall (seconds) no run is admitted after that time; the runs
        already admitted still finish and the others are reported unserved."""
        waiting = collections.deque(sorted(runs, key=lambda r: r.arrival))
        active = []
        used = 0
        batch = None
        rebuild = False
        t0 = clock()
        polls = 0
        while waiting or active:
            now = clock() - t0
            if max_wall is not None and now > max_wall and waiting:
                waiting.clear()
            while waiting and waiting[0].arrival <= now:
                r = waiting[0]
                need = self.bytes_cache.get(self._key(r.w, r.prec), 0)
                if active and used + need > self.budget:
                    break
                waiting.popleft()
                self._admit(r)
                r.admitted = clock() - t0
                used += r.bytes
                active.append(r)
                rebuild = True
            if not active:
                if waiting:
                    time.sleep(max(0.0, min(0.01, waiting[0].arrival - now)))
                continue
            if rebuild:
                if batch is not None:
                    batch.close()
                batch = adg.Batch([r.solver for r in active], self.stream)
                rebuild = False
            for _ in range(self.steps_per_poll):
                batch.step(cfl=0.0)
            polls += 1
            still, retry = [], []
            for r in active:
                t, n = r.solver.time()
                done = reached_end(t, r.t_end)
                # a run that took no step over a whole poll without reaching
                # its end time has stopped (its CFL step found no finite
                # positive dt): it is retired as failed
                stalled = not done and n == r.steps
                r.steps = n
                if done or stalled:
                    try:
                        status = r.solver.status()
                    except adg.AdgError as e:   # e.g. no admissible wave speed left
                        status = e.code
                    failed = stalled or status < 0
                    if failed and r.attempts < self.retries:
                        retry.append(r)
                    else:
                        r.finished = clock() - t0
                        r.status = status
                        r.failed = failed
                        if self.keep:
                            r.result = r.solver.read_full()
                    used -= r.bytes
                    rebuild = True
                else:
                    still.append(r)
            if rebuild:
                if batch is not None:
                    batch.close()
                    batch = None
                for r in active:
                    if (r.finished is not None or r in retry) and r.solver is not None:
                        r.solver.close()
                        r.solver = None
            # failed runs with retries left go back to the head of the queue
            # (their arrival is earlier than every waiting run's)
            for r in reversed(retry):
                r.attempts += 1
                r.cfl_scale *= self.retry_cfl_factor
                if self.retry_prec is not None:
                    r.prec = self.retry_prec
                r.wasted_steps += r.steps
                r.steps = 0
                waiting.appendleft(r)
            active = still
        wall = clock() - t0
        if batch is not None:
            batch.close()
        served = [r for r in runs if r.finished is not None and not r.failed]
        failed = [r for r in runs if r.failed]
        lat = np.array([r.finished - r.arrival for r in served]) if served else np.zeros(1)
        stdofs = sum(r.stdofs_per_step * r.steps for r in served)
        return {"runs": len(served), "failed": len(failed),
                "failed_ids": [r.rid for r in failed],
                "unserved": len(runs) - len(served) - len(failed), "wall_s": wall,
                "polls": polls,
                "latency_p50_s": float(np.percentile(lat, 50)),
                "latency_p99_s": float(np.percentile(lat, 99)),
                "latency_max_s": float(lat.max()),
                "stdof_updates": int(stdofs), "stdof_per_s": stdofs / wall,
                "steps": int(sum(r.steps for r in served)),
                "retried": sum(1 for r in runs if r.attempts > 0),
                "retried_served": sum(1 for r in served if r.attempts > 0),
                "retried_ids": [r.rid for r in runs if r.attempts > 0],
                "wasted_steps": int(sum(r.wasted_steps for r in runs) + sum(r.steps for r in failed))}


def reached_end(t, t_end):
    """The end-time test of the device step (a run takes no further step once
    the time left is at most 1e-12 t_end), in the same double arithmetic."""
    return not (t_end - t > 1e-12 * t_end)


def poisson_arrivals(count, rate, seed):
    """Arrival times of a Poisson process of `rate` per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
