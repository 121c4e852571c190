#!/usr/bin/env python
"""Throughput of one full ADER-DG + subcell-limiter time step on GB300.

Workload: 2D Euler, N = 5 (Ns = 11), 512 x 512 periodic cells on [-5, 5]^2,
seeded four-quadrant Riemann data with a superposed isentropic vortex
(strength 5) -- the paper's 2D Riemann / vortex test shapes (Sec. 5.2, 5.6).
A step is one adg_step: predictor, corrector, detection, subcell ADER-WENO3
of troubled cells, reconstruction and neighbour flux correction.

Metric: space-time DOF updates per second = cells * (N+1)^(d+1) * steps / s
(per conserved variable, as the paper counts).  `value` is the mixed-precision
path: FP32 Picard sweeps; for N <= 5 no FP64 sweep follows and the final stage
adds the FP32 space-time correction to the FP64 DOFs term by term, for N >= 6
one FP64 sweep follows; FP32 subcell scheme with an FP64 update; FP64
corrector, detector tests and flux correction, the detector's subcell
averages being the kept FP64 averages plus an FP32 projection of the step's
change (an FP64 projection every 16th step).  The FP64
path is reported beside it, with the L1 distance between the two after the
same steps against the stated tolerance of the workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: one independent replica per rank (weak scaling), launched by torchrun.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ORDER = 5
GRID = 512
GRID_SET = None
WORKLOAD = "quadvortex512"
METRIC = "space-time DOF updates/s"
UNIT = "ST-DOF/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz


def workload(n=None, N=N_ORDER):
    """The benchmark workload (default: 2D quadrants + vortex, N=5, 512^2)."""
    from paper_1406_7416_gb300 import inputs
    n = n or GRID_SET
    if WORKLOAD == "explosion2d":
        return inputs.explosion_2d(n=n or 32, N=3)
    if WORKLOAD == "explosion3d":
        return inputs.explosion_3d(n=n or 128, N=3)
    if WORKLOAD == "quadrants200":
        return inputs.quadrants_2d(n=n or 200, N=9)
    if WORKLOAD == "dmr":
        nx = n or 350
        return inputs.double_mach(nx=nx, ny=max(1, nx * 2 // 7), N=5)
    return inputs.quadrants_vortex_2d(n=n or GRID, N=N, steps=None)


def launch_mode(args):
    return ("plain kernel launches, limiter passes sized by the host after the DG phase"
            if args.host_passes else
            "one CUDA graph per step, limiter passes in a device-sized conditional loop")


def config_dict(w, extra=None):
    import numpy as np
    cells = int(np.prod(w["ncell"]))
    nv, nd = w["dim"] + 2, (w["N"] + 1) ** w["dim"]
    state = cells * nv * nd * 8
    traces = cells * w["dim"] * 2 * nv * (w["N"] + 1) ** w["dim"] * 8
    big = state + traces > 129e6
    c = {"workload": w["name"], "grid": "x".join(str(x) for x in w["ncell"]), "N": w["N"],
         "cells": cells, "dim": w["dim"],
         "l2": (f"inputs larger than L2: DOF state {state / 1e6:.0f} MB and face traces "
                f"{traces / 1e6:.0f} MB per step") if big else
               f"inputs smaller than L2 (state {state / 1e6:.1f} MB): steps run L2-warm"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# algorithmic operation counts (per cell), from the arithmetic the kernels do
# ---------------------------------------------------------------------------
def flux_flops(D):
    """Euler fluxes in all D directions at one node: 1 division, D + 2D for the
    velocities and kinetic term, 4 for pressure and E + p, D(D + 2) for F."""
    return D * D + 5 * D + 5


def flux_delta_flops(D):
    """F_k(U + dQ) - F_k(U) in all D directions at one node, in the form whose
    terms carry a factor of dQ: 2 divisions, velocities and their changes,
    m.v and its change, E + p and the pressure change, D (3D + 6) for the
    flux changes."""
    return 3 * D * D + 17 * D + 9


def predictor_flops(D, N, iters, fp64_sweeps):
    """(fp64, fp32) flops of the predictor kernel for one cell: `iters` Picard
    sweeps, `fp64_sweeps` of them in FP64 and the others in FP32, then the
    final stage.  After an FP64 sweep (and in the FP64 path) the final stage
    is FP64: fluxes at the space-time nodes, their time average, the volume
    term and the face traces.  With no FP64 sweep it splits: F(u) at the
    spatial nodes, the volume term and trace(u) in FP64; the flux changes at
    the space-time nodes, their weighted time sum and trace(q - u) in FP32;
    and the first sweep, from the time-constant u (x) 1, runs on the spatial
    nodes only."""
    n, nv = N + 1, D + 2
    nst, nd, nf = n ** (D + 1), n ** D, n ** (D - 1)
    it = nst * flux_flops(D) + nv * nst * D * (2 * n + 2) + nv * nd * n * (2 * n + 1)
    vol = nv * nd * D * (2 * n + 2)
    if fp64_sweeps > 0:
        final = nst * flux_flops(D) + D * nv * nd * 2 * n + vol + 2 * D * nv * nf * n * 2 * n
        return fp64_sweeps * it + final, (iters - fp64_sweeps) * it
    final64 = nd * flux_flops(D) + D * nv * nd + vol + 2 * D * nv * nf * 2 * n
    final32 = (nst * flux_delta_flops(D) + D * nv * nst * 2 + 2 * D * nv * nf * n * 2 * n
               + nv * nst * n * 2)
    # the first sweep from u (x) 1: fluxes and derivatives on the n^d spatial
    # nodes, then one FMA per space-time node (q1_m = u - kappa_m S)
    first = nd * flux_flops(D) + nv * nd * D * (2 * n + 2) + nv * nd * n * 2
    return final64, (iters - 1) * it + first + final32


def clocks_sampler():
    """nvidia-smi clock / throttle samples during the timed region."""
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
           "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"]
    if "CUDA_VISIBLE_DEVICES" in os.environ and os.environ["CUDA_VISIBLE_DEVICES"].strip():
        cmd += ["-i", os.environ["CUDA_VISIBLE_DEVICES"].split(",")[0]]
    try:
        return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def clocks_summary(proc, local_rank):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    proc.terminate()
    out, _ = proc.communicate(timeout=10)
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for nm, val in zip(names, f[5:9]):
            if val.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
            "samples": len(sm)}


def traffic_record():
    """DRAM bytes per predictor launch from the committed ncu summary, if it was
    taken on the current kernel source (else null)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "predictor_traffic.json")
    src = os.path.join(ROOT, "paper_1406_7416_gb300", "csrc", "kernels_pred.cuh")
    try:
        rec = json.load(open(path))
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("kernels_pred_sha256") == h:
            return rec
    except (OSError, ValueError):
        pass
    return None


# ---------------------------------------------------------------------------
# CPU oracle timing (test infrastructure, timed as a baseline only)
# ---------------------------------------------------------------------------
def oracle_sample(block=32):
    """The central block^d cells of the workload (quadrant corner and vortex
    core, or the centre of the explosion), transmissive at the block edges,
    projected by the oracle."""
    from oracle.dg import Grid
    from oracle.ic import initial_state, project_problem
    from oracle.step import Scheme
    w = workload()
    d = w["dim"]
    block = min(block, w["ncell"][0])
    i0 = [w["ncell"][k] // 2 - block // 2 for k in range(d)]
    x0 = tuple(w["x0"][k] + i0[k] * w["dx"][k] for k in range(d))
    g = Grid((block,) * d, x0, w["dx"], (1,) * (2 * d))
    if w["problem"].get("cell_rho_factor") is not None:
        w["problem"]["cell_rho_factor"] = w["problem"]["cell_rho_factor"][
            tuple(slice(i0[k], i0[k] + block) for k in range(d))]
    sch = Scheme(g, w["N"], w["gamma"])
    U0, V0 = project_problem(sch, w["problem"])
    return w, sch, initial_state(sch, U0, V0)


def oracle_rate(steps, warmup, block=32, budget_s=20.0):
    """Oracle ST-DOF/s on the central sample: up to `steps` timed steps, fewer
    when they would exceed budget_s seconds (at least one)."""
    import numpy as np
    from oracle.step import stable_dt, step
    w, sch, st = oracle_sample(block)
    dt = stable_dt(sch, st, w["cfl"])
    for _ in range(warmup):
        st, _ = step(sch, st, dt)
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        st, _ = step(sch, st, dt)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    steps = done
    el = time.perf_counter() - t0
    d = w["dim"]
    dofs = int(np.prod(sch.grid.ncell)) * (w["N"] + 1) ** (d + 1)
    return dofs * steps / el, el, steps


def run_cpu_baseline(steps, warmup, block, budget_s=20.0):
    """Times the oracle in a child process pinned to one BLAS thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-rate",
                        str(steps), str(warmup), str(block), WORKLOAD, str(budget_s)], env=env,
                       capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"failed: {r.stderr.strip()[-300:]}"}
    rate, el, steps = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} oracle steps (after {warmup} warm-up) on the central "
                      f"{block}^d cells of the same workload, transmissive block edges, "
                      f"{el:.1f} s, one BLAS thread"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
# Stated accuracy bar of the mixed-precision path per workload: the relative
# L1 distance to the FP64 path after the run's steps, per conserved variable,
# may be at most TOL.  Each TOL is at most 1% of the FP64 scheme's own
# relative L1 error on that workload over the steps the bench runs (3 + 20 for
# the default workload, 3 + 5 for the others): the error is estimated from
# the distance r to the FP64 solution on the grid refined by 2 by Richardson's
# rule with the first-order L1 convergence of discontinuous data, 2 r, so TOL
# <= 0.02 r, taken over the variables and rounded down (measured on one
# GB300: quadrants + vortex 512^2 N = 5, 23 steps, 0.02 r >= 8.5e-6; 2D
# quadrants 200^2 N = 9, 8 steps, >= 7.0e-6; 3D explosion 64^3 N = 3, 8 steps,
# >= 5.4e-5, finer grids halving it; 2D explosion 32^2 N = 3, 20 steps,
# >= 1.6e-4).
TOL = {"quadvortex512": 8e-6, "explosion2d": 1e-5, "explosion3d": 1e-5, "quadrants200": 7e-6,
       "dmr": None}


def measure(args, wname, grid, steps, warmup, stream, rep, clocks=False, keep=False,
            floor_run=False):
    """FP64 and mixed runs of one workload: timed CFL steps, phases, the
    mixed-vs-FP64 distance against the stated bar, troubled counts per step."""
    import numpy as np
    import torch
    from paper_1406_7416_gb300 import adg
    globals()["WORKLOAD"] = wname
    globals()["GRID_SET"] = grid
    w = workload()
    D, N = w["dim"], w["N"]
    n = N + 1
    cells = int(np.prod(w["ncell"]))
    stdofs = cells * n ** (D + 1)
    rank = rep.rank

    def make(prec, opts=None):
        s = adg.Solver.from_workload(w, prec)
        s.set_stream(stream.cuda_stream)
        if args.host_passes:
            s.set_option(adg.OPT_HOST_PASSES, 1)
        for k, v in (opts or {}).items():
            s.set_option(k, v)
        s.init_problem(w["problem"])
        return s

    results = {}
    precs = [("fp64", adg.PREC_FP64), ("mixed", adg.PREC_MIXED_FP32)]
    if args.only != "both":
        precs = [p for p in precs if p[0] == args.only]
    mixed_opts = {adg.OPT_PREDICTOR: args.predictor} if args.predictor is not None else {}
    for name, prec in precs:
        s = make(prec, mixed_opts if name == "mixed" else None)
        s.set_option(adg.OPT_PROFILE, 1)
        for _ in range(warmup):
            s.step_cfl(w["cfl"])
        s.phase_times()                             # discard warm-up phases
        torch.cuda.synchronize()
        rep.barrier()
        clk = clocks_sampler() if (clocks and name == "mixed" and rank == 0) else None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = s.info()["launches"]
        e0.record(stream)
        for _ in range(steps):
            s.step_cfl(w["cfl"])
        e1.record(stream)
        torch.cuda.synchronize()
        launches = s.info()["launches"] - l0
        rep.barrier()
        ms = e0.elapsed_time(e1) / steps
        r = dict(ms=rep.max_over_ranks(ms), solver=s, status=s.status(),
                 troubled=s.troubled_count(), info=s.info(), launches=launches,
                 clocks=clocks_summary(clk, 0) if clk is not None else None,
                 history=s.troubled_history(warmup + steps).tolist(), time=s.time()[0])
        phases, nsteps = s.phase_times()
        r["phases"] = {k: v / max(nsteps, 1) for k, v in phases.items()}
        results[name] = r
    out = dict(w=w, D=D, N=N, n=n, cells=cells, stdofs=stdofs, results=results)
    if args.only == "both":
        Wd = 0.5 * np.polynomial.legendre.leggauss(n)[1]
        W1 = Wd
        for _ in range(D - 1):
            Wd = np.outer(W1, Wd).ravel()
        U64 = results["fp64"]["solver"].read()
        Umx = results["mixed"]["solver"].read()
        num = np.einsum("cvl,l->v", np.abs(Umx - U64), Wd)
        den = np.einsum("cvl,l->v", np.abs(U64), Wd)
        d = (num / den).tolist()
        tol = TOL.get(wname)
        out["mixed_vs_fp64"] = {
            "l1_rel_per_variable": d, "l1_density_rel": d[0], "steps": warmup + steps,
            "tolerance_rel": tol, "pass": (max(d) <= tol) if tol else None,
            "bar": "relative L1 distance to the FP64 path per conserved variable after the same "
                   "number of CFL steps <= tolerance_rel, which is 1% of the FP64 scheme's own "
                   "relative L1 error on this workload (error against the 2x refined solution)",
            "final_time": {"fp64": results["fp64"]["time"], "mixed": results["mixed"]["time"]}}
    if floor_run:
        # the literal Eq. (relax) (no floor on the DMP relaxation) against the
        # default floor, same workload and steps, mixed precision (untimed)
        s = make(adg.PREC_MIXED_FP32, {**mixed_opts, adg.OPT_DMP_FLOOR: 0.0})
        for _ in range(warmup + steps):
            s.step_cfl(w["cfl"])
        h0 = s.troubled_history(warmup + steps).tolist()
        s.close()
        h4 = results["mixed"]["history"] if "mixed" in results else None
        out["dmp_floor"] = {"troubled_per_step_floor_1e-4": h4, "troubled_per_step_floor_0": h0,
                            "mean_floor_1e-4": float(np.mean(h4)) if h4 else None,
                            "mean_floor_0": float(np.mean(h0))}
    if not keep:
        for r in results.values():
            r["solver"].close()
            r["solver"] = None
    return out


def run_gpu(args):
    import torch
    from paper_1406_7416_gb300 import adg, build_lib
    from paper_1406_7416_gb300.replicas import Replicas

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    rep = Replicas("nccl", torch.device("cuda", local))
    world, rank = rep.world, rep.rank
    if rank == 0:
        build_lib.build()
    rep.barrier()
    adg.load_library()
    stream = torch.cuda.Stream()
    rates = adg.pipe_rates()            # measured arithmetic-pipe rates, beside the derived peaks
    main_wl, main_grid = WORKLOAD, GRID_SET
    m = measure(args, main_wl, main_grid, args.steps, args.warmup, stream, rep, clocks=True,
                keep=True, floor_run=(args.only == "both" and not args.no_extras))
    w, results = m["w"], m["results"]
    if args.only != "both":
        # profiling run of one precision: timings only
        if rank == 0:
            r = results[args.only]
            print(json.dumps({"profile_run": args.only, "ms_per_step": r["ms"],
                              "phases_ms": r["phases"], "troubled_cells": r["troubled"],
                              "predictor_shape": r["info"]["predictor"],
                              "config": config_dict(w, {"launch": launch_mode(args)})}), flush=True)
        for r in results.values():
            r["solver"].close()
        rep.close()
        return
    # end-to-end through the C ABI with host buffers (rank-local)
    e2e = None
    s = results["mixed"]["solver"]
    tune = None
    if not args.no_e2e:
        e2e = end_to_end(s, args, m["stdofs"], world, w["cfl"], rep.barrier, rep.max_over_ranks)
    tune = s.autotune(3)
    for r in results.values():
        r["solver"].close()
    # the other configurations (mixed and FP64, 3 warm-up + 5 steps each), on
    # the default workload only
    subs = {}
    if main_wl == "quadvortex512" and main_grid is None and not args.no_extras:
        for wl in ("explosion2d", "quadrants200", "explosion3d"):
            sm = measure(args, wl, None, 5, 3, stream, rep)
            mx, f64 = sm["results"]["mixed"], sm["results"]["fp64"]
            subs[wl] = {"workload": sm["w"]["name"], "cells": sm["cells"],
                        "mixed": {"value": sm["stdofs"] * world / (mx["ms"] / 1e3),
                                  "ms_per_step": mx["ms"], "phases_ms": mx["phases"],
                                  "predictor_shape": adg.PRED_NAMES[mx["info"]["predictor"]],
                                  "fp64_sweeps": mx["info"]["fp64_sweeps"]},
                        "fp64": {"value": sm["stdofs"] * world / (f64["ms"] / 1e3),
                                 "ms_per_step": f64["ms"]},
                        "mixed_vs_fp64": sm["mixed_vs_fp64"],
                        "troubled_per_step": mx["history"],
                        "troubled_fraction_per_step": [c / sm["cells"] for c in mx["history"]],
                        "status": mx["status"], "steps": 5, "warmup": 3}
    globals()["WORKLOAD"], globals()["GRID_SET"] = main_wl, main_grid
    if rank == 0:
        emit_line(args, m, e2e, world, tune, subs, rates)
    rep.close()


def end_to_end(s, args, stdofs, world, cfl, barrier, max_over_ranks):
    """The metric through the C ABI with host buffers: adg_load_full from pinned
    host memory, then per step adg_step_cfl + adg_flags to pinned host memory,
    then adg_read of the DOFs."""
    import numpy as np
    import torch
    from paper_1406_7416_gb300 import adg
    dofs, beta, sub = s.read_full()
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    hd, hb, hs = pin(dofs), pin(beta), pin(sub)
    flags = pin(np.empty(s.cells, dtype=np.uint8))
    out = pin(np.empty_like(dofs))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    s.load_full(hd, hb, hs)
    t1 = time.perf_counter()
    for _ in range(args.steps):
        s.step_cfl(cfl)
        s.lib.adg_flags(s.h, adg._u8ptr(flags))
    t2 = time.perf_counter()
    s.read(out)
    t3 = time.perf_counter()
    el = max_over_ranks(t3 - t0)
    h2d = (hd.nbytes + hb.nbytes + hs.nbytes) / args.steps + 8
    d2h = flags.nbytes + out.nbytes / args.steps
    return {"value": stdofs * args.steps * world / el, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "breakdown_ms": {"load": (t1 - t0) * 1e3, "steps": (t2 - t1) * 1e3,
                             "read": (t3 - t2) * 1e3},
            "timed": "adg_load_full from pinned host, then per step adg_step_cfl + adg_flags to "
                     "pinned host, then adg_read of the DOFs"}


def emit_line(args, m, e2e, world, tune, subs, rates=None):
    from paper_1406_7416_gb300 import adg
    w, results = m["w"], m["results"]
    D, N, n, cells, stdofs = m["D"], m["N"], m["n"], m["cells"], m["stdofs"]
    mx, f64 = results["mixed"], results["fp64"]
    value = stdofs * world / (mx["ms"] / 1e3)
    iters = int(mx["info"]["picard_iters"])
    fl64, fl32 = predictor_flops(D, N, iters, int(mx["info"]["fp64_sweeps"]))
    pred_ms = mx["phases"]["predictor"]
    # the predictor's bound: the pipe whose algorithmic flops take longer at its
    # derived peak (the FP64 and FP32 pipes run side by side)
    t64 = fl64 * cells / (FP64_PEAK_TFLOPS * 1e12)
    t32 = fl32 * cells / (FP32_PEAK_TFLOPS * 1e12)
    pipe, fl_dom, peak = (("fp64", fl64, FP64_PEAK_TFLOPS) if t64 >= t32 else
                          ("fp32", fl32, FP32_PEAK_TFLOPS))
    achieved = fl_dom * cells / (pred_ms / 1e3) / 1e12
    fl64f, _ = predictor_flops(D, N, iters, iters)
    achieved_f64 = fl64f * cells / (f64["phases"]["predictor"] / 1e3) / 1e12
    traffic = traffic_record() if (WORKLOAD == "quadvortex512" and GRID == 512) else None
    shape = adg.PRED_NAMES[mx["info"]["predictor"]]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mx["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": config_dict(w, {"precision": ("mixed: FP32 Picard sweeps (%d of %d in FP64; with "
                                                "none the final stage takes the FP64 u plus FP32 "
                                                "corrections), FP64 corrector/detector; subcell "
                                                "scheme: FP32 reconstruction, predictor and "
                                                "sub-face fluxes, FP64 update"
                                                % (int(mx["info"]["fp64_sweeps"]),
                                                   int(mx["info"]["picard_iters"]))),
                                  "predictor_shape": shape,
                                  "first_order_layer": "on: the extra MOOD layer of Sec. 6 "
                                                       "(ADG_OPT_CASCADE = 1) recomputes troubled "
                                                       "cells whose WENO3 result fails PAD",
                                  "launch": launch_mode(args),
                                  "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                  "time_step": f"CFL {w['cfl']:.6g} of Eq. (cfl), dt from the "
                                               "current subcell data every step"}),
        "fp64": {"value": stdofs * world / (f64["ms"] / 1e3), "ms_per_step": f64["ms"],
                 "dtype": "f64", "phases_ms": f64["phases"],
                 "predictor_shape": adg.PRED_NAMES[f64["info"]["predictor"]],
                 "roofline": {"bound": "alu", "achieved": achieved_f64,
                              "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": achieved_f64 / FP64_PEAK_TFLOPS}},
        "mixed_vs_fp64": m["mixed_vs_fp64"],
        "phases_ms": mx["phases"],
        "troubled_cells": mx["troubled"], "status": mx["status"],
        "troubled_per_step": mx["history"],
        "troubled_fraction_per_step": [c / cells for c in mx["history"]],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "pipe": pipe,
                     "kernel": "predictor (%s shape); bound by the %s pipe: its algorithmic flops "
                               "take the longer time at the derived peaks (FP64 %.3f, FP32 %.1f "
                               "TFLOP/s: 2 and 128 FMA per clock per SM at 2.07 GHz)"
                               % (shape, pipe.upper(), FP64_PEAK_TFLOPS, FP32_PEAK_TFLOPS),
                     "fp32_flops_per_launch": fl32 * cells,
                     "fp64_flops_per_launch": fl64 * cells,
                     "pipe_time_ms": {"fp64": t64 * 1e3, "fp32": t32 * 1e3},
                     "traffic": traffic["bytes_per_launch"] if traffic else None},
        "autotune_ms_per_launch": tune,
        "pipe_rates_measured": ({k: v for k, v in rates.items()} if rates else None),
        "e2e": e2e,
        "gpu_launches": int(mx["launches"]),
        "clocks": mx["clocks"],
    }
    if rates:
        # the same kernel against the measured pipe rate (adg_pipe_rates: FMA = 2 flop)
        meas = 2.0 * rates["dfma" if pipe == "fp64" else "ffma"] / 1e12
        line["roofline"]["peak_measured"] = meas
        line["roofline"]["frac_of_measured"] = achieved / meas
    if "dmp_floor" in m:
        line["dmp_floor"] = m["dmp_floor"]
    if subs:
        line["other_configs"] = subs
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_baseline(args.cpu_steps, 1, 32 if D == 2 else 6)
    print(json.dumps(line), flush=True)


def run_serving_solo(args):
    """Serving runs alone (ids from --serving-solo), each to min(--t-end, its
    final time) at the serving CFL number, in FP64, in mixed precision with
    the FP64 subcell scheme and in mixed precision: whether each reaches its
    end time, and how long it takes.  One JSON line per run and mode."""
    from paper_1406_7416_gb300 import adg, build_lib, inputs
    build_lib.build()
    adg.load_library()
    ids = [int(x) for x in args.serving_solo.split(",")]
    specs = inputs.serving_runs(count=max(args.runs, max(ids) + 1))
    modes = (("fp64", adg.PREC_FP64, {}),
             ("mixed_fp64_subcells", adg.PREC_MIXED_FP32,
              {adg.OPT_SUBCELL_FP32: 0, adg.OPT_SUBCELL_FP64_SWEEPS: 3}),
             ("mixed", adg.PREC_MIXED_FP32, {}))
    for rid in ids:
        w = specs[rid]
        t_end = min(w["t_end"], args.t_end)
        for name, prec, opts in modes:
            s = adg.Solver.from_workload(w, prec)
            for k, v in opts.items():
                s.set_option(k, v)
            s.set_option(adg.OPT_END_TIME, t_end)
            s.init_problem(w["problem"])
            t0 = time.perf_counter()
            ok = True
            try:
                while True:
                    for _ in range(64):
                        s.step_cfl(args.serving_cfl_factor * w["cfl"])
                    s.status()
                    if s.time()[0] >= t_end * (1 - 1e-12):
                        break
            except adg.AdgError:
                ok = False
            t, steps = s.time()
            print(json.dumps({"run": rid, "name": w["name"], "mode": name, "reached_end": ok,
                              "t": t, "t_end": t_end, "steps": steps,
                              "seconds": round(time.perf_counter() - t0, 2)}), flush=True)
            s.close()


def run_serving(args):
    """Serving: independent 2D runs (grids from {32,64,128,256}^2, N in {3,5},
    the 2D Riemann problems of Sec. 5.6 with seeded jitter, each to
    min(--t-end, its final time)) with Poisson arrivals, admitted by an HBM budget and
    stepped together in batched CUDA-graph launches; p50/p99 latency and the
    aggregate space-time DOF rate.  First a closed-loop pass (all runs at t=0)
    measures capacity, then an open-loop pass at 80% of it."""
    import torch
    from paper_1406_7416_gb300 import adg, build_lib, inputs
    from paper_1406_7416_gb300.serving import RunSpec, Server, poisson_arrivals
    build_lib.build()
    adg.load_library()
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.5 * free)
    specs = inputs.serving_runs(count=args.runs)
    for w in specs:
        w["t_end"] = min(w["t_end"], args.t_end)
        # runs of hundreds to thousands of steps take half the factor of
        # Eq. (cfl), as the paper's own long runs did (at the full factor the
        # one-step scheme's error grows over such runs)
        w["cfl"] *= args.serving_cfl_factor
    # capacity from a closed-loop pass (all runs at t = 0) over the first
    # --capacity-runs runs (all by default), scaled to the whole stream by work
    ncap = args.capacity_runs or len(specs)
    runs = [RunSpec(w, w["t_end"], 0.0, i) for i, w in enumerate(specs[:ncap])]
    retry = dict(retries=args.serving_retries,
                 retry_prec=adg.PREC_FP64 if args.serving_retry_prec == "fp64" else None,
                 retry_cfl_factor=args.serving_retry_cfl_factor)
    closed = Server(budget, adg.PREC_MIXED_FP32, **retry).serve(runs, max_wall=args.max_wall)
    print(json.dumps({"closed_loop": closed}), file=sys.stderr, flush=True)
    capacity = closed["runs"] / closed["wall_s"]
    rate = 0.8 * capacity
    # single-grid reference rates: one 256^2 run alone per degree, 20 CFL steps
    single = {}
    for N in (3, 5):
        w = inputs.riemann_2d(256, N, 3)
        sv = adg.Solver.from_workload(w, adg.PREC_MIXED_FP32)
        sv.init_problem(w["problem"])
        for _ in range(3):
            sv.step_cfl(w["cfl"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(20):
            sv.step_cfl(w["cfl"])
        sv.status()
        el = time.perf_counter() - t0
        single[f"256^2 N={N}"] = 256 * 256 * (N + 1) ** 3 * 20 / el
        sv.close()
    arrivals = poisson_arrivals(len(specs), rate, seed=1406 + 4)
    runs = [RunSpec(w, w["t_end"], a, i) for i, (w, a) in enumerate(zip(specs, arrivals))]
    opened = Server(budget, adg.PREC_MIXED_FP32, **retry).serve(runs, max_wall=args.max_wall)
    line = {"metric": METRIC, "value": opened["stdof_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": opened["steps"], "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"serving: {len(specs)} independent 2D Riemann-problem runs "
                                   f"(Sec. 5.6 RP1-RP5, 2% jitter), grids from "
                                   f"{{32,64,128,256}}^2, N in {{3,5}}, t_end={args.t_end}, "
                                   f"CFL {args.serving_cfl_factor} x 0.9/(d(2N+1)), "
                                   "Poisson arrivals at 80% of the measured capacity; "
                                   f"a failed run restarts in {args.serving_retry_prec} at "
                                   f"{args.serving_retry_cfl_factor} x its CFL number, "
                                   f"{args.serving_retries} time(s) at most",
                       "hbm_budget_bytes": budget, "mixed precision": True},
            "latency_p50_s": opened["latency_p50_s"], "latency_p99_s": opened["latency_p99_s"],
            "single_grid_rate": single, "closed_loop": closed, "open_loop": opened,
            "arrival_rate_per_s": rate, "capacity_runs": ncap}
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The oracle (plain FP64 CPU scheme) on the machine's host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload()
    block = 32 if w["dim"] == 2 else 6
    cb = run_cpu_baseline(args.steps, args.warmup, block, budget_s=120.0)
    rate = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w, {"sample": f"central {block}^d cells per step"}),
            "cpu_baseline": cb,
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if rate:
        d = w["dim"]
        line["ms_per_step"] = block ** d * (w["N"] + 1) ** (d + 1) / rate * 1e3
    print(json.dumps(line), flush=True)


def main():
    if len(sys.argv) >= 2 and sys.argv[1] == "--oracle-rate":
        steps, warmup, block = (int(x) for x in sys.argv[2:5])
        if len(sys.argv) > 5:
            globals()["WORKLOAD"] = sys.argv[5]
        budget = float(sys.argv[6]) if len(sys.argv) > 6 else 20.0
        print(json.dumps(list(oracle_rate(steps, warmup, block, budget_s=budget))))
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=15)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer timing")
    ap.add_argument("--host-passes", action="store_true",
                    help="plain kernel launches with host-sized limiter passes instead of one "
                         "CUDA graph per step (profilers skip kernels of graphs with "
                         "conditional nodes)")
    ap.add_argument("--grid", type=int, default=None,
                    help="cells per axis (profiling runs; default: the workload's own)")
    ap.add_argument("--only", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--predictor", type=int, default=None,
                    help="ADG_OPT_PREDICTOR of the mixed run (-1, -2 autotune; 0..4 a fixed shape)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations and the DMP floor comparison")
    ap.add_argument("--workload", default="quadvortex512",
                    choices=["quadvortex512", "explosion2d", "explosion3d", "quadrants200", "dmr",
                             "serving"])
    ap.add_argument("--runs", type=int, default=32, help="serving: number of runs")
    ap.add_argument("--t-end", type=float, default=0.02,
                    help="serving: end time cap of every run (each stops at min(cap, its final time))")
    ap.add_argument("--serving-retries", type=int, default=0,
                    help="serving: restarts of a failed run (see --serving-retry-*)")
    ap.add_argument("--serving-retry-prec", default="fp64", choices=["fp64", "same"],
                    help="serving: precision of a restarted run")
    ap.add_argument("--serving-retry-cfl-factor", type=float, default=1.0,
                    help="serving: factor on a restarted run's CFL number")
    ap.add_argument("--serving-cfl-factor", type=float, default=0.5,
                    help="serving: fraction of the CFL number of Eq. (cfl) the runs take")
    ap.add_argument("--capacity-runs", type=int, default=0,
                    help="serving: runs of the closed-loop capacity pass (0: all)")
    ap.add_argument("--serving-solo", default="",
                    help="serving: comma-separated run ids to run alone in FP64, mixed with FP64 "
                         "subcells and mixed, each to its end time")
    ap.add_argument("--max-wall", type=float, default=120.0,
                    help="serving: no admissions after this many seconds per pass")
    args = ap.parse_args()
    globals()["GRID"] = args.grid or GRID
    globals()["GRID_SET"] = args.grid
    globals()["WORKLOAD"] = args.workload
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving" and args.serving_solo:
        run_serving_solo(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
