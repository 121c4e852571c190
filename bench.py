#!/usr/bin/env python
"""Throughput of one full ADER-DG + subcell-limiter time step on GB300.

Workload: 2D Euler, N = 5 (Ns = 11), 512 x 512 periodic cells on [-5, 5]^2,
seeded four-quadrant Riemann data with a superposed isentropic vortex
(strength 5) -- the paper's 2D Riemann / vortex test shapes (Sec. 5.2, 5.6).
A step is one adg_step: predictor, corrector, detection, subcell ADER-WENO3
of troubled cells, reconstruction and neighbour flux correction.

Metric: space-time DOF updates per second = cells * (N+1)^(d+1) * steps / s
(per conserved variable, as the paper counts).  `value` is the mixed-precision
path (FP32 Picard sweeps + one FP64 sweep); the FP64 path is reported beside
it, with the L1 distance between the two after the same steps.

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
METRIC = "space-time DOF updates/s"
UNIT = "ST-DOF/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz


def workload(n=None, N=N_ORDER):
    from paper_1406_7416_gb300 import inputs
    return inputs.quadrants_vortex_2d(n=n or GRID, N=N, steps=None)


def config_dict(w, extra=None):
    c = {"workload": w["name"], "grid": f"{w['ncell'][0]}x{w['ncell'][1]}", "N": w["N"],
         "cells": int(w["ncell"][0] * w["ncell"][1]), "dim": w["dim"],
         "l2": "inputs larger than L2: DOF state 302 MB and face traces 1.2 GB per step"}
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


def predictor_flops(D, N, iters, mixed):
    """(fp64, fp32) flops of the predictor kernel for one cell."""
    n, nv = N + 1, D + 2
    nst, nd = n ** (D + 1), n ** D
    it = nst * flux_flops(D) + nv * nst * D * (2 * n + 2) + nv * nd * n * (2 * n + 1)
    final = (nst * flux_flops(D) + D * nv * nd * 2 * n + nv * nd * D * (2 * n + 2)
             + 2 * D * nv * n ** (D - 1) * n * 2 * n)
    n32 = (iters - 1) if mixed and iters > 1 else 0
    return (iters - n32) * it + final, n32 * it


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
    src = os.path.join(ROOT, "paper_1406_7416_gb300", "csrc", "kernels_dg.cuh")
    try:
        rec = json.load(open(path))
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("kernels_dg_sha256") == h:
            return rec
    except (OSError, ValueError):
        pass
    return None


# ---------------------------------------------------------------------------
# CPU oracle timing (test infrastructure, timed as a baseline only)
# ---------------------------------------------------------------------------
def oracle_sample(block=32):
    """The central block x block cells of the workload (quadrant corner and
    vortex core), transmissive at the block edges, projected by the oracle."""
    from oracle.dg import Grid
    from oracle.ic import initial_state, project_problem
    from oracle.step import Scheme
    w = workload()
    i0 = GRID // 2 - block // 2
    x0 = tuple(w["x0"][k] + i0 * w["dx"][k] for k in range(2))
    g = Grid((block, block), x0, w["dx"], (1, 1, 1, 1))
    sch = Scheme(g, w["N"], w["gamma"])
    U0, V0 = project_problem(sch, w["problem"])
    return w, sch, initial_state(sch, U0, V0)


def oracle_rate(steps, warmup, block=32):
    from oracle.step import stable_dt, step
    w, sch, st = oracle_sample(block)
    dt = stable_dt(sch, st, w["cfl"])
    for _ in range(warmup):
        st, _ = step(sch, st, dt)
    t0 = time.perf_counter()
    for _ in range(steps):
        st, _ = step(sch, st, dt)
    el = time.perf_counter() - t0
    dofs = block * block * (w["N"] + 1) ** 3
    return dofs * steps / el, el


def run_cpu_baseline(steps, warmup, block):
    """Times the oracle in a child process pinned to one BLAS thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-rate",
                        str(steps), str(warmup), str(block)], env=env, capture_output=True,
                       text=True, timeout=1800)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"failed: {r.stderr.strip()[-300:]}"}
    rate, el = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} oracle steps (after {warmup} warm-up) on the central "
                      f"{block}x{block} cells of the same workload, transmissive block edges, "
                      f"{el:.1f} s, one BLAS thread"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch
    from paper_1406_7416_gb300 import adg, build_lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build_lib.build()
    if dist:
        dist.barrier()
    adg.load_library()
    w = workload()
    D, N = w["dim"], w["N"]
    n = N + 1
    cells = w["ncell"][0] * w["ncell"][1]
    stdofs = cells * n ** (D + 1)
    stream = torch.cuda.Stream()

    def make(prec):
        s = adg.Solver.from_workload(w, prec)
        s.set_stream(stream.cuda_stream)
        s.init_problem(w["problem"])
        return s

    def barrier():
        if dist:
            dist.barrier()

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    results = {}
    fixed_dt = None
    precs = [("fp64", adg.PREC_FP64), ("mixed", adg.PREC_MIXED_FP32)]
    if args.only != "both":
        precs = [p for p in precs if p[0] == args.only]
    for name, prec in precs:
        s = make(prec)
        if fixed_dt is None:
            fixed_dt = s.max_dt(w["cfl"])          # same dt sequence for both precisions
        s.set_option(adg.OPT_PROFILE, 1)
        for _ in range(args.warmup):
            s.step(fixed_dt)
        s.phase_times()                             # discard warm-up phases
        torch.cuda.synchronize()
        barrier()
        clk = clocks_sampler() if (name == "mixed" and rank == 0) else None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            s.step(fixed_dt)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / args.steps
        clocks = clocks_summary(clk, local) if clk is not None else None
        phases, nsteps = s.phase_times()
        status = s.status()
        troubled = s.troubled_count()
        info = s.info()
        results[name] = dict(ms=max_over_ranks(ms), solver=s, phases={k: v / nsteps for k, v in phases.items()},
                             status=status, troubled=troubled, info=info, clocks=clocks)
    if args.only != "both":
        # profiling run of one precision: timings only
        if rank == 0:
            r = results[args.only]
            print(json.dumps({"profile_run": args.only, "ms_per_step": r["ms"],
                              "phases_ms": r["phases"], "troubled_cells": r["troubled"],
                              "config": config_dict(w)}), flush=True)
        for r in results.values():
            r["solver"].close()
        return
    # L1 distance of the density, mixed vs FP64, after warmup + steps equal steps
    W = 0.5 * np.polynomial.legendre.leggauss(n)[1]
    Wd = np.outer(W, W).ravel()
    rho64 = results["fp64"]["solver"].read()[:, 0, :]
    rhomx = results["mixed"]["solver"].read()[:, 0, :]
    area = w["dx"][0] * w["dx"][1]
    l1 = float(np.sum(np.abs(rhomx - rho64) @ Wd) * area)
    l1ref = float(np.sum(np.abs(rho64) @ Wd) * area)

    # end-to-end through the C ABI with host buffers (rank-local)
    e2e = None
    s = results["mixed"]["solver"]
    dofs, beta, sub = s.read_full()
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    hd, hb, hs = pin(dofs), pin(beta), pin(sub)
    flags = pin(np.empty(s.cells, dtype=np.uint8))
    out = pin(np.empty_like(dofs))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    s.load_full(hd, hb, hs)
    for _ in range(args.steps):
        s.step(fixed_dt)
        s.lib.adg_flags(s.h, adg._u8ptr(flags))
    s.read(out)
    el = max_over_ranks(time.perf_counter() - t0)
    h2d = (hd.nbytes + hb.nbytes + hs.nbytes) / args.steps + 8
    d2h = flags.nbytes + out.nbytes / args.steps
    e2e = {"value": stdofs * args.steps * world / el, "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "timed": "adg_load_full from pinned host, then per step adg_step(dt) + adg_flags to "
                    "pinned host, then adg_read of the DOFs"}

    if rank == 0:
        mx, f64 = results["mixed"], results["fp64"]
        value = stdofs * world / (mx["ms"] / 1e3)
        iters = N + 1
        fl64, fl32 = predictor_flops(D, N, iters, True)
        pred_ms = mx["phases"]["predictor"]
        achieved = fl64 * cells / (pred_ms / 1e3) / 1e12
        fl64f, _ = predictor_flops(D, N, iters, False)
        achieved_f64 = fl64f * cells / (f64["phases"]["predictor"] / 1e3) / 1e12
        traffic = traffic_record()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mx["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": config_dict(w, {"precision": "mixed: FP32 Picard sweeps + final FP64 sweep, "
                                                   "FP64 corrector/detector/limiter",
                                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                      "dt": fixed_dt}),
            "fp64": {"value": stdofs * world / (f64["ms"] / 1e3), "ms_per_step": f64["ms"],
                     "dtype": "f64", "phases_ms": f64["phases"],
                     "roofline": {"bound": "alu", "achieved": achieved_f64,
                                  "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                  "frac": achieved_f64 / FP64_PEAK_TFLOPS}},
            "mixed_vs_fp64": {"l1_density": l1, "l1_density_rel": l1 / l1ref,
                              "steps": args.warmup + args.steps},
            "phases_ms": mx["phases"],
            "troubled_cells": mx["troubled"], "status": mx["status"],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                         "kernel": "k_predictor (FP64 pipe: final sweep + corrector terms)",
                         "fp32_flops_per_launch": fl32 * cells,
                         "fp64_flops_per_launch": fl64 * cells,
                         "traffic": traffic["bytes_per_launch"] if traffic else None},
            "e2e": e2e,
            "gpu_launches": int(mx["info"]["launches_per_step"]) * args.steps,
            "clocks": mx["clocks"],
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = run_cpu_baseline(args.cpu_steps, 1, 32)
        print(json.dumps(line), flush=True)
    for r in results.values():
        r["solver"].close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    """The oracle (plain FP64 CPU scheme) on the machine's host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload()
    block = 32
    rate, el = oracle_rate(args.steps, args.warmup, block)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w, {"sample": f"central {block}x{block} cells per step"}),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} oracle steps on the central {block}x{block} "
                                       f"cells of the workload (numpy, default threads)"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    if len(sys.argv) >= 2 and sys.argv[1] == "--oracle-rate":
        steps, warmup, block = (int(x) for x in sys.argv[2:5])
        print(json.dumps(oracle_rate(steps, warmup, block)))
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=15)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, default=GRID, help="cells per axis (profiling runs)")
    ap.add_argument("--only", default="both", choices=["both", "mixed", "fp64"])
    args = ap.parse_args()
    globals()["GRID"] = args.grid
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
