#!/usr/bin/env python
"""Benchmark: cell-steps per second of the biofilm IBM time step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config c3]
                    [--impl ours|reference]

One step is one full time step of the method (momentum right-hand side,
viscous multigrid solve, divergence, pressure multigrid solve, projection,
interpolation and node move, springs, spreads, coefficient hierarchy) on the
chosen synthetic workload, replayed from a CUDA graph. ``value`` is
(cells x steps x ranks) / device time with every input resident on the GPU;
``e2e`` repeats the run through the public C ABI from host buffers (context
creation and node/spring upload included, node positions read back after
every step, fields read back at the end). Multi-GPU runs are independent
replicas (a single simulation does not shard): one process per GPU under
torchrun, max-over-ranks time.

``--impl reference`` times the FP64 CPU oracle (OpenMP, all host cores) on the
same workload and prints the same JSON line with "impl": "reference".
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s & V-cycle HBM roofline frac; served p50/p99 step latency vs FP64"
UNIT = "cell-steps/s"

# Solves run to a relative residual of 1e-11, which leaves max |div u| below
# 1e-10 after every projection; coarse-grid viscosity scaled by gamma = 0.8
# (Eq. ViscCoarseGrid, inside the recommended [0.7, 1]); V(3,3) cycles.
# Mixed precision only (the FP64 path ignores both): inner_cycles FP32
# V-cycles per FP64 residual, and krylov = 1 puts the viscous solve's FP32
# V-cycles inside a flexible conjugate-gradient iteration in FP64
TOL_SOLVER = {"vc_visc": 0, "vc_p": 0, "rtol": 1e-11, "max_cycles": 100, "gamma_coarse": 0.8,
              "nu1": 2, "nu2": 2, "inner_cycles": 2, "krylov": 1, "div_tol": 1e-10}
# the same with plain defect correction (3 V(3,3) cycles per FP64 residual)
DC_SOLVER = dict(TOL_SOLVER, nu1=3, nu2=3, inner_cycles=3, krylov=0)
DIV_TARGET = 1e-10
# ncu capture of the FP32 viscous sweep on the 128x128x256 grid (mean of the
# three components' dram__bytes_read.sum + dram__bytes_write.sum per launch)
# in the shape the autotuner chose (tile rows, planes per chunk, planes per
# phase, threads per row, kernel); claimed only while the tuner picks it
PROFILED_SWEEP_SHAPE = (6, 20, 1, 0, 1)
PROFILED_SWEEP_TRAFFIC = 171.8e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="c3")
    ap.add_argument("--precision", type=int, default=None,
                    help="0: FP64; 1: FP32 V-cycles in FP64 defect correction "
                         "(default: the workload's own, 1 for c3)")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain FP64 single-instance comparison run")
    ap.add_argument("--no-served", action="store_true",
                    help="skip the served-stream block of the default run")
    ap.add_argument("--instances", type=int, default=64, help="c4: batched instances")
    ap.add_argument("--requests", type=int, default=None, help="c5: requests served")
    ap.add_argument("--request-steps", type=int, default=None, help="c5: steps per request")
    ap.add_argument("--budget-frac", type=float, default=0.05,
                    help="c5: admission budget as a fraction of free device memory")
    ap.add_argument("--solver", choices=["tol", "fixed"], default="tol",
                    help="tol: V-cycles until max |div u| <= 1e-10 (relative residual "
                         "1e-11); fixed: the workload's own fixed V-cycle counts")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel directly instead of replaying the step graph "
                         "(same kernels; for profilers that cannot enter graphs with "
                         "conditional nodes)")
    ap.add_argument("--tma", type=int, choices=[0, 1, 2], default=1,
                    help="FP32 sweeps with TMA-staged inputs: 0 never, 1 where the autotuner "
                         "timed them faster (default), 2 wherever a level allows")
    ap.add_argument("--study", choices=["gamma", "work_units", "refinement"], default=None,
                    help="gamma: tune the coarse viscosity scaling per level (Eq. "
                         "ViscCoarseGrid) on the workload and time a step before and after; "
                         "work_units: cycles and work units of one solve against the number "
                         "of multigrid levels (Sec. 4.3.1); refinement: convergence rates in "
                         "time and space (Sec. 4.3.2-4.3.3) on the GPU")
    ap.add_argument("--save-plans", default=None,
                    help="write the FP32 sweep choices the autotuner made (JSON) after the "
                         "context is created")
    ap.add_argument("--load-plans", default=None,
                    help="pin FP32 sweep choices written by --save-plans instead of this "
                         "process's own tuning (a profiler distorts the tuner's timings)")
    ap.add_argument("--no-tune-gamma", action="store_true",
                    help="keep one coarse viscosity scaling for every level instead of tuning "
                         "it per level before the timed region")
    ap.add_argument("--forms", default="persistent,replay,fp64",
                    help="batched sweep: which of persistent, replay, fp64 to run")
    ap.add_argument("--unroll", type=int, default=0,
                    help="persistent batch: solve loops unrolled to this many iterations "
                         "(for a profiler that cannot see inside conditional graph nodes)")
    ap.add_argument("--tail", type=int, default=None,
                    help="cell threshold of the coarse-level cluster kernel (0: a launch per "
                         "phase on every level)")
    ap.add_argument("--batch-tail", type=int, default=None,
                    help="persistent batch: cell threshold of its coarse-level kernel (0: none)")
    ap.add_argument("--save-batch-shapes", default=None,
                    help="write the persistent batch's tuned sweep shapes to this JSON file")
    ap.add_argument("--load-batch-shapes", default=None,
                    help="pin the persistent batch's sweep shapes from this JSON file")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched sweep (64 uneven ducts, persistent vs replay)")
    ap.add_argument("--no-open", action="store_true",
                    help="skip the open-duct block of the default run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def solver_override(args):
    return dict(TOL_SOLVER) if args.solver == "tol" else {}


def load_workload(name, precision, args=None):
    from paper_1302_3663_gb300 import workloads as W
    inst = W.CONFIGS[name]()
    if precision is not None:
        inst["params"]["precision"] = precision
    if args is not None:
        inst["params"].update(solver_override(args))
    return inst


def describe(inst):
    from paper_1302_3663_gb300 import workloads as W
    p = inst["params"]
    n = p["n"][:p["dim"]]
    prec = ("fp64" if p.get("precision", 0) == 0 else
            "fp32 V-cycles in fp64 flexible CG (viscous) and defect correction (pressure)"
            if p.get("krylov", 0) else "fp32 V-cycles in fp64 defect correction")
    gl = [g for g in p.get("gamma_levels", [])[1:] if g > 0]
    vc = ("%d viscous + %d pressure V(%d,%d) cycles per step" %
          (p["vc_visc"], p["vc_p"], p["nu1"], p["nu2"]) if p["vc_visc"] > 0
          else "V(%d,%d) cycles until the relative residual is %.0e, coarse viscosity x %s%s%s"
          % (p["nu1"], p["nu2"], p["rtol"],
             ("%s per level (tuned)" % gl) if gl else "%g" % p["gamma_coarse"],
             (", %d FP32 V-cycles per FP64 residual" % p["inner_cycles"])
             if p.get("precision", 0) == 1 and p.get("inner_cycles", 1) > 1 else "",
             ", viscous solve: flexible CG in FP64 preconditioned by the FP32 V-cycles"
             if p.get("precision", 0) == 1 and p.get("krylov", 0) else ""))
    return {
        "workload": "%s: %s grid, %d nodes, %d springs, density ratio %g, viscosity ratio %g"
                    % (inst["name"], "x".join(map(str, n)), inst["X"].shape[0],
                       inst["ab"].shape[0], p["rho_ratio"], p["mu_ratio"]),
        "cells": W.cells(p),
        "precision": prec,
        "solver": vc,
        "dt": p["dt"],
        "parallelism": "replicas (one independent simulation per GPU)",
    }


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s)"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    """One process per GPU (torchrun's RANK / LOCAL_RANK / WORLD_SIZE): NCCL on
    GPUs; gloo where no GPU is visible (the host-side logic of the replica
    runs, which the CPU tests exercise)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    gpu = torch.cuda.is_available()
    if world > 1:
        import torch.distributed as dist
        if gpu:
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if gpu else "gloo")
    elif gpu:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def max_over_ranks(world, v):
    """The slowest rank's value (every rank gets it)."""
    import torch
    if world == 1:
        return v
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(cells, steps, world, ms_max):
    """Whole-job cell-steps per second of `world` independent replicas: the
    units every rank processed over the slowest rank's time."""
    return cells * steps * world / (ms_max / 1e3)


def alg_bytes_visc_sweep(dim, cells, elem):
    # one sweep of one component: u_d (read + write), rhs_d, m_d, mu_c, and per
    # other axis one edge-mu array and one cross component
    return (5 + 2 * (dim - 1)) * elem * cells


def cpu_baseline(inst, max_seconds=30.0):
    """The oracle as it stands, on the host cores: one time step of the same
    workload (a bounded sample), cell-steps per second."""
    from oracle import oracle as O
    from paper_1302_3663_gb300 import workloads as W
    prm = dict(inst["params"], precision=0)
    o = O.Oracle(prm, omp=True)
    o.set_nodes(inst["X"])
    o.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
    o.refresh()
    t0 = time.perf_counter()
    steps = 0
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el > max_seconds / 2 or steps >= 3:
            break
    cells = W.cells(prm)
    return {"value": cells * steps / el, "unit": UNIT, "cores": O.num_threads(True),
            "kind": "oracle",
            "sample": "%d full time step(s) of %s in FP64 (OpenMP oracle, %.1f s)"
                      % (steps, inst["name"], el)}


def timed_steps(ctx, stream, steps, world, label="timed"):
    """Device time (ms) of `steps` time steps replayed on `stream` (inside an
    NVTX range named `label`, so a profiler can select exactly these)."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.nvtx.range_push(label)
    e0.record(stream)
    ctx.step(steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    return max_over_ranks(world, e0.elapsed_time(e1))


def final_stats(ctx):
    """One more (untimed) step with statistics on: V-cycles of each solve,
    relative residuals and max |div u| after the projection."""
    from paper_1302_3663_gb300 import bfibm
    ctx.set_option(bfibm.OPT_STATS, 1)
    ctx.step(1)
    st = ctx.get_stats()
    return {"div_max": st["div_max"], "cycles_visc": st["cycles_visc"],
            "cycles_p": st["cycles_p"], "res_visc": st["res_visc"], "res_p": st["res_p"],
            "kinetic": st["kinetic"], "broken": st["broken_total"],
            "wait_timeouts": st["wait_timeouts"]}


def step_checks(ctx):
    """What the device recorded inside every step so far: the largest max
    |div u| of any projection, projections above div_tol, solves that stopped
    above their tolerance."""
    st = ctx.get_stats()
    return {"div_max_all_steps": st["div_max_steps"], "div_violations": st["div_violations"],
            "nonconverged_solves": st["nonconv_total"], "steps": st["step"]}


def sweep_roofline(ctx, stream, prm, cells):
    """The dominant kernel: one red-black sweep of one viscous component on
    the finest grid (FP32 in the mixed path, FP64 otherwise), timed alone with
    events on the context's stream."""
    import torch
    peak, peak_src = measured_peak()
    sweeps = 10
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    if prm.get("precision", 0) == 1:
        ctx.smooth_f32(1, 0, 2, sync=True)
        torch.cuda.nvtx.range_push("sweep")
        k0.record(stream)
        ctx.smooth_f32(1, 0, sweeps, sync=False)
        k1.record(stream)
        k1.synchronize()
        torch.cuda.nvtx.range_pop()
        nlaunch = sweeps * prm["dim"]
        alg = alg_bytes_visc_sweep(prm["dim"], cells, 4)
        plans = [ctx.tma_plan(0, d) for d in range(prm["dim"])]
        kinds = {(ctx.sweep_shape(0, d) or (0,) * 5)[4] for d in range(prm["dim"])}
        if any(p is not None for p in plans) or len(kinds) > 1:
            kname = ("k_rb_tma / k_v_rb_fused<float> / k_v_rb_pair (red-black sweep of one "
                     "viscous component, FP32, finest grid; per component the autotuned choice)")
        elif kinds == {1}:
            kname = ("k_v_rb_pair (pair red-black sweep of one viscous component, FP32, finest "
                     "grid: a thread per (red, black) pair of a row marching over the planes)")
        else:
            kname = ("k_v_rb_fused<float> (one-pass red-black sweep of one viscous component, "
                     "FP32, finest grid, inputs read from global memory)")
    else:
        ctx.smooth_viscous(0, 2, sync=True)
        torch.cuda.nvtx.range_push("sweep")
        k0.record(stream)
        ctx.smooth_viscous(0, sweeps, sync=False)
        k1.record(stream)
        k1.synchronize()
        torch.cuda.nvtx.range_pop()
        nlaunch = sweeps * 2 * prm["dim"]
        alg = alg_bytes_visc_sweep(prm["dim"], cells, 8) / 2.0
        plans = None
        kname = "k_v_rbgs<double> (one colour of one viscous component, FP64, finest grid)"
    launch_s = k0.elapsed_time(k1) / 1e3 / nlaunch
    achieved = alg / launch_s / 1e9
    roof = {"kernel": kname, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
            "alg_bytes_per_launch": alg, "launch_us": round(launch_s * 1e6, 2),
            "peak_source": peak_src}
    if plans is not None:
        roof["tma_plans"] = {"viscous_%d" % d: p for d, p in enumerate(plans)}
        roof["tma_plans"]["pressure"] = ctx.tma_plan(0, 3)
        # (tile rows, planes per chunk, planes per phase, threads per row)
        shapes = [ctx.sweep_shape(0, d) for d in range(prm["dim"])]
        roof["sweep_shapes"] = {"viscous_%d" % d: sh for d, sh in enumerate(shapes)}
        roof["sweep_shapes"]["pressure"] = ctx.sweep_shape(0, 3)
        # DRAM bytes per launch (read + write) from the ncu capture of this
        # kernel on this grid in the tuned shape; not claimed for any other
        if (prm["n"] == [128, 128, 256] and all(p is None for p in plans)
                and all(tuple(sh or ()) == PROFILED_SWEEP_SHAPE for sh in shapes)):
            roof["traffic"] = PROFILED_SWEEP_TRAFFIC
    return roof


def run_ours(args):
    import torch

    from paper_1302_3663_gb300 import bfibm, workloads as W

    world, rank, local = dist_setup(args)
    inst = load_workload(args.config, args.precision, args)
    prm = inst["params"]
    cells = W.cells(prm)
    stream = torch.cuda.Stream()
    ctx = bfibm.load_instance(inst, stream=stream)
    ctx.set_option(bfibm.OPT_STATS, 0)
    if args.no_graph:
        ctx.set_option(bfibm.OPT_GRAPH, 0)
    ctx.set_option(bfibm.OPT_TMA, args.tma)
    if args.tail is not None:
        ctx.set_option(bfibm.OPT_TAIL, args.tail)
    if args.load_plans:
        with open(args.load_plans) as f:
            ctx.pin_sweep_plans(json.load(f))
    if args.save_plans:
        with open(args.save_plans, "w") as f:
            json.dump(ctx.sweep_plans(), f)
    ctx.step(args.warmup)
    ctx.synchronize()
    if args.solver == "tol" and not args.no_tune_gamma:
        # gamma_lh of Eq. (ViscCoarseGrid) per coarse level, tuned on this
        # state before the timed region (the plain FP64 comparison reuses it)
        from paper_1302_3663_gb300 import tuning
        ctx.set_option(bfibm.OPT_GRAPH, 0)
        gl, _, _ = tuning.tune_gamma(ctx)
        ctx.set_option(bfibm.OPT_GRAPH, 0 if args.no_graph else 1)
        ctx.set_option(bfibm.OPT_STATS, 0)
        prm["gamma_levels"] = gl
        inst["params"]["gamma_levels"] = gl
        ctx.step(1)
        ctx.synchronize()
    lc0 = ctx.launch_counts()
    with Clocks(local) as clk:
        ms = timed_steps(ctx, stream, args.steps, world)
    lc1 = ctx.launch_counts()
    checks = step_checks(ctx)
    value = replica_throughput(cells, args.steps, world, ms)
    # kernels launched in the timed region: top-level graph nodes per step plus
    # the loop bodies times the iterations the device ran
    launches = None
    if lc1["top"] > 0:
        launches = (args.steps * lc1["top"] +
                    (lc1["iters_visc"] - lc0["iters_visc"]) * lc1["body_visc"] +
                    (lc1["iters_p"] - lc0["iters_p"]) * lc1["body_p"])
    roof = sweep_roofline(ctx, stream, prm, cells)
    fin = final_stats(ctx)
    ctx.close()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if prm.get("precision", 0) == 0 else "f64+f32",
           "data": "synthetic (seeded mounds standing in for the measured S. epidermidis "
                   "coordinates)",
           "config": dict(describe(inst), l2="working set larger than L2 (%.2f GB of grids); "
                          "no flush" % (bfibm.footprint(prm, inst['X'].shape[0],
                                                        inst['ab'].shape[0]) / 1e9)),
           "roofline": roof, "clocks": clk.summary(),
           "gpu_launches": launches,
           "final_stats": fin, "step_checks": checks}
    if args.solver == "tol":
        out["config"]["div_target"] = DIV_TARGET
        # checked inside every step (warm-up and timed), on the device
        out["div_target_met"] = (checks["div_max_all_steps"] <= DIV_TARGET and
                                 checks["div_violations"] == 0)

    if not args.no_fp64 and prm.get("precision", 0) == 1:
        out["fp64_single_instance"] = run_fp64(inst, args, world, stream)
    if args.solver == "tol" and prm.get("precision", 0) == 1 and prm.get("krylov", 0):
        out["mixed_defect_correction"] = run_dc(inst, args, world, stream)
    if args.solver == "tol":
        out["fixed_3_vcycles"] = run_fixed(inst, args, world, stream)
    if args.solver == "tol" and not args.no_open:
        out["open_duct"] = run_open(args, world, stream)
    if not args.no_e2e:
        out["e2e"] = run_e2e(inst, args, world, stream)
    if not args.no_batched and args.solver == "tol" and prm.get("precision", 0) == 1:
        out["batched"] = batched_forms(args, 64, 50, world, fp64_subset=8)
    if not args.no_served:
        # a reduced c5 stream: its first 16 requests (Poisson arrivals, mean 4 per
        # second) for 20 steps each instead of 128 requests for 200 steps
        nreq, nst = args.requests or 16, args.request_steps or 20
        out["served"] = run_served_stream(nreq, nst, args.budget_frac, fp64_subset=4,
                                          solver=solver_override(args))
        out["served"]["stream"] = ("reduced c5 stream: %d of its 128 requests, %d of its 200 "
                                   "steps each" % (nreq, nst))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(inst)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_fixed(inst, args, world, stream):
    """The same workload with 3 V-cycles per solve (no convergence check): the
    throughput of the loosest setting, for context."""
    from paper_1302_3663_gb300 import bfibm, workloads as W
    prm = dict(inst["params"], vc_visc=3, vc_p=3, nu1=2, nu2=2, gamma_coarse=1.0,
               gamma_levels=[], inner_cycles=1, krylov=0)
    ctx = bfibm.load_instance(dict(inst, params=prm), stream=stream)
    ctx.set_option(bfibm.OPT_STATS, 0)
    ctx.step(args.warmup)
    ctx.synchronize()
    steps = max(args.steps, 10)
    ms = timed_steps(ctx, stream, steps, world, "timed_fixed")
    fin = final_stats(ctx)
    ctx.close()
    return {"value": W.cells(prm) * steps * world / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / steps, "div_max": fin["div_max"]}


def run_open(args, world, stream):
    """The open duct of Sec. 3.6 (laminar inflow, du/dn = 0 and the pressure
    held at the outflow): the 64 x 64 x 128 tube with the 64^3 duct's mound,
    FP64, solves to the benchmark's tolerance and divergence target."""
    from paper_1302_3663_gb300 import bfibm, workloads as W
    inst = W.open_duct(e=64)
    prm = dict(inst["params"], **{k: v for k, v in TOL_SOLVER.items()
                                  if k not in ("inner_cycles", "krylov")})
    ctx = bfibm.load_instance(dict(inst, params=prm), stream=stream)
    ctx.set_option(bfibm.OPT_STATS, 0)
    ctx.step(args.warmup)
    ctx.synchronize()
    steps = max(args.steps, 10)
    ms = timed_steps(ctx, stream, steps, world, "timed_open")
    chk = step_checks(ctx)
    fin = final_stats(ctx)
    ctx.close()
    return {"workload": "open duct 64x64x128 (side 1, length 2), %d nodes, %d springs, density "
                        "ratio %g, viscosity ratio %g, FP64" % (inst["X"].shape[0],
                                                                inst["ab"].shape[0],
                                                                prm["rho_ratio"], prm["mu_ratio"]),
            "value": W.cells(prm) * steps * world / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / steps, "step_checks": chk, "cycles_visc": fin["cycles_visc"],
            "cycles_p": fin["cycles_p"]}


def run_dc(inst, args, world, stream):
    """Mixed precision with plain defect correction (no conjugate gradients)
    on the same workload, tolerance and coarse scaling."""
    from paper_1302_3663_gb300 import bfibm, workloads as W
    prm = dict(inst["params"], **{k: DC_SOLVER[k] for k in ("nu1", "nu2", "inner_cycles",
                                                             "krylov")})
    ctx = bfibm.load_instance(dict(inst, params=prm), stream=stream)
    ctx.set_option(bfibm.OPT_STATS, 0)
    ctx.step(args.warmup)
    ctx.synchronize()
    ms = timed_steps(ctx, stream, args.steps, world, "timed_dc")
    fin = final_stats(ctx)
    ctx.close()
    return {"value": W.cells(prm) * args.steps * world / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "div_max": fin["div_max"],
            "cycles_visc": fin["cycles_visc"], "cycles_p": fin["cycles_p"],
            "solver": "V(3,3), 3 FP32 V-cycles per FP64 residual, no conjugate gradients"}


def run_fp64(inst, args, world, stream):
    """The plain FP64 single-instance path on the same workload, solver
    settings and step count, for comparison at equal final divergence."""
    from paper_1302_3663_gb300 import bfibm, workloads as W
    prm = dict(inst["params"], precision=0)
    ctx = bfibm.load_instance(dict(inst, params=prm), stream=stream)
    ctx.set_option(bfibm.OPT_STATS, 0)
    ctx.step(args.warmup)
    ctx.synchronize()
    ms = timed_steps(ctx, stream, args.steps, world, "timed_fp64")
    fin = final_stats(ctx)
    ctx.close()
    return {"value": W.cells(prm) * args.steps * world / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "div_max": fin["div_max"],
            "cycles_visc": fin["cycles_visc"], "cycles_p": fin["cycles_p"]}


def run_e2e(inst, args, world, stream):
    """The same run through the public API from host buffers."""
    import numpy as np
    import torch

    from paper_1302_3663_gb300 import bfibm, workloads as W
    prm = inst["params"]
    cells = W.cells(prm)
    eta, dim = inst["X"].shape
    pinned = torch.empty((eta, dim), dtype=torch.float64, pin_memory=True).numpy()
    Xh = torch.empty((eta, dim), dtype=torch.float64, pin_memory=True).numpy()
    Xh[:] = inst["X"]
    barrier(world)
    t0 = time.perf_counter()
    ctx = bfibm.Context(prm, stream=stream)
    ctx.set_option(bfibm.OPT_STATS, 0)
    ctx.set_nodes(Xh)
    ctx.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
    for k in range(args.steps):
        ctx.step(1)
        ctx.get_nodes(pinned)
    fields = [ctx.get_velocity(d) for d in range(dim)] + [ctx.get_pressure()]
    ctx.close()
    el = time.perf_counter() - t0
    el = max_over_ranks(world, el)
    h2d = (Xh.nbytes + inst["ab"].nbytes + 3 * inst["rest"].nbytes) / args.steps
    d2h = pinned.nbytes + sum(f.nbytes for f in fields) / args.steps
    return {"value": cells * args.steps * world / el, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "note": "context creation, node/spring upload, every step's node positions "
                    "read back, final u and p read back; wall clock"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1302_3663_gb300 import workloads as W
    inst = load_workload(args.config, 0, args)
    prm = inst["params"]
    cells = W.cells(prm)
    o = O.Oracle(prm, omp=True)
    o.set_nodes(inst["X"])
    o.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
    o.refresh()
    # each step is one full oracle time step of the workload; the count is
    # bounded so that the whole run stays within a few minutes
    t_one = time.perf_counter()
    o.step(1)
    t_one = time.perf_counter() - t_one
    budget = 150.0
    k_timed = max(1, min(args.steps, int(budget / max(t_one, 1e-3)) - args.warmup))
    k_warm = max(0, min(args.warmup - 1, int(budget / max(t_one, 1e-3)) - k_timed - 1))
    o.step(k_warm)
    t0 = time.perf_counter()
    o.step(k_timed)
    el = time.perf_counter() - t0
    value = cells * k_timed / el
    cores = O.num_threads(True)
    sample = ("%d timed oracle time steps of %s (after %d warm-up), FP64, OpenMP"
              % (k_timed, inst["name"], k_warm + 1))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": world, "steps": k_timed, "warmup": k_warm + 1,
           "ms_per_step": el / k_timed * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": describe(inst),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_served_stream(nreq, steps, budget_frac, fp64_subset=None, solver=None, persistent=False):
    """A bounded Poisson stream of duct requests through the continuous-
    batching service, and the same requests run one after another alone in
    plain FP64 and in mixed precision (same solver settings)."""
    import torch

    from paper_1302_3663_gb300 import serve, workloads as W
    arr = W.c5_arrivals(count=nreq)
    reqs = []
    for i in range(nreq):
        inst = W.c5_request(i)
        inst["params"].update(solver or {})
        reqs.append(serve.Request(i, inst, steps, float(arr[i])))
    free, _ = torch.cuda.mem_get_info()
    budget = max(int(budget_frac * free), max(int(1.05 * r.footprint) + 1 for r in reqs))
    srv = serve.Server(budget, keep_results=False, persistent=persistent)
    done = srv.run(reqs)
    srv.close()
    out = serve.summarize(done, srv.elapsed, srv.busy)
    out["budget_bytes"] = budget
    out["steps_per_request"] = steps
    out["batching"] = ("persistent (lock step, one launch per multigrid level over the admitted "
                       "requests)" if persistent else "concurrent replay of each request's graph")
    if fp64_subset == 0:
        return out
    sub = reqs[:fp64_subset] if fp64_subset else reqs
    v, ms = serve.serial(sub, precision=0)
    out["serial_fp64"] = {"cell_steps_per_s": v, "requests": len(sub), "device_ms": ms}
    v32, ms32 = serve.serial(sub, precision=None)
    out["serial_mixed"] = {"cell_steps_per_s": v32, "requests": len(sub), "device_ms": ms32}
    return out


def div_summary(stats):
    """The per-step device checks of several simulations: the largest max
    |div u| after any projection, projections above div_tol, solves stopped
    above their tolerance."""
    return {"div_max_all_steps": max(st["div_max_steps"] for st in stats),
            "div_violations": sum(st["div_violations"] for st in stats),
            "nonconverged_solves": sum(st["nonconv_total"] for st in stats)}


def batch_form(insts, steps, warmup, persistent, world, args=None):
    """Every instance stepped together for `steps` steps after `warmup`:
    persistent (lock step, one launch per multigrid level and phase over all
    members, per-member masks) or concurrent replay of each member's own step
    graph on its own stream. Wall time around the queued steps and the final
    wait (the host queues faster than the device runs)."""
    from paper_1302_3663_gb300 import bfibm, workloads as W
    import torch
    ctxs = []
    pinned = persistent and args is not None and args.load_batch_shapes
    batch = bfibm.Batch(persistent=persistent, tune=not pinned)
    if persistent and args is not None and args.unroll:
        batch.set_option(bfibm.BATCH_UNROLL, args.unroll)
    if persistent and args is not None and args.batch_tail is not None:
        batch.set_option(bfibm.BATCH_TAIL, args.batch_tail)
    for inst in insts:
        c = bfibm.load_instance(inst)
        c.set_option(bfibm.OPT_STATS, 0)
        ctxs.append(c)
        batch.add(c)
    t = time.perf_counter()
    batch.step()                  # plan (tuned sweeps) or member graphs built here
    batch.wait()
    first_s = time.perf_counter() - t
    if pinned:
        with open(args.load_batch_shapes) as f:
            batch.pin_sweep_shapes(json.load(f))
    if persistent and args is not None and args.save_batch_shapes:
        with open(args.save_batch_shapes, "w") as f:
            json.dump(batch.sweep_shapes(), f)
    for _ in range(max(warmup - 1, 0)):
        batch.step()
    batch.wait()
    info0 = batch.info()
    lc0 = [c.launch_counts() for c in ctxs]
    barrier(world)
    torch.cuda.nvtx.range_push("timed_batch")
    t = time.perf_counter()
    for _ in range(steps):
        batch.step()
    batch.wait()
    el = max_over_ranks(world, time.perf_counter() - t)
    torch.cuda.nvtx.range_pop()
    info1 = batch.info()
    cells = sum(W.cells(i["params"]) for i in insts)
    out = {"value": cells * steps * world / el, "unit": UNIT, "ms_per_step": el / steps * 1e3,
           "first_step_s": first_s}
    if persistent:
        out["gpu_launches"] = (steps * info1["graph_kernels"] +
                               (info1["visc_iterations"] - info0["visc_iterations"]) *
                               info1["visc_body_kernels"] +
                               (info1["p_iterations"] - info0["p_iterations"]) *
                               info1["p_body_kernels"])
        out["loop_iterations_per_step"] = {
            "viscous": (info1["visc_iterations"] - info0["visc_iterations"]) / steps,
            "pressure": (info1["p_iterations"] - info0["p_iterations"]) / steps}
        out["sweep_shapes_finest"] = {"viscous": batch.sweep_shape(0, 0),
                                      "pressure": batch.sweep_shape(0, 1)}
    else:
        n = 0
        for c, a in zip(ctxs, lc0):
            b = c.launch_counts()
            n += (steps * b["top"] + (b["iters_visc"] - a["iters_visc"]) * b["body_visc"] +
                  (b["iters_p"] - a["iters_p"]) * b["body_p"])
        out["gpu_launches"] = n
    out["step_checks"] = div_summary([c.get_stats() for c in ctxs])
    batch.close()
    for c in ctxs:
        c.close()
    return out


def batched_forms(args, count, steps, world, fp64_subset=None):
    """The batched sweep (64 uneven ducts): the persistent form, concurrent
    graph replay, and each instance alone in plain FP64 (on the first
    fp64_subset instances), all with the tolerance solver and the per-step
    divergence check."""
    from paper_1302_3663_gb300 import serve, workloads as W
    insts = [W.c4_instance(i) for i in range(count)]
    for inst in insts:
        inst["params"].update(solver_override(args))
    cells = sum(W.cells(i["params"]) for i in insts)
    out = {"workload": "c4: %d independent ducts (edges 32-96, length 2 edges, %d cells in all), "
                       "500-8,000 nodes each, %d steps each" % (count, cells, steps),
           "cells": cells}
    forms = args.forms.split(",")
    if "persistent" in forms:
        out["persistent"] = batch_form(insts, steps, args.warmup, True, world, args)
    if "replay" in forms:
        out["replay"] = batch_form(insts, steps, args.warmup, False, world)
    if "fp64" in forms:
        sub = insts[:fp64_subset] if fp64_subset else insts
        reqs = [serve.Request(i, inst, steps, 0.0) for i, inst in enumerate(sub)]
        chk = []
        v64, _ = serve.serial(reqs, precision=0, checks=chk)
        out["fp64_single_instance_serial"] = {"value": v64, "unit": UNIT,
                                              "instances": len(reqs),
                                              "step_checks": div_summary(chk)}
    return out


def run_batched(args):
    """c4: independent ducts of uneven sizes stepped together; the line's
    value is the persistent form."""
    world, rank, local = dist_setup(args)
    with Clocks(local) as clk:
        res = batched_forms(args, args.instances, args.steps, world)
    per = res.get("persistent") or res.get("replay") or res["fp64_single_instance_serial"]
    out = {"metric": METRIC, "value": per["value"], "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
           "data": "synthetic", "config": {
               "workload": res["workload"], "cells": res["cells"],
               "precision": "fp32 V-cycles in fp64 flexible CG (viscous) and defect correction "
                            "(pressure)",
               "parallelism": "persistent batch: one launch per multigrid level and phase over "
                              "every instance, per-instance convergence masks, one graph per "
                              "batch step",
               "div_target": DIV_TARGET},
           "clocks": clk.summary(), "gpu_launches": per.get("gpu_launches"), "batched": res}
    if rank == 0:
        print(json.dumps(out))


def run_served(args):
    from paper_1302_3663_gb300 import workloads as W
    world, rank, local = dist_setup(args)
    nreq = args.requests or 32
    steps = args.request_steps or 20
    with Clocks(local) as clk:
        res = run_served_stream(nreq, steps, args.budget_frac, fp64_subset=8,
                                solver=solver_override(args))
        if args.solver == "tol":   # the persistent batch needs tolerance solves
            res["persistent_form"] = run_served_stream(nreq, steps, args.budget_frac,
                                                       fp64_subset=0, persistent=True,
                                                       solver=solver_override(args))
    out = {"metric": METRIC, "value": res["cell_steps_per_s"], "unit": UNIT, "n_gpus": world,
           "steps": steps, "warmup": 0, "ms_per_step": res["step_ms_p50"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
           "data": "synthetic", "config": {
               "workload": "c5: Poisson stream (mean 4 requests/s) of %d duct simulations, "
                           "edges 48-160, 500-50,000 nodes, %d steps each" % (nreq, steps),
               "admission": "device-memory footprint within %.0f%% of free memory" %
                            (100 * args.budget_frac)},
           "served": res, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(out))


def run_study(args):
    """Solver studies (not the benchmark line): one JSON line each."""
    import torch

    from paper_1302_3663_gb300 import bfibm, tuning, workloads as W
    dist_setup(args)
    if args.study == "work_units":
        out = {"study": "work_units", "rtol": 1e-10, "rows": {}}
        for name, levels in (("c1", range(1, 6)), ("c2", range(3, 7))):
            inst = W.CONFIGS[name]()
            for which in ("pressure", "viscous"):
                out["rows"]["%s_%s" % (name, which)] = tuning.work_units_vs_levels(
                    inst, levels, which=which)
        print(json.dumps(out))
        return
    if args.study == "refinement":
        import functools

        from paper_1302_3663_gb300 import refinement as R
        solver = {"vc_visc": 0, "vc_p": 0, "rtol": 1e-12, "max_cycles": 300, "precision": 0}
        out = {"study": "refinement", "solver": solver,
               # a smooth flow: the discretisation's own orders
               "spin_up_time_h1/256": R.temporal_rates(W.spin_up_channel(256), T=0.02,
                                                        dt0=2e-3, nruns=5, solver=solver),
               "spin_up_space": R.spatial_rates(W.spin_up_channel, [32, 64, 128, 256, 512],
                                                T=0.02, dt=1e-3, solver=solver),
               # the mound with the paper's refinement settings (Sec. 4.3.2-4.3.3):
               # h = 1/256 and dt = 1/5000 ... 1/80000 to T = 0.01; dt = 1e-4 and
               # h = 1/16 ... 1/256 to T = 0.01
               "mound_time_h1/256": R.temporal_rates(W.mound_2d(256), T=0.01, dt0=1.0 / 5000,
                                                      nruns=5, solver=solver)}
        for name, kw in (("const", {}), ("rho2", {"rho_ratio": 2.0}),
                         ("mu500", {"mu_ratio": 500.0})):
            out["mound_space_" + name] = R.spatial_rates(
                functools.partial(W.mound_2d, **kw), [16, 32, 64, 128, 256], T=0.01, dt=1e-4,
                solver=solver)
        print(json.dumps(out))
        return
    inst = load_workload(args.config, args.precision, args)
    cells = W.cells(inst["params"])
    stream = torch.cuda.Stream()
    ctx = bfibm.load_instance(inst, stream=stream)
    ctx.set_option(bfibm.OPT_STATS, 0)
    ctx.step(args.warmup)
    ctx.synchronize()
    ms0 = timed_steps(ctx, stream, args.steps, 1, "timed_gamma0")
    fin0 = final_stats(ctx)
    ctx.set_option(bfibm.OPT_GRAPH, 0)
    g, before, after = tuning.tune_gamma(ctx)
    ctx.set_option(bfibm.OPT_GRAPH, 1)
    ctx.set_option(bfibm.OPT_STATS, 0)
    ctx.step(1)
    ms1 = timed_steps(ctx, stream, args.steps, 1, "timed_gamma1")
    fin1 = final_stats(ctx)
    ctx.close()
    print(json.dumps({"study": "gamma", "config": describe(inst), "gamma_levels": g,
                      "viscous_cycles_trial": [before, after],
                      "before": {"ms_per_step": ms0 / args.steps,
                                 "cell_steps_per_s": cells * args.steps / (ms0 / 1e3), **fin0},
                      "after": {"ms_per_step": ms1 / args.steps,
                                "cell_steps_per_s": cells * args.steps / (ms1 / 1e3), **fin1}}))


def main():
    args = parse()
    if args.study:
        run_study(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "c4":
        run_batched(args)
    elif args.config == "c5":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
