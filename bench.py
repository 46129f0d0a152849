#!/usr/bin/env python3
"""Throughput benchmark of the fused well-balanced D2Q9 step on one GB300.

Workload (the large-domain throughput case): a 4096 x 4096 periodic lattice
with 64 droplets at seeded non-overlapping centres (radii U[16, 64]),
rho_l = 1, rho_g = 0.1 (density ratio 10), kappa = 0.01, W = 5, tau = 0.7,
well-balanced scheme.  One benchmark step = S lattice time steps (fused
collide-stream kernel) followed by one statistics pass (mass, max|u|, mu
range, kinetic energy, non-finite flag).  The headline is the FP32-shifted
path; the FP64 path is measured on the same lattice and reported beside it.

`value` is MLUPS (lattice-node updates per second / 1e6) with the state
resident in HBM; the population buffers (2 x 604 MB in FP32) are larger than
L2, so no flush is needed between steps.  `e2e` measures the same through the
C ABI with host buffers (wblbe_run_sequence): every step copies the initial
density in from pinned host memory, runs S steps and reads the density field
and stats back, its copies overlapping the neighbouring steps' computation.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (one lattice time step per benchmark step).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import numpy as np

METRIC = "MLUPS and HBM-roofline % (WB D2Q9, FP64 vs FP32); batched solve p50/p99"
UNIT = "MLUPS"
WORKLOAD = "large_domain_4096x4096_64droplets_ratio10_wb"
BYTES_PER_LU = {"f32": 72, "f64": 144}          # 9 reads + 9 writes per node update
SUBSTEPS = {"f32": 200, "f64": 40}              # lattice steps per benchmark step
# FP64 flops per lattice update of the FP64 step kernel, from the ncu
# instruction mix (2 x DFMA + DADD + DMUL per node, halo work included;
# 2048^2 well-balanced case: DADD 41.5, DMUL 21.2, DFMA 48.75)
FP64_FLOPS_PER_LU = 160.3
# FP64 flops per lattice update of the three D3Q19 kernels (density 18 DADD;
# chemical potential 19 DADD + 4 DMUL + 4 DFMA; collide 78 DADD + 32 DMUL +
# 81 DFMA; ncu op mix on a 128^3 droplet, one thread per node, no halo work)
D3_FLOPS_PER_LU = 321.0
# oldest state (lattice steps since initialisation) a timed step may start
# from; see time_device
MAX_STATE_AGE = 1200
PROFILE_JSON = ROOT / "profiles" / "lbm_step_traffic.json"
KERNEL_SOURCES = [ROOT / "paper_2012_11075_gb300" / "csrc" / "lbm_kernels.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(p.read_bytes())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return {}


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        if not self.lines:
            return None
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_problem(n=4096, ratio=10.0):
    from paper_2012_11075_gb300 import workloads as wl
    return wl.large_domain(n=n, count=64, ratio=ratio, width=5.0, kappa=0.01, tau=0.7)


# ---------------------------------------------------------------------------------
def run_reference(args, world, rank):
    """The oracle, as it stands, on the host cores: one FP64 lattice step of
    the full 4096^2 lattice per benchmark step."""
    if rank != 0:
        return 0
    from oracle.oracle import Oracle, Params as OParams
    pr = make_problem()
    o = Oracle(OParams(pr.nx, pr.ny, pr.tau, pr.kappa, pr.beta, pr.rho_l, pr.rho_g, 0.0, 1))
    f = o.init(pr.rho)
    for _ in range(args.warmup):
        o.step(f, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(f, 1)
    dt = time.perf_counter() - t0
    mlups = pr.nx * pr.ny * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": pr.nx, "ny": pr.ny, "lattice_steps_per_step": 1,
                   "scheme": "well_balanced", "precision": "fp64"},
        "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} FP64 lattice steps of the full {pr.nx}x{pr.ny} lattice, single thread"},
        "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample(pr, seconds_target=15.0):
    """Oracle MLUPS on the host (one thread) on a bounded sample: full lattice,
    as many FP64 steps as fit in about seconds_target (at least one)."""
    from oracle.oracle import Oracle, Params as OParams
    o = Oracle(OParams(pr.nx, pr.ny, pr.tau, pr.kappa, pr.beta, pr.rho_l, pr.rho_g, 0.0, 1))
    f = o.init(pr.rho)
    t0 = time.perf_counter()
    o.step(f, 1)
    dt1 = time.perf_counter() - t0
    n = max(1, min(5, int(seconds_target / max(dt1, 1e-3)) - 1))
    t0 = time.perf_counter()
    o.step(f, n)
    dt = time.perf_counter() - t0
    out = {"value": pr.nx * pr.ny * n / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{n} FP64 lattice steps (after 1 untimed) of the full {pr.nx}x{pr.ny} lattice, single thread"}
    out["all_cores"] = cpu_baseline_all_cores(pr)
    return out


def cpu_baseline_all_cores(pr, seconds_target=10.0):
    """The same oracle loops split over all host threads (its timing-only
    OpenMP build; every node computed as in the serial build)."""
    from oracle.oracle import Oracle, Params as OParams
    threads = os.cpu_count() or 1
    try:
        o = Oracle(OParams(pr.nx, pr.ny, pr.tau, pr.kappa, pr.beta, pr.rho_l, pr.rho_g, 0.0, 1),
                   openmp=True)
    except Exception as e:                      # no OpenMP in this compiler
        return {"value": None, "unit": UNIT, "cores": threads, "unavailable": str(e)[:200]}
    f = o.init(pr.rho)
    t0 = time.perf_counter()
    o.step(f, 1)
    dt1 = time.perf_counter() - t0
    n = max(1, min(40, int(seconds_target / max(dt1, 1e-3)) - 1))
    t0 = time.perf_counter()
    o.step(f, n)
    dt = time.perf_counter() - t0
    return {"value": pr.nx * pr.ny * n / dt / 1e6, "unit": UNIT, "cores": threads,
            "sample": f"{n} FP64 lattice steps (after 1 untimed) of the full {pr.nx}x{pr.ny} "
                      f"lattice, OpenMP over rows on {threads} threads"}


def time_device(solver, substeps, steps, warmup, stream, torch, rho_dev=None,
                max_age=MAX_STATE_AGE):
    """Device-resident timing of K benchmark steps, each S lattice steps and
    one stats pass, bracketed by CUDA events on the launching stream.

    The state is never older than max_age lattice steps: before a benchmark
    step that would take it past that age it is re-initialised from the
    device-resident density rho_dev, outside the event window (the
    large-domain case at tau = 0.7 becomes non-finite between lattice steps
    2000 and 5000, whatever the precision).  Returns total seconds inside
    the windows, seconds in the step kernels, kernel launches inside the
    windows and the health record (lattice age at the start of every timed
    step, and whether any timed step ended on a non-finite state)."""
    def renew():
        if rho_dev is not None and solver.steps + substeps > max_age:
            solver.init_rho(rho_dev)            # synchronises; outside the window

    for _ in range(warmup):
        renew()
        solver.step(substeps)
        solver.stats()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    ages, bad, launches = [], [], 0
    with torch.cuda.stream(stream):
        for k in range(steps):
            renew()
            ages.append(int(solver.steps))
            l0 = solver.kernel_launches
            ev[k][0].record(stream)
            solver.step(substeps)
            ev[k][1].record(stream)
            st = solver.stats()                 # synchronises: the step's result
            ev[k][2].record(stream)
            launches += solver.kernel_launches - l0
            bad.append(bool(st["nonfinite"]))
    torch.cuda.synchronize()
    total = sum(e[0].elapsed_time(e[2]) for e in ev) / 1e3
    kern = sum(e[0].elapsed_time(e[1]) for e in ev) / 1e3
    health = {"max_state_age": max_age, "state_age_at_timed_steps": ages,
              "nonfinite": any(bad)}
    return total, kern, launches, health


def measure_fp64_peak(stream, torch, blocks_per_sm=8, threads=256, iters=16384, reps=5):
    """The device's FP64 fused multiply-add rate (TFLOP/s, 2 flops per FMA)
    from the library's probe kernel: eight independent FMA chains per
    thread, a full-occupancy grid; best of reps launches by CUDA events,
    SM clocks sampled meanwhile."""
    from paper_2012_11075_gb300 import wblbe
    lib = wblbe.load_library()
    dev = torch.cuda.current_device()
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * blocks_per_sm
    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    sp = ctypes.c_void_p(stream.cuda_stream)
    for _ in range(2):
        assert lib.wblbe_probe_fp64_fma(ctypes.c_void_p(out.data_ptr()), blocks, threads, iters,
                                        sp) == wblbe.OK
    torch.cuda.synchronize()
    best = float("inf")
    with ClockSampler(dev) as clk:
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lib.wblbe_probe_fp64_fma(ctypes.c_void_p(out.data_ptr()), blocks, threads, iters, sp)
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b) / 1e3)
    flops = blocks * threads * iters * 8 * 2
    assert bool(torch.isfinite(out).all())
    return {"tflops": flops / best / 1e12, "unit": "TFLOP/s", "launch_ms": best * 1e3,
            "how": f"{blocks} CTAs x {threads} threads x {iters} iterations x 8 independent "
                   f"DFMA chains, best of {reps} launches (CUDA events)",
            "clocks": clk.summary()}


def time_e2e(solver, rho_pinned, rho_outs_pinned, substeps, steps, warmup, torch):
    """End to end through the C ABI with host buffers: one wblbe_run_sequence
    call relaxes `steps` initial states, each with the H2D copy of its
    density from page-locked memory, f = f^eq(rho, 0), `substeps` lattice
    steps, a moments pass, and the D2H copy of its density and statistics;
    one state's copies overlap the neighbouring states' steps."""
    outs = [rho_outs_pinned[k % len(rho_outs_pinned)] for k in range(max(steps, warmup))]
    if warmup:
        solver.run_sequence([rho_pinned] * warmup, substeps, outs[:warmup])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stats = solver.run_sequence([rho_pinned] * steps, substeps, outs[:steps])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert not any(st["nonfinite"] for st in stats), "a state ended non-finite"
    return dt


def run_slabs(args, stream, torch, single_kernel_mlups):
    """The headline lattice (4096^2, 64 droplets, ratio 10, FP32 WB) split into
    N row slabs on this one GPU (each slab with 3 ghost rows per side, one
    exchange per step; the slabs' kernels run side by side on forked streams
    and chunks of steps replay from a CUDA graph): MLUPS against the
    single-lattice step kernel, i.e. what the decomposition itself costs."""
    from paper_2012_11075_gb300 import wblbe
    pr = make_problem(args.lattice)
    params = wblbe.Params(pr.nx, pr.ny, pr.tau, pr.kappa, pr.beta, pr.rho_l, pr.rho_g,
                          scheme=wblbe.WELL_BALANCED, precision=wblbe.FP32_SHIFTED)
    out = []
    for n in (1, 2, 4, 8):
        s = wblbe.Slabs(params, n, stream=stream)
        s.init_rho(pr.rho)
        s.step(32)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        steps = 192
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            s.step(steps)
            ev[1].record(stream)
        torch.cuda.synchronize()
        dt = ev[0].elapsed_time(ev[1]) / 1e3
        st = s.stats()
        s.close()
        mlups = pr.nx * pr.ny * steps / dt / 1e6
        out.append({"nslabs": n, "mlups": mlups, "vs_single_kernel": mlups / single_kernel_mlups,
                    "nonfinite": bool(st["nonfinite"])})
    return {"workload": WORKLOAD + ", row slabs on one GPU", "steps": 192, "results": out}


def run_batched(args, stream, torch):
    """The uneven batched case mix: 512 independent cases (sides 64..512
    log-uniform, flat/droplet, ratio 2..50, tau 0.55..1.2), FP32-shifted
    state with FP64 reductions, 5000 steps each, one persistent launch per
    steps_per_launch steps, the launch configuration chosen by the
    autotuner on the same lattices.  Latency of a case = time from the
    start of the solve to the launch after which it stopped."""
    from paper_2012_11075_gb300 import autotune, wblbe
    from paper_2012_11075_gb300 import workloads as wl
    specs = wl.batched_case_specs(count=args.batch_cases, seed=4)
    if args.batch_uniform:
        # equal cases instead of the mix (to separate the costs of ragged
        # strips from those of the queue): droplets of radius side/5, W = 4,
        # ratio 10, tau = 1.0 (stable, so every case runs its full budget)
        ux, uy, count = (int(v) for v in args.batch_uniform.split(","))
        beta = wl.beta_for_width(0.01, 4.0, 1.0, 0.1)
        specs = [dict(k=k, nx=ux, ny=uy, kind="droplet", frac=0.2, rho_l=1.0, rho_g=0.1,
                      tau=1.0, kappa=0.01, width=4.0, beta=beta) for k in range(count)]
    gpu = torch.cuda.get_device_name()
    max_nodes = max(512 * 512, max(sp["nx"] * sp["ny"] for sp in specs))

    def params(sp, tau=None):
        return wblbe.Params(sp["nx"], sp["ny"], sp["tau"] if tau is None else tau, sp["kappa"],
                            sp["beta"], sp["rho_l"], sp["rho_g"], scheme=wblbe.WELL_BALANCED,
                            precision=wblbe.FP32_SHIFTED)

    probe = wblbe.Batch(max_cases=1, arena_bytes=1 << 20, stream=stream)
    case_bytes = [probe.case_bytes(params(sp)) for sp in specs]
    probe.close()
    if args.batch_config:
        tuned = {"config": [int(v) for v in args.batch_config.split(",")], "cached": False,
                 "candidates": None, "fixed": True}
    else:
        # tuned on the whole mix (a 64-case subsample ranked the tile
        # heights differently from the full mix), on a batch of its own whose
        # cases all keep running while the candidates are timed (the same
        # lattices with tau >= 0.9, above the WB stability limit: the work
        # per launch does not depend on tau)
        tb = wblbe.Batch(max_cases=len(specs), max_tiles=1 << 18, max_case_nodes=max_nodes,
                         arena_bytes=int(sum(case_bytes) * 1.02) + (1 << 20), stream=stream)
        for sp in specs:
            tb.admit(params(sp, max(sp["tau"], 0.9)), wl.case_field(sp), 0.0, 10 ** 9)
        tuned = autotune.tune(tb, [(sp["nx"], sp["ny"]) for sp in specs], gpu, launches=2,
                              sync=torch.cuda.synchronize)
        tb.close()
    cfg = tuned["config"]
    b = wblbe.Batch(max_cases=len(specs), max_tiles=1 << 18, max_case_nodes=max_nodes,
                    arena_bytes=int(sum(case_bytes) * 1.02) + (1 << 20), tile_x=cfg[0],
                    rows_per_tile=cfg[1], steps_per_launch=cfg[2], stream=stream)
    fields = [wl.case_field(sp) for sp in specs]
    t0 = time.perf_counter()
    ids = [b.admit(params(sp), f, 0.0, args.batch_steps) for sp, f in zip(specs, fields)]
    torch.cuda.synchronize()
    t_admit = time.perf_counter() - t0
    assert None not in ids
    nodes = {cid: sp["nx"] * sp["ny"] for cid, sp in zip(ids, specs)}
    done_at = {}
    l0 = b.kernel_launches
    t0 = time.perf_counter()
    while b.counts()["running"] > 0:
        b.advance(1)
        t = time.perf_counter() - t0
        for cid in b.poll():
            done_at[cid] = t
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    infos = {cid: b.info(cid) for cid in ids}
    node_steps = sum(nodes[cid] * infos[cid]["steps"] for cid in ids)
    states = {}
    for cid in ids:
        states[str(infos[cid]["state"])] = states.get(str(infos[cid]["state"]), 0) + 1
    lat = np.array([done_at.get(cid, t_solve) for cid in ids])
    by_state = {}
    for cid, l in zip(ids, lat):
        by_state.setdefault(str(infos[cid]["state"]), []).append(l)
    launches = b.kernel_launches - l0
    b.close()
    name = (f"batched_{len(specs)}_equal_{specs[0]['nx']}x{specs[0]['ny']}_cases_wb_fp32"
            if args.batch_uniform else f"batched_{len(specs)}_uneven_cases_wb_fp32")
    return {"workload": name,
            "cases": len(specs), "nodes": int(sum(nodes.values())),
            "steps_per_case": args.batch_steps, "config": cfg,
            "tuned_from_cache": tuned.get("cached", False), "tuning_mlups": tuned.get("candidates"),
            "admit_s": t_admit, "solve_s": t_solve, "mlups": node_steps / t_solve / 1e6,
            # whole solve (launch gaps, host checks and tile halos included)
            # against the same roofline as the headline: 72 B per update
            "hbm_frac": node_steps * BYTES_PER_LU["f32"] / t_solve / 1e9
            / (measured_peaks().get("hbm_gbs") or 6800.0),
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            # every case runs to its step budget unless it goes unstable (the
            # mix draws tau below the WB stability limit): latency per outcome
            "latency_by_state": {k: {"count": len(v), "p50_s": float(np.percentile(v, 50)),
                                     "p99_s": float(np.percentile(v, 99))}
                                 for k, v in sorted(by_state.items())},
            "states": states, "state_names": {"1": "converged", "2": "budget", "3": "unstable"},
            "gpu_launches": int(launches)}


def run_serving(args, stream, torch, cfg):
    """Continuous batching of relax-to-equilibrium requests arriving as a
    Poisson process (sides 32..1024 log-uniform, case parameters as the
    batched mix), each run to max|u| < 1e-6 (FP32) / 1e-10 (FP64) or 200000
    steps; requests are admitted as slots and memory free up.  Each arrival
    rate runs until serve_requests requests have completed or its window
    has passed, whichever comes first.  Latency percentiles are reported
    over all completed requests and per outcome (converged / budget /
    unstable: the mix draws tau down to 0.55, below the well-balanced
    scheme's linear stability limit)."""
    from paper_2012_11075_gb300 import serve, wblbe

    def batch(prec):
        return wblbe.Batch(precision=prec, max_cases=256, max_tiles=1 << 17,
                           max_case_nodes=1024 * 1024, arena_bytes=args.serve_arena_gb << 30,
                           tile_x=cfg[0], rows_per_tile=cfg[1], steps_per_launch=cfg[2],
                           stream=stream)

    out = {}
    windows = {"fp32": args.serve_window, "fp64": args.serve_window_fp64}
    for name, prec in (("fp32", wblbe.FP32_SHIFTED), ("fp64", wblbe.FP64)):
        out[name] = {}
        for rate in args.serve_rates:
            reqs = serve.make_requests(rate, windows[name], seed=5, precision=prec,
                                       scheme=wblbe.WELL_BALANCED)
            b = batch(prec)
            srv = serve.Server(b)
            rep = srv.run(reqs, duration=windows[name], drain=False,
                          stop_after=args.serve_requests)
            b.close()
            out[name][str(rate)] = rep.summary()
    # FP64 at 1e-10 converges nothing inside a window at these rates: the
    # offered load is far above what the GPU finishes (about 1-2 requests
    # per second), so the resident requests share it and none gets far.  A
    # small set of the same requests, all offered at once and served until
    # each has stopped (or the cap), gives the FP64 steps to the tolerance.
    reqs = serve.make_requests(args.serve_rates[0], 10.0, seed=5, precision=wblbe.FP64,
                               scheme=wblbe.WELL_BALANCED)[:args.serve_drained]
    for r in reqs:
        r.arrival = 0.0
    b = batch(wblbe.FP64)
    srv = serve.Server(b)
    rep = srv.run(reqs, duration=0.0, drain=True, stop_after=None, time_cap=args.serve_drain_cap)
    # requests still running at the cap: how far they got
    unfinished = []
    for cid, r in srv.resident.items():
        info = b.info(cid)
        unfinished.append({"nx": r.params.nx, "ny": r.params.ny, "tau": r.params.tau,
                           "state": "running at the cap", "steps": info["steps"],
                           "umax": info["stats"]["umax"]})
    b.close()
    drained = rep.summary()
    drained["requests"] = [{"nx": r.params.nx, "ny": r.params.ny, "tau": r.params.tau,
                            "state": r.state, "steps": r.steps,
                            "latency_s": None if math.isnan(r.finished) else r.finished - r.arrival}
                           for r in sorted(rep.completed, key=lambda q: q.rid)] + unfinished
    drained["policy"] = (f"the first {len(reqs)} requests of the FP64 serving stream, all "
                         f"offered at t = 0, served until each stopped (cap "
                         f"{args.serve_drain_cap} s)")
    return {"workload": "poisson_relax_to_equilibrium_wb",
            "window_s": windows,
            "stop_rule": f"each rate until {args.serve_requests} requests completed or "
                         f"its window passed",
            "fp64_drained": drained,
            "policy": "admit by slot and arena room, one launch per loop, stop at launch "
                      "boundaries (requests still queued or running at the end are "
                      "reported, not counted as completed)",
            "outcomes": {"1": "converged", "2": "budget", "3": "unstable"},
            "results": out}


def run_schemes(args, stream, torch):
    """Cost of the four schemes on the same 4096^2 droplet field (density
    ratio 5, where the standard scheme is stable too): Sec. III says the
    well-balanced LBE has the algorithmic structure of the standard one, so
    they should cost the same.  Step-kernel time by CUDA events."""
    from paper_2012_11075_gb300 import wblbe
    from paper_2012_11075_gb300 import workloads as wl
    pr = wl.large_domain(n=args.lattice, count=64, ratio=5.0, width=5.0, kappa=0.01, tau=0.7)
    names = {wblbe.STANDARD: "standard", wblbe.WELL_BALANCED: "well_balanced",
             wblbe.STANDARD_PRESSURE: "standard_pressure_form",
             wblbe.STANDARD_TEXTBOOK: "standard_textbook_forcing"}
    out = {"workload": f"large_domain_{pr.nx}x{pr.ny}_64droplets_ratio5", "results": {}}
    for prec_name, prec, S in (("f32", wblbe.FP32_SHIFTED, 100), ("f64", wblbe.FP64, 20)):
        for sch, name in names.items():
            params = wblbe.Params(pr.nx, pr.ny, pr.tau, pr.kappa, pr.beta, pr.rho_l, pr.rho_g,
                                  scheme=sch, precision=prec)
            solver = wblbe.Solver(params, stream=stream)
            solver.init_rho(pr.rho)
            total, kern, _, _ = time_device(solver, S, 2, 1, stream, torch)
            st = solver.stats()
            kern_avg = kern / (2 * S)
            out["results"][f"{prec_name}/{name}"] = {
                "mlups": pr.nx * pr.ny / kern_avg / 1e6, "kernel_us": kern_avg * 1e6,
                "hbm_frac": BYTES_PER_LU[prec_name] * pr.nx * pr.ny / kern_avg / 1e9 /
                (measured_peaks().get("hbm_gbs") or 6800.0),
                "nonfinite": bool(st["nonfinite"])}
            solver.close()
            del solver
            torch.cuda.empty_cache()
    return out


def run_d3q19(args, stream, torch, fp64_peak=None):
    """The three-dimensional (D3Q19) well-balanced path: a periodic n^3
    lattice with one droplet of radius n/4 (rho_l = 1, rho_g = 0.1,
    kappa = 0.01, W = 4, tau = 1.0); K benchmark steps of S lattice steps,
    timed by CUDA events on the launching stream, in FP64 and in
    FP32-shifted storage.  Three kernels per step (density, chemical
    potential, collide-stream); algorithmic bytes per update 19 populations
    read and written (304 in FP64, 152 in FP32); the kernels move about
    496 / 248 (the density and chemical-potential fields, and the
    populations read twice)."""
    from paper_2012_11075_gb300 import wblbe
    from paper_2012_11075_gb300 import workloads as wl
    n = args.d3_lattice
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - n // 2) ** 2 + (y - n // 2) ** 2 + (z - n // 2) ** 2)
    rho = 0.55 - 0.45 * np.tanh(2 * (r - n / 4) / 4.0)
    beta = wl.beta_for_width(0.01, 4.0, 1.0, 0.1)
    peak = measured_peaks().get("hbm_gbs") or 6800.0

    def timed(precision):
        s = wblbe.Solver3(wblbe.Params3(n, n, n, 1.0, 0.01, beta, 1.0, 0.1, 0.0,
                                        wblbe.WELL_BALANCED, precision), stream=stream)
        s.init_rho(rho)
        S = 20 if precision == wblbe.FP64 else 100
        K = max(1, min(args.steps, 5))
        for _ in range(2):
            s.step(S)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        l0 = s.kernel_launches
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            s.step(S * K)
            ev[1].record(stream)
        torch.cuda.synchronize()
        dt = ev[0].elapsed_time(ev[1]) / 1e3
        st = s.stats()
        launches = s.kernel_launches - l0
        s.close()
        return n ** 3 * S * K / dt, S * K, dt, launches, st

    lups, steps, dt, launches, st = timed(wblbe.FP64)
    if fp64_peak is None:
        fp64_peak = measure_fp64_peak(stream, torch)
    alu = lups * D3_FLOPS_PER_LU / 1e12
    l32, steps32, dt32, launches32, st32 = timed(wblbe.FP32_SHIFTED)
    return {"workload": f"d3q19_{n}^3_droplet_wb_fp64", "value": lups / 1e6, "unit": UNIT,
            "lattice_steps": steps, "seconds": dt, "gpu_launches": launches,
            "bytes_per_lattice_update": 304,
            "hbm_frac_algorithmic": 304 * lups / 1e9 / peak,
            "hbm_frac_moved": 496 * lups / 1e9 / peak,
            # the three kernels are bound by the FP64 pipe (83-87 % busy)
            "roofline_alu": {"bound": "alu", "achieved": alu, "peak": fp64_peak["tflops"],
                             "unit": "TFLOP/s", "frac": alu / fp64_peak["tflops"],
                             "flops_per_lattice_update": D3_FLOPS_PER_LU,
                             "peak_source": "of measured (FP64 FMA probe kernel, this run)"},
            "umax": st["umax"], "mass_drift_rel": st["mass_drift_rel"],
            "nonfinite": bool(st["nonfinite"]),
            "fp32": {"workload": f"d3q19_{n}^3_droplet_wb_fp32_shifted", "value": l32 / 1e6,
                     "unit": UNIT, "lattice_steps": steps32, "seconds": dt32,
                     "gpu_launches": launches32, "bytes_per_lattice_update": 152,
                     "roofline": {"bound": "hbm", "achieved": 152 * l32 / 1e9, "peak": peak,
                                  "unit": "GB/s", "frac": 152 * l32 / 1e9 / peak,
                                  "peak_source": "of measured"},
                     "hbm_frac_moved": 248 * l32 / 1e9 / peak,
                     "umax": st32["umax"], "mass_drift_rel": st32["mass_drift_rel"],
                     "nonfinite": bool(st32["nonfinite"])}}


def run_ours(args, world, rank, local):
    import torch
    from paper_2012_11075_gb300 import wblbe
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pr = make_problem(args.lattice)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    peak_note = "of measured" if hbm_peak else "of fallback"
    hbm_peak = hbm_peak or 6800.0
    stream = torch.cuda.Stream(device=dev)
    if args.only == "schemes":
        if rank == 0:
            print(json.dumps({"schemes": run_schemes(args, stream, torch)}), flush=True)
        return 0
    if args.only == "batched":
        # the batched leg alone (a partial run, not the benchmark line)
        if rank == 0:
            print(json.dumps({"batched": run_batched(args, stream, torch)}), flush=True)
        return 0
    if args.only == "d3q19":
        if rank == 0:
            print(json.dumps({"d3q19": run_d3q19(args, stream, torch)}), flush=True)
        return 0
    if args.only == "slabs":
        # against the single-lattice step kernel's rate measured here
        if rank == 0:
            sol = wblbe.Solver(wblbe.Params(pr.nx, pr.ny, pr.tau, pr.kappa, pr.beta, pr.rho_l,
                                            pr.rho_g, scheme=wblbe.WELL_BALANCED,
                                            precision=wblbe.FP32_SHIFTED), stream=stream)
            sol.init_rho(pr.rho)
            sol.step(32)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            with torch.cuda.stream(stream):
                ev[0].record(stream)
                sol.step(192)
                ev[1].record(stream)
            torch.cuda.synchronize()
            single = pr.nx * pr.ny * 192 / (ev[0].elapsed_time(ev[1]) / 1e3) / 1e6
            sol.close()
            print(json.dumps({"slabs": run_slabs(args, stream, torch, single),
                              "single_lattice_mlups": single}), flush=True)
        return 0
    results = {}
    precisions = [("f32", wblbe.FP32_SHIFTED, pr), ("f64", wblbe.FP64, pr)]
    if args.only != "both":
        precisions = [x for x in precisions if x[0] == args.only]
    elif not args.no_ratio50:
        # the same large-domain case at density ratio 50 (rho_g = 0.02)
        precisions.insert(1, ("f32_ratio50", wblbe.FP32_SHIFTED, make_problem(args.lattice, 50.0)))
    for prec_name, prec, prob in precisions:
        params = wblbe.Params(prob.nx, prob.ny, prob.tau, prob.kappa, prob.beta, prob.rho_l,
                              prob.rho_g, scheme=wblbe.WELL_BALANCED, precision=prec)
        solver = wblbe.Solver(params, stream=stream)
        rho_dev = torch.from_numpy(prob.rho).to(dev)
        solver.init_rho(rho_dev)
        bpl = BYTES_PER_LU["f64" if prec == wblbe.FP64 else "f32"]
        S = SUBSTEPS["f64" if prec == wblbe.FP64 else "f32"]
        K = args.steps if prec != wblbe.FP64 else max(1, min(args.steps, 5))
        barrier(world)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            total, kern, launches, health = time_device(solver, S, K, args.warmup, stream, torch,
                                                        rho_dev=rho_dev)
        total = max_over_ranks(world, total, dev)
        st = solver.stats()
        lu = prob.nx * prob.ny * S * K
        step_launches = S * K
        kern_avg = kern / step_launches
        achieved_gbs = bpl * prob.nx * prob.ny / kern_avg / 1e9
        health.update(umax=st["umax"], mass_drift_rel=st["mass_drift_rel"])
        results[prec_name] = dict(
            mlups=lu * world / total / 1e6, total=total, kern_avg=kern_avg,
            kern_mlups=prob.nx * prob.ny / kern_avg / 1e6,
            achieved_gbs=achieved_gbs, launches=launches, clocks=clk.summary(),
            launch=solver.get_launch(), health=health, S=S, K=K)
        if prec_name == "f32" and not args.no_e2e:
            rho_pinned = torch.from_numpy(pr.rho).pin_memory()
            rho_outs = [torch.empty_like(rho_pinned).pin_memory() for _ in range(2)]
            e2e_t = time_e2e(solver, rho_pinned, rho_outs, S, K, min(args.warmup, 2), torch)
            e2e_t = max_over_ranks(world, e2e_t, dev)
            # per state: its density in; its density and two statistics records
            # (initial and final state) out
            results["e2e"] = dict(mlups=lu * world / e2e_t / 1e6, seconds=e2e_t,
                                  h2d=pr.nx * pr.ny * 8, d2h=pr.nx * pr.ny * 8 + 2 * 6 * 8)
        solver.close()
        del solver
        torch.cuda.empty_cache()

    if rank != 0:
        return 0
    if args.only != "both" or args.no_e2e or args.lattice != 4096:
        # profiling / partial runs: a short summary, not the benchmark line
        print(json.dumps({k: {kk: vv for kk, vv in v.items() if kk != "clocks"}
                          for k, v in results.items()}, default=str), flush=True)
        return 0
    r32, r64 = results["f32"], results["f64"]
    traffic = None
    if PROFILE_JSON.exists():
        prof = json.loads(PROFILE_JSON.read_text())
        if prof.get("kernel_hash") == kernel_hash():
            traffic = prof.get("dram_bytes_per_launch_full_size")
    fp64_peak = measure_fp64_peak(stream, torch)
    # FP64 flops per lattice update, measured with ncu on the FP64 step kernel
    # (2 x DFMA + DADD + DMUL per node, 2048^2 case, halo work included)
    fp64_flops_per_lu = FP64_FLOPS_PER_LU
    line = {
        "metric": METRIC, "value": r32["mlups"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r32["total"] / r32["K"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": pr.nx, "ny": pr.ny, "droplets": 64,
                   "ratio": 10, "tau": pr.tau, "kappa": pr.kappa, "width": 5,
                   "scheme": "well_balanced", "precision": "fp32_shifted",
                   "lattice_steps_per_step": r32["S"], "tile_x": r32["launch"][0],
                   "rows_per_cta": r32["launch"][1],
                   "l2": "state (2 x 604 MB) larger than L2; no flush",
                   "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "achieved": r32["achieved_gbs"], "peak": hbm_peak,
                     "unit": "GB/s", "frac": r32["achieved_gbs"] / hbm_peak,
                     "traffic": traffic, "peak_source": peak_note,
                     "bytes_per_lattice_update": BYTES_PER_LU["f32"],
                     "kernel": "lbm_strip_kernel<float, WB>",
                     "kernel_ms": r32["kern_avg"] * 1e3},
        "e2e": {"value": results["e2e"]["mlups"], "unit": UNIT,
                "h2d_bytes_per_step": results["e2e"]["h2d"],
                "d2h_bytes_per_step": results["e2e"]["d2h"]},
        "gpu_launches": r32["launches"],
        "clocks": r32["clocks"],
        "fp64": {"value": r64["mlups"], "unit": UNIT, "lattice_steps_per_step": r64["S"],
                 "steps": r64["K"],
                 "roofline_hbm": {"achieved": r64["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                                  "frac": r64["achieved_gbs"] / hbm_peak},
                 "roofline_alu": {"bound": "alu",
                                  "achieved": r64["kern_mlups"] * 1e6 * fp64_flops_per_lu / 1e12,
                                  "peak": fp64_peak["tflops"], "unit": "TFLOP/s",
                                  "frac": r64["kern_mlups"] * 1e6 * fp64_flops_per_lu / 1e12
                                  / fp64_peak["tflops"],
                                  "flops_per_lattice_update": fp64_flops_per_lu,
                                  "peak_source": "of measured (FP64 FMA probe kernel, this run)",
                                  "peak_measurement": fp64_peak},
                 "gpu_launches": r64["launches"], "clocks": r64["clocks"]},
        "health": {k: v["health"] for k, v in results.items() if "health" in v},
    }
    line["health"]["nonfinite"] = any(h["nonfinite"] for h in line["health"].values())
    if "f32_ratio50" in results:
        r50 = results["f32_ratio50"]
        line["ratio50"] = {
            "workload": WORKLOAD.replace("ratio10", "ratio50"), "value": r50["mlups"],
            "unit": UNIT, "lattice_steps_per_step": r50["S"], "steps": r50["K"],
            "roofline": {"bound": "hbm", "achieved": r50["achieved_gbs"], "peak": hbm_peak,
                         "unit": "GB/s", "frac": r50["achieved_gbs"] / hbm_peak,
                         "peak_source": peak_note, "kernel_ms": r50["kern_avg"] * 1e3},
            "gpu_launches": r50["launches"], "clocks": r50["clocks"]}
    # the one-GPU legs: measured by an N = 1 run only (under torchrun the
    # other ranks have finished, and their GPUs would wait for rank 0)
    solo = world == 1
    if solo and not args.no_schemes:
        line["schemes"] = run_schemes(args, stream, torch)
    if solo and not args.no_d3q19:
        line["d3q19"] = run_d3q19(args, stream, torch, fp64_peak)
    if solo and not args.no_slabs:
        line["slabs"] = run_slabs(args, stream, torch, r32["kern_mlups"])
    if solo and not args.no_batched:
        line["batched"] = run_batched(args, stream, torch)
        if not args.no_serving:
            line["serving"] = run_serving(args, stream, torch, line["batched"]["config"])
    if not solo:
        line["one_gpu_legs"] = "measured at n_gpus = 1 only"
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_sample(pr)
    print(json.dumps(line), flush=True)
    if line["health"]["nonfinite"]:
        print("bench: a timed step ended on a non-finite state", file=sys.stderr, flush=True)
        return 1
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lattice", type=int, default=4096,
                    help="lattice side (4096 is the benchmark; smaller sides are for profiling)")
    ap.add_argument("--only", choices=["both", "f32", "f64", "batched", "schemes", "d3q19",
                                       "slabs"],
                    default="both")
    ap.add_argument("--no-d3q19", action="store_true")
    ap.add_argument("--d3-lattice", type=int, default=256)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-slabs", action="store_true")
    ap.add_argument("--no-schemes", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-ratio50", action="store_true")
    ap.add_argument("--batch-cases", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=5000)
    ap.add_argument("--batch-uniform", default=None,
                    help="NX,NY,COUNT: the batched leg on COUNT equal droplet cases instead "
                         "of the uneven mix")
    ap.add_argument("--batch-config", default=None,
                    help="tile_x,rows_per_tile,steps_per_launch for the batched leg "
                         "(default: chosen by the autotuner)")
    ap.add_argument("--serve-window", type=float, default=20.0)
    ap.add_argument("--serve-window-fp64", type=float, default=10.0)
    ap.add_argument("--serve-drained", type=int, default=16)
    ap.add_argument("--serve-drain-cap", type=float, default=90.0)
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[50.0, 200.0, 1000.0])
    ap.add_argument("--serve-arena-gb", type=int, default=24)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup(args)
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        return run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
