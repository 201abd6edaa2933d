#!/usr/bin/env python
"""Benchmark: DOF-updates/s per RK stage of the quadrature-free DG shallow
water solver (arXiv:1904.08684) on one GB300, through the libdgswe C-ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--proj fp64|fp32|df64|mixed] [--impl ours|reference]
                    [--no-cpu-baseline] [--no-fp64-plain]

Default workload: ensemble-256, the batched FP32 form of the headline metric:
256 seeded independent instances (nx, ny uniform in {64..384}, p uniform in
{1, 2, 3}, periodic, smooth bathymetry of depth 5-20 m, one Gaussian hump
each, SSP-RK3, per-instance CFL step), FP32 state and contractions with the
mixed velocity solve (FP32 factors refined once with a compensated FP32
residual: the FP64 solution to within FP32 rounding), tile-fused kernels,
one persistent launch per order class and RK stage, each step one CUDA
graph.  "e2e" times the same workload from host states to host states
(dg_batch_step_host: 4.1 GB of FP64 states up and down per step, copies
overlapped with the compute).  Beside it, in the
same JSON line, "fp64_plain" holds the plain FP64 path measured on
waves-p2-512 (512 x 512 quads -> 524,288 triangles, p = 2, periodic, h_b = 10
+ 2 sin(2 pi x) cos(2 pi y), 8 seeded Gaussians, q = 0, SSP-RK3, CFL 0.2), and
"speedup_vs_fp64_plain" the ratio of the two.  The metric counts 3 K E
updated coefficients per stage.  Inputs are synthetic (seeded), projected on
the device by the library's own set-up projection.

N > 1 (torchrun): the ensemble's independent instances are split across the
ranks (no data-path collective); single-instance workloads run as replicas.
value = all ranks' DOF-updates / the slowest rank's time.

--impl reference times the FP64 CPU oracle (the test reference) on the host
cores, on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1904_08684_gb300 import inputs as I  # noqa: E402

METRIC = "DOF-updates/s per RK stage"
UNIT = "DOF/s"
WORKLOADS = {
    "waves-p2-512": lambda: I.waves_p2_512(),
    "hump-p1-32": lambda: I.hump_p1_32(),
    "hump-p3-32": lambda: I.hump_p3_32(),
    "waves-p4-2048": lambda: I.waves_p4_2048(),
    "waves-p1-512-fp32": lambda: I.waves_p2_512(p=1, precision="fp32"),
    "waves-p2-512-fp32": lambda: I.waves_p2_512(precision="fp32"),
    "waves-p3-512-fp32": lambda: I.waves_p2_512(p=3, precision="fp32"),
    "ensemble-256": lambda: I.ensemble(),
    "ensemble-256-fp64": lambda: I.ensemble(precision="fp64"),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 FMA rate of GB300 from the profiling recipe's nominal table; the
# measured copy bandwidth comes from MEASURED_PEAKS.json
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 2 * 152 * 128 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x max clock


HBM_FALLBACK_GBS = 6800.0


def _hbm_peak():
    """measured copy bandwidth (GB/s) and where it comes from"""
    v = _peaks().get("hbm_gbs")
    if v:
        return float(v), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    return HBM_FALLBACK_GBS, "of fallback (6.8 TB/s, no MEASURED_PEAKS.json on this box)"


def _roofline(parts, precision, proj, launch_s, traffic, rk_order):
    """Roofline of the stage kernel.  parts: [(p, E)] of the instances of one
    launch; launch_s: seconds per stage launch (the step's CUDA-event time /
    its stage count).  Algorithmic flops per element and stage: 2 x the FMA
    counts of flops.ALGORITHMIC_FMA (velocity solve, rest).  FP64 path: all
    flops against the FP64 rate; FP32 state with the FP64 solve: the solve's
    flops against the FP64 rate (the pipe that binds), with the FP32 share
    beside it; FP32 state with a double-float, mixed or FP32 solve: all flops
    against the FP32 rate.  The HBM fraction uses the algorithmic bytes of
    flops.stage_bytes_avg (state, RK base from the second stage on,
    bathymetry in; state out) over the stages of one step."""
    from paper_1904_08684_gb300 import flops as FL
    fsolve = sum(2 * FL.ALGORITHMIC_FMA[p][0] * E for p, E in parts)
    frest = sum(2 * FL.ALGORITHMIC_FMA[p][1] * E for p, E in parts)
    word = 8 if precision == "fp64" else 4
    alg_bytes = sum(FL.stage_bytes_avg(p, word, rk_order) * E for p, E in parts)
    hbm_peak, hbm_src = _hbm_peak()
    fp64_src = "FP64 1.25 TFLOP/s nominal (recipe table; a probe measured 1.17-1.20)"
    fp32_src = "FP32 152 SM x 128 lanes x 2 x 2.07 GHz (nominal; a probe measured 73)"
    if precision == "fp64":
        ach, peak, src, what, pipe = ((fsolve + frest) / launch_s / 1e12, FP64_PEAK_TFLOPS, fp64_src,
                                      "all flops (FP64)", "fp64")
    elif proj == "fp64":
        ach, peak, src, what, pipe = (fsolve / launch_s / 1e12, FP64_PEAK_TFLOPS, fp64_src,
                                      "FP64 flops of the velocity solve", "fp64")
    else:
        ach, peak, src, what, pipe = ((fsolve + frest) / launch_s / 1e12, FP32_PEAK_TFLOPS, fp32_src,
                                      "all flops on the FP32 pipe (the %s solve counted at its algorithmic flops)"
                                      % proj, "fp32")
    hbm_ach = alg_bytes / launch_s / 1e9
    roof = {"bound": "alu", "pipe": pipe, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": traffic, "counted": what, "peak_source": src,
            "flops_per_launch": fsolve + frest,
            "hbm_algorithmic_bytes_per_launch": alg_bytes,
            "hbm_achieved_gbs": hbm_ach, "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src,
            "hbm_frac": hbm_ach / hbm_peak,
            "traffic_over_algorithmic": (traffic / alg_bytes) if traffic else None}
    if precision != "fp64" and proj == "fp64":
        roof["fp32_achieved_tflops"] = frest / launch_s / 1e12
        roof["fp32_frac"] = frest / launch_s / 1e12 / FP32_PEAK_TFLOPS
    return roof


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons (200 ms)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _measured_traffic(workload, src_hash):
    """DRAM bytes per stage launch from the last ncu capture of this exact
    kernel source (profiles/traffic.json), else None"""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(workload)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("src") != src_hash:
        return None
    return rec.get("bytes_per_launch")


def reduce_time_and_value(ms_local, dofs_per_step_local, steps, world):
    """Whole-job timing of replicas: every rank's time is replaced by the
    slowest rank's (all-reduce MAX over the default process group when
    world > 1); value = all ranks' DOF-updates / that time."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        tt = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
        tot = torch.tensor([float(dofs_per_step_local)], dtype=torch.float64, device=dev)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        total = float(tot.item())
    else:
        total = float(dofs_per_step_local)
    step_ms = ms / steps
    return ms, step_ms, total * 1e3 / step_ms


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _setup_device_inputs(B, torch, wl, cfg, stream):
    """seeded fields sampled at the library's set-up nodes, projected on the
    device (dg_proj_nodes + dg_project)"""
    E, K, Q = wl.E, wl.K, B.dg_proj_num_nodes(wl.p)
    coef = []
    chunk_fields = (wl.hb, wl.xi0)
    xy = torch.empty((2, Q, E), dtype=torch.float64, device="cuda")
    B.dg_proj_nodes(cfg, xy, stream)
    torch.cuda.synchronize()
    for f in chunk_fields:
        vals = f(xy[0], xy[1]).contiguous()
        c = torch.empty((K, E), dtype=torch.float64, device="cuda")
        B.dg_project(cfg, vals, c, stream)
        torch.cuda.synchronize()
        coef.append(c)
        del vals
    del xy
    zero = torch.zeros((K, E), dtype=torch.float64, device="cuda")
    return coef[0], coef[1], zero, zero


def _dtype(precision, proj):
    """arithmetic of the path: state/contractions, plus the velocity solve"""
    if precision == "fp64":
        return "f64"
    return {"fp64": "f32+f64solve", "fp32": "f32", "df64": "f32+df64solve", "mixed": "f32+f64refinedsolve"}[proj]


def _single_kernel_form(wl, args):
    """the kernel form a single context takes (the library's default rule
    for tile_shape 0: 8 x 8 tiles with the mixed and FP32 solves at p <= 3,
    8 x 4 tiles with the FP32 solve at p = 4, per-element otherwise)"""
    names = {1: "8x8", 2: "16x8", 3: "8x4"}
    if wl.precision != "fp32" or args.tile < 0:
        return "per-element"
    if args.tile > 0:
        return "tile-fused %s quads" % names[args.tile]
    if wl.p <= 3 and args.proj in ("mixed", "fp32"):
        return "tile-fused 8x8 quads"
    if wl.p == 4 and args.proj == "fp32":
        return "tile-fused 8x4 quads"
    return "per-element"


def _cfg_of(B, wl, args):
    return B.make_config(wl.nx, wl.ny, wl.p, bc=wl.bc, precision=wl.precision, rk_order=wl.rk_order,
                         cfl=wl.cfl, dt=wl.dt, g=wl.g, x0=wl.x0, y0=wl.y0, Lx=wl.Lx, Ly=wl.Ly,
                         proj_precision=args.proj, block_size=args.block, tile_shape=args.tile)


def shard_instances(n, world, rank):
    """Instances of an ensemble owned by one rank: a round-robin split of the
    index list (the list is ordered by seed, not by cost, so every rank gets
    a similar mix of sizes and orders).  The instances are independent: no
    data-path collective is needed."""
    return list(range(rank, n, world))


def run_batch(args, wls):
    """ensemble of independent instances, one persistent launch per stage;
    under torchrun the instances are split across the ranks"""
    import torch
    from paper_1904_08684_gb300 import binding as B
    from paper_1904_08684_gb300 import flops as FL
    world, rank, local = _dist()
    n_total = len(wls)
    if world > 1:
        wls = [wls[i] for i in shard_instances(n_total, world, rank)]
    B.load()
    stream = torch.cuda.current_stream()
    cfgs, fields = [], [[], [], [], []]
    for wl in wls:
        cfg = _cfg_of(B, wl, args)
        f = _setup_device_inputs(B, torch, wl, cfg, stream)
        cfgs.append(cfg)
        for k in range(4):
            fields[k].append(f[k])
    b = B.dg_batch_init_device(cfgs, *fields, stream=stream)
    del fields
    torch.cuda.empty_cache()
    S = wls[0].rk_order
    dofs = B.dg_batch_dofs(b)
    tiled = wls[0].precision == "fp32" and (args.tile > 0 or (args.tile == 0 and args.proj in ("mixed", "fp32")))
    shape_names = {1: "8x8 quads", 2: "16x8 quads", 3: "8x4 quads"}
    cand_names = [shape_names[k] for k in (1, 2, 3)] if tiled else ["%d elements" % k for k in (32, 64, 96, 128)]
    try:
        block, tune_ms = B.dg_batch_autotune(b, 2)
        cls_shapes = {"p%d" % q: shape_names[B.dg_batch_tile_shape(b, q)]
                      for q in (1, 2, 3) if B.dg_batch_tile_shape(b, q)}
        B.dg_batch_run(b, args.warmup)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(stream)
            tvals = B.dg_batch_run(b, args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
        ms, step_ms, value = reduce_time_and_value(e0.elapsed_time(e1), dofs * S, args.steps, world)
        # end to end through the public API with host buffers: per step every
        # instance's state goes host -> device, one SSP-RK step, and every
        # state comes back to the host (dg_batch_step_host: the three
        # pipelined over groups of instances); one untimed call first, which
        # allocates the staging area
        shapes = [(wl.E, wl.K) for wl in wls]
        host = B.HostStates(shapes, pinned=True)
        B.dg_batch_get_states(b, shapes, out=host.arrays)
        B.dg_batch_step_host(b, shapes, host, out=host)
        n_e2e = max(1, min(args.steps, args.e2e_steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            B.dg_batch_step_host(b, shapes, host, out=host)
        e2e_s = (time.perf_counter() - t0) / n_e2e
        d2h = sum(3 * wl.K * wl.E * 8 for wl in wls)
        del host
    finally:
        B.dg_batch_destroy(b)
    launch_s = step_ms * 1e-3 / S
    roof = _roofline([(wl.p, wl.E) for wl in wls], wls[0].precision, args.proj, launch_s,
                     _measured_traffic("ensemble-256-" + wls[0].precision + "-" + args.proj, FL.source_hash()),
                     S)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
           "scaling": "strong", "vs_baseline": None,
           "dtype": _dtype(wls[0].precision, args.proj),
           "data": "synthetic (seeded SplitMix64 fields, projected on device)",
           "config": {"workload": "ensemble-%d" % n_total, "instances": n_total,
                      "instances_this_rank": len(wls),
                      "elements_this_rank": sum(wl.E for wl in wls),
                      "p_counts": {str(q): sum(1 for wl in wls if wl.p == q) for q in (1, 2, 3)},
                      "dof_per_stage": dofs, "rk_stages": S, "precision": wls[0].precision,
                      "kernel_form": "tile-fused" if tiled else "per-element",
                      "launch_shape": cls_shapes if tiled else "%d elements per work item" % block,
                      "autotune_ms_per_step": {nm: float(m) for nm, m in zip(cand_names, tune_ms) if m > 0},
                      "l2": "working set per stage > L2 (no flush)",
                      "parallelism": ("instances split over %d ranks" % world) if world > 1 else "single GPU"},
           # one persistent launch per stage, per order class when tile-fused
           "gpu_launches": S * args.steps * (len({wl.p for wl in wls}) if tiled else 1), "roofline": roof,
           "e2e": {"value": dofs * S / e2e_s, "unit": UNIT, "h2d_bytes_per_step": d2h, "d2h_bytes_per_step": d2h},
           "clocks": clk.summary(), "gpu": torch.cuda.get_device_name(local), "host_cores": os.cpu_count(),
           "sim_time_range": [float(min(tvals)), float(max(tvals))]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        picks = [next(wl for wl in wls if wl.p == q) for q in (1, 2, 3) if any(w.p == q for w in wls)]
        parts = [cpu_baseline(wl, args.cpu_seconds / len(picks)) for wl in picks]
        # the whole ensemble at each order class's sampled rate, weighted by
        # the class's share of the ensemble's DOFs
        share = [sum(w.dofs() for w in wls if w.p == wl.p) for wl in picks]
        value = sum(share) / sum(sh / pp["value"] for sh, pp in zip(share, parts))
        out["cpu_baseline"] = {"value": value, "unit": UNIT, "cores": parts[0]["cores"], "kind": "oracle",
                               "sample": "; ".join(pp["sample"] for pp in parts)
                               + " (every order class weighted by its share of the ensemble's DOFs)"}
    return out


def run_ours(args, workload=None, proj=None):
    import torch
    from paper_1904_08684_gb300 import binding as B
    from paper_1904_08684_gb300 import flops as FL
    world, rank, local = _dist()
    B.load()
    wl = WORKLOADS[workload or args.workload]()
    if proj is not None:
        args = argparse.Namespace(**dict(vars(args), proj=proj))
    cfg = _cfg_of(B, wl, args)
    stream = torch.cuda.current_stream()
    hb, xi, qx, qy = _setup_device_inputs(B, torch, wl, cfg, stream)
    ctx = B.dg_init_device(cfg, hb, xi, qx, qy, stream)
    del hb, xi, qx, qy
    S = wl.rk_order
    dof_stage = wl.dofs()
    try:
        B.dg_run(ctx, args.warmup)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(stream)
            B.dg_run(ctx, args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms, step_ms, value = reduce_time_and_value(e0.elapsed_time(e1), dof_stage * S, args.steps, world)
        mass, energy = B.dg_diagnostics(ctx)
        # end-to-end through the public API with host buffers: per step the
        # state goes host -> device (dg_set_state), one dg_run step, and the
        # state comes back (dg_get_state)
        E, K = wl.E, wl.K
        host = [torch.empty((E, K), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
        B.dg_get_state(ctx, E, K, out=host)
        n_e2e = max(1, min(args.steps, args.e2e_steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            B.dg_set_state(ctx, *host, t=0.0)
            B.dg_run(ctx, 1)
            B.dg_get_state(ctx, E, K, out=host)
        e2e_s = (time.perf_counter() - t0) / n_e2e
    finally:
        B.dg_destroy(ctx)
    # roofline of the stage kernel (the only kernel of the timed graphs but
    # for the one-thread time advance)
    launch_s = step_ms * 1e-3 / S
    traffic_key = wl.name if wl.precision == "fp64" else wl.name + "-" + args.proj
    roof = _roofline([(wl.p, wl.E)], wl.precision, args.proj, launch_s,
                     _measured_traffic(traffic_key, FL.source_hash()), S)
    e2e_val = dof_stage * S / e2e_s
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": _dtype(wl.precision, args.proj),
           "data": "synthetic (seeded SplitMix64 fields, projected on device)",
           "config": {"workload": wl.name, "elements": wl.E, "p": wl.p, "K": wl.K, "rk_stages": S,
                      "kernel_form": _single_kernel_form(wl, args),
                      "dof_per_stage": dof_stage, "precision": wl.precision, "bc": wl.bc,
                      "l2": "working set per stage > L2 (no flush)",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           # per step: S stage kernels and the one-thread time-advance kernel
           "gpu_launches": (S + 1) * args.steps,
           "roofline": roof,
           "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 3 * wl.K * wl.E * 8,
                   "d2h_bytes_per_step": 3 * wl.K * wl.E * 8},
           "clocks": clk.summary(), "gpu": torch.cuda.get_device_name(local), "host_cores": os.cpu_count(),
           "diagnostics": {"mass": mass, "energy": energy}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    return out


def _oracle_sample(wl):
    """The FP64 oracle on a contiguous block of elements (1/16 of the mesh) of
    the workload, with the fields projected where the block and its
    neighbours need them."""
    import oracle
    o = oracle.Oracle(wl.nx, wl.ny, wl.p, bc=wl.bc, rk_order=wl.rk_order, cfl=wl.cfl, Lx=wl.Lx, Ly=wl.Ly)
    nsamp = max(1, o.E // 16)
    elems = np.arange(nsamp, dtype=np.int32)
    _, _, nb = o.geometry()
    need = np.zeros(o.E, bool)
    need[elems] = True
    need[nb[elems][nb[elems] >= 0]] = True
    xy = o.proj_nodes()
    vals_hb = np.zeros(xy.shape[:2])
    vals_xi = np.zeros(xy.shape[:2])
    vals_hb[need] = wl.hb(xy[need][..., 0], xy[need][..., 1])
    vals_xi[need] = wl.xi0(xy[need][..., 0], xy[need][..., 1])
    hb = o.project_hb_values(vals_hb)
    xi = o.project_values(vals_xi)
    return o, hb, xi, np.zeros_like(xi), elems


def _time_sample(sample, seconds):
    """repeat the oracle's RHS of the sample (one RK stage of those elements)
    for about ``seconds``; returns (updated DOFs, elapsed s, repetitions)"""
    o, hb, xi, z, elems = sample
    reps, t0 = 0, time.perf_counter()
    while True:
        o.rhs(hb, xi, z, z, elems=elems)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return 3 * o.K * len(elems) * reps, el, reps


def cpu_baseline(wl, seconds):
    """The FP64 oracle, as it stands, on the host cores: right-hand sides of a
    contiguous block of elements (1/16 of the mesh) of the same workload,
    repeated for about ``seconds``; one RHS evaluation is one RK stage."""
    sample = _oracle_sample(wl)
    dofs, el, reps = _time_sample(sample, seconds)
    return {"value": dofs / el, "unit": UNIT, "cores": sample[0].threads(), "kind": "oracle",
            "sample": "oracle RHS (one RK stage) of elements 0..%d of %s, %d repetitions, %.1f s"
                      % (len(sample[4]) - 1, wl.name, reps, el)}


def run_reference(args):
    world, rank, local = _dist()
    if rank != 0:
        return
    all_wls = WORKLOADS[args.workload]()
    ens = isinstance(all_wls, list)
    if ens:                                       # ensemble: one instance per order
        wls = [next(w for w in all_wls if w.p == q) for q in (1, 2, 3) if any(w.p == q for w in all_wls)]
    else:
        wls = [all_wls]
    samples = [_oracle_sample(w) for w in wls]
    per_step = max(0.5, args.cpu_seconds / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        for sm in samples:
            _time_sample(sm, per_step / len(samples))
    d_s = [0.0] * len(samples)
    e_s = [0.0] * len(samples)
    reps = 0
    for _ in range(args.steps):
        for k, sm in enumerate(samples):
            d, e, r = _time_sample(sm, per_step / len(samples))
            d_s[k] += d
            e_s[k] += e
            reps += r
    el = sum(e_s)
    if ens:
        # the whole ensemble's throughput: every order class's DOFs at the
        # rate measured on its sampled instance
        share = [sum(w.dofs() for w in all_wls if w.p == wl.p) for wl in wls]
        value = sum(share) / sum(sh * e / d for sh, d, e in zip(share, d_s, e_s))
        config = {"workload": args.workload, "instances": len(all_wls),
                  "p_counts": {str(q): sum(1 for w in all_wls if w.p == q) for q in (1, 2, 3)},
                  "dof_per_stage": sum(w.dofs() for w in all_wls), "rk_stages": wls[0].rk_order,
                  "precision": "fp64", "parallelism": "host cores"}
        how = "; every order class weighted by its share of the ensemble's DOFs"
    else:
        value = sum(d_s) / el
        wl = wls[0]
        config = {"workload": args.workload, "elements": wl.E, "p": wl.p, "K": wl.K,
                  "rk_stages": wl.rk_order, "precision": "fp64", "bc": wl.bc}
        how = ""
    sample = "oracle RHS (one RK stage) of 1/16 of the elements of %s, %d evaluations in %.1f s%s" % (
        ", ".join(w.name for w in wls), reps, el, how)
    # n_gpus: the launch's N (the oracle itself runs on rank 0's host cores)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "device": "host CPU cores (FP64 oracle)",
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "strong" if ens else "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded SplitMix64 fields)",
           "config": config,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": samples[0][0].threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ensemble-256", choices=sorted(WORKLOADS))
    ap.add_argument("--proj", default=None, choices=["fp64", "fp32", "df64", "mixed"],
                    help="velocity-solve arithmetic of the FP32 state path (default: mixed for "
                         "ensemble-256, fp64 otherwise)")
    ap.add_argument("--block", type=int, default=0, help="threads per block (0 = library default)")
    ap.add_argument("--tile", type=int, default=0, choices=[-1, 0, 1, 2, 3],
                    help="FP32 kernel form: 0 library default, tile shape 1 (8x8), 2 (16x8), 3 (8x4) quads, "
                         "or -1 per-element")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--instances", type=int, default=0, help="ensemble: use only the first N instances")
    ap.add_argument("--p-class", type=int, default=0, help="ensemble: use only the instances of this order")
    ap.add_argument("--no-fp64-plain", action="store_true",
                    help="ensemble: skip the nested plain FP64 measurement")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)      # timing rule: at least 3 untimed steps
    if args.proj is None:
        args.proj = "mixed" if args.workload == "ensemble-256" else "fp64"
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload.startswith("ensemble"):
        wls = WORKLOADS[args.workload]()
        if args.p_class:
            wls = [w for w in wls if w.p == args.p_class]
        out = run_batch(args, wls[:args.instances] if args.instances > 0 else wls)
        if not args.no_fp64_plain:
            # the plain FP64 path on waves-p2-512, same launch, same box
            plain_args = argparse.Namespace(**dict(vars(args), no_cpu_baseline=True))
            plain = run_ours(plain_args, workload="waves-p2-512", proj="fp64")
            keep = ("value", "unit", "ms_per_step", "dtype", "config", "gpu_launches", "roofline", "e2e", "clocks")
            out["fp64_plain"] = {k: plain[k] for k in keep}
            out["speedup_vs_fp64_plain"] = out["value"] / plain["value"]
    else:
        out = run_ours(args)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
