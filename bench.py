#!/usr/bin/env python3
"""Throughput of the compressible-Euler RK step on GB300: cell-updates per second.

One "step" is one midpoint-RK step of the whole hot path (CFL dt from the previous step's
fused epilogue, two fused MinBee/HLLC stage kernels) over the 3D periodic 512^3 blast in FP32
(uniform rho = 1, p = 1e-3, p = 10 within 8 cells of the centre, gamma = 1.4, CFL 0.4).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun (N > 1) every rank advances its own replica of
the grid (the step has no exchange between independent grids): value = all ranks' cell-updates
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK step (512^3 FP32) vs plain FP64; % HBM roofline"
N = 512
GAMMA, CFL, RADIUS = 1.4, 0.4, 8.0
WORKLOAD = "3D periodic 512^3 blast, FP32 stencil, FP64 dt/time/totals"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources each committed ncu record depends on: a record whose digest differs was taken on
# other kernel code and is not used
STAGE_SOURCES = ("hydro_device.cuh", "stage_kernel.cuh", "stage_launch.cuh", "stage_f32_d3.cu",
                 "stage_f32_d3b.cu")
BATCH_SOURCES = ("hydro_device.cuh", "stage_kernel.cuh", "batch_kernel.cuh", "batch_f32.cu")


def _kernel_digest(sources=STAGE_SOURCES) -> str:
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_1204_4779_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _ncu_record(field: str, kernel: str, name: str = "ncu_counters.json", sources=STAGE_SOURCES):
    """Per-launch figure (`per_launch_bytes` or `per_launch_warp_instructions`) of `kernel` in
    the benchmark's workload from a committed ncu summary (profiles/<name>), if it was taken on
    the current kernel source; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            rec = json.load(f)
        if rec.get("kernel_digest") != _kernel_digest(sources):
            return None
        return rec[field].get(kernel)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 100 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_replicas(ms_local: float, units_local: float, device=None):
    """Whole-job throughput of independent replicas: the units all ranks processed divided by
    the slowest rank's time.  Returns (units per second, slowest ms).  Works on any
    initialised process group (NCCL on the GPU machine, gloo in the CPU tests) or alone."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        mx = torch.tensor([ms_local], dtype=torch.float64, device=device)
        tot = torch.tensor([units_local], dtype=torch.float64, device=device)
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        ms, units = float(mx.item()), float(tot.item())
    else:
        ms, units = float(ms_local), float(units_local)
    return units / (ms * 1e-3), ms


def _gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    if ids and ids[min(local_rank, len(ids) - 1)].isdigit():
        return int(ids[min(local_rank, len(ids) - 1)])
    return local_rank


def _cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    try:
        import subprocess
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return os.uname().machine


def cpu_oracle_cups(budget_s: float = 12.0, n: int = 256, max_steps: int = 200, device=None):
    """The FP64 CPU oracle as it stands, on a bounded sample of the workload: the same blast
    at n^3 (radius 8 cells, periodic, CFL 0.4), all host cores, about `budget_s` of CPU work
    after one untimed step.  At 256^3 the oracle's arrays (state, primitives, face states and
    fluxes of every axis, about 520 bytes a cell) are 8.7 GB, far beyond the host's last-level
    cache, as the 512^3 workload is."""
    import oracle
    from paper_1204_4779_gb300 import inputs
    U = oracle.prim_to_cons(inputs.blast_3d(n, radius_cells=RADIUS), GAMMA)
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    U, _, s1, _ = oracle.run(U, GAMMA, CFL, 1, bc=(0, 0, 0), threads=threads)
    one = time.perf_counter() - t0
    steps = max(1, min(max_steps, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    Uo, _, done, _ = oracle.run(U, GAMMA, CFL, steps, bc=(0, 0, 0), threads=threads)
    el = time.perf_counter() - t0
    out = {"value": n ** 3 * done / el, "unit": "cell-updates/s", "cores": threads,
           "kind": "oracle", "cpu_model": _cpu_model(),
           "sample": f"{n}^3 blast (radius {RADIUS:g} cells), {done} FP64 RK steps after one "
                     f"untimed step, {el:.1f} s, OpenMP threads={threads}, "
                     f"host={os.uname().machine}; working set about {520 * n ** 3 / 1e9:.1f} GB "
                     f"(beyond the last-level cache)"}
    if device is not None:
        out["gpu_error_vs_oracle"] = _gpu_error(n, 1 + done, Uo, device)
    return out


def _gpu_error(n, steps, Uo, device):
    """The GPU's FP32 and FP64 results after the same steps from the same FP64 initial data as
    the oracle's sample: L1 density error (FP32) and max relative error (FP64, per field:
    elementwise for rho and E, normwise for the momenta)."""
    import numpy as np
    import torch

    from paper_1204_4779_gb300 import hydro, inputs
    V = torch.from_numpy(inputs.blast_3d(n, radius_cells=RADIUS)).to(device)
    U64 = hydro.prim_to_cons(V, GAMMA)
    res = {"steps": steps}
    for dt, key in ((torch.float32, "fp32_l1_rho"), (torch.float64, "fp64_max_rel")):
        U = U64.to(dt).contiguous()
        S = hydro.Solver((n, n, n), GAMMA, bc="periodic", dtype=dt, cfl=CFL, device=device)
        S.step(U, steps)
        G = U.double().cpu().numpy()
        S.close()
        if dt == torch.float32:
            res[key] = float(np.abs(G[0] - Uo[0]).sum() / np.abs(Uo[0]).sum())
        else:
            e = [float(np.max(np.abs(G[k] - Uo[k]) / np.abs(Uo[k]))) for k in (0, 4)]
            e += [float(np.max(np.abs(G[k] - Uo[k])) / max(float(np.max(np.abs(Uo[k]))), 1e-300))
                  for k in (1, 2, 3)]
            res[key] = max(e)
    return res


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, each step one RK step of a bounded
    128^3 sample of the blast workload (about 1.1 GB of oracle arrays, beyond the host's
    last-level cache)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1204_4779_gb300 import inputs
    n = args.ref_size
    U = oracle.prim_to_cons(inputs.blast_3d(n, radius_cells=RADIUS), GAMMA)
    threads = oracle.max_threads()
    U, *_ = oracle.run(U, GAMMA, CFL, args.warmup, bc=(0, 0, 0), threads=threads)
    t0 = time.perf_counter()
    _, _, done, _ = oracle.run(U, GAMMA, CFL, args.steps, bc=(0, 0, 0), threads=threads)
    el = time.perf_counter() - t0
    value = n ** 3 * done / el
    line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(done, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": f"{n}^3 blast per step on the host",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": threads,
                             "kind": "oracle", "cpu_model": _cpu_model(),
                             "sample": f"{n}^3 blast (radius {RADIUS:g} cells), {done} RK steps"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1204_4779_gb300 import hydro, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    n = args.size
    ncell = n ** 3
    V = inputs.blast_3d_torch(n, RADIUS, device=dev)
    U = hydro.prim_to_cons(V, GAMMA).to(torch.float32).contiguous()
    U_init = U.clone()
    del V
    S = hydro.Solver((n, n, n), GAMMA, bc="periodic", dtype=torch.float32, cfl=CFL,
                     variant=dict(staging=args.staging) if args.staging else None)
    variant = S.variant()
    variant = {"tile": list(variant["tile"]), "march": variant["march"],
               "split": "fused dt reduction" if variant["split"] == 2 else "separate CFL pass",
               "staging": {1: "look-ahead", 2: "at use", 3: "TMA"}[variant["staging"]],
               "occupancy": variant["occupancy"]}
    # measured FMA throughput of this GPU (the FP32 roofline's denominator), before the warm-up
    fma32 = hydro.fma_rate(torch.float32, dev)
    fma64 = hydro.fma_rate(torch.float64, dev)
    S.step(U, args.warmup)
    torch.cuda.synchronize()
    U_start = U.clone() if args.repeats > 0 else None

    # --- timed region: K RK steps, per-kernel CUDA events on the launching stream ----------
    S.set_profiling(True)
    S.kernel_times(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(_gpu_index(local)) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record()
        t_sim, done = S.step(U, args.steps)
        ev1.record()
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    kt = S.kernel_times(reset=True)
    S.set_profiling(False)
    if done != args.steps:
        raise RuntimeError(f"only {done} of {args.steps} steps ran")
    value, ms_max = aggregate_replicas(ms, ncell * args.steps, device=dev)

    # --- the paper's protocol: R runs of K steps replayed from CUDA graphs, mean and std ----
    repeats = None
    if args.repeats > 0:
        U.copy_(U_start)
        S.step(U, args.steps)  # capture the step graphs outside the timed runs
        runs = []
        for _ in range(args.repeats):
            U.copy_(U_start)
            barrier()
            torch.cuda.synchronize()
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            r0.record()
            S.step(U, args.steps, sync=False)
            r1.record()
            torch.cuda.synchronize()
            barrier()
            v, _ = aggregate_replicas(r0.elapsed_time(r1), ncell * args.steps, device=dev)
            runs.append(v)
        mu = sum(runs) / len(runs)
        sd = (sum((x - mu) ** 2 for x in runs) / max(len(runs) - 1, 1)) ** 0.5
        repeats = {"runs": len(runs), "steps_each": args.steps, "mean": mu, "std": sd,
                   "min": min(runs), "max": max(runs), "unit": "cell-updates/s",
                   "how": "state reset to the post-warm-up state before each run; steps replayed "
                          "from the context's CUDA graphs (no per-kernel events); CUDA events "
                          "around each run"}
        del U_start

    # --- roofline of the dominant kernel ---------------------------------------------------
    hbm, peak_kind = _peaks()
    nv = 5
    alg = {"stage1": 2 * nv * 4 * ncell, "stage2": 3 * nv * 4 * ncell}  # bytes per launch
    step_bytes = alg["stage1"] + alg["stage2"]
    dom = max(("stage1", "stage2"), key=lambda k: kt[k][0])
    avg_ms = kt[dom][0] / max(kt[dom][1], 1)
    achieved = alg[dom] / (avg_ms * 1e-3) / 1e9
    traffic = _ncu_record("per_launch_bytes", dom)
    winst = _ncu_record("per_launch_warp_instructions", dom)
    kernels = {k: {"avg_ms": v[0] / max(v[1], 1), "launches": v[1],
                   "alg_bytes_per_launch": alg.get(k, nv * 4 * ncell)} for k, v in kt.items()}

    # --- end to end through the C ABI with host buffers -------------------------------------
    e2e = None
    if args.e2e_steps > 0:
        host = U_init.cpu().pin_memory()
        dev_state = torch.empty_like(U_init)
        for _ in range(2):  # warm (copies + step)
            S.step_host(dev_state, host, host, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps + 1)]
        barrier()
        torch.cuda.synchronize()
        e0.record()
        marks[0].record()
        for i in range(args.e2e_steps):
            S.step_host(dev_state, host, host, 1)
            marks[i + 1].record()
        e1.record()
        torch.cuda.synchronize()
        barrier()
        e2e_value, _ = aggregate_replicas(e0.elapsed_time(e1), ncell * args.e2e_steps, device=dev)
        calls = [a.elapsed_time(b) for a, b in zip(marks, marks[1:])]
        per_call = sorted(calls)
        nbytes = nv * 4 * ncell
        # the CPU-GPU link alone: the same state copied each way (pinned memory, CUDA events)
        link = {}
        for name, dst, src in (("h2d_gbs", dev_state, host), ("d2h_gbs", host, dev_state)):
            best = None
            for _ in range(3):
                torch.cuda.synchronize()
                e0.record()
                dst.copy_(src, non_blocking=True)
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
            link[name] = nbytes / (best * 1e-3) / 1e9
        # two problems in flight: hydro_step_host_async on two contexts with their own streams,
        # the calls alternating, so that one problem's copy in runs during the other's copy
        # back (the link carries both directions at once); every step still copies its whole
        # state in and out
        S2 = hydro.Solver((n, n, n), GAMMA, bc="periodic", dtype=torch.float32, cfl=CFL,
                          variant=dict(staging=args.staging) if args.staging else None)
        solvers = (S, S2)
        hosts = (host, U_init.cpu().pin_memory())
        devs = (dev_state, torch.empty_like(U_init))
        streams = (torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev))

        def async_call(k):
            p = k % 2
            with torch.cuda.stream(streams[p]):
                solvers[p].step_host_async(devs[p], hosts[p], hosts[p], 1)

        for k in range(4):  # warm (graphs, copies)
            async_call(k)
        status = [sv.status() for sv in solvers]
        k_pipe = args.e2e_steps + (args.e2e_steps & 1)
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for k in range(k_pipe):
            async_call(k)
        status += [sv.status() for sv in solvers]
        w1 = time.perf_counter()
        barrier()
        pipe_value, _ = aggregate_replicas((w1 - w0) * 1e3, ncell * k_pipe, device=dev)
        pipelined = {"value": pipe_value, "unit": "cell-updates/s", "steps": k_pipe,
                     "problems_in_flight": 2, "ms_per_step": (w1 - w0) * 1e3 / k_pipe,
                     "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                     "status_ok": all(x == 0 for x in status),
                     "call": "hydro_step_host_async on two contexts and streams, calls "
                             "alternating: each call copies its problem's pinned host state in, "
                             "takes 1 RK step and copies it back in place; host wall clock "
                             "from the first call to both streams' completion"}
        del S2, solvers, hosts, devs
        e2e = {"value": e2e_value,
               "unit": "cell-updates/s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "steps": args.e2e_steps,
               "call": "hydro_step_host: pinned host state in, 1 RK step, host state out",
               "per_call_ms": {"min": per_call[0], "median": per_call[len(per_call) // 2],
                               "max": per_call[-1], "in_order": [round(c, 2) for c in calls]},
               "link": dict(link, note="plain copies of the state over the CPU-GPU link; the "
                                       "step's copies alone take nbytes/h2d + nbytes/d2h"),
               "pipelined": pipelined}

    # the kernel's real limit: instruction issue (4 warp-instructions per clock per SM)
    clocks = clk.summary()
    issue = None
    if winst is not None:
        props = torch.cuda.get_device_properties(dev)
        mhz = clocks.get("sm_mhz") or 2070.0
        peak = 4.0 * props.multi_processor_count * mhz * 1e6
        ach = winst / (avg_ms * 1e-3)
        issue = {"kernel": dom, "achieved": ach, "peak": peak, "unit": "warp-instructions/s",
                 "frac": ach / peak, "warp_instructions_per_launch": winst,
                 "source": "ncu smsp__inst_executed.sum (profiles/ncu_counters.json) / live "
                           "CUDA-event launch time; peak = 4 x SMs x sampled SM clock"}

    # FP64 throughput of the same workload (the FP64 form of the stage kernels), graph replay
    fp64 = None
    if args.fp64_steps > 0:
        del U_init
        V64 = inputs.blast_3d_torch(n, RADIUS, device=dev)
        U64 = hydro.prim_to_cons(V64, GAMMA)
        del V64
        S64 = hydro.Solver((n, n, n), GAMMA, bc="periodic", dtype=torch.float64, cfl=CFL, device=dev)
        S64.step(U64, args.fp64_steps)  # graphs and warm-up
        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        S64.step(U64, args.fp64_steps, sync=False)
        f1.record()
        torch.cuda.synchronize()
        barrier()
        v64, ms64 = aggregate_replicas(f0.elapsed_time(f1), ncell * args.fp64_steps, device=dev)
        fp64 = {"value": v64, "unit": "cell-updates/s", "steps": args.fp64_steps,
                "ms_per_step": ms64 / args.fp64_steps, "dtype": "f64"}
        S64.close()
        del U64, S64

    # FP32 roofline of the whole step: the FP32 lane operations the two stage kernels execute
    # per cell (FADD, FMUL, FFMA and the packed f32x2 forms counted twice, from the committed ncu
    # capture of the current kernels) times the cell-updates per second, against the FMA rate
    # measured live (one lane operation per lane per clock)
    fp32 = None
    lane = _ncu_record("fp32_lane_ops_per_cell", "stage1"), _ncu_record("fp32_lane_ops_per_cell", "stage2")
    if None not in lane:
        ops = lane[0] + lane[1]
        ach = ops * ncell * args.steps / (ms_max * 1e-3)
        fp32 = {"bound": "alu", "scope": "whole RK step (both stage kernels)", "achieved": ach,
                "peak": fma32, "unit": "FP32 lane-operations/s", "frac": ach / fma32,
                "ops_per_cell_update": ops, "fma_rate_f64": fma64,
                "source": "ncu-counted FP32 add/multiply/FMA lane operations of the stage kernels "
                          "per cell (profiles/ncu_counters.json fp32_lane_ops_per_cell, f32x2 "
                          "counted twice); peak = hydro_fma_rate measured live"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_cups(device=dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if n == N else WORKLOAD.replace("512^3", f"{n}^3"),
                       "grid": [n, n, n], "gamma": GAMMA, "cfl": CFL,
                       "blast_radius_cells": RADIUS, "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 ({5 * 4 * ncell / 2**30:.2f} GiB state vs 129 MB L2); no flush",
                       "host": "Python cyclic GC off during the run",
                       "variant": variant},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "kernel": dom,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "step_frac": step_bytes / (ms_max / args.steps * 1e-3) / 1e9 / hbm,
                         "step_frac_note": "the whole RK step time-weighted: 100 B per cell "
                                           "(stage 1 40 B, stage 2 60 B) over the step time"},
            "kernels": kernels,
            "gpu_launches": int(sum(v[1] for v in kt.values())),
            "clocks": clocks,
            "issue_roofline": issue,
            "fp32_roofline": fp32,
            "repeats": repeats,
            "fp64": fp64,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "sim_time": t_sim,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_wave(args):
    """The paper's linear-wave example (hydro_wave_run, f_t = g, g_t = c^2 f_xx on a periodic 1D
    grid) at --size cells (default 2^27) in FP32 (or --dtype f64): steps timed with CUDA events
    around the call, against the HBM roofline of its algorithmic traffic (read f and g, write
    both: 16 B per cell-update in FP32)."""
    import math

    import torch

    from paper_1204_4779_gb300 import hydro
    torch.cuda.set_device(0)
    n = args.size if args.size != N else 1 << 27
    f64 = args.dtype == "f64"
    dtype = torch.float64 if f64 else torch.float32
    esz = 8 if f64 else 4
    L, c = 2.0 * math.pi, 1.0
    dt = 0.5 * (L / n) / c
    x = torch.arange(n, dtype=torch.float64, device="cuda") * (L / n)
    f = torch.sin(x).to(dtype)
    g = torch.zeros(n, dtype=dtype, device="cuda")
    del x
    steps = args.steps + (args.steps & 1)  # even: the result ends in the caller's arrays
    hydro.wave_run(f, g, c, L, dt, 2 * args.warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(_gpu_index(0)) as clk:
        torch.cuda.synchronize()
        e0.record()
        E = hydro.wave_run(f, g, c, L, dt, steps)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    hbm, peak_kind = _peaks()
    achieved = 4 * esz * n * steps / (ms * 1e-3) / 1e9
    drift = max(abs(e - E[0]) for e in E) / abs(E[0])
    line = {"metric": f"cell-updates/s per step, linear wave {n} cells ({'FP64' if f64 else 'FP32'})",
            "value": n * steps / (ms * 1e-3), "unit": "cell-updates/s", "n_gpus": 1,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if f64 else "f32", "data": "synthetic",
            "config": {"workload": f"1D periodic linear wave (the paper's section 2.3 example), {n} cells, "
                                   "c = 1, dt = dx / 2, one sine period",
                       "l2": f"state {2 * esz * n / 2**20:.0f} MiB vs 129 MB L2; no flush",
                       "energy_drift": drift},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None,
                         "kernel": ("wave_step_kernel_f64v" if n % 2 == 0 else "wave_step_kernel")
                         if f64 else ("wave_step_kernel_f32v" if n % 4 == 0 else "wave_step_kernel_f32"),
                         "scope": "whole call (step kernels and the per-step energy sums)",
                         "bytes_per_cell_update": 4 * esz,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
            "gpu_launches": 2 * steps, "clocks": clk.summary(), "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def run_kh2d(args):
    """A 2D line: the shear layer (Kelvin-Helmholtz data, gamma 5/3, periodic, seed 1204477901) at
    --size^2 (default 2048) in FP32 (or --dtype f64) with the library's default 2D variant (FP32:
    row tiles; FP64: the 32 x 8 tile).  The value times hydro_step calls of --steps steps as a
    user makes them (graph replay, no per-launch events; the calls repeated, continuing the run,
    until about half a second has been timed, so that the clock sampler sees the load); the
    kernel times come from one more call with per-launch events."""
    import math

    import torch

    from paper_1204_4779_gb300 import hydro, inputs
    torch.cuda.set_device(0)
    n = args.size if args.size != N else 2048
    V = torch.from_numpy(inputs.kh_2d(n, seed=1204477901)).cuda()
    f64 = args.dtype == "f64"
    dtype = torch.float64 if f64 else torch.float32
    esz = 8 if f64 else 4
    U = hydro.prim_to_cons(V, 5.0 / 3.0).to(dtype).contiguous()
    del V
    S = hydro.Solver((n, n), 5.0 / 3.0, bc="periodic", dtype=dtype, cfl=CFL)
    variant = S.variant()
    S.step(U, args.warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_call():
        ev0.record()
        _, d = S.step(U, args.steps)
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), d

    ms0, _ = timed_call()  # sizes the repetition count (not timed)
    calls = max(1, min(1000, int(math.ceil(500.0 / max(ms0, 1e-3)))))
    total, done = 0.0, 0
    with ClockSampler(_gpu_index(0)) as clk:
        torch.cuda.synchronize()
        for _ in range(calls):
            ms_c, d = timed_call()
            total += ms_c
            done += d
    ms = total / calls
    S.set_profiling(True)
    S.kernel_times(reset=True)
    S.step(U, args.steps)
    torch.cuda.synchronize()
    kt = S.kernel_times(reset=True)
    S.set_profiling(False)
    ncell = n * n
    hbm, peak_kind = _peaks()
    alg = {"stage1": 2 * 4 * esz * ncell, "stage2": 3 * 4 * esz * ncell}
    dom = max(("stage1", "stage2"), key=lambda k: kt[k][0])
    avg_ms = kt[dom][0] / max(kt[dom][1], 1)
    achieved = alg[dom] / (avg_ms * 1e-3) / 1e9
    prec = "FP64" if f64 else "FP32"
    line = {"metric": f"cell-updates/s per RK step, 2D shear layer {n}^2 ({prec})",
            "value": ncell * args.steps / (ms * 1e-3), "unit": "cell-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if f64 else "f32", "data": "synthetic",
            "config": {"workload": f"2D periodic {n}^2 shear layer, gamma 5/3, {prec}",
                       "l2": f"state {4 * esz * ncell / 2**20:.0f} MiB vs 129 MB L2; no flush",
                       "variant": {"tile": list(variant["tile"]), "march": variant["march"],
                                   "split": variant["split"], "occupancy": variant["occupancy"]}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None, "kernel": dom,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
            "kernels": {k: {"avg_ms": v[0] / max(v[1], 1), "launches": v[1]} for k, v in kt.items()},
            "gpu_launches": calls * int(sum(v[1] for v in kt.values())),
            "clocks": clk.summary(), "timed_calls": calls, "steps_done": done}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """The batched configuration: 4096 independent 2D grids, sides log-uniform on [32, 512]
    (seed 1204477904), seeded smooth data, gamma 1.4, FP32, one persistent launch per RK
    stage, steps replayed from CUDA graphs (timed with per-launch events)."""
    import numpy as np
    import torch

    from paper_1204_4779_gb300 import hydro, inputs
    torch.cuda.set_device(0)
    shapes = [tuple(int(v) for v in s) for s in inputs.batch_shapes()]
    P = np.concatenate([inputs.batch_grid(nx, ny, 1204477904, i).reshape(4, -1)
                        for i, (nx, ny) in enumerate(shapes)], axis=1)
    U = hydro.prim_to_cons(torch.from_numpy(P).cuda().view(4, 1, -1), GAMMA).view(4, -1)
    U = U.to(torch.float32).contiguous()
    del P
    B = hydro.BatchSolver(shapes, GAMMA, dtype=torch.float32, cfl=CFL)
    ncell = B.total
    B.step(U, args.warmup)
    torch.cuda.synchronize()
    B.set_profiling(True)
    B.kernel_times(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(_gpu_index(0)) as clk:
        torch.cuda.synchronize()
        ev0.record()
        _, done = B.step(U, args.steps)
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    kt = B.kernel_times(reset=True)
    hbm, peak_kind = _peaks()
    alg = {"stage1": 2 * 4 * 4 * ncell, "stage2": 3 * 4 * 4 * ncell}
    dom = max(("stage1", "stage2"), key=lambda k: kt[k][0])
    avg_ms = kt[dom][0] / max(kt[dom][1], 1)
    achieved = alg[dom] / (avg_ms * 1e-3) / 1e9
    line = {"metric": "cell-updates/s per RK step, batched 4096 uneven 2D grids (FP32)",
            "value": ncell * args.steps / (ms * 1e-3), "unit": "cell-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "4096 independent 2D grids, sides log-uniform on [32, 512] "
                                   "(seed 1204477904), smooth seeded data, FP32",
                       "cells": ncell, "l2": "inputs larger than L2 (1.9 GB state); no flush",
                       "variant": "library default: row tiles of 32 columns marching 32 rows "
                                  "along y, one work item per strip and chunk"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm,
                         "traffic": _ncu_record("per_launch_bytes", dom, "ncu_counters_batched.json",
                                                BATCH_SOURCES),
                         "kernel": "batch_" + dom,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
            "kernels": {k: {"avg_ms": v[0] / max(v[1], 1), "launches": v[1]} for k, v in kt.items()},
            "gpu_launches": int(sum(v[1] for v in kt.values())), "clocks": clk.summary(),
            "steps_done_min": min(done)}
    print(json.dumps(line), flush=True)


def run_aux(args):
    """The two reductions of the step on their own, on the blast state (--size^3, FP32): the
    CFL pass (hydro_cfl_dt: max of the CFL signal over U, then dt; 20 B per cell read) and the
    FP64 totals audit (hydro_totals: fixed-order partial sums per CTA, then the final sum; 20 B
    per cell read).  Each call synchronises (its result comes back to the host); CUDA events
    around --steps calls after --warmup calls."""
    import torch

    from paper_1204_4779_gb300 import hydro, inputs
    torch.cuda.set_device(0)
    n = args.size
    V = inputs.blast_3d_torch(n, RADIUS, device="cuda")
    U = hydro.prim_to_cons(V, GAMMA).to(torch.float32).contiguous()
    del V
    S = hydro.Solver((n, n, n), GAMMA, bc="periodic", dtype=torch.float32, cfl=CFL)
    hbm, peak_kind = _peaks()
    nbytes = 5 * 4 * n ** 3
    out = {}
    with ClockSampler(_gpu_index(0)) as clk:
        for name, call in (("cfl_pass", lambda: S.cfl_dt(U)), ("totals", lambda: S.totals(U))):
            for _ in range(args.warmup):
                call()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(args.steps):
                call()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            out[name] = {"ms_per_call": ms, "achieved_gbs": nbytes / (ms * 1e-3) / 1e9,
                         "frac": nbytes / (ms * 1e-3) / 1e9 / hbm}
    S.close()
    line = {"metric": f"HBM throughput of the CFL pass and the totals audit, {n}^3 FP32 blast",
            "value": out["cfl_pass"]["achieved_gbs"], "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{n}^3 blast state, FP32 (20 B per cell read by each call)",
                       "l2": f"state {nbytes / 2**30:.2f} GiB vs 129 MB L2; no flush",
                       "timing": "CUDA events around whole calls (kernels, the 8-byte result "
                                 "copy and the synchronisation)"},
            "roofline": {"bound": "hbm", "peak": hbm, "unit": "GB/s",
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)", **out},
            "clocks": clk.summary(), "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def run_mlp(args):
    """The cost model's training (hydro_mlp_train: forward, loss, back-propagation and Adam of
    the 3-layer width-64 MLP on every record, epochs replayed from a CUDA graph) on a seeded
    synthetic record set of the tuner's size: --size records (default 4200) of the 3D feature
    width; epochs per second over --steps epochs after --warmup."""
    import numpy as np
    import torch

    from paper_1204_4779_gb300 import costmodel, tuner
    torch.cuda.set_device(0)
    n = args.size if args.size != N else 4200
    space = tuner.Space(3)
    d = len(tuner.features(space, space.default_genome(), (64, 64, 64)))
    rng = np.random.default_rng(1204477905)
    X = rng.normal(0.0, 1.0, (n, d)).astype(np.float32)
    t = rng.normal(0.0, 1.0, n).astype(np.float32)
    net = costmodel.MLP(d, 64, seed=0)
    net.train(X, t, max(args.warmup, 1))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    losses = net.train(X, t, args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    line = {"metric": f"cost-model training epochs/s ({n} records, width 64)",
            "value": args.steps / (ms * 1e-3), "unit": "epochs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": f"{n} seeded records x {d} features",
                                            "loss_first_last": [float(losses[0]), float(losses[-1])]},
            "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--e2e-steps", type=int, default=40,
                    help="timed hydro_step_host calls of one step each (mean over the calls)")
    ap.add_argument("--size", type=int, default=N, help="cube side (the benchmark config is 512)")
    ap.add_argument("--config", choices=("blast512", "batched", "kh2d", "wave", "aux", "mlp"),
                    default="blast512",
                    help="blast512: the benchmark line; batched: the 4096-grid configuration; "
                         "kh2d: the 2D shear layer (--size, default 2048); wave: the linear-wave "
                         "example (--size, default 2^27); aux: the CFL pass and the totals audit "
                         "alone (--size^3); mlp: the cost model's training (--size records)")
    ap.add_argument("--dtype", choices=("f32", "f64"), default="f32",
                    help="precision of the kh2d and wave lines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--staging", type=int, default=0, choices=(0, 1, 2, 3),
                    help="blast512: the stage kernels' staging (0 library default, 1 look-ahead "
                         "loads, 2 loads at use, 3 TMA)")
    ap.add_argument("--ref-size", type=int, default=128,
                    help="cube side of the reference arm's per-step sample (the oracle on the host)")
    ap.add_argument("--fp64-steps", type=int, default=10,
                    help="timed FP64 steps of the same workload after the FP32 run (0: none)")
    ap.add_argument("--repeats", type=int, default=30,
                    help="extra graph-replay runs of --steps steps for mean and std (0: none)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    # Python's cyclic garbage collector off for the run (as timeit does): its pauses stall the
    # host thread that issues the launches and copies, tens of milliseconds at a time
    gc.collect()
    gc.disable()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batched":
        run_batched(args)
    elif args.config == "kh2d":
        run_kh2d(args)
    elif args.config == "wave":
        run_wave(args)
    elif args.config == "aux":
        run_aux(args)
    elif args.config == "mlp":
        run_mlp(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
