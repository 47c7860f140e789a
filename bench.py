#!/usr/bin/env python
"""Benchmark of the GB300 RMT per-step update: FSI cell-updates/s.

Default workload: the 256^3 triply periodic active-swimmer scene (8 ellipsoids with an active
bending stress, FP32 bulk with two-float refinement of the projections).  One "step" is one full
timestep of the 13-step algorithm over the whole grid.  Inputs (fields of 256^3 cells, several
GB) are far larger than the 129 MB L2, so no cache flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config NAME]

N > 1 runs one independent replica per GPU (launched with torch.distributed.run); value is the
cell-updates/s of all replicas together, timed between barriers, max over ranks.
--impl reference times the FP64 CPU oracle on all host cores (OpenMP) on a bounded sample of the
same scene (the same bodies and constants on a 64^3 grid).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FSI cell-updates/s"
CONFIGS = {
    # name: (scene factory kwargs, description)
    "swimmers256": dict(kind="swimmers", n=256, precision="fp32",
                        desc="256^3 triply periodic unit box, 8 active-stress ellipsoid swimmers "
                             "(0.15,0.04,0.04), G=1, mu=mu_a=0.01, A=0.5, omega=2pi; FP32 bulk with "
                             "two-float refinement of the projections"),
    "swimmers256_fp64": dict(kind="swimmers", n=256, precision="fp64",
                             desc="the same 256^3 swimmer scene on the plain FP64 path"),
    "settling128": dict(kind="settling", n=128, precision="fp64",
                        desc="128^3 no-slip box, 20 settling ellipsoids (10 at 1.5, 10 at 0.5), FP64"),
    "cavity32": dict(kind="cavity", n=32, precision="fp64", desc="32^3 lid-driven cavity, one soft sphere, FP64"),
}
CPU_SAMPLE_N = 64


def make_scene(cfg: dict, n: int | None = None, nbodies: int | None = None):
    from paper_2104_00095_gb300 import scenes as S

    n = n or cfg["n"]
    kw = {} if nbodies is None else {"nbodies": nbodies}
    if cfg["kind"] == "swimmers":
        return S.swimmers(n=n, precision=cfg["precision"], **kw)
    if cfg["kind"] == "settling":
        return S.settling(n=n, precision=cfg["precision"], **kw)
    return S.cavity_sphere(n, precision=cfg["precision"])


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x of all ranks (x itself when world == 1)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, cells: int, steps: int, seconds: float) -> float:
    """Whole-job cell-updates/s: every replica advances its own grid of `cells` cells."""
    return world * cells * steps / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        self.skip = 0

    def _rows(self) -> list:
        with open(self.f.name) as f:
            return [r for r in f.read().splitlines() if r.strip()]

    def begin(self, timeout_s: float = 3.0):
        """Waits until the sampler has printed (NVML is up), then marks the start of the timed
        region: only samples taken after this point are reported."""
        if self.p is None:
            return
        t0 = time.perf_counter()
        while not self._rows() and time.perf_counter() - t0 < timeout_s and self.p.poll() is None:
            time.sleep(0.01)
        self.skip = len(self._rows())

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        lines = self._rows()
        os.unlink(self.f.name)
        # the samples of the timed region (the last earlier one if the region ended before the next)
        lines = lines[self.skip:] if len(lines) > self.skip else lines[-1:]
        rows = [r.split(",") for r in lines]
        sm, smax, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
                pw.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def dram_traffic(kernel: str, cells: int):
    """DRAM bytes per launch of `kernel` at `cells` cells, from the committed ncu record of a small
    case (profiles/dram_traffic_small_case.txt: bytes per launch measured on a grid of a few GB,
    scaled by the cell count, since the kernel moves a fixed number of bytes per cell), or None
    when there is no record or the kernel's source file changed since it was taken."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic_small_case.txt")) as f:
            lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    for name, nbytes, ncells, src, sha in lines:
        if name != kernel:
            continue
        try:
            with open(os.path.join(ROOT, src), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest()[:len(sha)] != sha:
                    return None
        except OSError:
            return None
        return float(nbytes) * cells / float(ncells)
    return None


def host_cores() -> int:
    """Threads the oracle's OpenMP loops use: OMP_NUM_THREADS, else every core this process may run on."""
    try:
        return int(os.environ["OMP_NUM_THREADS"])
    except (KeyError, ValueError):
        return len(os.sched_getaffinity(0))


def cpu_oracle_rate(cfg: dict, steps: int, warmup: int):
    """cell-updates/s of the FP64 oracle (OpenMP over all host cores) on the CPU_SAMPLE_N^3 copy
    of the scene."""
    import oracle as O

    sc = make_scene(cfg, CPU_SAMPLE_N)
    sc["precision"] = "fp64"
    o = O.Oracle(sc)
    o.read(O.F_RHO)  # initialisation outside the timed region
    for _ in range(warmup):
        o.step(1)
    t0 = time.perf_counter()
    rc = o.step(steps)
    dt = time.perf_counter() - t0
    if rc != 0:
        raise RuntimeError(f"oracle step failed: {o.error()}")
    return CPU_SAMPLE_N**3 * steps / dt, dt


def run_reference(args, cfg):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    rate, dt = cpu_oracle_rate(cfg, args.steps, args.warmup)
    sample = (f"{args.steps} timed steps (after {args.warmup} warm-up) of the same scene on a "
              f"{CPU_SAMPLE_N}^3 grid (all bodies), FP64 oracle, {host_cores()} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.config + f" (sampled at {CPU_SAMPLE_N}^3)"},
            "cpu_baseline": {"value": rate, "unit": "cell-updates/s", "cores": host_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(g, steps: int, stream) -> float:
    """ms per step of g over `steps` steps (CUDA events on the stream)."""
    import torch

    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    g.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def step_model_words(args) -> float:
    """Words moved per cell-step by the whole-step byte model: 55 outside the projections, and
    about 24 per V-cycle for 6 fine-level passes (2 + 2 sweeps, the residual and the transfers),
    scaled by the passes the schedule makes; 8/7 for the coarser levels."""
    mac_passes = 2 * args.mac_sweeps + 2
    fe_passes = args.fe_pre + args.fe_post + 2
    return 55 + 24 * (args.mg_cycles_mac * mac_passes / 6.0 + args.mg_cycles_fe * fe_passes / 6.0) * 8.0 / 7.0


def solver_options(args, graph: bool = True) -> dict:
    """The multigrid schedule of the timed configuration (rmt_set_option names)."""
    o = {"fe_inner": args.fe_inner, "mac_inner": args.mac_inner, "mac_warm": args.mac_warm, "fe_warm": args.fe_warm,
         "mac_pre": args.mac_sweeps, "mac_post": args.mac_sweeps, "mac_omega": args.mac_omega,
         "mac_coarse_pre": args.mac_coarse, "mac_coarse_post": args.mac_coarse,
         "fe_pre": args.fe_pre, "fe_post": args.fe_post, "fe_omega": args.fe_omega}
    if graph:
        o["graph"] = args.graph
    return o


def plain_fp64_leg(cfg: dict, args, stream) -> dict:
    """The same workload on the plain FP64 path (no mixed precision), same cycle counts."""
    from paper_2104_00095_gb300 import rmt

    sc = make_scene(cfg, n=args.n, nbodies=args.nbodies)
    sc.update(precision="fp64", mg_fixed_cycles=args.mg_cycles_mac, mg_fixed_cycles_fe=args.mg_cycles_fe,
              options=solver_options(args))
    g = rmt.Grid(sc, stream=stream.cuda_stream)
    g.step(3)
    k = max(3, args.steps // 2)
    ms = timed_steps(g, k, stream)
    n = int(np.prod(sc["n"]))
    g.close()
    return {"value": n / (ms / 1e3), "unit": "cell-updates/s", "ms_per_step": ms, "steps": k, "dtype": "f64"}


def settling_leg(args, stream) -> dict:
    """Config 2: the 128^3 settling mixture (20 ellipsoids, 10 heavy and 10 buoyant, gravity, no-slip
    walls) on the plain FP64 path and in the FP32 form side by side, with the bench's multigrid
    schedule; beside them the relative L2 difference of u between the two after the same steps."""
    from paper_2104_00095_gb300 import rmt, scenes as S

    out, us = {}, {}
    for prec in ("fp64", "fp32"):
        sc = S.settling(n=128, precision=prec)
        sc.update(mg_fixed_cycles=args.mg_cycles_mac, mg_fixed_cycles_fe=args.mg_cycles_fe,
                  options=solver_options(args))
        g = rmt.Grid(sc, stream=stream.cuda_stream)
        g.step(3)
        k = 5
        ms = timed_steps(g, k, stream)
        us[prec] = g.read(rmt.RMT_F_U)
        n = int(np.prod(sc["n"]))
        out[prec] = {"value": n / (ms / 1e3), "unit": "cell-updates/s", "ms_per_step": ms, "steps": k}
        g.close()
    out["workload"] = "settling128: 128^3 no-slip box, 20 ellipsoids (10 at 1.5, 10 at 0.5), gravity -z"
    out["u_rel_l2_fp32_vs_fp64_after_8_steps"] = float(np.linalg.norm(us["fp32"] - us["fp64"]) /
                                                       np.linalg.norm(us["fp64"]))
    return out


def batched_leg(args, stream) -> dict:
    """64 independent lid-driven cavities of {32..128}^3 with 1-6 spheres, FP32, advanced as one
    batch (one CUDA-graph launch per step).  The multigrid schedule of each grid size is picked by
    the autotuner (relative residual 1e-6) on one grid of that size.  Beside it: the same grids
    stepped one after another."""
    import torch

    from paper_2104_00095_gb300 import rmt, scenes as S

    scenes = S.batched(nsims=args.batch_sims)
    cells = sum(int(np.prod(sc["n"])) for sc in scenes)
    grids = [rmt.Grid(sc, stream=stream.cuda_stream) for sc in scenes]
    tuned = {}
    t0 = time.perf_counter()
    for g, sc in zip(grids, scenes):
        n = sc["n"][0]
        if n not in tuned:
            g.step(1)
            tuned[n] = g.autotune(1e-6)
    tune_s = time.perf_counter() - t0
    keys = ("mac_pre", "mac_post", "mac_inner", "mac_block", "mac_cycles", "fe_pre", "fe_post", "fe_inner",
            "fe_block", "fe_omega", "fe_cycles", "mac_zchunk", "fe_zchunk", "mac_omega")
    for g, sc in zip(grids, scenes):
        for k in keys:
            g.set_option(k, tuned[sc["n"][0]][k])
    # one after another, each grid launching its own kernels
    for g in grids:
        g.step(1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for g in grids:
        g.step(2)
    b.record(stream)
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(b) / 2
    bt = rmt.Batch(stream=stream.cuda_stream)
    for g in grids:
        bt.add(g)
    bt.step(3)  # captures both step graphs
    bt.sync()
    l0 = rmt.kernel_launches()
    k = args.batch_steps
    a.record(stream)
    bt.step(k)
    b.record(stream)
    torch.cuda.synchronize()
    bt.sync()
    ms = a.elapsed_time(b) / k
    launches = (rmt.kernel_launches() - l0) // k
    bt.close()
    for g in grids:
        g.close()
    return {"workload": f"{len(scenes)} lid-driven cavities, grids from {{32,48,64,96,128}}^3, 1-6 spheres, FP32",
            "value": cells / (ms / 1e3), "unit": "cell-updates/s", "ms_per_step": ms, "steps": k,
            "cells_per_step": cells, "kernels_per_step": launches, "graph_launches_per_step": 1,
            "autotune": {"seconds": tune_s, "per_size": {str(n): {k: tuned[n][k] for k in keys} for n in tuned}},
            "sequential": {"value": cells / (seq_ms / 1e3), "ms_per_step": seq_ms,
                           "note": "the same grids, same settings, stepped one after another, kernel by kernel"}}


def serving_leg(args, stream) -> dict:
    """Poisson arrivals (4 jobs/s) of settling / swimmer jobs of {48..192}^3 with 1-10 bodies under
    an 80 GB budget, served by continuous batching; beside it the same jobs run one after another
    on the plain FP64 path (per-step times measured on short runs, FIFO schedule)."""
    import torch

    from paper_2104_00095_gb300 import rmt, scenes as S

    lo, hi = args.serve_steps
    jobs = S.serving_stream(njobs=args.serve_jobs, steps=(lo, hi))
    for _, sc in jobs:
        sc.update(mg_fixed_cycles=args.mg_cycles_mac, mg_fixed_cycles_fe=args.mg_cycles_fe)
    srv = rmt.Server(80 * 10**9, stream=stream.cuda_stream, options=solver_options(args, graph=False))
    t_start = time.perf_counter()
    pending = list(jobs)
    ids, live, done = [], [], {}
    while True:
        now = time.perf_counter() - t_start
        while pending and pending[0][0] <= now:
            _, sc = pending.pop(0)
            ids.append(srv.submit(sc, sc["steps"]))
            live.append(ids[-1])
        r, q = srv.poll()
        # a finished job keeps its fields on the device until the client releases it: read its
        # record and release it, so that its memory returns to the budget for the queued jobs
        for i in list(live):
            info = srv.job(i)
            if info["state"] in (rmt.RMT_JOB_DONE, rmt.RMT_JOB_FAILED):
                done[i] = info
                srv.release(i)
                live.remove(i)
        if r == 0 and q == 0 and not pending:
            break
        if r == 0 and q == 0:
            time.sleep(max(0.0, pending[0][0] - (time.perf_counter() - t_start)))
    torch.cuda.synchronize()
    t_served = time.perf_counter() - t_start
    print(f"serving: {len(ids)} jobs served in {t_served:.1f} s", file=sys.stderr, flush=True)
    infos = [done[i] if i in done else srv.job(i) for i in ids]
    lat = np.array([i["t_done"] - i["t_submit"] for i in infos])
    failed = sum(1 for i in infos if i["state"] != rmt.RMT_JOB_DONE)
    first = min(i["t_submit"] for i in infos)
    span = max(i["t_done"] for i in infos) - first
    cell_steps = srv.cell_steps()
    stats = srv.stats()
    srv.close()
    # the same jobs one after another on the plain FP64 path: init + per-step time from short runs
    arr = np.array([t for t, _ in jobs])
    dur = []
    for _, sc in jobs:
        s64 = dict(sc, precision="fp64")
        t0 = time.perf_counter()
        g = rmt.Grid(s64, stream=stream.cuda_stream)
        g.step(1)
        torch.cuda.synchronize()
        init = time.perf_counter() - t0
        ms = timed_steps(g, 2, stream)
        g.close()
        dur.append(init + sc["steps"] * ms / 1e3)
    t_model = time.perf_counter() - t_start - t_served
    print(f"serving: serial FP64 model of {len(jobs)} jobs in {t_model:.1f} s", file=sys.stderr, flush=True)
    fin, t = [], 0.0
    for a_, d_ in zip(arr, dur):
        t = max(t, a_) + d_
        fin.append(t)
    slat = np.array(fin) - arr
    # the model checked against whole serial FP64 runs of the two smallest jobs
    small = sorted(range(len(jobs)), key=lambda q: np.prod(jobs[q][1]["n"]) * jobs[q][1]["steps"])[:2]
    checked = []
    for q in small:
        s64 = dict(jobs[q][1], precision="fp64")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = rmt.Grid(s64, stream=stream.cuda_stream)
        g.step(s64["steps"])
        torch.cuda.synchronize()
        checked.append({"grid": list(s64["n"]), "steps": s64["steps"], "measured_s": time.perf_counter() - t0,
                        "modelled_s": dur[q]})
        g.close()
    t_check = time.perf_counter() - t_start - t_served - t_model
    print(f"serving: whole FP64 runs checked in {t_check:.1f} s", file=sys.stderr, flush=True)
    return {"workload": f"{len(jobs)} jobs, Poisson 4/s, grids {{48..192}}^3, 1-10 bodies, steps U[{lo},{hi}], "
                        f"FP32, 80 GB budget",
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "value": cell_steps / span, "unit": "cell-updates/s", "makespan_s": span, "failed_jobs": failed,
            "runtime": stats,
            "leg_seconds": {"served": t_served, "serial_model": t_model, "whole_run_checks": t_check},
            "serial_fp64": {"p50_latency_s": float(np.percentile(slat, 50)),
                            "p99_latency_s": float(np.percentile(slat, 99)),
                            "value": float(sum(np.prod(sc["n"]) * sc["steps"] for _, sc in jobs) / (fin[-1] - arr[0])),
                            "method": "FIFO, one job at a time, FP64; duration = measured init + steps x measured "
                                      "per-step time (2-step sample)",
                            "whole_runs_checked": checked},
            "sample_note": ("the default run serves a sample of the mix (fewer jobs, shorter runs) so that the "
                            "bench ends within minutes; --serve-jobs 64 --serve-steps 100 2000 serves the full mix"
                            if (args.serve_jobs < 64 or lo != 100 or hi != 2000) else "the full mix")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="swimmers256", choices=sorted(CONFIGS))
    ap.add_argument("--mg-cycles-mac", type=int, default=5,
                    help="V-cycles per MAC solve (fixed, no host sync; 5 keep the MAC velocities divergence-free "
                         "to 1e-4 of their scale from the first step)")
    ap.add_argument("--mg-cycles-fe", type=int, default=4,
                    help="V-cycles per FE solve (fixed)")
    ap.add_argument("--mac-inner", type=int, default=5,
                    help="MAC V-cycles per high-precision residual (at least the cycle count: one residual, the "
                         "first, per solve)")
    ap.add_argument("--fe-inner", type=int, default=4,
                    help="FE V-cycles per high-precision residual (mixed-precision refinement)")
    ap.add_argument("--mac-warm", type=int, default=0, help="warm-start the MAC solve from the last step")
    ap.add_argument("--fe-warm", type=int, default=0, help="warm-start the FE solve from the last step")
    ap.add_argument("--mac-sweeps", type=int, default=2,
                    help="red-black sweeps before and after the coarse correction on the finest MAC level")
    ap.add_argument("--mac-omega", type=float, default=1.15,
                    help="over-relaxation factor of the MAC red-black sweeps")
    ap.add_argument("--mac-coarse", type=int, default=2,
                    help="red-black sweeps before and after the coarse correction on the MAC levels below the finest")
    ap.add_argument("--fe-pre", type=int, default=2, help="weighted Jacobi sweeps before the coarse correction (FE)")
    ap.add_argument("--fe-post", type=int, default=1, help="weighted Jacobi sweeps after the coarse correction (FE)")
    ap.add_argument("--fe-omega", type=float, default=1.0, help="weight of the FE Jacobi sweeps")
    ap.add_argument("--graph", type=int, default=1, help="replay each step as one captured CUDA graph")
    ap.add_argument("--nbodies", type=int, default=None,
                    help="override the body count (profiling captures only; changes the workload)")
    ap.add_argument("--n", type=int, default=None,
                    help="override the grid edge (profiling captures of a smaller case only; changes the workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the plain-FP64, batched and serving legs (profiling captures)")
    ap.add_argument("--batch-sims", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--serve-jobs", type=int, default=24)
    ap.add_argument("--serve-steps", type=int, nargs=2, default=(10, 200),
                    help="step-count range of the serving sample (the full mix draws from 100..2000)")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    cfg = CONFIGS[args.config]
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, cfg)
        return

    import torch
    import torch.distributed as dist

    from paper_2104_00095_gb300 import rmt

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    stream = torch.cuda.current_stream()
    scene = make_scene(cfg, n=args.n, nbodies=args.nbodies)
    scene["mg_fixed_cycles"] = args.mg_cycles_mac
    scene["mg_fixed_cycles_fe"] = args.mg_cycles_fe
    scene["options"] = solver_options(args)
    g = rmt.Grid(scene, stream=stream.cuda_stream)
    N = int(np.prod(scene["n"]))
    for _ in range(args.warmup):
        g.step(1)
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = str(local)
    clk = Clocks(uuid)
    clk.begin()
    barrier()
    torch.cuda.synchronize()
    l0 = rmt.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    launches = rmt.kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, world)
    value = job_rate(world, N, args.steps, ms / 1e3)

    # the same steps again with the library's CUDA-event profiler on: per-stage times and the
    # per-launch duration of the finest-level multigrid kernels
    g.profile(True)  # stage timing runs the same kernels launched one by one (no graph replay)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        g.step(1)
    p1.record(stream)
    torch.cuda.synchronize()
    prof = g.profile_read()
    g.profile(False)
    prof_ms = p0.elapsed_time(p1)
    kern = [p for p in prof if p[3] > 0 and p[2] > 0]
    peak, peak_kind = peaks()
    roofline = None
    if kern:
        name, tot, nl, byt = max(kern, key=lambda p: p[1])
        per = tot / nl
        ach = byt / (per / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "peak_source": peak_kind,
                    "traffic": dram_traffic(name, N),
                    "bytes_per_launch": byt, "launches": nl, "avg_launch_ms": per,
                    "share_of_step": tot / prof_ms, "profiled_ms_per_step": prof_ms / args.steps}
    stages = {p[0]: round(p[1] / args.steps, 4) for p in prof if p[1] > 0}
    # the whole step against the same peak, by the algorithmic byte model of one cell-step: 55 words
    # for the stages outside the projections plus 24 per V-cycle (six finest-level passes over x,
    # b and rho and one write), k_MAC + k_FE cycles, and 1/7 more for the coarse levels
    word = 4 if cfg["precision"] == "fp32" else 8
    model_words = step_model_words(args)
    step_achieved = model_words * word * N / (ms / args.steps / 1e3) / 1e9
    step_roofline = {"model_bytes_per_cell_step": model_words * word, "achieved": step_achieved, "peak": peak,
                     "unit": "GB/s", "frac": step_achieved / peak, "peak_source": peak_kind}

    # end to end through the C ABI with host buffers: every step uploads u from pinned host
    # memory, advances one step and reads u back, in the grid's storage precision (the float
    # calls for an FP32 grid, whose u they copy without conversion; the FP64 calls otherwise)
    e2e = None
    if not args.no_e2e:
        f32 = cfg["precision"] == "fp32"
        hd = torch.float32 if f32 else torch.float64
        esz = 4 if f32 else 8
        host_in = torch.empty(3 * N, dtype=hd, pin_memory=True)
        host_out = torch.empty(3 * N, dtype=hd, pin_memory=True)
        if f32:
            g.read_float(rmt.RMT_F_U, out=host_in.numpy())
        else:
            g.read(rmt.RMT_F_U, out=host_in.numpy())
        barrier()
        torch.cuda.synchronize()
        calls = np.zeros(3)  # host seconds in the write, step and read calls
        t0 = time.perf_counter()
        for _ in range(args.steps):
            c0 = time.perf_counter()
            if f32:
                g.write_float_ptr(rmt.RMT_F_U, host_in.data_ptr(), host_in.numel() * esz, 0)
            else:
                g.write_ptr(rmt.RMT_F_U, host_in.data_ptr(), host_in.numel() * esz, 0)
            c1 = time.perf_counter()
            g.step(1)
            c2 = time.perf_counter()
            if f32:
                g.read_float_ptr(rmt.RMT_F_U, host_out.data_ptr(), host_out.numel() * esz, 0)
            else:
                g.read(rmt.RMT_F_U, out=host_out.numpy())
            calls += (c1 - c0, c2 - c1, time.perf_counter() - c2)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        print("e2e host ms per step in write / step / read calls: " +
              " / ".join(f"{1e3 * v / args.steps:.2f}" for v in calls), file=sys.stderr)
        et = t1 - t0
        et = max_over_ranks(et, world)
        e2e = {"value": job_rate(world, N, args.steps, et), "unit": "cell-updates/s",
               "h2d_bytes_per_step": 3 * N * esz, "d2h_bytes_per_step": 3 * N * esz,
               "host_dtype": "f32" if f32 else "f64", "ms_per_step": 1e3 * et / args.steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, dt = cpu_oracle_rate(cfg, 2, 0)
        cpu = {"value": rate, "unit": "cell-updates/s", "cores": host_cores(), "kind": "oracle",
               "sample": f"2 steps of the same scene on a {CPU_SAMPLE_N}^3 grid (all bodies), FP64 oracle, "
                         f"{host_cores()} host threads ({dt:.1f} s)"}

    extra = {}
    if world == 1 and not args.no_extra:
        for key, leg in (("plain_fp64", lambda: plain_fp64_leg(cfg, args, stream)),
                         ("settling128", lambda: settling_leg(args, stream)),
                         ("batched", lambda: batched_leg(args, stream)), ("serving", lambda: serving_leg(args, stream))):
            try:
                extra[key] = leg()
            except Exception as ex:  # a failed side leg is reported, the headline line still prints
                extra[key] = {"error": f"{type(ex).__name__}: {ex}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if cfg["precision"] == "fp32" else "f64", "data": "synthetic",
                "config": {"workload": args.config if args.n is None else f"{args.config} resized to {args.n}^3",
                           "description": cfg["desc"], "grid": list(scene["n"]),
                           "bodies": len(scene["solids"]),
                           "mg_cycles_per_solve": {"mac": args.mg_cycles_mac, "fe": args.mg_cycles_fe,
                                                   "mac_inner": args.mac_inner, "fe_inner": args.fe_inner,
                                                   "mac_sweeps": args.mac_sweeps, "mac_omega": args.mac_omega,
                                                   "mac_coarse_sweeps": args.mac_coarse,
                                                   "fe_sweeps": [args.fe_pre, args.fe_post],
                                                   "fe_omega": args.fe_omega,
                                                   "mac_warm_start": bool(args.mac_warm),
                                                   "fe_warm_start": bool(args.fe_warm)},
                           "step_graph": bool(args.graph),
                           "dt": g.dt, "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (no flush needed)"},
                "gpu_launches": launches, "gpu_launches_before_timed": l0, "clocks": clocks, "roofline": roofline,
                "step_roofline": step_roofline, "stages_ms_per_step": stages,
                "e2e": e2e, "cpu_baseline": cpu}
        line.update(extra)
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
