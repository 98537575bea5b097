"""Benchmark of the Newton-multigrid Crank-Nicolson step on GB300.

Workload (default): five-lobed star phi = r - 0.6 - 0.2 sin(5 theta) on
[-1,1]^2 with 1025^2 nodes, the paper's model constants (Eq. dataeq), s0 = 0,
c0 = 10, s_ext = 1 (Eq. BCnumtests), dt = h, Newton tol 1e-10, V(2,2) red-black
collective Gauss-Seidel cycles to relative residual 1e-10, FP64.

One benchmark step = one Crank-Nicolson step (all Newton iterations and
multigrid cycles it needs).  Warm-up steps run from the initial data, then the
state is reset and K steps are timed from t = 0, each bracketed by CUDA events
on the library's stream, with the L2 cache flushed (a 512 MB write) between
steps outside the timed brackets.

Metric: fine-grid node-updates per second = (inside + ghost nodes) * steps /
time, summed over ranks (each rank runs its own replica: the path has no
exchange step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   (the CPU oracle, on host cores)
"""
from __future__ import annotations

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

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "fine-grid node-updates/s per CN step"
UNIT = "node-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Compulsory bytes of one inside-node relaxation (one colour) with the
# stencil coefficients precomputed per Newton iteration, 2-D: rhs 16, inverse
# of the 2x2 block 32, own edge coefficients 2*16, the other colour's edge
# coefficients 2*16 and x 16 (each read once per sweep), x written 16 -- in
# FP64; half in FP32.  About 23 flops per update: memory-bound (HBM or L2).
RELAX_BYTES_2D = {"fp64": 144, "mixed": 72}
RELAX_FLOPS_2D = 23


def whole_job_value(elapsed_ms_local: float, units_local: int, device=None) -> tuple[float, float]:
    """Replicas run independently; the job's time is the slowest rank's and its
    throughput the units of all ranks over that time.  Returns (value per
    second, max elapsed ms)."""
    import torch
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([elapsed_ms_local, float(units_local)], dtype=torch.float64, device=device)
        tmax = t[:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t[1:].clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        elapsed_ms, units = float(tmax.item()), float(tsum.item())
    else:
        elapsed_ms, units = elapsed_ms_local, float(units_local)
    return units / (elapsed_ms / 1e3), elapsed_ms


def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                mx.append(float(s[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_setup(name):
    w = workloads.WORKLOADS[name]
    N, dim = w["N"], w["dim"]
    phi = workloads.workload_levelset(name)
    return w, N, dim, phi, 2.0 / N


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cpu_baseline(name, budget_s=20.0, precision="fp64"):
    """The oracle as it stands, single-threaded, on a bounded sample: the first
    CN steps of the same workload until about budget_s seconds of CPU work."""
    import oracle

    w, N, dim, phi, dt = workload_setup(name)
    ref = oracle.Oracle(phi, dim, -1.0, 1.0, N)
    ref.set_model(workloads.PAPER_MODEL)
    ref.set_solver()
    info = ref.level_info(0)
    t = ref.level_type(0)
    nact = int(np.count_nonzero((t == 1) | (t == 2)))
    steps, t0 = 0, time.perf_counter()
    while True:
        ref.step(dt, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= w["steps"]:
            break
    del info
    return {"value": nact * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {steps} CN step(s) of {name} ({nact} active nodes), {el:.1f} s, 1 thread"}


def run_reference(args):
    r, world, _ = rank_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
        if r != 0:
            dist.barrier()
            dist.destroy_process_group()
            return
    import oracle

    w, N, dim, phi, dt = workload_setup(args.workload)
    ref = oracle.Oracle(phi, dim, -1.0, 1.0, N)
    ref.set_model(workloads.PAPER_MODEL)
    ref.set_solver()
    t = ref.level_type(0)
    nact = int(np.count_nonzero((t == 1) | (t == 2)))
    # warm-up (bounded) then reset, then time a bounded number of CN steps
    t0 = time.perf_counter()
    for _ in range(min(args.warmup, 1)):
        ref.step(dt, 1)
    per_step = max(time.perf_counter() - t0, 1e-3)
    ref.set_model(workloads.PAPER_MODEL)
    k_eff = max(1, min(args.steps, int(120.0 / per_step)))
    t0 = time.perf_counter()
    for _ in range(k_eff):
        ref.step(dt, 1)
    el = time.perf_counter() - t0
    value = nact * k_eff / el
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": k_eff, "warmup": args.warmup,
           "ms_per_step": 1e3 * el / k_eff, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload, "N": N, "dim": dim, "dt": "h", "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"first {k_eff} of {args.steps} requested CN steps of {args.workload}"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


def run_gpu(args):
    import torch

    import paper_1902_07029_gb300 as pkg

    r, world, lr = rank_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", lr))
    torch.cuda.set_device(lr)
    dev = torch.device("cuda", lr)
    pkg.build()
    w, N, dim, phi, dt = workload_setup(args.workload)
    dom = pkg.Domain(phi, dim, (-1.0, 1.0), N)
    dom.set_model(workloads.PAPER_MODEL)
    prec = 1 if args.precision == "mixed" else 0
    dom.set_solver(precision=prec)
    stream = torch.cuda.Stream(device=dev)
    dom.set_stream(stream.cuda_stream)
    st0 = dom.stats()
    nact = st0["n_inside"] + st0["n_ghost"]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # warm-up from the initial data, then reset
    for _ in range(args.warmup):
        dom.step(dt, 1)
    dom.set_model(workloads.PAPER_MODEL)
    torch.cuda.synchronize()

    sampler = ClockSampler(lr) if r == 0 else None
    if sampler:
        sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    dom.set_profiling(True)
    launches0 = dom.stats()["kernel_launches"]
    newton0, cyc0 = dom.stats()["newton_total"], dom.stats()["cycles_total"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    relax_ms, relax_n = 0.0, 0
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
            ev[k][0].record(stream)
        dom.step(dt, 1)
        with torch.cuda.stream(stream):
            ev[k][1].record(stream)
        ms, n = dom.kernel_time()
        relax_ms += ms
        relax_n += n
    torch.cuda.synchronize()
    dom.set_profiling(False)
    elapsed_ms = sum(a.elapsed_time(b) for a, b in ev)
    st1 = dom.stats()
    launches = st1["kernel_launches"] - launches0
    value, elapsed_ms = whole_job_value(elapsed_ms, nact * args.steps, device=dev)
    clocks = sampler.stop() if sampler else None

    # end to end through the C ABI with host buffers: each step uploads the
    # state, advances one CN step and downloads it (pinned host memory)
    e2e = None
    if r == 0:
        nn = dom.nn
        hs = torch.empty(nn, dtype=torch.float64, pin_memory=True).numpy()
        hc = torch.empty(nn, dtype=torch.float64, pin_memory=True).numpy()
        dom.set_model(workloads.PAPER_MODEL)
        dom.get_state_into(hs, hc)
        ke = min(args.steps, 20)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            dom.set_state(hs, hc, 0.0)
            dom.step(dt, 1)
            dom.get_state_into(hs, hc)
        el = time.perf_counter() - t0
        e2e = {"value": nact * ke / el, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * nn, "d2h_bytes_per_step": 2 * 8 * nn,
               "steps": ke}

    if r == 0:
        peaks = measured_peaks()
        avg_us = 1e3 * relax_ms / max(relax_n, 1)
        nodes_per_launch = st0["n_inside"] / 2.0
        nbytes = RELAX_BYTES_2D[args.precision] * nodes_per_launch
        achieved = nbytes / (avg_us * 1e-6) / 1e9 if dim == 2 and relax_n else None
        hbm = peaks.get("hbm_gbs")
        roofline = {"kernel": "k_relax_inside (finest level, one colour)", "bound": "hbm",
                    "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": (achieved / hbm) if (achieved and hbm) else None, "traffic": None,
                    "avg_launch_us": avg_us, "launches": relax_n,
                    "algorithmic": f"{RELAX_BYTES_2D[args.precision]} B and {RELAX_FLOPS_2D} flop per inside-node "
                                   f"update; {nodes_per_launch:.0f} nodes per launch",
                    "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json); the finest level's working "
                                 "set is partly L2-resident, so the fraction can exceed what HBM alone allows"}
        if prec == 1:
            roofline["kind"] = "fp32 relaxation inside fp64 defect correction"
        cb = cpu_baseline(args.workload, budget_s=args.cpu_budget) if args.cpu_budget > 0 else None
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f64+f32",
               "data": "synthetic",
               "config": {"workload": args.workload, "geometry": w["geometry"], "N": N, "dim": dim,
                          "nodes_active": nact, "dt": "h", "precision": args.precision,
                          "cycle": "V(2,2) red-black collective GS, 4 ghost passes",
                          "newton_tol": 1e-10, "lin_rtol": 1e-10, "l2": "flushed between CN steps (512 MB write)",
                          "newton_iters": st1["newton_total"] - newton0, "cycles": st1["cycles_total"] - cyc0},
               "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(out), flush=True)
    dom.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sulfmg", choices=["sulfmg", "reference"])
    ap.add_argument("--workload", default="star1025", choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle CPU work for cpu_baseline")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
