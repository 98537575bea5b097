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
# FP64; half in FP32.  22 flops per update (8 + 2 fused multiply-adds, 2
# multiplies): the minimum HBM time and the FP64-pipe time are both ~3 us per
# launch at 1025^2.
RELAX_BYTES_2D = {"fp64": 144, "mixed": 72}
RELAX_FLOPS_2D = 22
# 3-D: rhs 16, inverse 32, own edges 3*16, the other colour's edges 3*16, x 16
# read and 16 written (FP64); half in FP32
RELAX_BYTES_3D = {"fp64": 176, "mixed": 88}
RELAX_FLOPS_3D = 30
RELAX_BYTES = {2: RELAX_BYTES_2D, 3: RELAX_BYTES_3D}
# DRAM bytes (read + write) of one finest-level relaxation launch from an ncu
# capture of the current kernel (cold cache), per workload and precision
RELAX_TRAFFIC = {("star1025", "fp64"): (31.30e6 + 17.0e3, "profiles/relax_inside_fp64_star1025.md")}
RELAX_FLOPS = {2: RELAX_FLOPS_2D, 3: RELAX_FLOPS_3D}


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


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count()


def cpu_baseline(name, budget_s=20.0, precision="fp64"):
    """The oracle as it stands, single-threaded, on a bounded sample: the first
    CN steps of the same workload until about budget_s seconds of CPU work."""
    import oracle

    w, N, dim, phi, dt = workload_setup(name)
    ref = oracle.Oracle(phi, dim, -1.0, 1.0, N, w["coarsest"])
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
    return {"value": nact * steps / el, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle",
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
    ref = oracle.Oracle(phi, dim, -1.0, 1.0, N, w["coarsest"])
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
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle",
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
    dom = pkg.Domain(phi, dim, (-1.0, 1.0), N, w["coarsest"])
    dom.set_model(workloads.PAPER_MODEL)
    prec = 1 if args.precision == "mixed" else 0
    dom.set_solver(precision=prec)
    stream = torch.cuda.Stream(device=dev)
    dom.set_stream(stream.cuda_stream)
    st0 = dom.stats()
    nact = st0["n_inside"] + st0["n_ghost"]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # warm-up from the initial data, then reset; the last warm-up step runs
    # with the kernel-timing events, so that the cycle graphs of both modes
    # exist before the timed region
    for w_ in range(args.warmup):
        dom.set_profiling(1 if w_ == args.warmup - 1 else 0)
        dom.step(dt, 1)
    dom.set_profiling(0)
    dom.set_model(workloads.PAPER_MODEL)
    torch.cuda.synchronize()

    sampler = ClockSampler(lr) if r == 0 else None
    if sampler:
        sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = dom.stats()["kernel_launches"]
    newton0, cyc0 = dom.stats()["newton_total"], dom.stats()["cycles_total"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    relax_ms, relax_n = 0.0, 0
    # The relaxation launches of the last timed step are timed with CUDA
    # events on the library's stream (the first finest-level sweep of every
    # cycle).  Event nodes cannot sit inside the device-side cycle loop, so
    # that one step runs one graph launch and host test per cycle; the other
    # steps run each linear solve as one loop-graph launch.
    prof_step = args.steps - 1
    for k in range(args.steps):
        if k == prof_step:
            dom.set_profiling(1)
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
            ev[k][0].record(stream)
        dom.step(dt, 1)
        with torch.cuda.stream(stream):
            ev[k][1].record(stream)
        if k == prof_step:
            ms, n = dom.kernel_time()
            relax_ms += ms
            relax_n += n
            dom.set_profiling(0)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    elapsed_ms = sum(step_ms)
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
        nbytes = RELAX_BYTES[dim][args.precision] * nodes_per_launch
        achieved = nbytes / (avg_us * 1e-6) / 1e9 if relax_n else None
        hbm = peaks.get("hbm_gbs")
        roofline = {"kernel": "k_relax_inside (finest level, one colour)", "bound": "hbm",
                    "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": (achieved / hbm) if (achieved and hbm) else None,
                    "traffic": RELAX_TRAFFIC.get((args.workload, args.precision), (None,))[0],
                    "traffic_source": RELAX_TRAFFIC.get((args.workload, args.precision), (None, None))[1],
                    "avg_launch_us": avg_us, "launches": relax_n,
                    "algorithmic": f"{RELAX_BYTES[dim][args.precision]} B and {RELAX_FLOPS[dim]} flop per "
                                   f"inside-node update; {nodes_per_launch:.0f} nodes per launch",
                    "sample": "one event bracket around the two back-to-back colour launches of the first "
                              "finest-level sweep of every cycle of the last timed step",
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
               "step_latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                                   "p99": float(np.percentile(step_ms, 99)), "max": float(max(step_ms))},
               "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(out), flush=True)
    dom.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def run_batch(args):
    """256 random-star instances, sizes uniform in {129, 257, 513, 1025}^2,
    mixed precision, advanced together by the batching runtime; compared with
    the same instances advanced one after the other in plain FP64."""
    import torch

    import paper_1902_07029_gb300 as pkg

    pkg.build()
    rng = np.random.default_rng(4)
    n_inst = args.instances
    sizes = rng.choice([128, 256, 512, 1024], size=n_inst)
    params = [workloads.random_star_params(rng) for _ in range(n_inst)]

    def make(precision):
        doms = []
        for N, (a, p, s_ext) in zip(sizes, params):
            d = pkg.Domain(workloads.random_star(int(N), a, p), 2, (-1.0, 1.0), int(N))
            m = list(workloads.PAPER_MODEL)
            m[6] = s_ext
            d.set_model(m)
            d.set_solver(precision=precision)
            doms.append(d)
        return doms

    dts = [2.0 / float(N) for N in sizes]
    steps = args.steps
    out = {}
    for label, precision, batched in (("batched_mixed", 1, True), ("sequential_fp64", 0, False)):
        doms = make(precision)
        nact = sum(d.stats()["n_inside"] + d.stats()["n_ghost"] for d in doms)
        if batched:
            b = pkg.Batch(doms, nstreams=args.streams)
            b.step(dts, 1)  # warm-up: graphs, cluster kernels
            for d in doms:
                d.set_model(d_model(d, doms, sizes, params))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.step(dts, steps)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            b.close()
        else:
            for d, dt in zip(doms, dts):
                d.step(dt, 1)
            for d in doms:
                d.set_model(d_model(d, doms, sizes, params))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for d, dt in zip(doms, dts):
                d.step(dt, steps)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
        out[label] = {"value": nact * steps / el, "seconds": el}
        for d in doms:
            d.close()
    line = {"metric": METRIC, "value": out["batched_mixed"]["value"], "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic",
            "config": {"workload": f"batch of {n_inst} random stars, sizes uniform in {{129,257,513,1025}}^2",
                       "precision": "mixed", "streams": args.streams, "cn_steps_per_instance": steps},
            "sequential_fp64": out["sequential_fp64"], "batched_mixed": out["batched_mixed"]}
    print(json.dumps(line), flush=True)


def d_model(d, doms, sizes, params):
    i = doms.index(d)
    m = list(workloads.PAPER_MODEL)
    m[6] = params[i][2]
    return m


def run_serve(args):
    """Poisson arrivals (seed 5) of jobs: 70% 2-D random stars with
    N in {256, 512, 1024, 2048}, 30% 3-D random rounded boxes with N in
    {64, 128}; 20-100 CN steps each (dt = h in 2-D, h/2 at 129^3, h/4 at
    65^3), mixed precision, HBM budget 150 GB."""
    import paper_1902_07029_gb300 as pkg

    pkg.build()
    rng = np.random.default_rng(5)
    jobs = []
    for _ in range(args.jobs):
        if rng.random() < 0.7:
            N = int(rng.choice([256, 512, 1024, 2048]))
            a, p, s_ext = workloads.random_star_params(rng)
            phi = workloads.random_star(N, a, p)
            dim, cN = 2, 8
            m = list(workloads.PAPER_MODEL)
            m[6] = s_ext
        else:
            N = int(rng.choice([64, 128]))
            phi, _, _ = workloads.random_rounded_box(N, rng)
            dim, cN = 3, 4
            m = list(workloads.PAPER_MODEL)
        nsteps = int(rng.integers(20, 101))
        # 3-D: dt = h/2 at 129^3; at 65^3 some rounded boxes have no discrete
        # solution at dt = h/2 (as the 65^2 disk at dt = h), so dt = h/4 there
        dt = 2.0 / N if dim == 2 else (0.5 if N >= 128 else 0.25) * 2.0 / N
        jobs.append((phi, dim, N, cN, m, dt, nsteps))
    rates = [float(r) for r in str(args.rate).split(",")]
    gap_rng = np.random.default_rng(6)
    unit_gaps = gap_rng.exponential(1.0, size=len(jobs))  # the same arrival pattern, scaled per rate
    runs = []
    for rate in rates:
        srv = pkg.Server(budget_bytes=150 << 30, nworkers=args.streams)
        t0 = time.perf_counter()
        ids = []
        for (phi, dim, N, cN, m, dt, nsteps), g in zip(jobs, unit_gaps):
            time.sleep(g / rate)
            ids.append(srv.submit(phi, dim, N, m, dt, nsteps, coarsest_N=cN, precision=1))
        failed = []
        nodes = 0.0
        for i, (phi, dim, N, cN, m, dt, nsteps) in zip(ids, jobs):
            try:
                s, c, res = srv.wait(i)
                nodes += float(np.count_nonzero(phi < 0)) * nsteps
            except pkg.SulfError as e:
                failed.append({"dim": dim, "N": N, "nsteps": nsteps, "error": str(e)[:160]})
        el = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        runs.append({"arrival_rate_per_s": rate, "jobs_per_s": st["completed"] / el, "p50_ms": st["p50_ms"],
                     "p99_ms": st["p99_ms"], "completed": st["completed"], "failed": len(failed), "failures": failed,
                     "max_running": st["max_running"], "peak_reserved_GB": st["peak_reserved_bytes"] / 2 ** 30,
                     "inside_node_updates_per_s": nodes / el, "wall_s": el})
    r0 = runs[0]
    line = {"metric": "jobs/s and p50/p99 job latency", "value": r0["jobs_per_s"], "unit": "jobs/s",
            "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic",
            "config": {"workload": "Poisson-arrival serving of random star / rounded-box jobs", "jobs": len(jobs),
                       "arrival_rate_per_s": r0["arrival_rate_per_s"], "workers": args.streams, "budget_GB": 150},
            "p50_ms": r0["p50_ms"], "p99_ms": r0["p99_ms"], "completed": r0["completed"], "failed": r0["failed"],
            "failures": r0["failures"], "max_running": r0["max_running"],
            "peak_reserved_GB": r0["peak_reserved_GB"], "inside_node_updates_per_s": r0["inside_node_updates_per_s"],
            "wall_s": r0["wall_s"], "sweep": runs if len(runs) > 1 else None}
    print(json.dumps(line), flush=True)


def run_rho(args):
    """Multigrid convergence factors: the paper's W(2,1) and the default V(2,2),
    collective and pointwise red-black smoothing, on the star at several N.
    rho is the geometric mean of the defect ratios of cycles 4..12 of a linear
    solve with the Jacobian at the state after one CN step and a seeded random
    right-hand side."""
    import torch

    import paper_1902_07029_gb300 as pkg

    pkg.build()
    rows = []
    for N in (128, 256, 512, 1024):
        phi = workloads.star(N)
        dt = 2.0 / N
        for name, kw in (("V(2,2) collective", dict()), ("W(2,1) collective", dict(cycle=2, nu1=2, nu2=1)),
                         ("V(2,2) pointwise", dict(smoother=1)),
                         ("W(2,1) pointwise", dict(cycle=2, nu1=2, nu2=1, smoother=1))):
            dom = pkg.Domain(phi, 2, (-1.0, 1.0), N)
            dom.set_model(workloads.PAPER_MODEL)
            dom.step(dt, 1)
            dom.set_solver(**kw)
            s, c, t = dom.get_state()
            W = np.zeros(2 * s.size)
            W[0::2] = s.ravel()
            W[1::2] = c.ravel()
            act = ((t == 1) | (t == 2)).ravel()
            rng = np.random.default_rng(7)
            rhs = np.zeros_like(W)
            rhs[0::2][act] = rng.standard_normal(act.sum())
            rhs[1::2][act] = rng.standard_normal(act.sum())
            torch.cuda.synchronize()
            _, rn = dom.cycles(dt, W, rhs, 12)
            ratios = rn[3:] / rn[2:-1]
            rows.append({"N": N, "cycle": name, "rho": float(np.exp(np.mean(np.log(ratios))))})
            dom.close()
    line = {"metric": "multigrid convergence factor", "value": None, "unit": "defect ratio per cycle",
            "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "star r - 0.6 - 0.2 sin 5 theta, Jacobian after one CN step, dt = h"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sulfmg", choices=["sulfmg", "reference"])
    ap.add_argument("--workload", default="star1025", choices=sorted(workloads.WORKLOADS) + ["batch", "serve", "rho"])
    ap.add_argument("--instances", type=int, default=256, help="batch: number of instances")
    ap.add_argument("--streams", type=int, default=8, help="batch/serve: worker streams")
    ap.add_argument("--jobs", type=int, default=40, help="serve: number of jobs")
    ap.add_argument("--rate", default="4.0",
                    help="serve: Poisson arrival rate(s) in jobs/s, comma-separated for a sweep")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle CPU work for cpu_baseline")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "rho":
        run_rho(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
