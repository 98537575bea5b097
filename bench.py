"""Benchmark of the Newton-multigrid Crank-Nicolson step on GB300.

Workload (default): the 3-D rounded box phi = ||max(|x| - 0.6, 0)||_2 - 0.2 on
[-1,1]^3 with 257^3 nodes (coarsest level 5^3), the paper's model constants
(Eq. dataeq), s0 = 0, c0 = 10, s_ext = 1 (Eq. BCnumtests), dt = h, Newton tol
1e-10, V(2,2) red-black collective Gauss-Seidel cycles to relative residual
1e-10.  The plain FP64 form is the headline; the same run also measures the
mixed-precision form (FP32 cycles inside FP64 defect correction) and reports it
beside it.  Other workloads: the 1025^2 star (star1025), the 65^2 disk
(disk65), and the batch / serve / rho studies.

One benchmark step = one Crank-Nicolson step (all Newton iterations and
multigrid cycles it needs).  Warm-up steps run from the initial data, then the
state is reset and K steps are timed from t = 0, each bracketed by CUDA events
on the library's stream, with the L2 cache flushed (a 512 MB write) between
steps outside the timed brackets.

Metric: fine-grid node-updates per second = (inside + ghost nodes) * steps /
time, summed over ranks (each rank runs its own replica: the path has no
exchange step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision both|fp64|mixed]
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

# Algorithmic bytes of one relaxation sweep per active node with the stencil
# coefficients recomputed from (s, c): read (s, c), the right-hand side and the
# unknown, write the unknown -- 64 B in FP64, 32 B in FP32 (2-D and 3-D alike).
# One colour launch updates half of the inside nodes; per updated node it is
# charged these bytes.
SWEEP_BYTES = {"fp64": 64, "mixed": 32}
# Compulsory bytes of one colour update as this library streams it.  FP64:
# the stencil coefficients precomputed once per Newton iteration -- rhs, the
# rows of the inverse 2x2 block, the own and the other colour's edge
# coefficients and the unknown read and written: 2-D 16 + 32 + 2*16 + 2*16 +
# 32 = 144 B, 3-D 16 + 32 + 3*16 + 3*16 + 32 = 176 B.  FP32 (coefficients
# recomputed from (s, c)): (s, c) of the node and of one node of the other
# colour, x of the other colour, rhs, x written: 5 * 8 = 40 B.
STREAM_BYTES = {2: {"fp64": 144, "mixed": 40}, 3: {"fp64": 176, "mixed": 40}}
# FP64/FP32 arithmetic of one update: per axis four fused multiply-adds for
# the off-diagonal part, then two fused multiply-adds and two multiplies for
# the 2x2 block solve: 2-D 10 FMA + 2 MUL = 22 flop, 3-D 14 FMA + 2 MUL = 30.
RELAX_FLOPS = {2: 22, 3: 30}
# FP64 peak from the unit counts and clock: 152 SMs x 2 FP64 FMA lanes per
# clock x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# Per CN step and active node (Sec. 8 byte model): old-time part 32 B, per
# Newton iteration the residual 48 B and the update 32 B, per V(2,2) cycle
# 4 * 64 + 52 + 36 = 344 B on one level times the hierarchy factor 4/3 (2-D)
# or 8/7 (3-D); FP32 cycles half of that.
CYCLE_BYTES = {2: 344.0 * 4 / 3, 3: 344.0 * 8 / 7}
# DRAM bytes (read + write) of one finest-level relaxation launch from an ncu
# capture of the current kernel (cold cache), per workload and precision
RELAX_TRAFFIC = {
    # 129^3 capture (profiles/relax_inside_fp64_rbox129.md): 103.9 MB per
    # 521 488 updates = 199.2 B per update, scaled to the 257^3 launch
    ("rbox257", "fp64"): (199.2 * 4142122, "profiles/relax_inside_fp64_rbox129.md (199.2 B per update measured at "
                                           "129^3, scaled to the 4 142 122 updates of a 257^3 launch)"),
    ("star1025", "fp64"): (23.52e6 + 2.0e3, "profiles/relax_inside_fp64_star1025.md"),
    # 129^3 capture of the matrix-free FP32 kernel (profiles/relax_mf_fp32_rbox129.md): 31.6 MB per
    # 521 488 updates = 60.6 B per update, scaled to the 257^3 launch
    ("rbox257", "mixed"): (60.6 * 4142122, "profiles/relax_mf_fp32_rbox129.md (60.6 B per update measured at "
                                          "129^3, scaled to the 4 142 122 updates of a 257^3 launch)"),
}


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
    return w, N, dim, phi, w.get("dt_factor", 1.0) * 2.0 / N


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


def _oracle_for(name):
    import oracle

    w, N, dim, phi, dt = workload_setup(name)
    ref = oracle.Oracle(phi, dim, -1.0, 1.0, N, w["coarsest"])
    ref.set_model(workloads.PAPER_MODEL)
    ref.set_solver()
    t = ref.level_type(0)
    nact = int(np.count_nonzero((t == 1) | (t == 2)))
    return ref, w, N, dim, dt, nact


def _oracle_cycle_sample(ref, dt, ncycles):
    """Seconds per multigrid cycle of the oracle on the workload's Jacobian at
    the initial state (a seeded random right-hand side)."""
    import oracle

    s, c, t = ref.get_state()
    W = oracle.interleave(s, c)
    act = ((t == 1) | (t == 2)).ravel()
    rhs = np.zeros_like(W)
    rhs[0::2][act] = np.random.default_rng(1).standard_normal(int(act.sum()))
    t0 = time.perf_counter()
    ref.cycles(dt, W, rhs, np.zeros_like(W), ncycles)
    return (time.perf_counter() - t0) / ncycles


def cpu_baseline(name, budget_s=20.0, cycles_per_step=None):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    same workload.  Where a CN step fits the budget: the first CN steps until
    about budget_s seconds of CPU work.  Otherwise (the 257^3 box: ~4-5 s per
    oracle cycle, ~55 cycles per step): a few multigrid cycles of the oracle on
    the workload's Jacobian, scaled to a CN step by the cycles per step of the
    same workload (cycles_per_step: the GPU run's own count, which equals the
    oracle's cycle count in FP64)."""
    ref, w, N, dim, dt, nact = _oracle_for(name)
    if w.get("oracle_step_s_estimate", 0.0) > budget_s and cycles_per_step:
        k = 3
        tc = _oracle_cycle_sample(ref, dt, k)
        value = nact / (tc * cycles_per_step)
        return {"value": value, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle",
                "sample": f"{k} V(2,2) cycles of the oracle on {name} ({nact} active nodes) at the initial state, "
                          f"{tc:.2f} s per cycle, scaled by {cycles_per_step:.1f} cycles per CN step (counted by "
                          f"this run); 1 thread"}
    steps, t0 = 0, time.perf_counter()
    while True:
        ref.step(dt, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= w["steps"]:
            break
    return {"value": nact * steps / el, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle",
            "sample": f"first {steps} CN step(s) of {name} ({nact} active nodes), {el:.1f} s, 1 thread"}


def run_reference(args):
    """The oracle on the host cores, on the GPU arm's workload and metric: each
    timed step is one CN step of the oracle where that takes less than a
    minute, else a bounded sample (one oracle multigrid cycle, scaled by the
    cycles per CN step the oracle counted on this workload's first step)."""
    r, world, _ = rank_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
        if r != 0:
            dist.barrier()
            dist.destroy_process_group()
            return
    ref, w, N, dim, dt, nact = _oracle_for(args.workload)
    cps = w.get("oracle_cycles_per_step")
    sampled = w.get("oracle_step_s_estimate", 0.0) > 60.0 and cps
    times = []
    if sampled:
        for _ in range(min(args.warmup, 1)):
            _oracle_cycle_sample(ref, dt, 1)
        k_eff = max(1, min(args.steps, 20))
        for _ in range(k_eff):
            times.append(_oracle_cycle_sample(ref, dt, 3) * cps)
        sample = (f"{k_eff} steps, each three oracle V(2,2) cycles on {args.workload} at the initial state (with one "
                  f"Jacobian set-up) per cycle scaled by the {cps} cycles the oracle counted on its first CN step")
    else:
        t0 = time.perf_counter()
        for _ in range(min(args.warmup, 1)):
            ref.step(dt, 1)
        per_step = max(time.perf_counter() - t0, 1e-3)
        ref.set_model(workloads.PAPER_MODEL)
        k_eff = max(1, min(args.steps, int(120.0 / per_step)))
        for _ in range(k_eff):
            t0 = time.perf_counter()
            ref.step(dt, 1)
            times.append(time.perf_counter() - t0)
        sample = f"first {k_eff} of {args.steps} requested CN steps of {args.workload}"
    el = sum(times)
    value = nact * len(times) / el
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(times),
           "warmup": args.warmup, "ms_per_step": 1e3 * el / len(times), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload, "geometry": w["geometry"], "N": N, "dim": dim,
                      "nodes_active": nact, "dt": f"{w.get('dt_factor', 1.0):g} h", "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


def _measure(pkg, args, name, precision, dev, rank, world, e2e_steps):
    """Time K CN steps of one precision (0 FP64, 1 mixed) after W warm-up
    steps; returns the measurements of this rank."""
    import torch

    w, N, dim, phi, dt = workload_setup(name)
    dom = pkg.Domain(phi, dim, (-1.0, 1.0), N, w["coarsest"])
    dom.set_model(workloads.PAPER_MODEL)
    dom.set_solver(precision=precision)
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
    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    st_a = dom.stats()
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
    st_b = dom.stats()
    clocks = sampler.stop() if sampler else None
    value, elapsed_ms = whole_job_value(sum(step_ms), nact * args.steps, device=dev)
    s_gpu, c_gpu, _ = dom.get_state()
    e2e = None
    if rank == 0 and e2e_steps > 0:
        # end to end through the C ABI with host buffers: each step uploads the
        # state, advances one CN step and downloads it (pinned host memory)
        nn = dom.nn
        hs = torch.empty(nn, dtype=torch.float64, pin_memory=True).numpy()
        hc = torch.empty(nn, dtype=torch.float64, pin_memory=True).numpy()
        dom.set_model(workloads.PAPER_MODEL)
        dom.get_state_into(hs, hc)
        ke = min(args.steps, e2e_steps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            dom.set_state(hs, hc, 0.0)
            dom.step(dt, 1)
            dom.get_state_into(hs, hc)
        el = time.perf_counter() - t0
        e2e = {"value": nact * ke / el, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * nn,
               "d2h_bytes_per_step": 2 * 8 * nn, "steps": ke}
    dom.close()
    del flush
    return dict(w=w, N=N, dim=dim, nact=nact, n_inside=st0["n_inside"], value=value, elapsed_ms=elapsed_ms,
                step_ms=step_ms, relax_ms=relax_ms, relax_n=relax_n, clocks=clocks, e2e=e2e,
                newton=st_b["newton_total"] - st_a["newton_total"], cycles=st_b["cycles_total"] - st_a["cycles_total"],
                launches=st_b["kernel_launches"] - st_a["kernel_launches"], state=(s_gpu, c_gpu))


def _roofline(m, name, prec_name, peaks):
    """The dominant kernel (finest-level inside relaxation, one colour launch)
    against its binding roof: the FP64 pipe for the FP64 form, HBM for the FP32
    relaxation of the mixed form; both byte models are reported."""
    dim = m["dim"]
    avg_us = 1e3 * m["relax_ms"] / max(m["relax_n"], 1)
    n = m["n_inside"] / 2.0
    hbm = peaks.get("hbm_gbs")
    sec = avg_us * 1e-6 if m["relax_n"] else None
    ach_sweep = SWEEP_BYTES[prec_name] * n / sec / 1e9 if sec else None
    ach_stream = STREAM_BYTES[dim][prec_name] * n / sec / 1e9 if sec else None
    ach_flops = RELAX_FLOPS[dim] * n / sec / 1e12 if sec else None
    traffic = RELAX_TRAFFIC.get((name, prec_name), (None, None))
    hbm_part = {"achieved": ach_sweep, "peak": hbm, "unit": "GB/s",
                "frac": (ach_sweep / hbm) if (ach_sweep and hbm) else None,
                "algorithmic": f"{SWEEP_BYTES[prec_name]} B per updated node (Sec. 8 sweep bytes, coefficients "
                               f"recomputed); {n:.0f} nodes per launch",
                "achieved_stream_bytes": ach_stream,
                "frac_stream_bytes": (ach_stream / hbm) if (ach_stream and hbm) else None,
                "stream_bytes": f"{STREAM_BYTES[dim][prec_name]} B per update as streamed ("
                                + ("precomputed coefficients)" if prec_name == "fp64" else
                                   "coefficients recomputed from (s, c))"),
                "traffic": traffic[0], "traffic_source": traffic[1]}
    kname = "k_relax_inside" if prec_name == "fp64" else "k_relax_mf (coefficients from (s, c))"
    common = {"kernel": f"{kname} (finest level, one colour)", "avg_launch_us": avg_us,
              "launches": m["relax_n"], "sample": "one event bracket around the two back-to-back colour launches of "
              "the first finest-level sweep of every cycle of the last timed step (library stream)"}
    if prec_name == "fp64":
        # the FP64 pipe binds: 16 FP64 instructions per 3-D update at two
        # lanes per SM per clock take longer than the update's bytes at HBM speed
        return {**common, "bound": "alu", "achieved": ach_flops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": (ach_flops / FP64_PEAK_TFLOPS) if ach_flops else None,
                "peak_note": "FP64 peak derived from 152 SMs x 2 FP64 FMA lanes/clock x 2 flop x 2.07 GHz",
                "algorithmic": f"{RELAX_FLOPS[dim]} flop per update; {n:.0f} updates per launch",
                "traffic": traffic[0], "hbm": hbm_part}
    return {**common, "bound": "hbm", **{k: hbm_part[k] for k in ("achieved", "peak", "unit", "frac", "algorithmic",
                                                                    "traffic")},
            "achieved_stream_bytes": ach_stream, "frac_stream_bytes": hbm_part["frac_stream_bytes"],
            "stream_bytes": hbm_part["stream_bytes"], "traffic_source": traffic[1],
            "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json)",
            "kind": "fp32 relaxation inside fp64 defect correction"}


def _step_bandwidth(m, prec_name, peaks):
    """Sec. 8 algorithmic bytes of a whole CN step over its measured time."""
    nn_step = m["newton"] / max(len(m["step_ms"]), 1)
    nv_step = m["cycles"] / max(len(m["step_ms"]), 1)
    cyc = CYCLE_BYTES[m["dim"]] * (0.5 if prec_name == "mixed" else 1.0)
    per_node = 32.0 + nn_step * (48.0 + 32.0) + nv_step * cyc
    gbs = per_node * m["nact"] / (m["elapsed_ms"] / len(m["step_ms"]) * 1e-3) / 1e9
    hbm = peaks.get("hbm_gbs")
    return {"bytes_per_node_step": per_node, "newton_per_step": nn_step, "cycles_per_step": nv_step,
            "achieved_GBps": gbs, "frac": gbs / hbm if hbm else None}


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
    precs = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    res = {}
    for i, pn in enumerate(precs):
        res[pn] = _measure(pkg, args, args.workload, 1 if pn == "mixed" else 0, dev, r, world,
                           e2e_steps=20 if i == 0 else 0)
    if r == 0:
        peaks = measured_peaks()
        head = precs[0]
        m = res[head]
        w, N, dim, nact = m["w"], m["N"], m["dim"], m["nact"]
        cps = m["cycles"] / len(m["step_ms"])
        cb = cpu_baseline(args.workload, budget_s=args.cpu_budget, cycles_per_step=cps) if args.cpu_budget > 0 else None

        def leg(pn):
            x = res[pn]
            return {"value": x["value"], "ms_per_step": x["elapsed_ms"] / args.steps,
                    "step_latency_ms": {"p50": float(np.percentile(x["step_ms"], 50)),
                                        "p99": float(np.percentile(x["step_ms"], 99)), "max": float(max(x["step_ms"]))},
                    "newton_iters": x["newton"], "cycles": x["cycles"], "gpu_launches": x["launches"],
                    "roofline": _roofline(x, args.workload, pn, peaks),
                    "step_bandwidth": _step_bandwidth(x, pn, peaks), "clocks": x["clocks"]}

        out = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": m["elapsed_ms"] / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64" if head == "fp64" else "f64+f32",
               "data": "synthetic",
               "config": {"workload": args.workload, "geometry": w["geometry"], "N": N, "dim": dim,
                          "nodes_active": nact, "dt": f"{w.get('dt_factor', 1.0):g} h", "precision": head,
                          "cycle": "V(2,2) red-black collective GS, 4 ghost passes", "coarsest_N": w["coarsest"],
                          "newton_tol": 1e-10, "lin_rtol": 1e-10,
                          "l2": "flushed between CN steps (512 MB write); the working set exceeds L2",
                          "newton_iters": m["newton"], "cycles": m["cycles"]},
               "step_latency_ms": leg(head)["step_latency_ms"], "roofline": leg(head)["roofline"],
               "step_bandwidth": leg(head)["step_bandwidth"], "cpu_baseline": cb, "e2e": m["e2e"],
               "gpu_launches": m["launches"], "clocks": m["clocks"]}
        if "mixed" in res and head != "mixed":
            mx = leg("mixed")
            sf, cf = res["fp64"]["state"]
            sm, cm = res["mixed"]["state"]
            mask = np.abs(sf) + np.abs(cf) > 0
            mx["max_rel_diff_vs_fp64"] = {
                "s": float(np.abs(sm[mask] - sf[mask]).max() / np.abs(sf[mask]).max()),
                "c": float(np.abs(cm[mask] - cf[mask]).max() / np.abs(cf[mask]).max())}
            mx["speedup_vs_fp64"] = mx["value"] / m["value"]
            out["mixed"] = mx
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def run_batch(args):
    """256 random-star instances, sizes uniform in {129, 257, 513, 1025}^2
    (--instances, --sizes),
    s_ext ~ U(0.5, 1), dt = h, advanced together by the batching runtime after
    the autotuner has picked each size's speed-only controls.  Arms: batched
    mixed precision, batched FP64, the same two in lock-step mode (the
    instances of one size advance together, one launch per cycle phase for all
    of them; default controls) and the instances advanced one after the other
    in FP64.  Accuracy: each arm's state after two CN steps on an 8-instance
    subset (two per size) against the CPU oracle."""
    import torch

    import oracle
    import paper_1902_07029_gb300 as pkg

    pkg.build()
    rng = np.random.default_rng(4)
    n_inst = args.instances
    size_set = [int(x) for x in args.sizes.split(",")]
    sizes = [int(x) for x in rng.choice(size_set, size=n_inst)]
    params = [workloads.random_star_params(rng) for _ in range(n_inst)]
    dts = [2.0 / N for N in sizes]

    def model_of(i):
        m = list(workloads.PAPER_MODEL)
        m[6] = params[i][2]
        return m

    def make(idx, precision):
        doms = []
        for i in idx:
            d = pkg.Domain(workloads.random_star(sizes[i], *params[i][:2]), 2, (-1.0, 1.0), sizes[i])
            d.set_model(model_of(i))
            d.set_solver(precision=precision)
            doms.append(d)
        return doms

    # accuracy on the subset: two instances per size, two CN steps, each arm
    subset = []
    for N in size_set:
        subset += [i for i in range(n_inst) if sizes[i] == N][:2]
    ref = {}
    for i in subset:
        o = oracle.Oracle(workloads.random_star(sizes[i], *params[i][:2]), 2, -1.0, 1.0, sizes[i])
        o.set_model(model_of(i))
        o.set_solver()
        o.step(dts[i], 2)
        ref[i] = o.get_state()
    arms = (("batched_mixed", 1, "batched"), ("batched_fp64", 0, "batched"), ("lockstep_mixed", 1, "lockstep"),
            ("lockstep_fp64", 0, "lockstep"), ("sequential_fp64", 0, "sequential"))
    if args.arms:
        keep = args.arms.split(",")
        arms = tuple(a for a in arms if a[0] in keep)
    acc = {}
    for label, precision, mode in arms:
        doms = make(subset, precision)
        if mode != "sequential":
            b = pkg.Batch(doms, nstreams=args.streams, lockstep=mode == "lockstep")
            if mode == "batched":
                b.autotune([dts[i] for i in subset])
            b.step([dts[i] for i in subset], 2)
            b.close()
        else:
            for d, i in zip(doms, subset):
                d.step(dts[i], 2)
        err = 0.0
        for d, i in zip(doms, subset):
            s, c, _ = d.get_state()
            rs, rc, rt = ref[i]
            act = (rt == 1) | (rt == 2)
            err = max(err, float(np.abs(s[act] - rs[act]).max() / np.abs(rs[act]).max()),
                      float(np.abs(c[act] - rc[act]).max() / np.abs(rc[act]).max()))
            d.close()
        acc[label] = err

    steps = args.steps
    seq_steps = max(1, min(steps, args.seq_steps))
    out, tuned = {}, None
    for label, precision, mode in arms:
        doms = make(range(n_inst), precision)
        nact = sum(d.stats()["n_inside"] + d.stats()["n_ghost"] for d in doms)
        k = steps if mode != "sequential" else seq_steps
        if mode != "sequential":
            b = pkg.Batch(doms, nstreams=args.streams, lockstep=mode == "lockstep")
            t0 = time.perf_counter()
            res = b.autotune(dts) if mode == "batched" else None
            t_tune = time.perf_counter() - t0
            if precision == 1 and mode == "batched":
                tuned = {}
                for N, r in zip(sizes, res):
                    if N not in tuned or not r["cached"]:
                        tuned[N] = {kk: r[kk] for kk in ("fuse_below", "ghost_compose", "pdl", "relax_occupancy",
                                                          "ms_per_cycle",
                                                          "ms_per_cycle_default")}
            b.step(dts, 1)  # warm-up: graphs
            for i, d in enumerate(doms):
                d.set_model(model_of(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.step(dts, k)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            b.close()
        else:
            t_tune = 0.0
            for d, dt in zip(doms, dts):
                d.step(dt, 1)
            for i, d in enumerate(doms):
                d.set_model(model_of(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for d, dt in zip(doms, dts):
                d.step(dt, k)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
        out[label] = {"value": nact * k / el, "seconds": el, "cn_steps_per_instance": k,
                      "autotune_seconds": t_tune, "max_rel_err_vs_oracle_subset": acc[label]}
        for d in doms:
            d.close()
    def ratio(a, b):
        return out[a]["value"] / out[b]["value"] if a in out and b in out else None

    head = next(a for a in ("lockstep_mixed", "batched_mixed", "lockstep_fp64", "batched_fp64", "sequential_fp64")
                if a in out)
    sizes_txt = ",".join(str(N + 1) for N in size_set)
    line = {"metric": METRIC, "value": out[head]["value"], "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if head.endswith("fp64") else "f64+f32", "data": "synthetic",
            "config": {"workload": f"batch of {n_inst} random stars, sizes uniform in {{{sizes_txt}}}^2, dt = h",
                       "value_arm": head, "lockstep_chunks": "at most 32 instances",
                       "streams": args.streams, "cn_steps_per_instance": steps,
                       "sequential_arm_steps": seq_steps,
                       "accuracy": "max relative difference from the oracle over s and c, subset of two "
                                   "instances per size, 2 CN steps"},
            "tuned": {str(k): v for k, v in sorted(tuned.items())} if tuned else None,
            "mixed_vs_fp64_batched": ratio("batched_mixed", "batched_fp64"),
            "lockstep_vs_batched": {"mixed": ratio("lockstep_mixed", "batched_mixed"),
                                    "fp64": ratio("lockstep_fp64", "batched_fp64")},
            "batched_vs_sequential_fp64": ratio("batched_fp64", "sequential_fp64")}
    for a in out:
        line[a] = out[a]
    print(json.dumps(line), flush=True)


def serve_jobs(n_jobs, max_steps, seed=5):
    """The job stream of the serving workload: 70 % 2-D random stars with N in
    {256, 512, 1024, 2048} (s_ext ~ U(0.5, 1)), 30 % 3-D random rounded boxes
    with N in {64, 128, 256}; CN steps uniform in {20 .. max_steps} (500 in the
    full workload); dt = h, except dt = h/2 at 129^3 and h/4 at 65^3, where
    some random boxes have no discrete solution at larger steps (as the 65^2
    disk at dt = h)."""
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(n_jobs):
        if rng.random() < 0.7:
            N = int(rng.choice([256, 512, 1024, 2048]))
            a, p, s_ext = workloads.random_star_params(rng)
            phi = workloads.random_star(N, a, p)
            dim, cN = 2, 8
            m = list(workloads.PAPER_MODEL)
            m[6] = s_ext
        else:
            N = int(rng.choice([64, 128, 256]))
            phi, _, _ = workloads.random_rounded_box(N, rng)
            dim, cN = 3, 4
            m = list(workloads.PAPER_MODEL)
        nsteps = int(rng.integers(20, max_steps + 1))
        dt = 2.0 / N if (dim == 2 or N >= 256) else (0.5 if N >= 128 else 0.25) * 2.0 / N
        jobs.append((phi, dim, N, cN, m, dt, nsteps))
    return jobs


def _serve_once(pkg, jobs, rate, budget_bytes, workers, gaps):
    """Submit the jobs with Poisson arrivals at `rate` (inf: all at once), wait
    for all, and return the run's statistics."""
    srv = pkg.Server(budget_bytes=budget_bytes, nworkers=workers)
    t0 = time.perf_counter()
    ids = []
    for (phi, dim, N, cN, m, dt, nsteps), g in zip(jobs, gaps):
        if np.isfinite(rate):
            time.sleep(g / rate)
        ids.append(srv.submit(phi, dim, N, m, dt, nsteps, coarsest_N=cN, precision=1))
    failed, nodes, queue_ms, run_ms = [], 0.0, [], []
    for i, (phi, dim, N, cN, m, dt, nsteps) in zip(ids, jobs):
        try:
            s, c, res = srv.wait(i)
            nodes += float(np.count_nonzero(phi < 0)) * nsteps
            queue_ms.append(res["queue_ms"])
            run_ms.append(res["run_ms"])
        except pkg.SulfError as e:
            failed.append({"dim": dim, "N": N, "nsteps": nsteps, "error": str(e)[:160]})
    el = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    return {"arrival_rate_per_s": None if not np.isfinite(rate) else rate, "jobs_per_s": st["completed"] / el,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "completed": st["completed"], "failed": len(failed),
            "failures": failed, "max_running": st["max_running"], "budget_GB": budget_bytes / 2 ** 30,
            "peak_reserved_GB": st["peak_reserved_bytes"] / 2 ** 30,
            "queue_ms_p50": float(np.percentile(queue_ms, 50)) if queue_ms else None,
            "queue_ms_max": float(max(queue_ms)) if queue_ms else None,
            "inside_node_updates_per_s": nodes / el, "wall_s": el}


def run_serve(args):
    """Serving: Poisson arrivals (seed 6) of the job stream above, mixed
    precision, continuous batching under an HBM budget.  The service capacity
    is measured first (every job submitted at once), then the arrival rate is
    swept over 0.5x, 1x and 2x of it at the 150 GB budget; a last run at 2x
    with a tight budget shows admission by memory (jobs queue although workers
    are free)."""
    import paper_1902_07029_gb300 as pkg

    pkg.build()
    jobs = serve_jobs(args.jobs, args.max_steps)
    gaps = np.random.default_rng(6).exponential(1.0, size=len(jobs))
    budget = int(args.budget_gb * 2 ** 30)
    cap = _serve_once(pkg, jobs, float("inf"), budget, args.streams, gaps)
    capacity = cap["jobs_per_s"]
    if args.no_sweep:
        rates, runs, tight = [], [], None
    else:
        rates = [f * capacity for f in (0.5, 1.0, 2.0)] if args.rate == "auto" else \
            [float(r) for r in str(args.rate).split(",")]
        runs = [_serve_once(pkg, jobs, r, budget, args.streams, gaps) for r in rates]
        tight = _serve_once(pkg, jobs, rates[-1], int(args.tight_budget_gb * 2 ** 30), args.streams, gaps)
    est = [pkg.estimate_device_bytes(dim, N, cN, 1) / 2 ** 30 for (_, dim, N, cN, _, _, _) in jobs]
    r0 = runs[1] if len(runs) > 1 else (runs[0] if runs else cap)
    line = {"metric": "jobs/s and p50/p99 job latency", "value": r0["jobs_per_s"], "unit": "jobs/s",
            "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic",
            "config": {"workload": "Poisson-arrival serving of random star / rounded-box jobs (mixed precision)",
                       "jobs": len(jobs), "steps": f"uniform in 20..{args.max_steps}"
                       + ("" if args.max_steps >= 500 else " (scaled down from 20..500)"),
                       "sizes": "2-D N in {256,512,1024,2048} (70 %), 3-D N in {64,128,256} (30 %)",
                       "workers": args.streams, "budget_GB": args.budget_gb,
                       "job_estimates_GB": {"sum": float(sum(est)), "max": float(max(est))}},
            "capacity_jobs_per_s": capacity, "saturated": cap, "p50_ms": r0["p50_ms"], "p99_ms": r0["p99_ms"],
            "sweep": runs, "tight_budget": tight}
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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sulfmg", choices=["sulfmg", "reference"])
    ap.add_argument("--workload", default="rbox257", choices=sorted(workloads.WORKLOADS) + ["batch", "serve", "rho"])
    ap.add_argument("--instances", type=int, default=256, help="batch: number of instances")
    ap.add_argument("--streams", type=int, default=16,
                    help="batch/serve: worker streams (256-instance batch, 10 steps: 42.8 M node-updates/s with 8, "
                         "58.1 M with 16, 58.9 M with 32)")
    ap.add_argument("--seq-steps", type=int, default=10, help="batch: CN steps of the sequential FP64 arm")
    ap.add_argument("--sizes", default="128,256,512,1024", help="batch: grid sizes N the instances draw from")
    ap.add_argument("--arms", default="", help="batch: comma list of arms to run (default all: batched_mixed, "
                                                "batched_fp64, lockstep_mixed, lockstep_fp64, sequential_fp64)")
    ap.add_argument("--jobs", type=int, default=32, help="serve: number of jobs")
    ap.add_argument("--rate", default="auto",
                    help="serve: Poisson arrival rate(s) in jobs/s, comma-separated; auto = 0.5, 1, 2 x capacity")
    ap.add_argument("--max-steps", type=int, default=200, help="serve: CN steps per job uniform in 20..max")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serve: HBM budget")
    ap.add_argument("--tight-budget-gb", type=float, default=16.0, help="serve: budget of the admission run")
    ap.add_argument("--no-sweep", action="store_true", help="serve: the saturated run only (every job at once)")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="both: the FP64 form as the headline and the mixed form beside it")
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
