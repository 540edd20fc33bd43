#!/usr/bin/env python3
"""Benchmark of the fused hot path on one GB300 (or N GPUs, weak scaling).

Default workload: Black-Scholes call+put pricing of 2^26 FP32 options issued
as the 23-task array program, fused by the runtime into one sm_103a kernel.
One step = issue the task window through the API + flush + the fused kernel,
inputs resident in HBM (1.34 GB per step, larger than the 129 MB L2, so no
flush of L2 is needed between steps).  Also measured in the same run: the
unfused per-task path (23 kernels, every temporary in HBM), the end-to-end
path with host buffers (H2D of S,K,T and D2H of call,put every step), and the
CPU oracle on a bounded sample.

  python bench.py [--steps K] [--warmup W] [--workload bs|cg|jacobi]
  python bench.py --impl reference     # the CPU oracle as the reference arm
Prints one JSON line.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2406_18109_gb300 import configs  # noqa: E402
from synth import inputs  # noqa: E402

METRIC_BS = "Black-Scholes options/s (fused window, 2^26 FP32)"
METRIC_CG = "CG iterations/s (fused windows, 256^2 Poisson FP64)"
METRIC_JAC = "Jacobi sweeps/s (fused windows, 8192^2 FP32)"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


class Clocks:
    """Samples nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle
def oracle_rate(workload: str, budget_s: float = 10.0):
    """CPU oracle throughput on a bounded sample (the reference / cpu_baseline)."""
    from oracle import programs
    t_end = time.perf_counter() + budget_s
    if workload == "bs":
        cfg = configs.BLACK_SCHOLES
        m = 1 << 20
        S, K, T = inputs.bs_inputs(m, seed=cfg["seed"])
        done, t0 = 0, time.perf_counter()
        while True:
            programs.black_scholes(S, K, T, cfg["r"], cfg["sigma"], np.float32)
            done += m
            if time.perf_counter() > t_end:
                break
        dt = time.perf_counter() - t0
        return done / dt, "options/s", f"{done} options in batches of 2^20 from the 2^26-option seed-1 draw law"
    if workload == "cg":
        cfg = configs.CG
        rp, col, val, xs = inputs.cg_inputs(m=cfg["m"], seed=cfg["seed"])
        b = programs.spmv(rp, col, val, xs)
        done, t0 = 0, time.perf_counter()
        while True:
            programs.cg(rp, col, val, b, 10)
            done += 10
            if time.perf_counter() > t_end:
                break
        dt = time.perf_counter() - t0
        return done / dt, "iterations/s", f"{done} CG iterations on the 256^2 Poisson system"
    cfg = configs.JACOBI
    g = inputs.jacobi_grid(2046, seed=cfg["seed"])
    done, t0 = 0, time.perf_counter()
    while True:
        programs.jacobi(g, 2, np.float32)
        done += 2
        if time.perf_counter() > t_end:
            break
    dt = time.perf_counter() - t0
    scale = (2046 * 2046) / (cfg["N"] * cfg["N"])
    return done / dt * scale, "sweeps/s", f"{done} sweeps of a 2048^2 grid, scaled by area to 8192^2"


# ---------------------------------------------------------------- GPU arms
def run_bs(rt_kwargs, steps, warmup, torch, stream, e2e=False):
    from paper_2406_18109_gb300 import arrays as A
    from paper_2406_18109_gb300 import workloads as W
    cfg = configs.BLACK_SCHOLES
    n = cfg["n"]
    S, K, T = inputs.bs_inputs(n, seed=cfg["seed"])
    rt = A.Runtime(device=torch.cuda.current_device(), stream=stream.cuda_stream, **rt_kwargs)
    dS, dK, dT = rt.array(S), rt.array(K), rt.array(T)
    rt.sync()
    h2d = d2h = 0
    if e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        hS, hK, hT = pin(S), pin(K), pin(T)
        hc = torch.empty(n, dtype=torch.float32).pin_memory().numpy()
        hp = torch.empty(n, dtype=torch.float32).pin_memory().numpy()

    def step():
        nonlocal h2d, d2h
        if e2e:
            dS.write(hS)
            dK.write(hK)
            dT.write(hT)
        call, put = W.black_scholes(dS, dK, dT, cfg["r"], cfg["sigma"])
        rt.flush()
        if e2e:
            call.read_into(hc)
            put.read_into(hp)
        return call, put

    for _ in range(warmup):
        step()
    rt.sync()
    launches0 = rt.stats()["launches"]
    k_ev = []
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    t0 = time.perf_counter()
    keep = None
    for _ in range(steps):
        if not e2e:
            # events around the flush time its launch(es) on the launching stream
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            c_, p_ = W.black_scholes(dS, dK, dT, cfg["r"], cfg["sigma"])
            a.record(stream)
            rt.flush()
            b.record(stream)
            k_ev.append((a, b))
            keep = (c_, p_)
        else:
            keep = step()
    end.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = start.elapsed_time(end)
    launches = rt.stats()["launches"] - launches0
    kern_ms = [a.elapsed_time(b) for a, b in k_ev]
    if e2e:
        h2d = 3 * n * 4
        d2h = 2 * n * 4
    del keep
    st = rt.stats()
    rt.close()
    return {"ms": ms, "wall_s": wall, "launches": launches, "kernel_ms": kern_ms, "stats": st,
            "h2d": h2d, "d2h": d2h, "units": n * steps}


def run_cg(rt_kwargs, steps, warmup, torch, stream):
    from paper_2406_18109_gb300 import arrays as A
    from paper_2406_18109_gb300 import workloads as W
    cfg = configs.CG
    rp, col, val, xs = inputs.cg_inputs(m=cfg["m"], seed=cfg["seed"])
    rt = A.Runtime(device=torch.cuda.current_device(), stream=stream.cuda_stream, **rt_kwargs)
    Am = A.CSR(rt, rp, col, val)
    b = Am @ rt.array(xs)
    rt.sync()

    def solve():
        st = W.cg_start(b)
        rt.flush()
        for _ in range(cfg["iters"]):
            W.cg_iteration(Am, st)
            rt.flush()
        return st

    for _ in range(warmup):
        solve()
    rt.sync()
    l0 = rt.stats()["launches"]
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        st = solve()
    end.record(stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    launches = rt.stats()["launches"] - l0
    out = {"ms": ms, "launches": launches, "stats": rt.stats(), "units": cfg["iters"] * steps,
           "kernel_ms": [ms / (steps * cfg["iters"])]}
    rt.close()
    return out


def run_jacobi(rt_kwargs, steps, warmup, torch, stream):
    from paper_2406_18109_gb300 import arrays as A
    from paper_2406_18109_gb300 import workloads as W
    cfg = configs.JACOBI
    grid = inputs.jacobi_grid(cfg["N"], seed=cfg["seed"])
    rt = A.Runtime(device=torch.cuda.current_device(), stream=stream.cuda_stream, **rt_kwargs)
    g = rt.array(grid)
    views = W.jacobi_views(g)
    rt.sync()
    sweeps = cfg["sweeps"]

    def run(k):
        for s in range(k):
            W.jacobi_sweep(views)
            if (s + 1) % cfg["sweeps_per_flush"] == 0:
                rt.flush()
        rt.flush()

    run(warmup)
    rt.sync()
    l0 = rt.stats()["launches"]
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        run(sweeps)
    end.record(stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    out = {"ms": ms, "launches": rt.stats()["launches"] - l0, "stats": rt.stats(), "units": sweeps * steps,
           "kernel_ms": [ms / (steps * sweeps)]}
    rt.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bs", choices=["bs", "cg", "jacobi"])
    ap.add_argument("--quick", action="store_true", help="skip the comparison arms (for profiling)")
    ap.add_argument("--bs-n", type=int, default=0, help="Black-Scholes batch size (profiling a smaller case)")
    args = ap.parse_args()
    if args.bs_n:
        configs.BLACK_SCHOLES["n"] = args.bs_n
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    metric, unit = {"bs": (METRIC_BS, "options/s"), "cg": (METRIC_CG, "iterations/s"),
                    "jacobi": (METRIC_JAC, "sweeps/s")}[args.workload]
    workload_name = {"bs": "black-scholes-2^26-fp32", "cg": "cg-poisson2d-256x256-fp64-50it",
                     "jacobi": "jacobi-fig1-stencil-8192x8192-fp32-200sweeps"}[args.workload]

    if args.impl == "reference":
        if rank != 0:
            return
        v, u, sample = oracle_rate(args.workload, budget_s=max(5.0, min(60.0, 2.0 * args.steps)))
        line = {"metric": metric, "value": v, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.workload != "cg" else "f64", "data": "synthetic",
                "impl": "reference", "config": {"workload": workload_name},
                "cpu_baseline": {"value": v, "unit": u, "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": u, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    cache = os.path.join(ROOT, "gpurun_out", "cubins") if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else None

    from paper_2406_18109_gb300 import _build
    _build.build()

    if args.workload == "bs":
        cfg = configs.BLACK_SCHOLES
        base = dict(tile=cfg["tile"], block=cfg["block"], unroll=cfg["unroll"], sms=sms, cache_dir=cache)
        runner = lambda kw, s, w, **x: run_bs(kw, s, w, torch, stream, **x)
    elif args.workload == "cg":
        cfg = configs.CG
        base = dict(tile=cfg["tile"], block=cfg["block"], unroll=cfg["unroll"], sms=sms, cache_dir=cache)
        runner = lambda kw, s, w, **x: run_cg(kw, s, w, torch, stream)
    else:
        cfg = configs.JACOBI
        base = dict(rows=cfg["rows"], block=cfg["block"], unroll=cfg["unroll"], sms=sms, cache_dir=cache)
        runner = lambda kw, s, w, **x: run_jacobi(kw, s, w, torch, stream)

    clocks = Clocks(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks.start()
    fused = runner(dict(base, fusion=True, launch="persistent"), args.steps, args.warmup)
    clk = clocks.stop()
    ms_step = fused["ms"] / args.steps
    if world > 1:
        t = torch.tensor([fused["ms"]], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        fused["ms"] = float(t.item())
        ms_step = fused["ms"] / args.steps
    value = fused["units"] * world / (fused["ms"] / 1e3)

    extra = {}
    if not args.quick:
        k2 = max(3, args.steps // 4)
        unf = runner(dict(base, fusion=False, launch="per_task"), k2, 2)
        pt = runner(dict(base, fusion=True, launch="per_task"), k2, 2)
        extra["unfused"] = {"value": unf["units"] / (unf["ms"] / 1e3), "ms_per_step": unf["ms"] / k2,
                            "launches_per_step": unf["launches"] / k2}
        extra["fused_per_task"] = {"value": pt["units"] / (pt["ms"] / 1e3), "ms_per_step": pt["ms"] / k2,
                                   "launches_per_step": pt["launches"] / k2}
        extra["fused_vs_unfused"] = value / world / extra["unfused"]["value"]
        if args.workload == "bs":
            e = runner(dict(base, fusion=True, launch="persistent"), max(3, args.steps // 4), 2, e2e=True)
            extra["e2e"] = {"value": e["units"] / (e["ms"] / 1e3), "unit": unit,
                            "h2d_bytes_per_step": e["h2d"], "d2h_bytes_per_step": e["d2h"]}

    peaks = load_peaks()
    if args.workload == "bs":
        n = configs.BLACK_SCHOLES["n"]
        alg_bytes = 20 * n
        kern_ms = statistics.mean(fused["kernel_ms"])
    elif args.workload == "cg":
        m = configs.CG["m"]
        nn = m * m
        nnz = 5 * nn - 4 * m
        alg_bytes = 12 * nnz + 4 * (nn + 1) + 96 * nn
        kern_ms = statistics.mean(fused["kernel_ms"])
    else:
        N = configs.JACOBI["N"]
        alg_bytes = 16 * N * N
        kern_ms = statistics.mean(fused["kernel_ms"])
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "peak_source": peaks["source"], "kernel_ms": kern_ms, "algorithmic_bytes": alg_bytes}

    cpu = None
    if rank == 0 and world == 1 and not args.quick:
        v, u, sample = oracle_rate(args.workload, budget_s=10.0)
        cpu = {"value": v, "unit": u, "cores": 1, "kind": "oracle", "sample": sample}

    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.workload != "cg" else "f64",
            "data": "synthetic (seeded generators of synth/inputs.py)",
            "config": {"workload": workload_name, "l2": "inputs larger than L2" if args.workload != "cg"
                       else "working set L2-resident (10 MB); no flush", "launch": "persistent fused",
                       "parallelism": f"replicas x{world}"},
            "e2e": extra.get("e2e"), "gpu_launches": fused["launches"], "roofline": roofline,
            "cpu_baseline": cpu, "clocks": clk}
    line.update({k: v for k, v in extra.items() if k != "e2e"})
    line["runtime_stats"] = {k: fused["stats"].get(k) for k in ("compile_s", "kernels_compiled", "plan_hits",
                                                                  "plan_misses", "kernel_disk_hits", "last_regs",
                                                                  "last_occupancy", "last_grid", "last_block")}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
