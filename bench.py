"""Benchmark of the multigroup M1 radiation-hydrodynamics stage update on GB300.

Metric: zone-group updates per second per RK stage (each RK stage updates every zone-group of
the grid once), for the FP32 form (headline `value`) and the plain FP64 path (`fp64` object), on
the 2-d periodic Kelvin-Helmholtz workload, 1024 x 1024 cells x 16 groups (synthetic seeded
input; inputs are larger than L2, so no flush is needed between timed steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  Under torchrun each rank runs an independent replica (weak scaling);
the stage update is not decomposed across GPUs in this build.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1806_07390_gb300 import workloads as W  # noqa: E402

METRIC = "zone-group updates/s per RK stage"
UNIT = "zone-group-stages/s"
# DRAM bytes per stage launch from the committed ncu captures (profiles/); None until captured
# for the current kernel.
TRAFFIC_PER_LAUNCH = {"fp32": None, "fp32n64": None, "fp64": None}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        loaded = [s for s in sm if mx is None or s >= 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def time_form(pb, prim, steps, warmup, dist):
    """Device-timed K steps of one precision form with inputs resident in HBM."""
    import torch

    from paper_1806_07390_gb300 import fx

    g = fx.Grid(pb)
    g.init_equilibrium(prim)
    g.sync()
    for _ in range(warmup):
        g.step(pb.dt, 1)
    g.sync()
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    s = g.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        g.step(pb.dt, 1)
    e1.record(s)
    e1.synchronize()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = g.status()
    if dist:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    launches = g.launches_per_step() * steps
    return g, ms, st, launches


def time_e2e(g, pb, steps, warmup):
    """Same metric through the public API with host buffers: every step uploads the state from
    pinned host memory, advances one step and downloads the result to pinned host memory."""
    import torch

    n = g.nelem
    dt_t = torch.float64 if pb.precision == "fp64" else torch.float32
    h_in = torch.empty(n, dtype=dt_t, pin_memory=True)
    h_out = torch.empty(n, dtype=dt_t, pin_memory=True)
    prec = 0 if pb.precision == "fp64" else 1
    import ctypes
    L = g.L

    def one():
        g._check(L.fx_state_upload(g.h, ctypes.c_void_p(h_in.data_ptr()), prec, 0))
        g.step(pb.dt, 1)
        g._check(L.fx_state_download(g.h, ctypes.c_void_p(h_out.data_ptr()), prec, 0))

    g._check(L.fx_state_download(g.h, ctypes.c_void_p(h_in.data_ptr()), prec, 0))
    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
        h_in.copy_(h_out)  # next step's input is this step's result
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    return sec, n * h_in.element_size(), n * h_out.element_size()


def cpu_baseline(pb_full, prim_full, budget_s=15.0):
    """The FP64 oracle, as it stands, on the host cores: a 256 x 256-cell window of the same
    workload (same spacing, c and dt, outflow window edges), stepped until ~budget_s."""
    import oracle
    from tests import helpers as H

    cores = os.cpu_count() or 1
    sub, sprim = H.window(pb_full, prim_full, (384, 384), (256 - 8, 256 - 8), 4)
    s = oracle.init_equilibrium(sub, sprim)
    t0 = time.perf_counter()
    nst = 0
    while True:
        s, _ = oracle.run(sub, s, sub.dt, 1, nthreads=cores)
        nst += 1
        if time.perf_counter() - t0 > budget_s or nst >= 50:
            break
    sec = time.perf_counter() - t0
    zgs = sub.ncell * sub.ngroups * 2 * nst
    return {"value": zgs / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sub.n[0]}x{sub.n[1]} cells x {sub.ngroups} groups window of the "
                      f"1024^2 workload, {nst} FP64 steps, OpenMP over cells"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pb, prim = W.kh_2d(precision="fp64")
    steps, warmup = args.steps, args.warmup
    import oracle

    from tests import helpers as H
    cores = os.cpu_count() or 1
    sub, sprim = H.window(pb, prim, (384, 384), (120, 120), 4)
    s = oracle.init_equilibrium(sub, sprim)
    for _ in range(warmup):
        s, _ = oracle.run(sub, s, sub.dt, 1, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(steps):
        s, _ = oracle.run(sub, s, sub.dt, 1, nthreads=cores)
    sec = time.perf_counter() - t0
    zgs = sub.ncell * sub.ngroups * 2 * steps
    val = zgs / sec
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * sec / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "kh2d 1024x1024 cells x 16 groups, periodic (oracle sample "
                                   f"{sub.n[0]}x{sub.n[1]} window)", "precision": "fp64"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sub.n[0]}x{sub.n[1]} cells x 16 groups window, "
                                       f"{steps} steps"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    dev = torch.cuda.current_device()

    pb32, prim = W.kh_2d(precision="fp32")
    forms = {"fp32n64": W.kh_2d(precision="fp32n64")[0]}
    if not args.no_fp64:
        forms["fp64"] = W.kh_2d(precision="fp64")[0]
    pb64 = W.kh_2d(precision="fp64")[0]
    zg = pb32.ncell * pb32.ngroups
    peak, peak_kind = load_peaks()

    results = {}
    with ClockSampler(dev) as clk:
        g32, ms32, st32, launches32 = time_form(pb32, prim, args.steps, args.warmup, dist)
        for name, pbf in forms.items():
            gf, msf, stf, lf = time_form(pbf, prim, args.steps, args.warmup, dist)
            results[name] = (msf, stf, lf)
            gf.close()
    clocks = clk.summary()

    sec32 = ms32 / 1e3
    value = world * zg * 2 * args.steps / sec32
    nv = pb32.nvar

    def roofline(kind, sec, steps):
        b = 8 if kind == "fp64" else 4
        per_launch = 2.5 * b * nv * pb32.ncell  # algorithmic bytes per stage launch (2.5 N_v words)
        achieved = per_launch / (sec / (2 * steps)) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": TRAFFIC_PER_LAUNCH.get(kind),
                "peak_kind": peak_kind, "bytes_per_launch": per_launch}

    e2e_steps = max(5, args.steps // 4)
    e2e_sec, h2d, d2h = time_e2e(g32, pb32, e2e_steps, 2)
    g32.close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "kh2d: 2-d periodic Kelvin-Helmholtz, 1024x1024 cells x 16 "
                                   "groups, FP32 form", "cells": pb32.ncell, "groups": pb32.ngroups,
                       "l2": "inputs larger than L2 (no flush)", "precision": "fp32",
                       "parallelism": f"replicas{world}"},
            "roofline": roofline("fp32", sec32, args.steps),
            "e2e": {"value": world * zg * 2 * e2e_steps / e2e_sec, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches32 + sum(r[2] for r in results.values()),
            "clocks": clocks, "status": int(st32), "forms": {}}
    for name, (msf, stf, lf) in results.items():
        secf = msf / 1e3
        line["forms"][name] = {"value": world * zg * 2 * args.steps / secf, "unit": UNIT,
                               "ms_per_step": msf / args.steps,
                               "roofline": roofline(name, secf, args.steps), "status": int(stf),
                               "fp32_speedup": msf / ms32}
    if rank == 0 and not args.no_cpu and not dist:
        line["cpu_baseline"] = cpu_baseline(pb64, prim)
    elif rank == 0 and not args.no_cpu and dist:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line))
    if dist:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
