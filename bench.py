"""Benchmark of the multigroup M1 radiation-hydrodynamics stage update on GB300.

Metric: zone-group updates per second per RK stage (each RK stage updates every zone-group of
the grid once).  Headline `value`: the FP32 form with the FP64 Newton (FP32 state, reconstruction
and fluxes; FP64 temperature iterate, residual and energy/momentum bookkeeping); the `forms`
object reports the all-FP32 variant and the plain FP64 path.  Workload: 2-d periodic
Kelvin-Helmholtz, 1024 x 1024 cells x 16 groups (synthetic seeded input; inputs are larger than
L2, so no flush is needed between timed steps).  The `adjoint` object times the differentiation
form (forward + hand-written adjoint) on the 512 x 512 x 8 blob-screen workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]

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
# DRAM bytes per launch (mean of the two RK stages) of the radiation/update kernel and of the
# interaction kernel, from the committed ncu capture profiles/traffic_kh2d_1024x1024x16.txt; None
# where not captured for the current kernels.
TRAFFIC_PER_LAUNCH = {"kh2d": {"fp32n64": 570.6e6}}
TRAFFIC_INTERACTION = {"kh2d": {"fp32n64": 370.9e6}}
# FP64 lane operations (DFMA + DADD + DMUL thread instructions) per zone-group of the FP64 form's
# radiation/update and interaction kernels, from the committed ncu capture
# profiles/fp64_pipe_kh2d_512x512x16.txt (kh2d recipe at 512 x 512 cells x 16 groups).
FP64_OPS_PER_ZG = {"kh2d": {"stage": 315.8, "interaction": 217.3}}


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


def max_over_ranks(x: float) -> float:
    """Maximum of x over the ranks of the default process group (x itself without one): the
    timed region of a multi-GPU run ends when its slowest rank ends."""
    import torch
    import torch.distributed as tdist

    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return x
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units all ranks processed (each rank runs its own replica) per second of the slowest rank."""
    return world * units_per_rank / seconds


def time_form(pb, prim, steps, warmup, dist, graph_replay=False):
    """Device-timed K steps of one precision form with inputs resident in HBM.  The timed region
    carries the per-kernel CUDA events (the roofline's kernel durations), so fx_step launches
    the kernels one by one there.  With graph_replay, K more steps follow without the per-kernel
    events, which fx_step replays as a captured CUDA graph of a step (returned in kt)."""
    import torch

    from paper_1806_07390_gb300 import fx

    g = fx.Grid(pb)
    g.init_equilibrium(prim)
    if getattr(pb, "layers", None):
        g.boundary_layers(pb.layers)
    g.sync()
    for _ in range(warmup):
        g.step(pb.dt, 1)
    g.sync()
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    s = g.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.kernel_timing(True)  # per-kernel CUDA events on the launching stream, inside the timed region
    e0.record(s)
    for _ in range(steps):
        g.step(pb.dt, 1)
    e1.record(s)
    e1.synchronize()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = g.kernel_times()
    g.kernel_timing(False)
    if graph_replay:
        g.step(pb.dt, 1)  # the first step without events captures the graph
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(s)
        for _ in range(steps):
            g.step(pb.dt, 1)
        f1.record(s)
        f1.synchronize()
        kt["graph_ms"] = max_over_ranks(f0.elapsed_time(f1)) if dist else f0.elapsed_time(f1)
    st = g.status()
    if dist:
        ms = max_over_ranks(ms)
    launches = g.launches_per_step() * steps
    return g, ms, st, launches, kt


def time_e2e(g, pb, steps, warmup):
    """Same metric through the public API with host buffers: every step uploads the state from
    pinned host memory, advances one step and downloads the result to pinned host memory."""
    import torch

    n = g.nelem
    dt_t = torch.float64 if pb.precision == "fp64" else torch.float32
    # two pinned host buffers used in turn: each step uploads the previous step's result
    bufs = [torch.empty(n, dtype=dt_t, pin_memory=True) for _ in range(2)]
    prec = 0 if pb.precision == "fp64" else 1
    import ctypes
    L = g.L

    def one(i):
        h_in, h_out = bufs[i % 2], bufs[(i + 1) % 2]
        g._check(L.fx_state_upload(g.h, ctypes.c_void_p(h_in.data_ptr()), prec, 0))
        g.step(pb.dt, 1)
        g._check(L.fx_state_download(g.h, ctypes.c_void_p(h_out.data_ptr()), prec, 0))

    g._check(L.fx_state_download(g.h, ctypes.c_void_p(bufs[0].data_ptr()), prec, 0))
    for i in range(warmup):
        one(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(warmup, warmup + steps):
        one(i)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    return sec, n * bufs[0].element_size(), n * bufs[0].element_size()


# Workloads: generator, default headline precision form, description, and the oracle sample used
# for the CPU baseline (window start, interior size, halo) or None for the whole grid.
WORKLOADS = {
    "kh2d": (W.kh_2d, "fp32n64", "2-d periodic Kelvin-Helmholtz, 1024x1024 cells x 16 groups",
             ((384, 384), (248, 248), 4)),
    "lognormal3d": (W.lognormal_3d, "fp32n64",
                    "3-d periodic lognormal density, 256^3 cells x 12 groups",
                    ((100, 100, 100), (40, 40, 40), 4)),
    "sph2d": (W.spherical_2d, "fp32",
              "2-d spherical (r, theta) log-r atmosphere, 640x128 cells x 20 groups", None),
    "blobs2d": (W.blobs_2d, "fp32", "2-d density blobs, 512x512 cells x 8 groups",
                ((128, 128), (248, 248), 4)),
    "sod1d": (W.sod_1d, "fp64", "1-d radiating Sod tube, 512 cells x 12 groups", None),
    "nu2d": (W.neutrino_2d, "fp32n64", "2-d periodic box, three neutrino species, 512x512 cells x "
             "(3 x 8) channels, two-equation (T, Y_e) interaction", None),
    "dmr": (lambda precision, nx=520, ny=160: _with_layers(W.double_mach(nx=nx, ny=ny, precision=precision)),
            "fp32", "double Mach reflection, 520x160 cells (+ boundary layers) x 1 inert group, "
            "HLLC with the carbuncle guard", None),
}


def _with_layers(res):
    """(problem, prim) of a workload with boundary layers, the layers kept on the problem."""
    pb, prim, layers = res
    pb.layers = layers
    return pb, prim


def sized(name, gen, shape):
    """The workload's generator at another grid size (same recipe)."""
    if name == "kh2d":
        return lambda precision: W.kh_2d(nx=shape[0], ny=shape[1], precision=precision)
    if name == "sph2d":
        return lambda precision: W.spherical_2d(nr=shape[0], nth=shape[1], precision=precision)
    if name == "sod1d":
        return lambda precision: W.sod_1d(n=shape[0], precision=precision)
    if name == "dmr":
        return lambda precision: gen(precision, nx=shape[0], ny=shape[1])
    if name == "nu2d":
        return lambda precision: W.neutrino_2d(nx=shape[0], ny=shape[1], precision=precision)
    return lambda precision: gen(shape=tuple(shape), precision=precision)


FORM_DTYPE = {"fp32": "f32", "fp32n64": "f32+f64-newton", "fp64": "f64"}
FORM_NOTE = {"fp32": "FP32 state, fluxes and coupling (anchored FP32 Newton), FP64 totals",
             "fp32n64": "FP32 state and fluxes, FP64 Newton and energy bookkeeping, FP64 totals",
             "fp64": "FP64 throughout"}


def time_adjoint(steps_rep: int = 3):
    """The differentiation form on its own workload (blobs2d: 512 x 512 cells x 8 groups, FP32,
    a beam along +x through density blobs): J = radiation energy leaving through +x over 50
    steps, gradients with respect to rho(x, 0) and kappa0 with a checkpoint every 10 steps.
    Times (CUDA events on the handle's stream) the plain forward with the objective, the
    adjoint's forward pass (objective + checkpoints) and its backward pass (recomputation +
    stage adjoints); the median of steps_rep repetitions after one warm-up."""
    import torch

    from paper_1806_07390_gb300 import fx

    nsteps, k = 50, 10
    pb, prim = W.blobs_2d(precision="fp32")
    g = fx.Grid(pb)
    g.init_equilibrium(prim)
    s0 = W.streaming_flux(pb, g.download().astype(np.float64), 0.5)
    # the initial state stays resident on the device; every run restores it with a device copy
    # outside its timed region
    s0_dev = torch.tensor(s0.astype(np.float32), device=g.workspace.device)
    ws = g.adjoint_workspace(nsteps, k)
    st = g.stream

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def fwd_plain():
        g.step(pb.dt, nsteps)

    res = {"fwd": [], "adj_fwd": [], "adj_bwd": []}
    out = {}
    for rep in range(steps_rep + 1):
        g.upload(s0_dev)
        g.objective(True)
        tf = timed(fwd_plain)
        J_plain = g.boundary_energy_out()
        g.objective(False)
        g.upload(s0_dev)
        ta = timed(lambda: out.__setitem__("J", g.adjoint_forward(ws, pb.dt, nsteps, k)))
        tb = timed(lambda: out.__setitem__("g", g.adjoint_backward(ws, pb.dt, nsteps, k)))
        if rep > 0:
            res["fwd"].append(tf)
            res["adj_fwd"].append(ta)
            res["adj_bwd"].append(tb)
    med = {kk: statistics.median(v) for kk, v in res.items()}
    gs, gr, dk = out["g"]
    g.close()
    return {"workload": "blobs2d: 512x512 cells x 8 groups, FP32 form, beam along +x, 50 steps, "
                        "checkpoint every 10 steps",
            "J": out["J"], "J_plain_forward": J_plain, "dJ_dkappa0": dk,
            "grad_rho_norm": float(gr.double().norm()),
            "forward_ms": med["fwd"], "adjoint_forward_ms": med["adj_fwd"],
            "adjoint_backward_ms": med["adj_bwd"],
            "adjoint_step_over_forward_step": med["adj_bwd"] / med["fwd"],
            "gradient_over_forward": (med["adj_fwd"] + med["adj_bwd"]) / med["fwd"],
            "note": "adjoint step = recomputation of its checkpoint segment + the two stage adjoints"}


def oracle_sample(pb64, prim, spec):
    if spec is None:
        return pb64, prim, f"whole {'x'.join(str(n) for n in pb64.n[:pb64.dims])} grid"
    start, size, halo = spec
    sub, sprim = W.window(pb64, prim, start, size, halo)
    return sub, sprim, (f"{'x'.join(str(n) for n in sub.n[:sub.dims])}-cell window "
                        f"({halo}-cell halo, outflow edges) of the full grid")


def cpu_baseline(pb64, prim, spec, budget_s=15.0):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of the same workload
    (same spacing, c and dt), stepped until ~budget_s."""
    import oracle

    cores = os.cpu_count() or 1
    sub, sprim, what = oracle_sample(pb64, prim, spec)
    s = oracle.init_equilibrium(sub, sprim)
    lay = getattr(sub, "layers", None)
    t0 = time.perf_counter()
    nst = 0
    while True:
        s, _ = oracle.run(sub, s, sub.dt, 1, nthreads=cores, layers=lay, t0=nst * sub.dt)
        nst += 1
        if time.perf_counter() - t0 > budget_s or nst >= 50:
            break
    sec = time.perf_counter() - t0
    zgs = sub.ncell * sub.nchan * 2 * nst
    return {"value": zgs / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what} x {sub.nchan} groups, {nst} FP64 steps, OpenMP over cells"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    gen, form, desc, spec = WORKLOADS[args.workload]
    pb, prim = gen(precision="fp64")
    if spec is not None and args.workload == "kh2d":
        spec = ((384, 384), (120, 120), 4)  # smaller sample: each timed step stays ~1 s
    elif spec is not None and args.workload == "lognormal3d":
        spec = ((100, 100, 100), (24, 24, 24), 4)
    steps, warmup = args.steps, args.warmup
    import oracle

    cores = os.cpu_count() or 1
    sub, sprim, what = oracle_sample(pb, prim, spec)
    s = oracle.init_equilibrium(sub, sprim)
    lay = getattr(sub, "layers", None)
    for i in range(warmup):
        s, _ = oracle.run(sub, s, sub.dt, 1, nthreads=cores, layers=lay, t0=i * sub.dt)
    t0 = time.perf_counter()
    for i in range(steps):
        s, _ = oracle.run(sub, s, sub.dt, 1, nthreads=cores, layers=lay, t0=(warmup + i) * sub.dt)
    sec = time.perf_counter() - t0
    zgs = sub.ncell * sub.nchan * 2 * steps
    val = zgs / sec
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * sec / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc} (oracle sample: {what})",
                       "precision": "fp64"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{what} x {sub.nchan} groups, {steps} FP64 steps"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kh2d", choices=sorted(WORKLOADS))
    ap.add_argument("--form", default=None, choices=["fp32", "fp32n64", "fp64"],
                    help="precision form of the headline value (default: the workload's)")
    ap.add_argument("--forms", default="fp32,fp32n64,fp64",
                    help="extra precision forms timed beside the headline (comma list)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-vterms", action="store_true",
                    help="skip the headline form timed with the velocity-dependent terms on")
    ap.add_argument("--shape", default=None,
                    help="cells per direction, comma list (a smaller grid of the same recipe, for "
                         "profiler captures; the default is the workload's full size)")
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

    gen, form0, desc, spec = WORKLOADS[args.workload]
    if args.shape:
        gen = sized(args.workload, gen, [int(x) for x in args.shape.split(",")])
        desc = f"{desc.split(',')[0]} at {args.shape.replace(',', 'x')} cells (profiling size)"
        spec = None
    head = args.form or form0
    pbh, prim = gen(precision=head)
    forms = {}
    for name in [f for f in args.forms.split(",") if f and f != head]:
        if name == "fp64" and args.no_fp64:
            continue
        forms[name] = gen(precision=name)[0]
    zg = pbh.ncell * pbh.nchan  # zone-groups (zone-channels with three species)
    peak, peak_kind = load_peaks()
    # the headline form once more with the velocity-dependent radiation terms (Cartesian grids)
    pbv = None
    if not args.no_vterms and pbh.geom == "cart" and pbh.species == 1:
        pbv = gen(precision=head)[0]
        pbv.vterms = 1

    results = {}
    with ClockSampler(dev) as clk:
        gh, msh, sth, launchesh, kth = time_form(pbh, prim, args.steps, args.warmup, dist,
                                                 graph_replay=True)
        for name, pbf in forms.items():
            gf, msf, stf, lf, ktf = time_form(pbf, prim, args.steps, args.warmup, dist)
            results[name] = (msf, stf, lf, ktf)
            gf.close()
        if pbv is not None:
            gv, msv, stv, lv, ktv = time_form(pbv, prim, args.steps, args.warmup, dist)
            gv.close()
    clocks = clk.summary()

    sech = msh / 1e3
    value = whole_job_rate(zg * 2 * args.steps, world, sech)
    nv = pbh.nvar - pbh.ncomp  # the variables the radiation/update kernel moves

    sm_max = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            sm_max = float(json.load(f).get("sm_max_mhz", sm_max))
    except (OSError, ValueError):
        pass
    # FP64 pipe of GB300: 2 FP64 lane operations per cycle per SM (a warp instruction holds the
    # pipe 16 cycles), 152 SMs at the maximum SM clock
    fp64_peak = 152 * 2 * sm_max * 1e6

    def roofline(kind, kt):
        """Radiation/update kernel (the dominant one): algorithmic bytes per launch over its
        average CUDA-event launch duration in the timed region.  In the FP64 form the kernels are
        bound by the FP64 pipe: the line reports that bound (FP64 lane operations per second
        against the pipe's peak) and keeps the HBM figures under "hbm"."""
        b = 8 if kind == "fp64" else 4
        per_launch = 2.5 * b * nv * pbh.ncell  # 2.5 N_v words per cell per stage
        avg_s = kt["stage_ms"] / max(kt["stage_launches"], 1) / 1e3
        achieved = per_launch / avg_s / 1e9
        trafficd = TRAFFIC_PER_LAUNCH.get(args.workload, {})
        total = max(kt["stage_ms"] + kt["face_ms"] + kt["couple_ms"], 1e-30)
        out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
               "frac": achieved / peak, "traffic": trafficd.get(kind),
               "peak_kind": peak_kind, "kernel": "stage_kernel (radiation/update)",
               "bytes_per_launch": per_launch, "avg_launch_ms": avg_s * 1e3,
               "face_kernel_avg_ms": kt["face_ms"] / max(kt["face_launches"], 1),
               "stage_share_of_step": kt["stage_ms"] / total}
        cs = kt["couple_ms"] / kt["couple_launches"] / 1e3 if kt["couple_launches"] else None
        if cs:
            # the interaction kernel reads and writes the state once per stage
            cb = 2.0 * b * nv * pbh.ncell
            out["interaction_kernel"] = {
                "kernel": "couple_kernel / couple64_kernel (interaction, one thread per cell)",
                "bytes_per_launch": cb, "avg_launch_ms": cs * 1e3, "achieved": cb / cs / 1e9,
                "frac": cb / cs / 1e9 / peak, "share_of_step": kt["couple_ms"] / total,
                "traffic": TRAFFIC_INTERACTION.get(args.workload, {}).get(kind)}
        ops = FP64_OPS_PER_ZG.get(args.workload)
        if kind == "fp64" and ops:
            hbm = {k: out[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "peak_kind")}
            a64 = ops["stage"] * zg / avg_s
            out.update({"bound": "alu", "achieved": a64, "peak": fp64_peak, "unit": "FP64 lane-op/s",
                        "frac": a64 / fp64_peak, "peak_kind": "FP64 pipe: 152 SMs x 2 lane-ops/clk x max SM clock",
                        "ops_per_zone_group": ops["stage"], "hbm": hbm})
            if cs:
                ai = ops["interaction"] * zg / cs
                out["interaction_kernel"].update({"alu_achieved": ai, "alu_frac": ai / fp64_peak,
                                                  "ops_per_zone_group": ops["interaction"]})
        return out

    e2e_steps = max(5, args.steps // 4)
    if args.no_e2e:
        e2e_sec, h2d, d2h = float("nan"), 0, 0
    else:
        e2e_sec, h2d, d2h = time_e2e(gh, pbh, e2e_steps, 2)
    chunk_h = gh.march_chunk()
    gh.close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": msh / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": FORM_DTYPE[head],
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc}, {head} form", "cells": pbh.ncell,
                       "groups": pbh.ngroups, "form": FORM_NOTE[head],
                       "l2": ("inputs larger than L2 (no flush)"
                              if pbh.state_size() * (8 if head == "fp64" else 4) * 2 > 129e6
                              else "state fits in L2 (no flush): L2-resident figure"),
                       "precision": head, "parallelism": f"replicas{world}",
                       "march_chunk": chunk_h},
            "roofline": roofline(head, kth),
            "e2e": {"value": world * zg * 2 * e2e_steps / e2e_sec, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launchesh,  # the headline form's timed region
            "gpu_launches_all_timed_regions": launchesh + sum(r[2] for r in results.values()) +
                                              (lv if pbv is not None else 0),
            "clocks": clocks, "status": int(sth), "forms": {}}
    if "graph_ms" in kth:
        line["graph_replay"] = {
            "note": "the same form and steps right after the timed region, without the per-kernel "
                    "events: fx_step replays one captured CUDA graph per step",
            "ms_per_step": kth["graph_ms"] / args.steps,
            "value": whole_job_rate(zg * 2 * args.steps, world, kth["graph_ms"] / 1e3), "unit": UNIT}
    for name, (msf, stf, lf, ktf) in results.items():
        secf = msf / 1e3
        line["forms"][name] = {"value": whole_job_rate(zg * 2 * args.steps, world, secf), "unit": UNIT,
                               "ms_per_step": msf / args.steps, "note": FORM_NOTE[name],
                               "roofline": roofline(name, ktf), "status": int(stf),
                               "speedup_of_headline": msf / msh}
    if pbv is not None:
        # velocity-term kernel: reads the stage input's radiation rows and reads and writes the
        # stage output's (3 G (1 + D) words per cell per launch); its time is the interval after
        # the radiation/update kernel less the interaction kernel's time without the terms
        b = 8 if head == "fp64" else 4
        vb = 3.0 * b * pbh.ngroups * (1 + pbh.dims) * pbh.ncell
        per = lambda kt: kt["couple_ms"] / max(kt["couple_launches"], 1)  # noqa: E731
        vms = per(ktv) - per(kth)
        line["vterms"] = {
            "note": "headline form with the velocity-dependent radiation terms (work terms and "
                    "frequency-space fluxes) in each stage's operator: one more kernel per stage",
            "value": whole_job_rate(zg * 2 * args.steps, world, msv / 1e3), "unit": UNIT,
            "ms_per_step": msv / args.steps, "extra_ms_per_step": (msv - msh) / args.steps,
            "status": int(stv),
            "kernel": {"name": "vterm_kernel2" if head != "fp64" and pbh.nchan > 8 else "vterm_kernel",
                       "avg_launch_ms": vms, "bytes_per_launch": vb,
                       "achieved": vb / (vms / 1e3) / 1e9 if vms > 0 else None, "unit": "GB/s",
                       "frac": vb / (vms / 1e3) / 1e9 / peak if vms > 0 else None}}
    if not args.no_adjoint and args.workload == "kh2d":
        line["adjoint"] = time_adjoint()
    if rank == 0 and not args.no_cpu and not dist:
        pb64 = gen(precision="fp64")[0]
        line["cpu_baseline"] = cpu_baseline(pb64, prim, spec)
    elif rank == 0 and not args.no_cpu and dist:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line))
    if dist:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
