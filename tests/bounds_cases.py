"""Small runs of every kernel path of the stage update, for the index checks of the debug build.

Each case builds a small seeded problem, runs it through the library that the binding loads (the
normal build, or the debug build with index checks when FX_LIBRARY names libfx_bc.so) and
returns its outputs and the status of the run.  The cases span the kernel variants: 1-d, 2-d and
3-d grids with ragged tiles, the three precision forms, one and two groups per lane, odd group
counts, spherical grids, the velocity-dependent terms, three species, the carbuncle guard and the
alternative solvers, the parabolic radiation reconstruction, budgets on open boundaries, boundary
layers with graph replay, per-kernel timing, the objective, and the adjoint's forward and
backward passes.

Run as a script (python tests/bounds_cases.py OUT.npz) it saves every case's outputs, and status
under the key "<case>/status"; with --full it runs FULL_CASES instead: one step of the full-size
kh2d and lognormal3d workloads, whose states it keeps as SHA-256 digests.
"""
from __future__ import annotations

import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1806_07390_gb300 import fx  # noqa: E402
from paper_1806_07390_gb300 import workloads as W  # noqa: E402


def _forward(pb, prim=None, state=None, nsteps=2, budgets=False, layers=None, timing=False,
             objective=False):
    g = fx.Grid(pb)
    try:
        if layers is not None:
            g.boundary_layers(layers)
        if state is not None:
            g.upload(state)
        else:
            g.init_equilibrium(prim)
        if budgets:
            g.budgets_enable(True)
        if timing:
            g.kernel_timing(True)
        if objective:
            g.objective(True)
        g.step(pb.dt, nsteps)
        st = g.status()
        if st != 0:
            return st, {}
        out = {"state": g.download()}
        out["totals"] = g.totals()
        if budgets:
            out["budgets"] = g.budgets()
        if objective:
            out["J"] = np.array([g.boundary_energy_out()])
        return st, out
    finally:
        g.close()


def _adjoint(precision):
    pb, _ = W.blobs_2d(shape=(16, 12), ngroups=3, nsteps=2, precision=precision)
    s0 = W.random_state(pb, seed=9, flux_frac=0.3)
    g = fx.Grid(pb)
    try:
        g.upload(s0.astype(g.np_dtype))
        try:
            J, gs, gr, dk = g.adjoint(pb.dt, 2, 1)
        except fx.FxError as e:
            return e.status, {}
        st = g.status()
        return st, {"J": np.array([J, dk]), "grad_state": gs.cpu().numpy(), "grad_rho": gr.cpu().numpy()}
    finally:
        g.close()


def _kh(nx, ny, G, precision, **kw):
    pb, prim = W.kh_2d(nx=nx, ny=ny, ngroups=G, nsteps=2, precision=precision)
    for k, v in kw.items():
        setattr(pb, k, v)
    return pb, prim


def _blast(precision, riemann, guard):
    pb, prim = W.kh_2d(nx=44, ny=38, ngroups=5, nsteps=2, precision=precision)
    prim = prim.copy()
    y, x = np.divmod(np.arange(pb.ncell), 44)
    r2 = ((x + 0.5) / 44 - 0.45) ** 2 + ((y + 0.5) / 38 - 0.55) ** 2
    prim[1] = np.where(r2 < 0.04, 30.0, 1.0)
    prim[-1] = prim[1] / prim[0]
    pb.riemann, pb.shock_guard = riemann, guard
    return pb, prim


def _open_kh(precision, G):
    # kh2d with outflow and reflecting sides and some radiation flux: budgets on open boundaries
    pb, prim = W.kh_2d(nx=26, ny=18, ngroups=G, nsteps=2, precision=precision)
    pb.bc_lo = ("outflow", "reflect", "periodic")
    pb.bc_hi = ("outflow", "outflow", "periodic")
    return _forward(pb, state=W.random_state(pb, seed=4, flux_frac=0.3), budgets=True)


def case_names():
    return list(CASES)


def run_case(name):
    return CASES[name]()


CASES = {
    "sod1d_fp64": lambda: _forward(*W.sod_1d(n=40, ngroups=6, nsteps=2)),
    "sod1d_fp32": lambda: _forward(*W.sod_1d(n=40, ngroups=6, nsteps=2, precision="fp32")),
    "sod1d_fp32n64_g20": lambda: _forward(*W.sod_1d(n=37, ngroups=20, nsteps=2, precision="fp32n64")),
    "kh2d_fp64": lambda: _forward(*_kh(24, 20, 8, "fp64")),
    "kh2d_fp32n64_g16_vterms": lambda: _forward(*_kh(24, 20, 16, "fp32n64", vterms=1)),
    "kh2d_fp32_g5_vterms": lambda: _forward(*_kh(23, 21, 5, "fp32", vterms=1)),
    "kh2d_fp32_g20_recon2": lambda: _forward(*_kh(24, 20, 20, "fp32", rad_recon_order=2)),
    "kh2d_fp64_timing_objective": lambda: _forward(*_kh(24, 20, 4, "fp64"), timing=True, objective=True),
    "kh2d_fp32n64_timing": lambda: _forward(*_kh(24, 20, 16, "fp32n64", vterms=1), timing=True),
    "open2d_fp64_budgets": lambda: _open_kh("fp64", 6),
    "open2d_fp32n64_budgets": lambda: _open_kh("fp32n64", 17),
    "ln3d_fp64": lambda: _forward(*W.lognormal_3d(shape=(13, 11, 9), ngroups=5, nsteps=2, precision="fp64")),
    "ln3d_fp32n64": lambda: _forward(*W.lognormal_3d(shape=(13, 11, 9), ngroups=12, nsteps=2, precision="fp32n64")),
    "ln3d_fp32_vterms": lambda: _forward(*_ln3d_vterms()),
    "sph_fp64_vterms": lambda: _forward(*_sph("fp64", 6)),
    "sph_fp32_g20_vterms_budgets": lambda: _forward(*_sph("fp32", 20), budgets=True),
    "nu2d_fp32n64_vterms_budgets": lambda: _forward(*_nu2d("fp32n64"), budgets=True),
    "nu2d_fp64": lambda: _forward(*W.neutrino_2d(nx=16, ny=12, ngroups=4, nsteps=2)),
    "nu_sph_fp32": lambda: _forward(*W.neutrino_sph2d(nr=16, nth=8, ngroups=3, nsteps=2, precision="fp32")),
    "blast_fp32_hllc_guard": lambda: _forward(*_blast("fp32", "hllc", 0.5)),
    "blast_fp64_llf": lambda: _forward(*_blast("fp64", "llf", 0.0)),
    "blast_fp32n64_hlle": lambda: _forward(*_blast("fp32n64", "hlle", 0.0)),
    "dmr_fp32n64_layers": lambda: _dmr("fp32n64"),
    "dmr_fp64_layers": lambda: _dmr("fp64"),
    "adjoint_fp64": lambda: _adjoint("fp64"),
    "adjoint_fp32": lambda: _adjoint("fp32"),
}


def _ln3d_vterms():
    pb, prim = W.lognormal_3d(shape=(13, 11, 9), ngroups=7, nsteps=2, precision="fp32")
    pb.vterms = 1
    return pb, prim


def _sph(precision, G):
    pb, prim = W.spherical_2d(nr=24, nth=12, ngroups=G, nsteps=2, precision=precision)
    pb.vterms = 1
    return pb, prim


def _nu2d(precision):
    pb, prim = W.neutrino_2d(nx=16, ny=12, ngroups=4, nsteps=2, precision=precision)
    pb.vterms = 1
    return pb, prim


def _dmr(precision):
    # boundary layers; fx_step replays the captured step graph (no timing, no objective)
    pb, prim, layers = W.double_mach(nx=130, ny=40, t_end=0.05, precision=precision)
    return _forward(pb, prim, nsteps=3, layers=layers)


def _full(pb, prim):
    # one step at full size in the benchmark's launch configuration: the state's SHA-256 (the
    # arrays are gigabytes) and the totals
    st, out = _forward(pb, prim, nsteps=1)
    if st == 0:
        out["sha256"] = np.frombuffer(hashlib.sha256(out.pop("state").tobytes()).digest(), dtype=np.uint8)
    return st, out


FULL_CASES = {
    "kh2d_1024x1024x16_fp32n64": lambda: _full(*W.kh_2d(nx=1024, ny=1024, ngroups=16, nsteps=1,
                                                       precision="fp32n64")),
    "lognormal3d_256x256x256x12_fp32n64": lambda: _full(*W.lognormal_3d(n=256, ngroups=12, nsteps=1,
                                                                        precision="fp32n64")),
}


def main(path, full=False):
    cases = FULL_CASES if full else CASES
    out = {}
    for name in cases:
        st, arrs = cases[name]()
        out[f"{name}/status"] = np.array([st])
        for k, v in arrs.items():
            out[f"{name}/{k}"] = v
    np.savez(path, **out)
    print(f"ran {len(cases)} cases with {fx.LIB_PATH}")


if __name__ == "__main__":
    main(sys.argv[1], full="--full" in sys.argv[2:])
