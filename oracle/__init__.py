"""Python binding of the FP64 CPU oracle (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg load this package.
It shares no code with the CUDA library; the only module both sides use is the seeded input
generator `paper_1806_07390_gb300.workloads`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from paper_1806_07390_gb300.workloads import BC_CODES, GEOM_CODES, MAP_CODES, RIEMANN_CODES, Problem

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fx_oracle.cpp")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrcLayer(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("d", ctypes.c_int), ("m", ctypes.c_int),
                ("lo", ctypes.c_int * 3), ("hi", ctypes.c_int * 3), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("cot_alpha", ctypes.c_double), ("speed", ctypes.c_double),
                ("A", ctypes.c_double * 6), ("B", ctypes.c_double * 6)]


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int), ("n", ctypes.c_int * 3), ("geom", ctypes.c_int),
        ("map1", ctypes.c_int), ("x_lo", ctypes.c_double * 3), ("x_hi", ctypes.c_double * 3),
        ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3), ("ngroups", ctypes.c_int),
        ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double), ("gamma", ctypes.c_double),
        ("c_light", ctypes.c_double), ("a_rad", ctypes.c_double), ("kappa0", ctypes.c_double),
        ("kap_rho_exp", ctypes.c_double), ("kap_T_exp", ctypes.c_double),
        ("kap_eps_exp", ctypes.c_double), ("sigma0", ctypes.c_double),
        ("rad_recon_order", ctypes.c_int), ("r3_literal", ctypes.c_int), ("couple", ctypes.c_int),
        ("newton_maxit", ctypes.c_int), ("bisect_maxit", ctypes.c_int),
        ("newton_rtol", ctypes.c_double), ("rho_floor", ctypes.c_double),
        ("p_floor", ctypes.c_double), ("E_floor", ctypes.c_double), ("nthreads", ctypes.c_int),
        ("map_rt", ctypes.c_double), ("r10_full_dt", ctypes.c_int), ("riemann", ctypes.c_int),
        ("shock_guard", ctypes.c_double), ("vterms", ctypes.c_int), ("frozen_gas", ctypes.c_int),
        ("edges", ctypes.c_void_p), ("inflow", ctypes.c_void_p), ("nlayers", ctypes.c_int),
        ("layers", ctypes.c_void_p), ("t0", ctypes.c_double), ("species", ctypes.c_int),
        ("xi0", ctypes.c_double),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(OrcParams)
        L.orc_run.argtypes = [P, _DP, ctypes.c_double, ctypes.c_int]
        L.orc_run_tangent.argtypes = [P, _DP, _DP, ctypes.c_double, ctypes.c_int]
        L.orc_run_budget.argtypes = [P, _DP, ctypes.c_double, ctypes.c_int, _DP]
        L.orc_run_objective.argtypes = [P, _DP, _DP, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, _DP]
        L.orc_rhs.argtypes = [P, _DP, _DP]
        L.orc_couple.argtypes = [P, _DP, ctypes.c_double]
        L.orc_totals.argtypes = [P, _DP, _DP]
        L.orc_init_equilibrium.argtypes = [P, _DP, _DP]
        L.orc_state_size.argtypes = [P]
        L.orc_state_size.restype = ctypes.c_size_t
        for f in ("orc_planck_band",):
            getattr(L, f).argtypes = [ctypes.c_double, ctypes.c_double]
            getattr(L, f).restype = ctypes.c_double
        for f in ("orc_planck_lower", "orc_planck_upper", "orc_m1_chi"):
            getattr(L, f).argtypes = [ctypes.c_double]
            getattr(L, f).restype = ctypes.c_double
        L.orc_m1_pressure_row.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _DP,
                                          ctypes.c_int, _DP]
        L.orc_recon_cell.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, _DP, _DP]
        L.orc_hllc.argtypes = [ctypes.c_int, ctypes.c_double, _DP, _DP, _DP, _DP]
        L.orc_gas_flux.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _DP, _DP, _DP, _DP]
        L.orc_planck_group.argtypes = [P, ctypes.c_int, ctypes.c_double, _DP, _DP]
        L.orc_geometry.argtypes = [P, ctypes.c_int, _DP, _DP, _DP]
        L.orc_christoffel.argtypes = [P, _DP, _DP, _DP, _DP, _DP]
        L.orc_vterms.argtypes = [P, _DP, _DP, _DP]
        L.orc_vterms.restype = ctypes.c_double
        L.orc_vgrad.argtypes = [P, _DP, _DP]
        _lib = L
    return _lib


def layer_structs(layers):
    """Boundary layers (reading R29) as oracle structs: dictionaries with kind "front" or
    "mirror", box lo/hi, and the front (x0, y0, cot_alpha, speed, primitive states A, B) or mirror
    (d, m) parameters."""
    arr = (OrcLayer * max(len(layers), 1))()
    for q, ly in enumerate(layers):
        L = arr[q]
        L.kind = {"front": 0, "mirror": 1}[ly["kind"]]
        for d in range(3):
            L.lo[d], L.hi[d] = ly["lo"][d], ly["hi"][d]
        L.d, L.m = ly.get("d", 0), ly.get("m", 0)
        L.x0, L.y0 = ly.get("x0", 0.0), ly.get("y0", 0.0)
        L.cot_alpha, L.speed = ly.get("cot_alpha", 0.0), ly.get("speed", 0.0)
        for k, v in enumerate(ly.get("A", ())):
            L.A[k] = v
        for k, v in enumerate(ly.get("B", ())):
            L.B[k] = v
    return arr


def params(pb: Problem, nthreads: int = 1, r3_literal: int = 0, r10_full_dt: int = 0,
           edges=None, inflow=None, frozen_gas: int = 0, layers=None, t0: float = 0.0) -> OrcParams:
    """Oracle parameters of a problem.  edges (G + 1 group edges), inflow (E_g then the normal
    F_g of a radiation inflow through the lower x boundary) and frozen_gas are the oracle-only
    test aids of reading R28."""
    P = OrcParams()
    P.dims = pb.dims
    for d in range(3):
        P.n[d] = pb.n[d] if d < pb.dims else 1
        P.x_lo[d] = pb.x_lo[d]
        P.x_hi[d] = pb.x_hi[d]
        P.bc_lo[d] = BC_CODES[pb.bc_lo[d]]
        P.bc_hi[d] = BC_CODES[pb.bc_hi[d]]
    P.geom = GEOM_CODES[pb.geom]
    P.map1 = MAP_CODES[pb.map1]
    P.map_rt = pb.map_rt
    P.ngroups = pb.ngroups
    P.eps_min, P.eps_max = pb.eps_min, pb.eps_max
    P.gamma, P.c_light, P.a_rad = pb.gamma, pb.c_light, pb.a_rad
    P.kappa0, P.kap_rho_exp, P.kap_T_exp = pb.kappa0, pb.kap_rho_exp, pb.kap_T_exp
    P.kap_eps_exp, P.sigma0 = pb.kap_eps_exp, pb.sigma0
    P.rad_recon_order, P.r3_literal, P.couple = pb.rad_recon_order, r3_literal, pb.couple
    P.newton_maxit, P.bisect_maxit, P.newton_rtol = pb.newton_maxit, pb.bisect_maxit, pb.newton_rtol
    P.rho_floor, P.p_floor, P.E_floor = pb.rho_floor, pb.p_floor, pb.E_floor
    P.nthreads = nthreads
    P.r10_full_dt = r10_full_dt
    P.riemann = RIEMANN_CODES[pb.riemann]
    P.shock_guard = pb.shock_guard
    P.vterms = pb.vterms
    P.frozen_gas = frozen_gas
    P.species, P.xi0 = pb.species, pb.xi0
    if pb.species > 1 and layers:
        raise ValueError("three species: without boundary layers")
    keep = []
    if edges is not None:
        e = np.ascontiguousarray(edges, dtype=np.float64)
        assert e.shape == (pb.ngroups + 1,)
        keep.append(e)
        P.edges = e.ctypes.data
    if inflow is not None:
        f = np.ascontiguousarray(inflow, dtype=np.float64)
        assert f.shape == (2 * pb.ngroups,)
        keep.append(f)
        P.inflow = f.ctypes.data
        P.bc_lo[0] = 4  # ORC_INFLOW
    if layers:
        arr = layer_structs(layers)
        keep.append(arr)
        P.nlayers = len(layers)
        P.layers = ctypes.addressof(arr)
        P.t0 = t0
    P._keep = keep  # the arrays must outlive the calls that read P
    return P


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def init_equilibrium(pb: Problem, prim: np.ndarray) -> np.ndarray:
    P = params(pb)
    state = np.zeros(pb.state_size())
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    lib().orc_init_equilibrium(ctypes.byref(P), _ptr(prim), _ptr(state))
    return state


def run(pb: Problem, state: np.ndarray, dt: float, nsteps: int, nthreads: int = 1,
        **kw) -> tuple[np.ndarray, int]:
    P = params(pb, nthreads=nthreads, **kw)
    out = np.array(state, dtype=np.float64, copy=True)
    st = lib().orc_run(ctypes.byref(P), _ptr(out), dt, nsteps)
    return out, st


def run_budget(pb: Problem, state: np.ndarray, dt: float, nsteps: int, nthreads: int = 1):
    """orc_run with the budget terms of reading R13: returns (state, status, budget) with budget =
    boundary outflows [mass, momentum 1..3 (incl. radiation / c^2), total energy, radiation
    energy], the coupling work, the energy the positivity floor of E_g added and the radiation
    energy the velocity-dependent terms added, accumulated over the steps."""
    P = params(pb, nthreads=nthreads)
    out = np.array(state, dtype=np.float64, copy=True)
    bud = np.zeros(9)
    st = lib().orc_run_budget(ctypes.byref(P), _ptr(out), dt, nsteps, _ptr(bud))
    return out, st, bud


def run_tangent(pb: Problem, state: np.ndarray, tangent: np.ndarray, dt: float, nsteps: int):
    P = params(pb)
    out = np.array(state, dtype=np.float64, copy=True)
    tan = np.array(tangent, dtype=np.float64, copy=True)
    st = lib().orc_run_tangent(ctypes.byref(P), _ptr(out), _ptr(tan), dt, nsteps)
    return out, tan, st


def run_objective(pb: Problem, state: np.ndarray, dt: float, nsteps: int, tangent=None,
                  dkappa0: float = 0.0, signature: bool = False, nthreads: int = 1, **kw):
    """Advance nsteps steps accumulating the boundary outflow objective J (R19).

    Returns (final state, J, dJ, signature, status): dJ is the tangent of J along the initial-state
    tangent `tangent` and the kappa0 tangent `dkappa0` (0 when `tangent` is None); the signature
    (a Python int, or None) hashes every branch decision of the run in order."""
    P = params(pb, nthreads=nthreads, **kw)
    out = np.array(state, dtype=np.float64, copy=True)
    res = np.zeros(3)
    tan = None
    if tangent is not None:
        tan = np.array(tangent, dtype=np.float64, copy=True)
    st = lib().orc_run_objective(ctypes.byref(P), _ptr(out), _ptr(tan) if tan is not None else None,
                                 float(dkappa0), dt, nsteps, int(signature), _ptr(res))
    sig = int(res[2:3].view(np.uint64)[0]) if signature else None
    return out, float(res[0]), float(res[1]), sig, st


def rhs(pb: Problem, state: np.ndarray) -> np.ndarray:
    P = params(pb)
    s = np.ascontiguousarray(state, dtype=np.float64)
    out = np.zeros_like(s)
    lib().orc_rhs(ctypes.byref(P), _ptr(s), _ptr(out))
    return out


def couple(pb: Problem, state: np.ndarray, dt: float) -> tuple[np.ndarray, int]:
    P = params(pb)
    out = np.array(state, dtype=np.float64, copy=True)
    st = lib().orc_couple(ctypes.byref(P), _ptr(out), dt)
    return out, st


def totals(pb: Problem, state: np.ndarray) -> np.ndarray:
    P = params(pb)
    s = np.ascontiguousarray(state, dtype=np.float64)
    out = np.zeros(6)
    lib().orc_totals(ctypes.byref(P), _ptr(s), _ptr(out))
    return out


def planck_group(pb: Problem, g: int, T: float) -> tuple[float, float]:
    P = params(pb)
    B, dB = ctypes.c_double(), ctypes.c_double()
    lib().orc_planck_group(ctypes.byref(P), g, T, ctypes.byref(B), ctypes.byref(dB))
    return B.value, dB.value


def recon_cell(pb: Problem, d: int, i: int, pm: float, p0: float, pp: float, kind: int = 2,
               r3_literal: int = 0) -> tuple[float, float]:
    P = params(pb, r3_literal=r3_literal)
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_recon_cell(ctypes.byref(P), d, i, pm, p0, pp, kind, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def hllc(D: int, gamma: float, WL, WR) -> tuple[np.ndarray, float]:
    wl = np.zeros(5)
    wr = np.zeros(5)
    wl[: len(WL)] = WL
    wr[: len(WR)] = WR
    fl = np.zeros(5)
    vs = ctypes.c_double()
    lib().orc_hllc(D, gamma, _ptr(wl), _ptr(wr), _ptr(fl), ctypes.byref(vs))
    return fl[: 2 + D], vs.value


def gas_flux(solver: str, D: int, gamma: float, WL, WR) -> tuple[np.ndarray, float]:
    """Gas flux of one face by the solver "hllc", "hlle" or "llf" (states as for hllc)."""
    wl = np.zeros(5)
    wr = np.zeros(5)
    wl[: len(WL)] = WL
    wr[: len(WR)] = WR
    fl = np.zeros(5)
    vs = ctypes.c_double()
    lib().orc_gas_flux(RIEMANN_CODES[solver], D, gamma, _ptr(wl), _ptr(wr), _ptr(fl), ctypes.byref(vs))
    return fl[: 2 + D], vs.value


def m1_pressure_row(D: int, c: float, E: float, F, n: int) -> np.ndarray:
    f = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(D)
    lib().orc_m1_pressure_row(D, c, E, _ptr(f), n, _ptr(out))
    return out


def geometry(pb: Problem, d: int):
    P = params(pb)
    n = pb.n[d]
    vol, cen, m2 = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_geometry(ctypes.byref(P), d, _ptr(vol), _ptr(cen), _ptr(m2))
    return vol, cen, m2


def christoffel(pb: Problem):
    P = params(pb)
    nr, nt = pb.n[0], pb.n[1]
    a, b, c = np.zeros(nr), np.zeros(nr), np.zeros(nr)
    d, e = np.zeros(nt), np.zeros(nt)
    lib().orc_christoffel(ctypes.byref(P), _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(e))
    return {"G111": a, "G221": b, "G122": c, "G222": d, "G332": e}


# ---- external state layout helpers ----
def split_state(pb: Problem, state: np.ndarray):
    """(gas [NG, ncell], rad [(1+D), ncell, G]) views of an external-layout state vector."""
    NG = 2 + pb.dims
    gas = state[: NG * pb.ncell].reshape(NG, pb.ncell)
    rad = state[NG * pb.ncell:].reshape(1 + pb.dims, pb.ncell, pb.ngroups)
    return gas, rad


def vterms(pb: Problem, V, rad, edges=None) -> tuple[np.ndarray, float]:
    """Velocity-dependent radiation terms of one cell (readings R23-R27): V = <v^i_;j> (D x D),
    rad = [G, 1 + D] (E_g, physical F_g).  Returns (their time derivatives [G, 1 + D],
    sum_g dE_g/dt)."""
    P = params(pb, edges=edges)
    Vm = np.zeros((3, 3))
    Va = np.asarray(V, dtype=np.float64)
    Vm[: Va.shape[0], : Va.shape[1]] = Va
    r = np.ascontiguousarray(rad, dtype=np.float64)
    out = np.zeros_like(r)
    s = lib().orc_vterms(ctypes.byref(P), _ptr(np.ascontiguousarray(Vm.ravel())), _ptr(r), _ptr(out))
    return out, s


def vgrad(pb: Problem, state: np.ndarray) -> np.ndarray:
    """<v^i_;j> of every cell (readings R24-R25), [ncell, 3, 3] in x-fastest cell order."""
    P = params(pb)
    s = np.ascontiguousarray(state, dtype=np.float64)
    out = np.zeros((pb.ncell, 3, 3))
    lib().orc_vgrad(ctypes.byref(P), _ptr(s), _ptr(out.reshape(-1)))
    return out
