"""Thin Python binding of the C ABI in include/fx.h (argument marshalling only).

Every step of the stage update runs in the CUDA library libfx.so; this module only converts
arguments, owns the torch-allocated workspace and forwards calls.  Importing it does not need a
GPU; creating a bound Grid does, and fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from .workloads import BC_CODES, GEOM_CODES, MAP_CODES, RIEMANN_CODES, Problem

_HERE = os.path.dirname(os.path.abspath(__file__))
# FX_LIBRARY selects another build of the library (the debug build with index checks, libfx_bc.so)
LIB_PATH = os.environ.get("FX_LIBRARY") or os.path.join(_HERE, "libfx.so")

FX_OK = 0
STATUS_NAMES = {0: "FX_OK", -1: "FX_ERR_ARG", -2: "FX_ERR_CUDA", -3: "FX_ERR_WORKSPACE",
                -4: "FX_ERR_NEWTON", -5: "FX_ERR_FLOOR", -6: "FX_ERR_NONFINITE",
                -7: "FX_ERR_UNSUPPORTED", -8: "FX_ERR_BOUNDS"}
FX_FP64, FX_FP32, FX_FP32_F64NEWTON = 0, 1, 2
NTOTALS = 6
NBUDGET = 9

# every symbol include/fx.h declares
EXPORTS = ["fx_grid_create", "fx_bind_workspace", "fx_state_elems", "fx_state_upload",
           "fx_state_init_equilibrium", "fx_step", "fx_sync", "fx_conserved_totals",
           "fx_state_download", "fx_launches_per_step", "fx_march_chunk", "fx_debug_table", "fx_debug_ntab",
           "fx_debug_planck_table", "fx_state_init_equilibrium_noalloc",
           "fx_kernel_timing_enable", "fx_kernel_timing_read", "fx_objective_enable",
           "fx_boundary_energy_out", "fx_set_kappa0", "fx_state_set_density",
           "fx_adjoint_workspace_bytes", "fx_adjoint_forward", "fx_adjoint_backward", "fx_adjoint",
           "fx_budgets_enable", "fx_budgets", "fx_boundary_layers", "fx_last_error", "fx_clear_error",
           "fx_grid_destroy"]


class FxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class FxLayer(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("d", ctypes.c_int), ("m", ctypes.c_int),
                ("lo", ctypes.c_int64 * 3), ("hi", ctypes.c_int64 * 3), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("cot_alpha", ctypes.c_double), ("speed", ctypes.c_double),
                ("A", ctypes.c_double * 6), ("B", ctypes.c_double * 6)]


class FxParams(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("geom", ctypes.c_int),
        ("map1", ctypes.c_int), ("x_lo", ctypes.c_double * 3), ("x_hi", ctypes.c_double * 3),
        ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3), ("ngroups", ctypes.c_int),
        ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double), ("gamma", ctypes.c_double),
        ("c_light", ctypes.c_double), ("a_rad", ctypes.c_double), ("kappa0", ctypes.c_double),
        ("kap_rho_exp", ctypes.c_double), ("kap_T_exp", ctypes.c_double),
        ("kap_eps_exp", ctypes.c_double), ("sigma0", ctypes.c_double), ("precision", ctypes.c_int),
        ("rad_recon_order", ctypes.c_int), ("couple", ctypes.c_int),
        ("newton_maxit", ctypes.c_int), ("bisect_maxit", ctypes.c_int),
        ("newton_rtol", ctypes.c_double), ("rho_floor", ctypes.c_double),
        ("p_floor", ctypes.c_double), ("E_floor", ctypes.c_double), ("map_rt", ctypes.c_double),
        ("riemann", ctypes.c_int), ("shock_guard", ctypes.c_double), ("vterms", ctypes.c_int),
        ("species", ctypes.c_int), ("xi0", ctypes.c_double),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libfx.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: build it with "
                               "paper_1806_07390_gb300.build.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, dp = ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)
        L.fx_grid_create.argtypes = [ctypes.POINTER(FxParams), ctypes.POINTER(vp), ctypes.POINTER(sz)]
        L.fx_bind_workspace.argtypes = [vp, vp, sz, vp]
        L.fx_state_elems.argtypes = [vp]
        L.fx_state_elems.restype = sz
        L.fx_state_upload.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
        L.fx_state_init_equilibrium.argtypes = [vp, vp, ctypes.c_int]
        L.fx_step.argtypes = [vp, ctypes.c_double, ctypes.c_int]
        L.fx_sync.argtypes = [vp]
        L.fx_conserved_totals.argtypes = [vp, dp]
        L.fx_state_download.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
        L.fx_launches_per_step.argtypes = [vp]
        L.fx_march_chunk.argtypes = [vp]
        L.fx_debug_table.argtypes = [vp, ctypes.c_int, dp, sz]
        L.fx_debug_ntab.argtypes = []
        L.fx_debug_planck_table.argtypes = [vp, ctypes.POINTER(ctypes.c_float), sz,
                                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
        L.fx_state_init_equilibrium_noalloc.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        L.fx_state_init_equilibrium_noalloc.restype = ctypes.c_int
        L.fx_kernel_timing_enable.argtypes = [vp, ctypes.c_int]
        L.fx_kernel_timing_read.argtypes = [vp, dp]
        L.fx_objective_enable.argtypes = [vp, ctypes.c_int]
        L.fx_boundary_energy_out.argtypes = [vp, dp]
        L.fx_set_kappa0.argtypes = [vp, ctypes.c_double]
        L.fx_state_set_density.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
        L.fx_adjoint_workspace_bytes.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(sz)]
        L.fx_adjoint_forward.argtypes = [vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, sz, dp]
        L.fx_adjoint_backward.argtypes = [vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, sz,
                                          ctypes.c_double, vp, vp, dp]
        L.fx_adjoint.argtypes = [vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, sz, vp, vp, dp, dp]
        L.fx_budgets_enable.argtypes = [vp, ctypes.c_int]
        L.fx_boundary_layers.argtypes = [vp, ctypes.POINTER(FxLayer), ctypes.c_int, ctypes.c_double]
        L.fx_budgets.argtypes = [vp, dp]
        L.fx_last_error.argtypes = [vp]
        L.fx_last_error.restype = ctypes.c_char_p
        L.fx_clear_error.argtypes = [vp]
        L.fx_grid_destroy.argtypes = [vp]
        for f in ("fx_grid_create", "fx_bind_workspace", "fx_state_upload",
                  "fx_state_init_equilibrium", "fx_step", "fx_sync", "fx_conserved_totals",
                  "fx_state_download", "fx_kernel_timing_enable", "fx_kernel_timing_read",
                  "fx_objective_enable", "fx_boundary_energy_out", "fx_set_kappa0",
                  "fx_state_set_density", "fx_adjoint_workspace_bytes", "fx_adjoint_forward",
                  "fx_adjoint_backward", "fx_adjoint", "fx_budgets_enable", "fx_budgets"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def params(pb: Problem) -> FxParams:
    P = FxParams()
    P.dims = pb.dims
    for d in range(3):
        P.n[d] = pb.n[d] if d < pb.dims else 1
        P.x_lo[d], P.x_hi[d] = pb.x_lo[d], pb.x_hi[d]
        P.bc_lo[d], P.bc_hi[d] = BC_CODES[pb.bc_lo[d]], BC_CODES[pb.bc_hi[d]]
    P.geom, P.map1 = GEOM_CODES[pb.geom], MAP_CODES[pb.map1]
    P.map_rt = pb.map_rt
    P.ngroups, P.eps_min, P.eps_max = pb.ngroups, pb.eps_min, pb.eps_max
    P.gamma, P.c_light, P.a_rad = pb.gamma, pb.c_light, pb.a_rad
    P.kappa0, P.kap_rho_exp, P.kap_T_exp = pb.kappa0, pb.kap_rho_exp, pb.kap_T_exp
    P.kap_eps_exp, P.sigma0 = pb.kap_eps_exp, pb.sigma0
    P.precision = {"fp64": FX_FP64, "fp32": FX_FP32, "fp32n64": FX_FP32_F64NEWTON}[pb.precision]
    P.rad_recon_order, P.couple = pb.rad_recon_order, pb.couple
    P.newton_maxit, P.bisect_maxit, P.newton_rtol = pb.newton_maxit, pb.bisect_maxit, pb.newton_rtol
    P.rho_floor, P.p_floor, P.E_floor = pb.rho_floor, pb.p_floor, pb.E_floor
    P.riemann, P.shock_guard = RIEMANN_CODES[pb.riemann], pb.shock_guard
    P.vterms = pb.vterms
    P.species, P.xi0 = pb.species, pb.xi0
    return P


class Grid:
    """One handle of the CUDA stage update with a torch-owned workspace on `device`."""

    def __init__(self, pb: Problem, device: str = "cuda", stream=None, bind: bool = True):
        import torch

        self.pb = pb
        self.L = lib()
        self._P = params(pb)
        h = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        st = self.L.fx_grid_create(ctypes.byref(self._P), ctypes.byref(h), ctypes.byref(ws))
        if st != FX_OK:
            raise FxError(st, "fx_grid_create rejected the parameters")
        self.h = h
        self.ws_bytes = ws.value
        self.workspace = None
        if bind:
            self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
            self._check(self.L.fx_bind_workspace(h, ctypes.c_void_p(self.workspace.data_ptr()),
                                                 self.ws_bytes, ctypes.c_void_p(self.stream.cuda_stream)))

    # -- helpers
    def _check(self, st: int) -> None:
        if st != FX_OK:
            msg = self.L.fx_last_error(self.h).decode()
            raise FxError(st, msg)

    @property
    def nelem(self) -> int:
        return int(self.L.fx_state_elems(self.h))

    @property
    def np_dtype(self):
        return np.float64 if self.pb.precision == "fp64" else np.float32

    def debug_table(self, d: int) -> np.ndarray:
        ntab = self.L.fx_debug_ntab()
        n = ntab * (self.pb.n[d] + 4)
        out = np.zeros(n)
        self.L.fx_debug_table(self.h, d, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
        return out.reshape(ntab, self.pb.n[d] + 4)

    # -- state
    def init_equilibrium(self, prim) -> None:
        import torch

        if isinstance(prim, torch.Tensor):
            assert prim.dtype == torch.float64 and prim.is_contiguous() and prim.is_cuda
            self._check(self.L.fx_state_init_equilibrium(self.h, ctypes.c_void_p(prim.data_ptr()), 1))
        else:
            p = np.ascontiguousarray(prim, dtype=np.float64)
            self._check(self.L.fx_state_init_equilibrium(self.h, p.ctypes.data_as(ctypes.c_void_p), 0))

    def upload(self, state) -> None:
        import torch

        if isinstance(state, torch.Tensor):
            assert state.is_contiguous() and state.is_cuda and state.numel() == self.nelem
            prec = FX_FP64 if state.dtype == torch.float64 else FX_FP32
            self._check(self.L.fx_state_upload(self.h, ctypes.c_void_p(state.data_ptr()), prec, 1))
        else:
            s = np.ascontiguousarray(state)
            assert s.size == self.nelem
            prec = FX_FP64 if s.dtype == np.float64 else FX_FP32
            self._check(self.L.fx_state_upload(self.h, s.ctypes.data_as(ctypes.c_void_p), prec, 0))

    def download(self, out=None, precision: Optional[int] = None) -> np.ndarray:
        import torch

        if isinstance(out, torch.Tensor):
            prec = FX_FP64 if out.dtype == torch.float64 else FX_FP32
            self._check(self.L.fx_state_download(self.h, ctypes.c_void_p(out.data_ptr()), prec, 1))
            return out
        prec = FX_FP64 if precision is None else precision
        arr = np.empty(self.nelem, dtype=np.float64 if prec == FX_FP64 else np.float32)
        self._check(self.L.fx_state_download(self.h, arr.ctypes.data_as(ctypes.c_void_p), prec, 0))
        return arr

    def step(self, dt: float, nsteps: int = 1) -> None:
        self._check(self.L.fx_step(self.h, float(dt), int(nsteps)))

    def sync(self) -> None:
        self._check(self.L.fx_sync(self.h))

    def status(self) -> int:
        return int(self.L.fx_sync(self.h))

    def totals(self) -> np.ndarray:
        out = np.zeros(NTOTALS)
        self._check(self.L.fx_conserved_totals(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def boundary_layers(self, layers, t0: float = 0.0) -> None:
        """Set the boundary layers (dictionaries: kind "front" or "mirror", box lo/hi, and the
        front's x0, y0, cot_alpha, speed and primitive states A, B, or the mirror's d, m)."""
        arr = (FxLayer * max(len(layers), 1))()
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
        self._check(self.L.fx_boundary_layers(self.h, arr, len(layers), float(t0)))

    def budgets_enable(self, on: bool = True) -> None:
        """Start (zeroing them) or stop accumulating the budgets of reading R13 in fx_step."""
        self._check(self.L.fx_budgets_enable(self.h, int(bool(on))))

    def budgets(self) -> np.ndarray:
        """Budget terms accumulated since the reset (synchronising): boundary outflows of mass,
        momentum 1..3, total energy and radiation energy; coupling work; floor energy; the
        radiation energy the velocity-dependent terms add."""
        out = np.zeros(NBUDGET)
        self._check(self.L.fx_budgets(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def launches_per_step(self) -> int:
        return int(self.L.fx_launches_per_step(self.h))

    def march_chunk(self) -> int:
        """Planes per block of the radiation/update kernel's march (fitted to the bound device)."""
        return int(self.L.fx_march_chunk(self.h))

    def kernel_timing(self, on: bool) -> None:
        """Start (or stop) recording per-kernel CUDA-event durations of the stages fx_step enqueues."""
        self._check(self.L.fx_kernel_timing_enable(self.h, int(bool(on))))

    def kernel_times(self) -> dict:
        """Synchronising read of the recorded durations: total ms and launch counts per kernel."""
        out = np.zeros(6)
        self._check(self.L.fx_kernel_timing_read(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return {"stage_ms": float(out[0]), "stage_launches": int(out[1]),
                "face_ms": float(out[2]), "face_launches": int(out[3]),
                "couple_ms": float(out[4]), "couple_launches": int(out[5])}

    # -- objective and adjoint
    def objective(self, on: bool = True) -> None:
        """Accumulate the boundary outflow J during subsequent steps (resets it to 0)."""
        self._check(self.L.fx_objective_enable(self.h, int(bool(on))))

    def boundary_energy_out(self) -> float:
        out = ctypes.c_double()
        self._check(self.L.fx_boundary_energy_out(self.h, ctypes.byref(out)))
        return out.value

    def set_kappa0(self, kappa0: float) -> None:
        self._check(self.L.fx_set_kappa0(self.h, float(kappa0)))
        self.pb.kappa0 = float(kappa0)

    def set_density(self, rho) -> None:
        """Replace the density at fixed pressure, velocity and radiation (torch CUDA tensor or
        host array of the state's precision)."""
        import torch

        prec = FX_FP64 if self.pb.precision == "fp64" else FX_FP32
        if isinstance(rho, torch.Tensor):
            assert rho.is_cuda and rho.is_contiguous() and rho.numel() == self.pb.ncell
            assert rho.dtype == (torch.float64 if prec == FX_FP64 else torch.float32)
            self._check(self.L.fx_state_set_density(self.h, ctypes.c_void_p(rho.data_ptr()), prec, 1))
        else:
            r = np.ascontiguousarray(rho, dtype=self.np_dtype)
            assert r.size == self.pb.ncell
            self._check(self.L.fx_state_set_density(self.h, r.ctypes.data_as(ctypes.c_void_p), prec, 0))

    def adjoint_workspace(self, nsteps: int, k: int):
        import torch

        nb = ctypes.c_size_t()
        self._check(self.L.fx_adjoint_workspace_bytes(self.h, int(nsteps), int(k), ctypes.byref(nb)))
        return torch.empty(max(nb.value, 1), dtype=torch.uint8, device=self.workspace.device)

    def adjoint_forward(self, ws, dt: float, nsteps: int, k: int) -> float:
        J = ctypes.c_double()
        self._check(self.L.fx_adjoint_forward(self.h, float(dt), int(nsteps), int(k),
                                              ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(J)))
        return J.value

    def adjoint_backward(self, ws, dt: float, nsteps: int, k: int, seed: float = 1.0):
        """Returns (dJ/dU^0 as a device tensor in the state layout, dJ/drho(x,0), dJ/dkappa0)."""
        import torch

        tdt = torch.float64 if self.pb.precision == "fp64" else torch.float32
        gs = torch.empty(self.nelem, dtype=tdt, device=self.workspace.device)
        gr = torch.empty(self.pb.ncell, dtype=tdt, device=self.workspace.device)
        dk = ctypes.c_double()
        self._check(self.L.fx_adjoint_backward(self.h, float(dt), int(nsteps), int(k),
                                               ctypes.c_void_p(ws.data_ptr()), ws.numel(), float(seed),
                                               ctypes.c_void_p(gs.data_ptr()), ctypes.c_void_p(gr.data_ptr()),
                                               ctypes.byref(dk)))
        return gs, gr, dk.value

    def adjoint(self, dt: float, nsteps: int, k: int):
        """Both passes: (J, dJ/dU^0, dJ/drho(x,0), dJ/dkappa0)."""
        import torch

        ws = self.adjoint_workspace(nsteps, k)
        tdt = torch.float64 if self.pb.precision == "fp64" else torch.float32
        gs = torch.empty(self.nelem, dtype=tdt, device=self.workspace.device)
        gr = torch.empty(self.pb.ncell, dtype=tdt, device=self.workspace.device)
        J, dk = ctypes.c_double(), ctypes.c_double()
        self._check(self.L.fx_adjoint(self.h, float(dt), int(nsteps), int(k), ctypes.c_void_p(ws.data_ptr()),
                                      ws.numel(), ctypes.c_void_p(gs.data_ptr()), ctypes.c_void_p(gr.data_ptr()),
                                      ctypes.byref(J), ctypes.byref(dk)))
        return J.value, gs, gr, dk.value

    def clear_error(self) -> None:
        self.L.fx_clear_error(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            self.L.fx_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
