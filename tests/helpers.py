"""Shared test helpers: field-wise error norms and gathers of window cells."""
from __future__ import annotations

import numpy as np

from paper_1806_07390_gb300.workloads import Problem, sub_cells, window, window_cells  # noqa: F401


def fields(pb: Problem, state: np.ndarray):
    """Yield (name, array) per conserved field of an external-layout state."""
    N, G, D = pb.ncell, pb.nchan, pb.dims
    NG = 2 + D
    names = ["rho"] + [f"m{q}" for q in range(D)] + ["rhoe"]
    for v in range(NG):
        yield names[v], state[v * N:(v + 1) * N]
    rad = state[NG * N:(NG + (1 + D) * G) * N].reshape(1 + D, N, G)
    yield "E", rad[0].reshape(-1)
    for q in range(D):
        yield f"F{q}", rad[1 + q].reshape(-1)
    if pb.ncomp:
        yield "rhoYe", state[(NG + (1 + D) * G) * N:]


def natural_scales(pb: Problem, ref: np.ndarray):
    """Per field, the magnitude each field is naturally measured against: rho, rho e and E
    themselves; momentum against sqrt(rho * rho e); radiation flux against c E."""
    f = dict(fields(pb, ref))
    mom = np.sqrt(np.abs(f["rho"] * f["rhoe"]))
    sc = {"rho": f["rho"], "rhoe": f["rhoe"], "E": f["E"]}
    if "rhoYe" in f:
        sc["rhoYe"] = f["rhoYe"]
    for q in range(pb.dims):
        sc[f"m{q}"] = mom
        sc[f"F{q}"] = pb.c_light * f["E"]
    return sc


def field_errors(pb: Problem, got: np.ndarray, ref: np.ndarray, natural: bool = False):
    """Per field: (L1 error, max-norm error), relative to the field itself, or with
    natural=True relative to the field's natural scale (see natural_scales)."""
    out = {}
    sc = natural_scales(pb, ref) if natural else None
    for (name, a), (_, b) in zip(fields(pb, np.asarray(got, dtype=np.float64)), fields(pb, ref)):
        s = sc[name] if natural else b
        den1 = np.sum(np.abs(s))
        denm = np.max(np.abs(s)) if s.size else 0.0
        l1 = np.sum(np.abs(a - b)) / den1 if den1 > 0 else np.max(np.abs(a - b))
        mx = np.max(np.abs(a - b)) / denm if denm > 0 else np.max(np.abs(a - b))
        out[name] = (float(l1), float(mx))
    return out


def assert_parity(pb, got, ref, l1_tol, max_tol=None, skip=(), natural=False):
    """Per-field L1 (and optionally max-norm) gate.  natural=True measures each field against its
    natural scale (see natural_scales), except momentum wherever it is O(1) next to that scale
    (max |m| >= 0.1 max sqrt(rho rho e)): there it is gated relative to itself.  The assertion
    message reports both the natural-scale and the self-relative errors of every field."""
    own = field_errors(pb, got, ref, natural=False)
    errs = dict(own)
    if natural:
        errs = field_errors(pb, got, ref, natural=True)
        f = dict(fields(pb, ref))
        sc = natural_scales(pb, ref)
        for q in range(pb.dims):
            k = f"m{q}"
            if f[k].size and np.max(np.abs(f[k])) >= 0.1 * np.max(sc[k]):
                errs[k] = own[k]
    bad = {k: v for k, v in errs.items() if k not in skip and (v[0] > l1_tol or (max_tol is not None and v[1] > max_tol))}
    nat = field_errors(pb, got, ref, natural=True) if natural else None
    assert not bad, (f"parity failed (l1 tol {l1_tol}, max tol {max_tol}): {bad}; gated: {errs}; "
                     f"self-relative: {own}; natural-scale: {nat}")
    return errs


def gather_cells(pb: Problem, state: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """External-layout state restricted to the given cells (same layout, ncell = len(cells))."""
    N, G, D = pb.ncell, pb.nchan, pb.dims
    NG = 2 + D
    gas = state[: NG * N].reshape(NG, N)[:, cells]
    rad = state[NG * N:(NG + (1 + D) * G) * N].reshape(1 + D, N, G)[:, cells, :]
    comp = state[(NG + (1 + D) * G) * N:].reshape(pb.ncomp, N)[:, cells]
    return np.concatenate([gas.reshape(-1), rad.reshape(-1), comp.reshape(-1)])


def rho_tangent(pb: Problem, state: np.ndarray, drho: np.ndarray) -> np.ndarray:
    """State tangent of a density perturbation drho (per cell) that holds the pressure, the
    velocity and the radiation variables fixed (Cartesian): d rho = drho, d m = v drho,
    d(rho e) = |v|^2/2 drho, zero elsewhere."""
    D, N = pb.dims, pb.ncell
    rho = state[:N]
    out = np.zeros_like(state)
    out[:N] = drho
    ke = np.zeros(N)
    for q in range(D):
        v = state[(1 + q) * N:(2 + q) * N] / rho
        out[(1 + q) * N:(2 + q) * N] = v * drho
        ke += 0.5 * v * v
    out[(1 + D) * N:(2 + D) * N] = ke * drho
    return out


def with_rho(pb: Problem, state: np.ndarray, rho_new: np.ndarray) -> np.ndarray:
    """The state with density rho_new and the same pressure, velocity and radiation (Cartesian)."""
    D, N = pb.dims, pb.ncell
    out = np.array(state, copy=True)
    rho = state[:N]
    ke_old = np.zeros(N)
    ke_new = np.zeros(N)
    for q in range(D):
        v = state[(1 + q) * N:(2 + q) * N] / rho
        out[(1 + q) * N:(2 + q) * N] = rho_new * v
        ke_old += 0.5 * rho * v * v
        ke_new += 0.5 * rho_new * v * v
    out[:N] = rho_new
    out[(1 + D) * N:(2 + D) * N] = state[(1 + D) * N:(2 + D) * N] - ke_old + ke_new
    return out
