"""Shared test helpers: field-wise error norms and oracle windows of large grids."""
from __future__ import annotations

import copy

import numpy as np

from paper_1806_07390_gb300.workloads import Problem


def fields(pb: Problem, state: np.ndarray):
    """Yield (name, array) per conserved field of an external-layout state."""
    N, G, D = pb.ncell, pb.ngroups, pb.dims
    NG = 2 + D
    names = ["rho"] + [f"m{q}" for q in range(D)] + ["rhoe"]
    for v in range(NG):
        yield names[v], state[v * N:(v + 1) * N]
    rad = state[NG * N:].reshape(1 + D, N, G)
    yield "E", rad[0].reshape(-1)
    for q in range(D):
        yield f"F{q}", rad[1 + q].reshape(-1)


def natural_scales(pb: Problem, ref: np.ndarray):
    """Per field, the magnitude each field is naturally measured against: rho, rho e and E
    themselves; momentum against sqrt(rho * rho e); radiation flux against c E."""
    f = dict(fields(pb, ref))
    mom = np.sqrt(np.abs(f["rho"] * f["rhoe"]))
    sc = {"rho": f["rho"], "rhoe": f["rhoe"], "E": f["E"]}
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
    errs = field_errors(pb, got, ref, natural=natural)
    bad = {k: v for k, v in errs.items() if k not in skip and (v[0] > l1_tol or (max_tol is not None and v[1] > max_tol))}
    assert not bad, f"parity failed (l1 tol {l1_tol}, max tol {max_tol}): {bad}; all: {errs}"
    return errs


def window(pb: Problem, prim: np.ndarray, start, size, halo):
    """Sub-problem of `size` cells per active direction starting at `start` (interior index), with
    `halo` extra cells on each side taken with the grid's own boundary rules, outflow boundaries
    at the window edge.  Cells farther than the dependency radius from the edge are exact."""
    D = pb.dims
    sub = copy.deepcopy(pb)
    idx = []
    n_sub = []
    for d in range(D):
        n = pb.n[d]
        m = size[d] + 2 * halo
        raw = np.arange(start[d] - halo, start[d] - halo + m)
        if pb.bc_lo[d] == "periodic":
            ii = raw % n
        else:
            ii = np.clip(raw, 0, n - 1)
        idx.append(ii)
        n_sub.append(m)
    dx = [(pb.x_hi[d] - pb.x_lo[d]) / pb.n[d] for d in range(D)]
    sub.n = tuple(n_sub) + (1,) * (3 - D)
    sub.x_lo = (0.0, 0.0, 0.0)
    sub.x_hi = tuple(n_sub[d] * dx[d] for d in range(D)) + (1.0,) * (3 - D)
    sub.bc_lo = ("outflow",) * 3
    sub.bc_hi = ("outflow",) * 3
    shape = pb.shape
    grids = np.ix_(*reversed(idx))  # numpy axes are (z, y, x)
    sub_prim = np.stack([p.reshape(shape)[grids].reshape(-1) for p in prim])
    return sub, sub_prim


def window_cells(pb: Problem, start, size):
    """Flat cell indices (x fastest) of the window interior in the full grid."""
    D = pb.dims
    axes = [np.arange(start[d], start[d] + size[d]) % pb.n[d] for d in range(D)]
    if D == 1:
        return axes[0]
    if D == 2:
        y, x = np.meshgrid(axes[1], axes[0], indexing="ij")
        return (y * pb.n[0] + x).reshape(-1)
    z, y, x = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return ((z * pb.n[1] + y) * pb.n[0] + x).reshape(-1)


def sub_cells(sub: Problem, size, halo):
    """Flat indices of the window interior inside the sub-problem."""
    D = sub.dims
    axes = [np.arange(halo, halo + size[d]) for d in range(D)]
    if D == 1:
        return axes[0]
    if D == 2:
        y, x = np.meshgrid(axes[1], axes[0], indexing="ij")
        return (y * sub.n[0] + x).reshape(-1)
    z, y, x = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return ((z * sub.n[1] + y) * sub.n[0] + x).reshape(-1)


def gather_cells(pb: Problem, state: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """External-layout state restricted to the given cells (same layout, ncell = len(cells))."""
    N, G, D = pb.ncell, pb.ngroups, pb.dims
    NG = 2 + D
    gas = state[: NG * N].reshape(NG, N)[:, cells]
    rad = state[NG * N:].reshape(1 + D, N, G)[:, cells, :]
    return np.concatenate([gas.reshape(-1), rad.reshape(-1)])


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
