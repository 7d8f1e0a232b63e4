"""Seeded synthetic workloads for the multigroup M1 radiation-hydrodynamics stage update.

This module only builds inputs: grid parameters and the primitive initial fields
(rho, p, physical velocity, radiation temperature).  It holds none of the method's arithmetic;
turning primitives into the conserved state (including the Planck group energies) is done by
the CUDA library and, independently, by the CPU oracle.

The five workloads follow the structure of the paper's radiation-hydrodynamics applications
(Sec. 3.2, Sec. 4: 8-20 logarithmically spaced groups, power-law absorption opacities, 2-d
spherical grids of a few hundred by ~128 zones).  The paper's own core-collapse progenitors,
nuclear equations of state and neutrino opacity tables are not available, so these seeded
fields stand in for them.

Units are dimensionless: k_B = mu = 1, T = p / rho, photon energies in units of k T0 = 1,
radiation constant a_R = 0.1, and the (reduced) speed of light c = 10 max(|v| + a_s) over the
initial state (the paper's example choice c = 10 (v0 + a0), Sec. 9.5).
"""
from __future__ import annotations

import copy
import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

BC_CODES = {"outflow": 0, "periodic": 1, "reflect": 2, "axis": 3}
GEOM_CODES = {"cart": 0, "sph": 1}
MAP_CODES = {"id": 0, "exp": 1, "sinh": 2}
RIEMANN_CODES = {"hllc": 0, "hlle": 1, "llf": 2}


@dataclasses.dataclass
class Problem:
    """Grid, physics and run parameters of one workload (shared by the library and the oracle)."""

    name: str
    dims: int
    n: Tuple[int, int, int]
    x_lo: Tuple[float, float, float]
    x_hi: Tuple[float, float, float]
    bc_lo: Tuple[str, str, str]
    bc_hi: Tuple[str, str, str]
    ngroups: int
    gamma: float
    kappa0: float
    kap_rho_exp: float
    kap_T_exp: float
    kap_eps_exp: float
    eps_min: float = 0.01
    eps_max: float = 10.0
    sigma0: float = 0.0
    a_rad: float = 0.1
    c_light: float = 0.0
    geom: str = "cart"
    map1: str = "id"
    map_rt: float = 1.0  # r_t of the sinh map r = r_t sinh(x1 / r_t)
    rad_recon_order: int = 1
    riemann: str = "hllc"      # gas Riemann solver: "hllc", "hlle" or "llf" (Sec. 5.2)
    shock_guard: float = 0.0   # carbuncle guard pressure-jump threshold (0: off)
    vterms: int = 0            # 1: velocity-dependent radiation terms (Sec. 3.2, 5.2; Cartesian)
    species: int = 1           # 1 (photons) or 3 (neutrino species; composition rho Y_e)
    xi0: float = 0.0           # lepton number per unit energy (three species)
    couple: int = 1
    newton_maxit: int = 50
    bisect_maxit: int = 200
    newton_rtol: float = 1e-13
    rho_floor: float = 1e-12
    p_floor: float = 1e-12
    E_floor: float = 1e-300
    cfl: float = 0.5
    dt: float = 0.0
    nsteps: int = 1
    precision: str = "fp64"

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n[: self.dims]))

    @property
    def nchan(self) -> int:
        """Radiation channels: species x groups (species-major)."""
        return self.species * self.ngroups

    @property
    def ncomp(self) -> int:
        """Composition variables after the radiation block (rho Y_e with three species)."""
        return 1 if self.species > 1 else 0

    @property
    def nvar(self) -> int:
        return 2 + self.dims + self.nchan * (1 + self.dims) + self.ncomp

    @property
    def shape(self) -> Tuple[int, ...]:
        """numpy shape of one cell field, slowest axis first (z, y, x)."""
        return tuple(reversed(self.n[: self.dims]))

    def state_size(self) -> int:
        return self.ncell * self.nvar

    def cell_centres(self, d: int) -> np.ndarray:
        lo, hi, n = self.x_lo[d], self.x_hi[d], self.n[d]
        return lo + (np.arange(n) + 0.5) * (hi - lo) / n

    def cell_lower_faces(self, d: int) -> np.ndarray:
        lo, hi, n = self.x_lo[d], self.x_hi[d], self.n[d]
        return lo + np.arange(n) * (hi - lo) / n

    def zone_groups(self) -> int:
        return self.ncell * self.ngroups


def _finish(pb: Problem, prim: np.ndarray) -> Tuple[Problem, np.ndarray]:
    """Set c from the initial state (c = 10 max(|v| + a_s)) and dt from the light-crossing limit."""
    D = pb.dims
    rho, p = prim[0], prim[1]
    vmag = np.sqrt(sum(prim[2 + q] ** 2 for q in range(D)))
    a_s = np.sqrt(pb.gamma * p / rho)
    if pb.c_light <= 0.0:
        pb.c_light = float(10.0 * np.max(vmag + a_s))
    pb.dt = float(pb.cfl / _max_inverse_crossing(pb, prim))
    return pb, prim


def _max_inverse_crossing(pb: Problem, prim: np.ndarray) -> float:
    """max over cells of sum_d lambda_d / (h_d dx^d), lambda_d = max(|v_d| + a_s, c)."""
    D = pb.dims
    rho, p = prim[0], prim[1]
    a_s = np.sqrt(pb.gamma * p / rho)
    tot = np.zeros(pb.shape)
    for d in range(D):
        dx = (pb.x_hi[d] - pb.x_lo[d]) / pb.n[d]
        lam = np.maximum(np.abs(prim[2 + d]).reshape(pb.shape) + a_s.reshape(pb.shape), pb.c_light)
        if pb.geom == "sph":
            xl = pb.cell_lower_faces(0)
            if pb.map1 == "exp":
                r, dr = np.exp(xl), np.exp(xl)
            elif pb.map1 == "sinh":
                r, dr = pb.map_rt * np.sinh(xl / pb.map_rt), np.cosh(xl / pb.map_rt)
            else:
                r, dr = np.maximum(xl, 1e-300), np.ones_like(xl)
            h = dr if d == 0 else r  # h_1 = dr/dx1, h_2 = r (identity theta map)
            hb = np.broadcast_to(h[np.newaxis, :], pb.shape) if D > 1 else h
            tot = tot + lam / (hb * dx)
        else:
            tot = tot + lam / dx
    return float(np.max(tot))


def _flat(*fields: np.ndarray) -> np.ndarray:
    return np.stack([np.ascontiguousarray(f, dtype=np.float64).reshape(-1) for f in fields])


# ---------------------------------------------------------------------------------------------
# The five workloads.  Each returns (Problem, prim) with prim of shape (3 + D, ncell):
# rows rho, p, vhat_1..vhat_D, T_rad; cells in x-fastest order.
# ---------------------------------------------------------------------------------------------
def sod_1d(n: int = 512, ngroups: int = 12, nsteps: int = 200, gamma: float = 5.0 / 3.0,
           precision: str = "fp64") -> Tuple[Problem, np.ndarray]:
    """Sod-like 1-d shock tube with multigroup radiation in local equilibrium (Sec. 8.3 states)."""
    pb = Problem(name=f"sod1d_{n}x{ngroups}g", dims=1, n=(n, 1, 1), x_lo=(0.0, 0.0, 0.0),
                 x_hi=(1.0, 1.0, 1.0), bc_lo=("outflow",) * 3, bc_hi=("outflow",) * 3,
                 ngroups=ngroups, gamma=gamma, kappa0=1.0, kap_rho_exp=1.0, kap_T_exp=-1.5,
                 kap_eps_exp=-2.0, nsteps=nsteps, precision=precision)
    x = pb.cell_centres(0)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    v = np.zeros(n)
    return _finish(pb, _flat(rho, p, v, p / rho))


def kh_2d(nx: int = 1024, ny: int = 1024, ngroups: int = 16, nsteps: int = 100, seed: int = 1,
          precision: str = "fp64") -> Tuple[Problem, np.ndarray]:
    """Periodic Kelvin-Helmholtz shear layer (a variant of Sec. 8.6) with equilibrium radiation."""
    pb = Problem(name=f"kh2d_{nx}x{ny}x{ngroups}g", dims=2, n=(nx, ny, 1), x_lo=(0.0, 0.0, 0.0),
                 x_hi=(1.0, 1.0, 1.0), bc_lo=("periodic",) * 3, bc_hi=("periodic",) * 3,
                 ngroups=ngroups, gamma=1.4, kappa0=10.0, kap_rho_exp=1.0, kap_T_exp=-1.5,
                 kap_eps_exp=-2.0, nsteps=nsteps, precision=precision)
    rng = np.random.default_rng(seed)
    y = pb.cell_centres(1)[:, None] * np.ones((1, nx))
    band = (y >= 0.25) & (y < 0.75)
    rho = np.where(band, 2.0, 1.0)
    vx = np.where(band, 0.5, -0.5)
    vy = 0.01 * rng.uniform(-1.0, 1.0, size=(ny, nx))
    p = np.full((ny, nx), 2.5)
    return _finish(pb, _flat(rho, p, vx, vy, p / rho))


def gaussian_random_field(shape: Tuple[int, ...], slope: float, seed: int) -> np.ndarray:
    """Periodic Gaussian random field with power spectrum P(k) ~ k^slope, zero mean, unit std."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    kk = np.meshgrid(*[np.fft.fftfreq(m) * m for m in shape], indexing="ij")
    k = np.sqrt(sum(q ** 2 for q in kk))
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (slope / 2.0)
    field = np.real(np.fft.ifftn(np.fft.fftn(white) * amp))
    field -= field.mean()
    return field / field.std()


def lognormal_3d(n: int = 256, ngroups: int = 12, nsteps: int = 20, seed: int = 2,
                 shape: Optional[Tuple[int, int, int]] = None,
                 precision: str = "fp32") -> Tuple[Problem, np.ndarray]:
    """Periodic 3-d lognormal density (k^-11/3 spectrum), uniform p, radiation at twice T."""
    nx, ny, nz = shape if shape is not None else (n, n, n)
    pb = Problem(name=f"lognormal3d_{nx}x{ny}x{nz}x{ngroups}g", dims=3, n=(nx, ny, nz),
                 x_lo=(0.0, 0.0, 0.0), x_hi=(1.0, 1.0, 1.0), bc_lo=("periodic",) * 3,
                 bc_hi=("periodic",) * 3, ngroups=ngroups, gamma=5.0 / 3.0, kappa0=1.0,
                 kap_rho_exp=1.0, kap_T_exp=-3.5, kap_eps_exp=-3.0, nsteps=nsteps,
                 precision=precision)
    delta = gaussian_random_field((nz, ny, nx), -11.0 / 3.0, seed)
    rho = np.exp(delta - 0.5)
    p = np.ones_like(rho)
    z = np.zeros_like(rho)
    return _finish(pb, _flat(rho, p, z, z, z, 2.0 * p / rho))


def blobs_2d(n: int = 512, ngroups: int = 8, nsteps: int = 50, seed: int = 3, nblobs: int = 16,
             shape: Optional[Tuple[int, int]] = None,
             precision: str = "fp32") -> Tuple[Problem, np.ndarray]:
    """Gaussian density blobs (peak 10, width 0.03) in a uniform medium; kappa ~ rho^3 gives a
    1e3 thin/thick contrast.  The blob centres lie in the strip 0.9 <= x <= 1 next to the outflow
    boundary whose energy outflow is the objective: in 50 steps at CFL 0.5 light crosses ~13 of
    the 512 cells, so only that strip can change the outflow.  Pair with `streaming_flux`."""
    nx, ny = shape if shape is not None else (n, n)
    pb = Problem(name=f"blobs2d_{nx}x{ny}x{ngroups}g", dims=2, n=(nx, ny, 1), x_lo=(0.0, 0.0, 0.0),
                 x_hi=(1.0, 1.0, 1.0), bc_lo=("outflow", "periodic", "periodic"),
                 bc_hi=("outflow", "periodic", "periodic"), ngroups=ngroups, gamma=5.0 / 3.0,
                 kappa0=1.0, kap_rho_exp=3.0, kap_T_exp=-1.5, kap_eps_exp=-2.0, nsteps=nsteps,
                 precision=precision)
    rng = np.random.default_rng(seed)
    centres = np.stack([rng.uniform(0.9, 1.0, nblobs), rng.uniform(0.0, 1.0, nblobs)], axis=1)
    x = pb.cell_centres(0)[None, :]
    y = pb.cell_centres(1)[:, None]
    rho = np.ones((ny, nx))
    for cx, cy in centres:
        rho = rho + 9.0 * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * 0.03 ** 2))
    p = np.ones_like(rho)
    z = np.zeros_like(rho)
    return _finish(pb, _flat(rho, p, z, z, p / rho))


def spherical_2d(nr: int = 640, nth: int = 128, ngroups: int = 20, nsteps: int = 200,
                 seed: int = 4, precision: str = "fp32", map1: str = "exp",
                 map_rt: float = 10.0) -> Tuple[Problem, np.ndarray]:
    """2-d spherical (r, theta) atmosphere over r in [1, 1000], rho ~ r^-2, p ~ r^-2.5: a log-r grid,
    or (map1 = "sinh") r = r_t sinh(x1 / r_t), nearly uniform inside r_t and logarithmic outside."""
    if map1 == "sinh":
        x0, x1 = map_rt * math.asinh(1.0 / map_rt), map_rt * math.asinh(1000.0 / map_rt)
    else:
        x0, x1 = 0.0, math.log(1000.0)
    pb = Problem(name=f"sph2d_{nr}x{nth}x{ngroups}g", dims=2, n=(nr, nth, 1),
                 x_lo=(x0, 0.0, 0.0), x_hi=(x1, math.pi, 1.0),
                 bc_lo=("reflect", "axis", "periodic"), bc_hi=("outflow", "axis", "periodic"),
                 ngroups=ngroups, gamma=5.0 / 3.0, kappa0=1e3, kap_rho_exp=2.0, kap_T_exp=-1.5,
                 kap_eps_exp=-2.0, geom="sph", map1=map1, map_rt=map_rt, nsteps=nsteps,
                 precision=precision)
    rng = np.random.default_rng(seed)
    xi = rng.uniform(-1.0, 1.0, size=nth)
    xc = pb.cell_centres(0)
    r = (map_rt * np.sinh(xc / map_rt) if map1 == "sinh" else np.exp(xc))[None, :]
    rho = r ** -2.0 * (1.0 + 1e-3 * xi[:, None])
    p = r ** -2.5 * np.ones((nth, 1))
    z = np.zeros_like(rho)
    return _finish(pb, _flat(rho, p, z, z, p / rho))


def double_mach(nx: int = 520, ny: int = 160, t_end: float = 0.2, ngroups: int = 1,
                shock_guard: float = 0.5, precision: str = "fp64"):
    """Double Mach reflection (Sec. 8.4; Woodward & Colella 1984): a Mach-10 oblique shock at
    alpha = 60 degrees to a reflecting wall, on [0, 3.25 nx/520] x [0, 1] with nx x ny cells
    (gamma = 1.4; pre-shock (rho, p, v) = (1.4, 1, 0, 0), post-shock (8, 116.5, 8.25 sin alpha,
    -8.25 cos alpha)).  The grid carries two extra cell layers on the left, bottom and top sides
    that the boundary layers overwrite before each stage: the post-shock state on the left and on
    the bottom for x <= x0 = 1/6, the mirror image of the interior (reflecting wall) on the bottom
    for x > x0, and on the top the post-shock state behind the shock's exact position
    x0 + y cot(alpha) + 10 t / sin(alpha), the pre-shock state ahead of it; outflow on the right.
    One group of inert radiation (kappa = 0, no interaction) at T_rad = 0.01.

    Returns (problem, prim, layers): the layers as plain dictionaries (kind "front" or "mirror",
    box lo/hi in cell indices, and the front or mirror parameters)."""
    dx = 1.0 / ny
    alpha = math.pi / 3.0
    pre = (1.4, 1.0, 0.0, 0.0)
    post = (8.0, 116.5, 8.25 * math.sin(alpha), -8.25 * math.cos(alpha))
    tr = 0.01
    n = (nx + 2, ny + 4, 1)
    pb = Problem(name=f"dmr_{nx}x{ny}", dims=2, n=n, x_lo=(-2 * dx, -2 * dx, 0.0),
                 x_hi=(nx * dx, 1.0 + 2 * dx, 1.0), bc_lo=("outflow",) * 3, bc_hi=("outflow",) * 3,
                 ngroups=ngroups, gamma=1.4, kappa0=0.0, kap_rho_exp=0.0, kap_T_exp=0.0,
                 kap_eps_exp=0.0, c_light=20.0, couple=0, riemann="hllc", shock_guard=shock_guard,
                 precision=precision)
    x0, cot, speed = 1.0 / 6.0, 1.0 / math.tan(alpha), 10.0 / math.sin(alpha)
    x = pb.cell_centres(0)[None, :] * np.ones((n[1], 1))
    y = pb.cell_centres(1)[:, None] * np.ones((1, n[0]))
    behind = x - x0 - y * cot <= 0.0
    fields = [np.where(behind, post[q], pre[q]) for q in range(4)]
    prim = _flat(*fields, np.full(x.shape, tr))
    pb.dt = float(pb.cfl / _max_inverse_crossing(pb, prim))
    pb.nsteps = int(math.ceil(t_end / pb.dt))
    ifront = int(np.searchsorted(pb.cell_centres(0), x0, side="right"))  # first cell with x > x0
    A, B = post + (tr,), pre + (tr,)
    fixed = dict(kind="front", x0=1e30, y0=0.0, cot_alpha=0.0, speed=0.0, A=A, B=A)
    layers = [
        dict(fixed, lo=(0, 0, 0), hi=(2, n[1], 1)),                        # left: post-shock
        dict(fixed, lo=(2, 0, 0), hi=(ifront, 2, 1)),                      # bottom, x <= x0
        dict(kind="mirror", d=1, m=2, lo=(ifront, 0, 0), hi=(n[0], 2, 1)),  # bottom wall
        dict(kind="front", lo=(2, n[1] - 2, 0), hi=(n[0], n[1], 1), x0=x0, y0=0.0,
             cot_alpha=cot, speed=speed, A=A, B=B),                        # top: moving shock
    ]
    return pb, prim, layers


def neutrino_2d(nx: int = 512, ny: int = 512, ngroups: int = 8, nsteps: int = 50, seed: int = 5,
                precision: str = "fp64"):
    """Three neutrino species in a periodic 2-d box for the two-equation (T, Y_e) interaction:
    groups over eps in [0.01, 10] kT0, rho = exp(0.5 delta), a seeded Gaussian random field
    delta (k^-3), p = 1, Y_e = 0.3 + 0.1 sin(2 pi x) sin(2 pi y), shear flow v_x = 0.3 sin(2 pi y),
    radiation at 1.5 T in the Y_e-weighted equilibrium, kappa = 3 rho T^-1.5 eps^-2, xi0 = 0.05.
    prim rows: rho, p, v_x, v_y, T_rad, Y_e."""
    pb = Problem(name=f"nu2d_{nx}x{ny}x{ngroups}g", dims=2, n=(nx, ny, 1), x_lo=(0.0, 0.0, 0.0),
                 x_hi=(1.0, 1.0, 1.0), bc_lo=("periodic",) * 3, bc_hi=("periodic",) * 3,
                 ngroups=ngroups, gamma=4.0 / 3.0, kappa0=3.0, kap_rho_exp=1.0, kap_T_exp=-1.5,
                 kap_eps_exp=-2.0, nsteps=nsteps, species=3, xi0=0.05, precision=precision)
    delta = gaussian_random_field((ny, nx), -3.0, seed)
    rho = np.exp(0.5 * delta)
    x = pb.cell_centres(0)[None, :] * np.ones((ny, 1))
    y = pb.cell_centres(1)[:, None] * np.ones((1, nx))
    p = np.ones((ny, nx))
    vx = 0.3 * np.sin(2 * np.pi * y)
    vy = np.zeros((ny, nx))
    ye = 0.3 + 0.1 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    pb, prim = _finish(pb, _flat(rho, p, vx, vy, 1.5 * p / rho))
    return pb, np.concatenate([prim, _flat(ye)])


def neutrino_sph2d(nr: int = 320, nth: int = 64, ngroups: int = 8, nsteps: int = 50, seed: int = 6,
                   precision: str = "fp64"):
    """Three neutrino species on the 2-d spherical (r, theta) grid: the log-r atmosphere of
    spherical_2d (r in [1, 1000], rho ~ r^-2, p ~ r^-2.5, reflecting centre, outflow outer
    boundary, polar axes) with a slow radial outflow v_r = 0.02 c_s (r / 1000) (1 + 0.1 cos theta),
    Y_e falling from 0.45 at the centre to 0.2 outside, radiation at 1.2 T in the Y_e-weighted
    equilibrium, xi0 = 0.02.  prim rows: rho, p, v_r, v_theta, T_rad, Y_e."""
    x0, x1 = 0.0, math.log(1000.0)
    pb = Problem(name=f"nusph2d_{nr}x{nth}x{ngroups}g", dims=2, n=(nr, nth, 1),
                 x_lo=(x0, 0.0, 0.0), x_hi=(x1, math.pi, 1.0),
                 bc_lo=("reflect", "axis", "periodic"), bc_hi=("outflow", "axis", "periodic"),
                 ngroups=ngroups, gamma=4.0 / 3.0, kappa0=1e2, kap_rho_exp=2.0, kap_T_exp=-1.5,
                 kap_eps_exp=-2.0, geom="sph", map1="exp", nsteps=nsteps, species=3, xi0=0.02,
                 precision=precision)
    rng = np.random.default_rng(seed)
    xi = rng.uniform(-1.0, 1.0, size=nth)
    r = np.exp(pb.cell_centres(0))[None, :]
    th = pb.cell_centres(1)[:, None]
    rho = r ** -2.0 * (1.0 + 1e-3 * xi[:, None])
    p = r ** -2.5 * np.ones((nth, 1))
    cs = np.sqrt(pb.gamma * p / rho)
    vr = 0.02 * cs * (r / 1000.0) * (1.0 + 0.1 * np.cos(th))
    vt = np.zeros_like(rho)
    ye = 0.2 + 0.25 * np.exp(-np.log(r) / 2.0) * np.ones((nth, 1))
    pb, prim = _finish(pb, _flat(rho, p, vr, vt, 1.2 * p / rho))
    return pb, np.concatenate([prim, _flat(ye)])


WORKLOADS = {
    "sod1d": sod_1d,
    "kh2d": kh_2d,
    "lognormal3d": lognormal_3d,
    "blobs2d": blobs_2d,
    "sph2d": spherical_2d,
    "nu2d": neutrino_2d,
}


def streaming_flux(pb: Problem, state: np.ndarray, frac: float = 0.5, axis: int = 0) -> np.ndarray:
    """Copy of a conserved state (external layout) whose radiation flux is replaced by a beam
    along `axis`: F_g = frac * c * E_g (Cartesian components), every other component zero."""
    D, G, N = pb.dims, pb.ngroups, pb.ncell
    NG = 2 + D
    out = np.array(state, dtype=np.float64, copy=True)
    rad = out[NG * N:].reshape(1 + D, N, G)
    for q in range(D):
        rad[1 + q] = frac * pb.c_light * rad[0] if q == axis else 0.0
    return out


def random_state(pb: Problem, seed: int, flux_frac: float = 0.5) -> np.ndarray:
    """A generic random conserved state (external layout) for unit-level parity tests.

    rho in [0.5, 2], physical velocity in [-0.3, 0.3], internal energy in [0.5, 2], E_g in
    [0.05, 1] and |F| up to flux_frac * c * E.  Covariant momentum/flux for Cartesian grids only.
    """
    rng = np.random.default_rng(seed)
    D, G, N = pb.dims, pb.ngroups, pb.ncell
    rho = rng.uniform(0.5, 2.0, N)
    v = rng.uniform(-0.3, 0.3, (D, N))
    u = rng.uniform(0.5, 2.0, N)
    out = [rho]
    for q in range(D):
        out.append(rho * v[q])
    out.append(u + 0.5 * rho * (v ** 2).sum(0))
    gas = np.stack(out).reshape(-1)
    E = rng.uniform(0.05, 1.0, (N, G))
    dirs = rng.standard_normal((D, N, G))
    dirs /= np.maximum(np.sqrt((dirs ** 2).sum(0)), 1e-12)
    mag = rng.uniform(0.0, flux_frac, (N, G)) * pb.c_light * E
    rad = [E.reshape(-1)] + [(dirs[q] * mag).reshape(-1) for q in range(D)]
    return np.concatenate([gas, np.concatenate(rad)])


# ---------------------------------------------------------------------------------------------
# Windows of a large grid: sub-problems that the oracle can run in seconds, for the sampled
# parity checks of full-size grids and the CPU baseline.  Input slicing only.
# ---------------------------------------------------------------------------------------------
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
