"""GPU parity of the velocity-dependent radiation terms (Sec. 3.2, the group form of the moment
equations; Sec. 5.2; Step 2 of Sec. 6) with the FP64 oracle, through the C ABI.

Bars as for the rest of the path: FP64 relative L1 <= 1e-10 and max-norm <= 1e-8 per field; the
FP32 forms at 1e-4 against each field's natural scale.  The inputs have strong velocity
gradients: a shear layer (kh2d) and random states whose velocities change sign from cell to
cell, on periodic, outflow and reflecting boundaries, in 1, 2 and 3 dimensions, with odd group
counts and the largest group count (32); on the spherical (r, theta) grid (log-r and sinh radial
maps, reflecting inner boundary, both polar axes) with random velocities and fluxes.
"""
import numpy as np
import pytest

import oracle
from paper_1806_07390_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

FP64_L1, FP64_MAX = 1e-10, 1e-8


@pytest.fixture(scope="module")
def fxmod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07390_gb300 import build, fx
    build.build()
    return fx


def case(name, precision):
    """(problem, initial state) with vterms on."""
    if name == "kh":
        pb, prim = W.kh_2d(nx=44, ny=38, ngroups=16, nsteps=3, precision=precision)
        pb.vterms = 1
        return pb, oracle.init_equilibrium(pb, prim)
    if name == "kh_g32":
        pb, prim = W.kh_2d(nx=26, ny=22, ngroups=32, nsteps=2, precision=precision)
        pb.vterms = 1
        return pb, oracle.init_equilibrium(pb, prim)
    if name in ("rand1d", "rand1d_g12"):
        pb, _ = W.sod_1d(n=70, ngroups=7 if name == "rand1d" else 12, precision=precision)
        pb.bc_lo = ("reflect", "outflow", "outflow")
        pb.c_light, pb.nsteps = 6.0, 4
    elif name == "rand2d":
        pb, _ = W.blobs_2d(shape=(37, 29), ngroups=13, nsteps=3, precision=precision)
        pb.bc_lo = ("reflect", "periodic", "periodic")
        pb.bc_hi = ("outflow", "periodic", "periodic")
        pb.c_light = 5.0
    else:
        pb, _ = W.lognormal_3d(shape=(11, 9, 8), ngroups=5 if name == "rand3d" else 11, nsteps=2,
                               precision=precision)
        pb.bc_lo = ("outflow", "reflect", "periodic")
        pb.bc_hi = ("reflect", "outflow", "periodic")
        pb.c_light = 5.0
    pb.dt = 0.3 / max(pb.n[: pb.dims]) / pb.c_light
    pb.vterms = 1
    return pb, W.random_state(pb, seed=23, flux_frac=0.6)


def run_both(fxmod, pb, s):
    g = fxmod.Grid(pb)
    g.upload(s)
    g.step(pb.dt, pb.nsteps)
    st = g.status()
    got = g.download()
    g.close()
    ref, rst = oracle.run(pb, s, pb.dt, pb.nsteps, nthreads=8)
    assert st == 0 and rst == 0
    return got, ref


@pytest.mark.parametrize("name", ["kh", "kh_g32", "rand1d", "rand2d", "rand3d", "rand3d_g11"])
def test_velocity_terms_fp64(fxmod, name):
    pb, s = case(name, "fp64")
    got, ref = run_both(fxmod, pb, s)
    H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)
    # the terms change the result by far more than the bar
    pb.vterms = 0
    plain, _ = oracle.run(pb, s, pb.dt, pb.nsteps, nthreads=8)
    rad = slice((2 + pb.dims) * pb.ncell, None)
    assert np.abs(plain[rad] - ref[rad]).max() > 1e3 * FP64_MAX * np.abs(ref[rad]).max()


@pytest.mark.parametrize("form", ["fp32", "fp32n64"])
@pytest.mark.parametrize("name", ["kh", "kh_g32", "rand1d", "rand1d_g12", "rand2d", "rand3d", "rand3d_g11"])
def test_velocity_terms_fp32_forms(fxmod, name, form):
    # from 9 groups the FP32 forms take two groups per lane (8 lanes per cell for kh's 16,
    # rand2d's 13, rand1d_g12's 12 and rand3d_g11's 11 groups, 16 lanes for 32 groups); rand1d
    # (7) and rand3d (5) one group per lane
    pb, s = case(name, form)
    got, ref = run_both(fxmod, pb, s)
    H.assert_parity(pb, got, ref, 1e-4, natural=True)


def test_velocity_terms_budget(fxmod):
    # the radiation energy the terms add (budget entry 8) equals the oracle's, and the energy
    # budget closes with it
    pb, s = case("rand2d", "fp64")
    ref, rst, rbud = oracle.run_budget(pb, s, pb.dt, 3, nthreads=8)
    g = fxmod.Grid(pb)
    g.upload(s)
    t0 = g.totals()
    g.budgets_enable(True)
    g.step(pb.dt, 3)
    assert g.status() == 0 and rst == 0
    bud = g.budgets()
    t1 = g.totals()
    g.close()
    assert abs(bud[8]) > 1e-6 * abs(t0[4])
    assert np.all(np.abs(bud - rbud) <= 1e-12 * abs(t0[4])), (bud, rbud)
    assert abs(t0[4] - t1[4] - bud[4] - bud[6] + bud[7] + bud[8]) <= 1e-13 * abs(t0[4])


def test_velocity_terms_have_no_adjoint(fxmod):
    pb, s = case("rand2d", "fp64")
    g = fxmod.Grid(pb)
    g.upload(s)
    ws = g.adjoint_workspace(2, 1)
    with pytest.raises(fxmod.FxError) as ei:
        g.adjoint_forward(ws, pb.dt, 2, 1)
    assert ei.value.status == -7
    g.close()


def sph_case(map1, precision, seed=31, ngroups=9):
    """Spherical grid with random physical velocities (up to 0.3 of the sound speed, changing
    sign from cell to cell) and random physical fluxes (|F| up to 0.6 cE), stored covariant."""
    pb, prim = W.spherical_2d(nr=40, nth=22, ngroups=ngroups, nsteps=3, precision=precision, map1=map1)
    pb.vterms = 1
    rng = np.random.default_rng(seed)
    N, G = pb.ncell, pb.ngroups
    prim = np.array(prim, copy=True)
    cs = np.sqrt(pb.gamma * prim[1] / prim[0])
    prim[2] = rng.uniform(-0.3, 0.3, N) * cs
    prim[3] = rng.uniform(-0.3, 0.3, N) * cs
    s = oracle.init_equilibrium(pb, prim)
    # the cell scale factors: the covariant momentum of rho = 1, vhat = (1, 1)
    unit = np.array(prim, copy=True)
    unit[0], unit[2], unit[3] = 1.0, 1.0, 1.0
    hs = oracle.init_equilibrium(pb, unit)[N:3 * N].reshape(2, N)
    E = s[4 * N:4 * N + N * G].reshape(N, G)
    ang = rng.uniform(0, 2 * np.pi, (N, G))
    mag = rng.uniform(0, 0.6, (N, G)) * pb.c_light * E
    s[4 * N + N * G:4 * N + 2 * N * G] = (hs[0][:, None] * mag * np.cos(ang)).ravel()
    s[4 * N + 2 * N * G:] = (hs[1][:, None] * mag * np.sin(ang)).ravel()
    return pb, s


@pytest.mark.parametrize("map1", ["exp", "sinh"])
def test_velocity_terms_spherical_fp64(fxmod, map1):
    pb, s = sph_case(map1, "fp64")
    got, ref = run_both(fxmod, pb, s)
    H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)
    pb.vterms = 0
    plain, _ = oracle.run(pb, s, pb.dt, pb.nsteps, nthreads=8)
    rad = slice(4 * pb.ncell, None)
    assert np.abs(plain[rad] - ref[rad]).max() > 1e3 * FP64_MAX * np.abs(ref[rad]).max()


@pytest.mark.parametrize("ngroups", [9, 20])
@pytest.mark.parametrize("form", ["fp32", "fp32n64"])
def test_velocity_terms_spherical_fp32_forms(fxmod, form, ngroups):
    # two groups per lane on 8 (9 groups) and 16 (20 groups, the spherical workload's) lanes
    pb, s = sph_case("exp", form, ngroups=ngroups)
    got, ref = run_both(fxmod, pb, s)
    H.assert_parity(pb, got, ref, 1e-4, natural=True)


def test_velocity_terms_spherical_budget(fxmod):
    # the radiation energy the terms add on the spherical grid (cell volumes from the geometry)
    pb, s = sph_case("exp", "fp64")
    _, rst, rbud = oracle.run_budget(pb, s, pb.dt, 2, nthreads=8)
    g = fxmod.Grid(pb)
    g.upload(s)
    t0 = g.totals()
    g.budgets_enable(True)
    g.step(pb.dt, 2)
    assert g.status() == 0 and rst == 0
    bud = g.budgets()
    t1 = g.totals()
    g.close()
    assert abs(bud[8]) > 1e-8 * abs(t0[4])
    assert abs(bud[8] - rbud[8]) <= 1e-10 * abs(rbud[8]), (bud[8], rbud[8])
    # energy closes with it (the boundary fluxes, absorption work, floor and velocity terms)
    assert abs(t0[4] - t1[4] - bud[4] - bud[6] + bud[7] + bud[8]) <= 1e-13 * abs(t0[4])
