"""Parity of the CUDA stage update (through the C ABI) with the FP64 CPU oracle.

Bar (FP64 path): relative L1 error <= 1e-10 and max-norm error <= 1e-8 per field; conserved
totals <= 1e-13.  FP32 form: L1 error <= 1e-5 on smooth problems and <= 1e-4 with shocks, each
field measured against its natural scale (momentum against sqrt(rho rho e), radiation flux
against c E): near equilibrium the flux is many orders below c E and below FP32 resolution, so
an error relative to the flux itself would measure FP32 rounding noise, not the method.
"""
import numpy as np
import pytest

import oracle
from paper_1806_07390_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

FP64_L1, FP64_MAX, TOT = 1e-10, 1e-8, 1e-13


@pytest.fixture(scope="module")
def fxmod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07390_gb300 import build, fx
    build.build()
    return fx


def run_gpu(fxmod, pb, prim=None, state=None, nsteps=None, dt=None):
    g = fxmod.Grid(pb)
    if state is not None:
        g.upload(np.asarray(state, dtype=np.float64))
    else:
        g.init_equilibrium(prim)
    g.step(pb.dt if dt is None else dt, pb.nsteps if nsteps is None else nsteps)
    st = g.status()
    out = g.download()
    tot = g.totals()
    g.close()
    return out, st, tot


def run_oracle(pb, prim=None, state=None, nsteps=None, dt=None):
    s0 = oracle.init_equilibrium(pb, prim) if state is None else np.asarray(state, dtype=np.float64)
    out, st = oracle.run(pb, s0, pb.dt if dt is None else dt, pb.nsteps if nsteps is None else nsteps,
                         nthreads=8)
    return out, st


def check_totals(pb, tot_gpu, out_ref):
    ref = oracle.totals(pb, out_ref)
    scale = np.array([abs(ref[0]), abs(ref[0]), abs(ref[0]), abs(ref[0]), abs(ref[4]), abs(ref[5])])
    err = np.abs(tot_gpu - ref) / scale
    assert np.all(err[[0, 4, 5]] <= TOT), (tot_gpu, ref, err)


def test_sod1d_full_config_fp64(fxmod):
    # 512 cells, 12 groups, 200 steps (the 1-d workload at full size)
    pb, prim = W.sod_1d()
    got, st, tot = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)
    # totals of the GPU state by the library vs the oracle's on the oracle state
    check_totals(pb, tot, ref)


@pytest.mark.parametrize("shape,G,steps", [((40, 36), 16, 4), ((37, 70), 5, 3), ((21, 19), 20, 3),
                                           ((33, 9), 12, 2)])
def test_kh2d_small_fp64(fxmod, shape, G, steps):
    # ragged tiles, several march chunks (ny > 32), all lane-segment widths (G = 5, 12, 16, 20)
    pb, prim = W.kh_2d(nx=shape[0], ny=shape[1], ngroups=G, nsteps=steps)
    got, st, tot = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)
    check_totals(pb, tot, ref)


def test_blobs2d_outflow_periodic_fp64(fxmod):
    pb, prim = W.blobs_2d(shape=(36, 34), ngroups=8, nsteps=3, precision="fp64")
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)


def test_lognormal3d_small_fp64(fxmod):
    pb, prim = W.lognormal_3d(shape=(14, 10, 9), ngroups=12, nsteps=2, precision="fp64")
    got, st, tot = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)
    check_totals(pb, tot, ref)


@pytest.mark.parametrize("form", ["fp32", "fp32n64"])
@pytest.mark.parametrize("G", [8, 16, 21])
def test_reflecting_walls_fp32_forms(fxmod, form, G):
    # mirror ghosts (negated normal components of v and F) on both x walls and the upper march
    # wall, with one group per lane (G = 8) and two (G = 16, 21: 32-cell and 16-cell tiles whose
    # planes are ordered by warp-to-warp hand-offs); three tiles across x with a ragged last one
    pb, prim = W.kh_2d(nx=70, ny=30, ngroups=G, nsteps=3, precision=form)
    pb.bc_lo = ("reflect", "outflow", "periodic")
    pb.bc_hi = ("reflect", "reflect", "periodic")
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, 1e-4, natural=True)


def test_reflecting_walls_and_random_state_fp64(fxmod):
    pb, _ = W.kh_2d(nx=20, ny=18, ngroups=6, nsteps=2)
    pb.bc_lo = ("reflect", "outflow", "periodic")
    pb.bc_hi = ("reflect", "reflect", "periodic")
    pb.c_light = 12.0
    pb.dt = 2e-4
    s = W.random_state(pb, seed=5)
    got, st, _ = run_gpu(fxmod, pb, state=s)
    ref, rst = run_oracle(pb, state=s)
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)


@pytest.mark.parametrize("form", ["fp32", "fp32n64"])
@pytest.mark.parametrize("maker,tol", [("kh", 1e-4), ("blobs", 1e-4), ("lognormal", 1e-5)])
def test_fp32_form_small(fxmod, maker, tol, form):
    if maker == "kh":
        pb, prim = W.kh_2d(nx=48, ny=40, ngroups=16, nsteps=4, precision=form)
    elif maker == "blobs":
        pb, prim = W.blobs_2d(shape=(40, 36), ngroups=8, nsteps=4, precision=form)
    else:
        pb, prim = W.lognormal_3d(shape=(12, 10, 9), ngroups=12, nsteps=2, precision=form)
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, tol, natural=True)


@pytest.mark.parametrize("form", ["fp32", "fp32n64"])
@pytest.mark.parametrize("G", [9, 13, 21])
def test_fp32_forms_odd_group_counts(fxmod, form, G):
    # odd group counts: padded lanes of each cell (G = 9, 13: one group per lane), and two groups
    # per lane with one group in the cell's last lane (G = 21, 32 padded groups)
    pb, prim = W.kh_2d(nx=44, ny=38, ngroups=G, nsteps=3, precision=form)
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, 1e-4, natural=True)


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_L1), ("fp32", 1e-5), ("fp32n64", 1e-5)])
def test_rayleigh_jeans_groups(fxmod, precision, tol):
    # every group far below kT (eps/T < 2^-14 at all band edges): the FP32 Planck path leaves its
    # tables for the series x^3/3 - x^4/8 of each band (whose upper edge is the group's own), the
    # FP64 path takes its small-x series
    pb, prim = W.kh_2d(nx=24, ny=20, ngroups=6, nsteps=3, precision=precision)
    pb.eps_min, pb.eps_max = 1e-6, 1e-5
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    if precision == "fp64":
        H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)
    else:
        H.assert_parity(pb, got, ref, tol, natural=True)


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_L1), ("fp32", 1e-4), ("fp32n64", 1e-4)])
def test_kh2d_full_size_sampled_windows(fxmod, precision, tol):
    # 1024^2 x 16 groups, one step in the benchmark's launch configuration; windows of 8x8 cells
    # (+4 halo: the two-stage dependency radius) recomputed by the oracle
    pb, prim = W.kh_2d(precision=precision)
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    g.step(pb.dt, 1)
    assert g.status() == 0
    out = g.download()
    g.close()
    rng = np.random.default_rng(7)
    starts = [(0, 0), (1016, 1016), (508, 252)] + [tuple(rng.integers(0, 1017, 2)) for _ in range(3)]
    for start in starts:
        sub, sprim = H.window(pb, prim, start, (8, 8), 4)
        ref, _ = run_oracle(sub, sprim, nsteps=1)
        r = H.gather_cells(sub, ref, H.sub_cells(sub, (8, 8), 4))
        gcell = H.gather_cells(pb, out, H.window_cells(pb, start, (8, 8)))
        small = W.Problem(**{**sub.__dict__, "n": (8, 8, 1)})
        if precision == "fp64":
            H.assert_parity(small, gcell, r, tol, FP64_MAX)
        else:
            H.assert_parity(small, gcell, r, tol, natural=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32n64"])
@pytest.mark.parametrize("where", ["gas", "E", "F"])
def test_nonfinite_state_is_reported(fxmod, precision, where):
    # one NaN in a gas variable, a group energy or a group flux of one cell: every form reports it
    pb, prim = W.kh_2d(nx=16, ny=16, ngroups=4, nsteps=1, precision=precision)
    s = oracle.init_equilibrium(pb, prim)
    ncell, G, NG = 16 * 16, 4, 4
    c = 37
    idx = {"gas": c, "E": NG * ncell + c * G + 2, "F": NG * ncell + (ncell + c) * G + 1}[where]
    s[idx] = np.nan
    g = fxmod.Grid(pb)
    g.upload(s)
    g.step(pb.dt, 1)
    assert g.status() == -6
    g.close()


def test_newton_failure_is_reported(fxmod):
    # an opacity far too large for a two-iteration cap and no bisection: the status says so and
    # the GPU stays usable
    pb, prim = W.kh_2d(nx=16, ny=16, ngroups=4, nsteps=1)
    pb.kappa0 = 1e9
    pb.newton_maxit = 1
    pb.bisect_maxit = 0
    prim = prim.copy()
    prim[-1] *= 3.0  # radiation far from equilibrium
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    g.step(pb.dt, 1)
    assert g.status() == -4
    g.close()
    pb2, prim2 = W.kh_2d(nx=16, ny=16, ngroups=4, nsteps=1)
    out, st, _ = run_gpu(fxmod, pb2, prim2)
    assert st == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32n64"])
def test_bisection_fallback(fxmod, precision):
    # one Newton iteration allowed, strong coupling, radiation twice the gas temperature: every
    # cell falls back to the bisection on its bracket (reading R11), on both sides
    pb, prim = W.kh_2d(nx=20, ny=16, ngroups=6, nsteps=2, precision=precision)
    pb.kappa0, pb.newton_maxit = 1e4, 1
    prim = prim.copy()
    prim[-1] *= 2.0
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    if precision == "fp64":
        H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)
    else:
        H.assert_parity(pb, got, ref, 1e-4, natural=True)


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_L1), ("fp32", 1e-5), ("fp32n64", 1e-5)])
def test_spherical_2d_small(fxmod, precision, tol):
    # log-r x theta grid with reflecting inner radius, outflow outer radius, polar-axis parity;
    # coordinate moments, curvilinear face factors and geometric sources all active
    pb, prim = W.spherical_2d(nr=36, nth=20, ngroups=20, nsteps=3, precision=precision)
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    if precision == "fp64":
        H.assert_parity(pb, got, ref, tol, FP64_MAX)
    else:
        H.assert_parity(pb, got, ref, tol, natural=True)


@pytest.mark.parametrize("maker", ["kh", "lognormal", "spherical"])
def test_second_order_radiation_reconstruction_fp64(fxmod, maker):
    # rad_recon_order = 2: the gas's n = 2 parabola with its limiters for E and F, per group
    # (reading R1), on a Cartesian 2-d, a 3-d and the spherical grid
    if maker == "kh":
        pb, prim = W.kh_2d(nx=40, ny=36, ngroups=6, nsteps=3)
    elif maker == "lognormal":
        pb, prim = W.lognormal_3d(shape=(12, 10, 9), ngroups=5, nsteps=2, precision="fp64")
    else:
        pb, prim = W.spherical_2d(nr=30, nth=16, ngroups=6, nsteps=3, precision="fp64")
    pb.rad_recon_order = 2
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)


@pytest.mark.parametrize("form", ["fp32", "fp32n64"])
@pytest.mark.parametrize("G", [8, 16])
def test_second_order_radiation_reconstruction_fp32_forms(fxmod, form, G):
    pb, prim = W.kh_2d(nx=48, ny=40, ngroups=G, nsteps=3, precision=form)
    pb.rad_recon_order = 2
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, 1e-4, natural=True)


def test_second_order_radiation_reconstruction_has_no_adjoint(fxmod):
    pb, prim = W.blobs_2d(shape=(24, 20), ngroups=4, nsteps=2, precision="fp64")
    pb.rad_recon_order = 2
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    with pytest.raises(fxmod.FxError) as e:
        g.adjoint_forward(g.adjoint_workspace(2, 1), pb.dt, 2, 1)
    assert e.value.status == -7
    g.close()


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_L1), ("fp32n64", 1e-5)])
def test_spherical_2d_sinh_map(fxmod, precision, tol):
    # the sinh radial map r = r_t sinh(x1 / r_t): nearly uniform in r at the inner boundary,
    # logarithmic outside r_t; the kernels see it only through the geometry tables
    pb, prim = W.spherical_2d(nr=36, nth=20, ngroups=20, nsteps=3, precision=precision, map1="sinh")
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    if precision == "fp64":
        H.assert_parity(pb, got, ref, tol, FP64_MAX)
    else:
        H.assert_parity(pb, got, ref, tol, natural=True)


def test_spherical_static_atmosphere_gpu(fxmod):
    # uniform p and E, v = F = 0: flux divergence and geometric sources cancel (Eqs. 84-85)
    pb, _ = W.spherical_2d(nr=24, nth=16, ngroups=3, nsteps=1, precision="fp64")
    pb.couple = 0
    N = pb.ncell
    s = np.zeros(pb.state_size())
    s[:N] = np.linspace(0.5, 2.0, N)
    s[3 * N: 4 * N] = 0.7 / (pb.gamma - 1)
    s[4 * N: 4 * N + N * 3] = 0.3
    got, st, _ = run_gpu(fxmod, pb, state=s, nsteps=2)
    assert st == 0
    assert np.max(np.abs(got - s)) < 1e-12


@pytest.mark.parametrize("case", ["blobs", "sod", "box3d"])
def test_budgets_match_the_oracle_and_close(fxmod, case):
    # reading R13: boundary outflows, coupling work and floor energy accumulated by the kernels
    # equal the oracle's, and with the library's own totals every budget closes to round-off
    if case == "blobs":
        pb, _ = W.blobs_2d(shape=(40, 34), ngroups=6, nsteps=4, precision="fp64")
        pb.c_light, pb.kappa0 = 6.0, 5.0
    elif case == "sod":
        pb, _ = W.sod_1d(n=64, ngroups=5)
        pb.c_light = 8.0
    else:
        pb, _ = W.lognormal_3d(shape=(14, 10, 9), ngroups=4, precision="fp64")
        pb.bc_lo = ("outflow", "reflect", "periodic")
        pb.bc_hi = ("reflect", "outflow", "periodic")
        pb.c_light = 5.0
    pb.dt = 0.2 / pb.n[0] / pb.c_light
    s = W.random_state(pb, seed=17, flux_frac=0.6)
    ref, rst, rbud = oracle.run_budget(pb, s, pb.dt, 4, nthreads=8)
    g = fxmod.Grid(pb)
    g.upload(s)
    t0 = g.totals()
    g.budgets_enable(True)
    g.step(pb.dt, 4)
    assert g.status() == 0 and rst == 0
    bud = g.budgets()
    t1 = g.totals()
    g.close()
    scale = np.array([abs(t0[0])] * 4 + [abs(t0[4])] * 5)
    assert np.all(np.abs(bud - rbud) <= 1e-12 * scale), (bud, rbud)
    assert abs(t0[0] - t1[0] - bud[0]) <= 1e-13 * abs(t0[0])
    for q in range(pb.dims):
        assert abs(t0[1 + q] - t1[1 + q] - bud[1 + q]) <= 1e-13 * abs(t0[0])
    assert abs(t0[4] - t1[4] - bud[4] - bud[6] + bud[7]) <= 1e-13 * abs(t0[4])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32n64"])
def test_density_floor_is_reported(fxmod, precision):
    # reading R18: a host-uploaded state with a block of cells below the density floor (at the
    # temperature of their neighbours; wide enough that transport cannot lift its centre above
    # the floor in one stage) is floored by the interaction and the status says so; the oracle
    # applies the same floor and flags it
    pb, prim = W.kh_2d(nx=24, ny=24, ngroups=4, nsteps=1, precision=precision)
    pb64 = W.Problem(**{**pb.__dict__, "precision": "fp64"})
    s = oracle.init_equilibrium(pb64, prim)
    N = pb.ncell
    y, x = np.divmod(np.arange(N), 24)
    blk = (x >= 5) & (x < 19) & (y >= 5) & (y < 19)
    T = prim[1] / prim[0]
    rho = 0.5 * pb.rho_floor
    s[:N][blk] = rho
    s[N:2 * N][blk] = 0.0
    s[2 * N:3 * N][blk] = 0.0
    s[3 * N:4 * N][blk] = rho * T[blk] / (pb.gamma - 1.0)
    _, rst = oracle.run(pb64, s, pb.dt, 1)
    assert rst & 2  # the oracle's floor bit
    g = fxmod.Grid(pb)
    g.upload(s)
    g.step(pb.dt, 1)
    assert g.status() == -5
    g.close()


def _blast(precision, solver, guard, nx=44, ny=38, G=5, nsteps=3):
    # strong shocks in every direction: pressure 30 inside a disk, 1 outside, radiation in
    # equilibrium with the gas; ragged tiles and several march chunks
    pb, prim = W.kh_2d(nx=nx, ny=ny, ngroups=G, nsteps=nsteps, precision=precision)
    prim = prim.copy()
    y, x = np.divmod(np.arange(pb.ncell), nx)
    r2 = ((x + 0.5) / nx - 0.45) ** 2 + ((y + 0.5) / ny - 0.55) ** 2
    prim[1] = np.where(r2 < 0.04, 30.0, 1.0)
    prim[-1] = prim[1] / prim[0]
    pb.riemann, pb.shock_guard = solver, guard
    return pb, prim


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32n64"])
@pytest.mark.parametrize("solver,guard", [("hlle", 0.0), ("llf", 0.0), ("hllc", 0.5)])
def test_riemann_options_match_the_oracle(fxmod, precision, solver, guard):
    pb, prim = _blast(precision, solver, guard)
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    if precision == "fp64":
        H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)
    else:
        H.assert_parity(pb, got, ref, 1e-4, natural=True)
    if guard > 0 and precision == "fp64":
        # the guard changes the result (the blast's shocks are tagged)
        pb2, _ = _blast(precision, solver, 0.0)
        plain, _, _ = run_gpu(fxmod, pb2, prim)
        assert np.max(np.abs(plain - got)) > 1e-8


def test_carbuncle_guard_on_the_gpu(fxmod):
    # Quirk's odd-even decoupling (as the oracle pin): a Mach-6 shock along a periodic channel
    # with an odd-even perturbation of 1e-3 on its centre row; one weakly coupled radiation group
    nx, ny, g = 160, 24, 1.4

    def setup(guard):
        pb = W.Problem(name="quirk", dims=2, n=(nx, ny, 1), x_lo=(0, 0, 0), x_hi=(nx / ny, 1, 1),
                       bc_lo=("outflow", "periodic", "periodic"), bc_hi=("outflow", "periodic", "periodic"),
                       ngroups=1, gamma=g, kappa0=1e-3, kap_rho_exp=0.0, kap_T_exp=0.0,
                       kap_eps_exp=0.0, c_light=60.0, a_rad=1e-6, couple=1)
        pb.shock_guard = guard
        y, x = np.divmod(np.arange(pb.ncell), nx)
        M = 6.0
        r2 = (g + 1) * M ** 2 / ((g - 1) * M ** 2 + 2)
        p2 = (2 * g * M ** 2 - (g - 1)) / (g + 1)
        u2 = M * np.sqrt(g) * (1 - 1 / r2)
        rho = np.where(x < 10, r2, 1.0)
        mid = y == ny // 2
        rho[mid] *= 1 + 1e-3 * (2 * (x[mid] % 2) - 1)
        p = np.where(x < 10, p2, 1.0)
        prim = np.stack([rho, p, np.where(x < 10, u2, 0.0), np.zeros(pb.ncell), p / rho])
        pb.dt = 0.3 / ny / pb.c_light
        return pb, prim

    vy = {}
    for guard in (0.0, 1.0):
        pb, prim = setup(guard)
        got, st, _ = run_gpu(fxmod, pb, prim, nsteps=2700)
        assert st == 0
        vy[guard] = np.max(np.abs(got[2 * pb.ncell: 3 * pb.ncell] / got[: pb.ncell]))
        if guard > 0:
            ref, rst = run_oracle(pb, prim, nsteps=2700)
            assert rst == 0
            # (the transverse momentum is perturbation-sized: measured against sqrt(rho rho e))
            H.assert_parity(pb, got, ref, FP64_L1, natural=True)
    assert vy[0.0] > 1e-2 and vy[1.0] < 1e-4, vy


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32n64"])
def test_scattering_matches_the_oracle(fxmod, precision):
    # scattering sigma = sigma0 rho in the flux absorption (Eq. 28) and the optical depth of the
    # HLL correction (R9), beside absorption, on the shear layer with a flux-carrying state
    pb, prim = W.kh_2d(nx=40, ny=36, ngroups=8, nsteps=3, precision=precision)
    pb.sigma0 = 25.0
    got, st, _ = run_gpu(fxmod, pb, prim)
    ref, rst = run_oracle(pb, prim)
    assert st == 0 and rst == 0
    if precision == "fp64":
        H.assert_parity(pb, got, ref, FP64_L1, FP64_MAX)
    else:
        H.assert_parity(pb, got, ref, 1e-4, natural=True)
    pb.sigma0 = 0.0
    plain, _, _ = run_gpu(fxmod, pb, prim)
    assert np.max(np.abs(plain - got)) > 1e-6 * np.max(np.abs(got))  # sigma changes the result
