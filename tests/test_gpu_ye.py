"""GPU parity of the three-species form (neutrinos: the composition rho Y_e and the two-equation
(T, Y_e) interaction of Sec. 5.3; readings R30-R33) with the FP64 oracle, through the C ABI.

FP64 bars (relative L1 <= 1e-10, max-norm <= 1e-8 per field, rho Y_e included) on the neutrino
box in 2-d, a 1-d tube with reflecting and outflow ends and a 3-d box; total lepton number
rho Y_e - sum xi E conserved to round-off on the periodic box; the equilibrium initial state
against the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_1806_07390_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fxmod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07390_gb300 import build, fx
    build.build()
    return fx


def xi_of(pb):
    e = pb.eps_min * (pb.eps_max / pb.eps_min) ** (np.arange(pb.ngroups + 1) / pb.ngroups)
    cen = np.sqrt(e[:-1] * e[1:])
    return np.concatenate([-pb.xi0 / cen, pb.xi0 / cen, np.zeros(pb.ngroups)])


def lepton(pb, s):
    N, G, D = pb.ncell, pb.nchan, pb.dims
    NG = 2 + D
    E = s[NG * N:(NG + G) * N].reshape(N, G)
    X = s[(NG + (1 + D) * G) * N:]
    return X.sum() - (E * xi_of(pb)[None, :]).sum()


def case(name):
    if name == "box2d":
        pb, prim = W.neutrino_2d(nx=44, ny=36, ngroups=8, nsteps=5)
    elif name == "tube1d":
        pb, prim = W.neutrino_2d(nx=4, ny=4, ngroups=6)
        pb = W.Problem(**{**pb.__dict__, "dims": 1, "n": (90, 1, 1), "bc_lo": ("reflect",) * 3,
                          "bc_hi": ("outflow",) * 3, "nsteps": 6})
        x = pb.cell_centres(0)
        rho = 1.0 + 0.5 * np.tanh((x - 0.5) / 0.05)
        p = np.ones_like(x)
        prim = np.stack([rho, p, 0.2 * np.sin(2 * np.pi * x), 1.5 * p / rho, 0.25 + 0.15 * x])
    else:
        pb, prim = W.neutrino_2d(nx=4, ny=4, ngroups=4)
        n = (10, 9, 8)
        pb = W.Problem(**{**pb.__dict__, "dims": 3, "n": n, "nsteps": 3})
        rng = np.random.default_rng(9)
        N = int(np.prod(n))
        rho = rng.uniform(0.6, 1.8, N)
        p = rng.uniform(0.7, 1.3, N)
        v = rng.uniform(-0.2, 0.2, (3, N))
        prim = np.vstack([rho, p, v, 1.4 * p / rho, rng.uniform(0.15, 0.45, N)])
    # the light-crossing step of this grid (the generator's step was for its own grid)
    pb.dt = 0.3 * min(1.0 / pb.n[d] for d in range(pb.dims)) / pb.c_light / pb.dims
    return pb, np.ascontiguousarray(prim, dtype=np.float64)


@pytest.mark.parametrize("name", ["box2d", "tube1d", "box3d"])
def test_three_species_fp64(fxmod, name):
    pb, prim = case(name)
    s0 = oracle.init_equilibrium(pb, prim)
    ref, rst = oracle.run(pb, s0, pb.dt, pb.nsteps, nthreads=8)
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    init = g.download()
    g.step(pb.dt, pb.nsteps)
    st = g.status()
    got = g.download()
    g.close()
    assert st == 0 and rst == 0
    np.testing.assert_allclose(init, s0, rtol=1e-13, atol=1e-300)
    H.assert_parity(pb, got, ref, 1e-10, 1e-8)
    if name == "box2d":  # periodic: total lepton number conserved
        L0, L1 = lepton(pb, s0), lepton(pb, got)
        assert abs(L1 - L0) <= 1e-13 * abs(L0)
        # and the interaction moved it between gas and radiation
        X0 = s0[-pb.ncell:].sum()
        assert abs(got[-pb.ncell:].sum() - X0) > 1e-6 * abs(X0)


@pytest.mark.parametrize("form", ["fp32", "fp32n64"])
@pytest.mark.parametrize("name", ["box2d", "box3d"])
def test_three_species_fp32_forms(fxmod, name, form):
    pb, prim = case(name)
    pb.precision = form
    s0 = oracle.init_equilibrium(pb, prim)
    ref, rst = oracle.run(pb, s0, pb.dt, pb.nsteps, nthreads=8)
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    g.step(pb.dt, pb.nsteps)
    st = g.status()
    got = g.download()
    g.close()
    assert st == 0 and rst == 0
    H.assert_parity(pb, got, ref, 1e-5, natural=True)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32n64", 1e-5)])
def test_three_species_spherical(fxmod, precision, tol):
    # the spherical grid: composition fluxes with the area/volume factors, covariant momentum
    # and flux in the interaction, and the initial momentum with the scale factors
    pb, prim = W.neutrino_sph2d(nr=48, nth=20, ngroups=6, nsteps=6, precision=precision)
    s0 = oracle.init_equilibrium(pb, prim)
    ref, rst = oracle.run(pb, s0, pb.dt, pb.nsteps, nthreads=8)
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    init = g.download()
    g.step(pb.dt, pb.nsteps)
    st = g.status()
    got = g.download()
    g.close()
    assert st == 0 and rst == 0
    if precision == "fp64":
        np.testing.assert_allclose(init, s0, rtol=1e-13, atol=1e-300)
        H.assert_parity(pb, got, ref, tol, 1e-8)
    else:
        H.assert_parity(pb, got, ref, tol, natural=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_spherical_initial_momentum_is_covariant(fxmod, precision):
    # a spherical grid with flow: the equilibrium initialisation stores rho vhat_q h_q, as the
    # oracle does (host-staged, device and no-allocation paths)
    import torch
    pb, prim = W.spherical_2d(nr=40, nth=16, ngroups=5, precision=precision)
    prim = np.array(prim, copy=True)
    prim[2] = 0.1 * np.sqrt(pb.gamma * prim[1] / prim[0])
    prim[3] = 0.05 * np.sqrt(pb.gamma * prim[1] / prim[0])
    ref = oracle.init_equilibrium(pb, prim)
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    host = g.download()
    g.init_equilibrium(torch.from_numpy(np.ascontiguousarray(prim)).cuda())
    dev = g.download()
    dt = torch.float64 if precision == "fp64" else torch.float32
    st = torch.empty(g.nelem, dtype=dt, device="cuda")
    code = g.L.fx_state_init_equilibrium_noalloc(g.h, np.ascontiguousarray(prim).ctypes.data_as(
        __import__("ctypes").c_void_p), __import__("ctypes").c_void_p(st.data_ptr()),
        0 if precision == "fp64" else 1, __import__("ctypes").c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert code == 0
    na = st.double().cpu().numpy()
    g.close()
    tol = 1e-13 if precision == "fp64" else 2e-7
    for a in (host, dev, na):
        np.testing.assert_allclose(a, ref, rtol=tol, atol=1e-300)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32n64"])
@pytest.mark.parametrize("name", ["box2d", "sph"])
def test_three_species_with_velocity_terms(fxmod, name, precision):
    # reading R35: each species' groups their own frequency chain.  box2d: random gas, E and F
    # per channel, 5 groups per species (15 channels: with two groups per lane, lane pairs
    # straddle the species boundaries); sph: the spherical neutrino atmosphere, 6 groups per
    # species (18 channels, 16 lanes per cell)
    from tests.test_oracle_ye import species_vterms_problem, species_vterms_state
    if name == "box2d":
        pb = species_vterms_problem(couple=1)
        pb.precision = precision
        s0 = species_vterms_state(pb, seed=3)
        pb.dt, pb.nsteps = 0.3 / max(pb.n[:2]) / pb.c_light, 4
    else:
        pb, prim = W.neutrino_sph2d(nr=48, nth=20, ngroups=6, nsteps=4, precision=precision)
        pb.vterms = 1
        s0 = oracle.init_equilibrium(pb, prim)
    ref, rst = oracle.run(pb, s0, pb.dt, pb.nsteps, nthreads=8)
    g = fxmod.Grid(pb)
    g.upload(s0)
    g.step(pb.dt, pb.nsteps)
    st = g.status()
    got = g.download()
    g.close()
    assert st == 0 and rst == 0
    if precision == "fp64":
        H.assert_parity(pb, got, ref, 1e-10, 1e-8)
    else:
        H.assert_parity(pb, got, ref, 1e-4, natural=True)
    # the terms change the radiation by far more than the bar
    pb.vterms = 0
    plain, _ = oracle.run(pb, s0, pb.dt, pb.nsteps, nthreads=8)
    rad = slice((2 + pb.dims) * pb.ncell, -pb.ncell)
    assert np.abs(plain[rad] - ref[rad]).max() > 1e-6 * np.abs(ref[rad]).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32n64", 1e-6)])
def test_three_species_budgets(fxmod, precision, tol):
    # budgets with three species and the velocity terms: the flux-absorption work and the E floor
    # of the two-equation interaction and the terms' radiation energy equal the oracle's, and the
    # total energy closes with them (periodic box)
    from tests.test_oracle_ye import species_vterms_problem, species_vterms_state
    pb = species_vterms_problem(couple=1)
    pb.precision = precision
    s0 = species_vterms_state(pb, seed=3)
    dt = 0.3 / max(pb.n[:2]) / pb.c_light
    _, rst, rbud = oracle.run_budget(pb, s0, dt, 3, nthreads=8)
    g = fxmod.Grid(pb)
    g.upload(s0)
    t0 = g.totals()
    g.budgets_enable(True)
    g.step(dt, 3)
    assert g.status() == 0 and rst == 0
    bud = g.budgets()
    t1 = g.totals()
    g.close()
    assert abs(bud[6]) > 1e-6 * abs(t0[4]) and abs(bud[8]) > 1e-6 * abs(t0[4])
    assert np.all(np.abs(bud - rbud) <= tol * abs(t0[4])), (bud, rbud)
    closure = abs(t0[4] - t1[4] - bud[4] - bud[6] + bud[7] + bud[8])
    assert closure <= (1e-13 if precision == "fp64" else 1e-6) * abs(t0[4]), closure


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32n64"])
def test_three_species_totals_after_upload(fxmod, precision):
    # the conserved totals of an uploaded three-species state, every form, on a grid small enough
    # that a write past the Planck table's workspace region would reach the totals' cell volumes
    from tests.test_oracle_ye import species_vterms_problem, species_vterms_state
    pb = species_vterms_problem(couple=1)
    pb.precision = precision
    s0 = species_vterms_state(pb, seed=3)
    g = fxmod.Grid(pb)
    g.upload(s0)
    t = g.totals()
    g.close()
    ref = oracle.totals(pb, s0)
    np.testing.assert_allclose(t, ref, rtol=1e-13 if precision == "fp64" else 1e-6,
                               atol=1e-12 * np.abs(ref).max())
