"""Pins of the oracle's three-species form: the two-equation (T, Y_e) interaction and the
composition rho Y_e (Sec. 5.3 in the core-collapse form; Sec. 3.2's composition equation;
readings R30-R33).

- Total energy and total lepton number rho Y_e - sum xi E are conserved to round-off on a
  periodic grid with the interaction on (the lepton total computed here from xi's definition:
  the interaction changes rho Y_e by sum xi dE, so a nu_e, xi < 0, carries lepton number
  -xi E).
- The interaction's result solves the implicit system: every channel satisfies the inner
  backward-Euler update at the accepted (T, Y_e), with B_g from an independent quadrature.
- Equilibrium (E = w_s(Y_e) B_g(T), F = 0) is a fixed point.
- In the stiff limit the state reaches the equilibrium (T*, Y_e*) that conserves energy and
  lepton number, found here by an independent root finder.
- rho Y_e is advected at third order in a uniform flow.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
from paper_1806_07390_gb300 import workloads as W


def planck_int(a, b):
    f = lambda t: t ** 3 / math.expm1(t) if t > 0 else 0.0  # noqa: E731
    return integrate.quad(f, a, b, epsabs=0, epsrel=1e-13, limit=200)[0]


def groups(pb):
    e = pb.eps_min * (pb.eps_max / pb.eps_min) ** (np.arange(pb.ngroups + 1) / pb.ngroups)
    return e, np.sqrt(e[:-1] * e[1:])


def xi_of(pb):
    """xi per channel (species-major): -xi0/eps_g, +xi0/eps_g, 0 at the group centre (R30)."""
    _, cen = groups(pb)
    return np.concatenate([-pb.xi0 / cen, pb.xi0 / cen, np.zeros(pb.ngroups)])


def w_of(Ye):
    return np.array([2 * Ye, 2 * (1 - Ye), 1.0])


def B_of(pb, T):
    e, _ = groups(pb)
    return np.array([pb.a_rad * 15 / math.pi ** 4 * T ** 4 * planck_int(e[g] / T, e[g + 1] / T)
                     for g in range(pb.ngroups)])


def unpack(pb, s):
    N, G, D = pb.ncell, pb.nchan, pb.dims
    NG = 2 + D
    gas = s[:NG * N].reshape(NG, N)
    rad = s[NG * N:(NG + (1 + D) * G) * N].reshape(1 + D, N, G)
    X = s[(NG + (1 + D) * G) * N:]
    return gas, rad, X


def lepton_total(pb, s):
    gas, rad, X = unpack(pb, s)
    V = np.prod([(pb.x_hi[d] - pb.x_lo[d]) / pb.n[d] for d in range(pb.dims)])
    return V * (X.sum() - (rad[0] * xi_of(pb)[None, :]).sum())


def test_energy_and_lepton_number_are_conserved():
    pb, prim = W.neutrino_2d(nx=20, ny=16, ngroups=5, nsteps=6)
    s0 = oracle.init_equilibrium(pb, prim)
    out, st, bud = oracle.run_budget(pb, s0, pb.dt, pb.nsteps)
    assert st == 0
    t0, t1 = oracle.totals(pb, s0), oracle.totals(pb, out)
    assert abs(t1[0] - t0[0]) <= 1e-13 * t0[0]
    # total energy: periodic, so only the flux-absorption work on the moving gas and the E floor
    # change it (reading R13)
    assert abs(t0[4] - t1[4] - bud[6] + bud[7]) <= 1e-13 * t0[4]
    L0, L1 = lepton_total(pb, s0), lepton_total(pb, out)
    assert abs(L1 - L0) <= 1e-13 * abs(L0)
    # lepton number really moved between the gas and the radiation
    X0, X1 = unpack(pb, s0)[2], unpack(pb, out)[2]
    V = 1.0 / pb.ncell
    assert abs(V * (X1.sum() - X0.sum())) > 1e-6 * abs(L0)


def random_cells(pb, seed, ye=(0.1, 0.45)):
    """Random cells at rest (no kinetic energy: the flux absorption does no work, and the gas
    energy after the interaction is u itself), three-species radiation and composition."""
    rng = np.random.default_rng(seed)
    N, G, D = pb.ncell, pb.nchan, pb.dims
    s = W.random_state(pb, seed=seed, flux_frac=0.3)
    NG = 2 + D
    rho = s[:N]
    s[(1 + D) * N:NG * N] -= 0.5 * (s[N:(1 + D) * N].reshape(D, N) ** 2).sum(0) / rho
    s[N:(1 + D) * N] = 0.0
    E = rng.uniform(0.05, 1.0, (N, G))
    dirs = rng.standard_normal((D, N, G))
    dirs /= np.sqrt((dirs ** 2).sum(0))
    F = dirs * rng.uniform(0, 0.3, (N, G)) * pb.c_light * E
    Ye = rng.uniform(*ye, N)
    out = np.concatenate([s[:NG * N], E.reshape(-1), F.reshape(-1), rho * Ye])
    assert out.size == pb.state_size()
    return out


def one_cell_problem(kappa0=3.0, xi0=0.002, c=4.0):
    # (random cells with a larger xi0 can carry more lepton number than Y_e in [0, 1] admits)
    return W.Problem(name="nu1", dims=1, n=(6, 1, 1), x_lo=(0, 0, 0), x_hi=(1, 1, 1),
                     bc_lo=("periodic",) * 3, bc_hi=("periodic",) * 3, ngroups=4, gamma=4 / 3,
                     kappa0=kappa0, kap_rho_exp=1.0, kap_T_exp=-1.5, kap_eps_exp=-2.0, c_light=c,
                     species=3, xi0=xi0)


def test_interaction_solves_the_implicit_two_equation_system():
    pb = one_cell_problem()
    dt = 0.05
    s = random_cells(pb, seed=3)
    out, st = oracle.couple(pb, s, dt)
    assert st == 0
    gas0, rad0, X0 = unpack(pb, s)
    gas1, rad1, X1 = unpack(pb, out)
    N, G = pb.ncell, pb.nchan
    _, cen = groups(pb)
    xi = xi_of(pb)
    for c in range(N):
        rho = gas1[0, c]
        T = gas1[2, c] * (pb.gamma - 1) / rho  # at rest: rho e = u
        Ye = X1[c] / rho
        B = B_of(pb, T)
        kap = pb.kappa0 * rho * T ** -1.5 * cen ** -2.0
        tau = pb.c_light * dt * np.tile(kap, 3)
        Eq = np.concatenate([w * B for w in w_of(Ye)])
        Ein = rad0[0, c]
        np.testing.assert_allclose(rad1[0, c], (Ein + tau * Eq) / (1 + tau), rtol=1e-9)
        # energy (incl. the flux-absorption work) and lepton number by conservation
        assert abs((X1[c] - xi @ rad1[0, c]) - (X0[c] - xi @ Ein)) <= 1e-13 * abs(X0[c] + np.abs(xi) @ Ein)
        # the flux is absorbed with the opacity at the accepted T
        np.testing.assert_allclose(rad1[1, c], rad0[1, c] / (1 + tau), rtol=1e-12)


def test_equilibrium_is_a_fixed_point():
    pb = one_cell_problem()
    N, G = pb.ncell, pb.nchan
    rng = np.random.default_rng(8)
    rho, T, Ye = rng.uniform(0.5, 2, N), rng.uniform(0.5, 2, N), rng.uniform(0.1, 0.45, N)
    E = np.stack([np.concatenate([w * B_of(pb, T[c]) for w in w_of(Ye[c])]) for c in range(N)])
    s = np.concatenate([rho, np.zeros(N), rho * T / (pb.gamma - 1), E.reshape(-1), np.zeros(N * G), rho * Ye])
    out, st = oracle.couple(pb, s, 0.3)
    assert st == 0
    np.testing.assert_allclose(out, s, rtol=1e-12, atol=1e-15)


def test_stiff_limit_reaches_the_conserving_equilibrium():
    pb = one_cell_problem(kappa0=1e7)
    dt = 1.0
    s = random_cells(pb, seed=12)
    out, st = oracle.couple(pb, s, dt)
    assert st == 0
    gas0, rad0, X0 = unpack(pb, s)
    gas1, rad1, X1 = unpack(pb, out)
    xi = xi_of(pb)
    cv = 1 / (pb.gamma - 1)
    for c in range(pb.ncell):
        rho = gas0[0, c]
        ke = 0.5 * gas0[1, c] ** 2 / rho
        u0 = gas0[2, c] - ke
        Etot = u0 + rad0[0, c].sum()
        Ltot = X0[c] - xi @ rad0[0, c]

        def res(z):
            T, Ye = z
            Eq = np.concatenate([w * B_of(pb, T) for w in w_of(Ye)])
            return [(rho * cv * T + Eq.sum() - Etot) / Etot, (rho * Ye - xi @ Eq - Ltot) / abs(Ltot)]

        T0 = u0 / (rho * cv)
        Ts, Yes = optimize.fsolve(res, [T0, X0[c] / rho], xtol=1e-13)
        T1 = gas1[2, c] / (rho * cv)  # at rest: rho e = u (the absorbed flux's momentum aside)
        assert abs(T1 - Ts) <= 1e-6 * Ts, (T1, Ts)
        assert abs(X1[c] / rho - Yes) <= 1e-6, (X1[c] / rho, Yes)


def test_composition_advects_at_third_order():
    # uniform rho, p, v = 1 and Y_e = 0.3 + 0.1 tanh((x - x0 - t)/w): rho Y_e is an exact contact
    # solution moving with v (monotone, so the limiter's extremum clipping stays out of the
    # measurement); cell averages of the exact profile, dt ~ dx^1.5 so that the second-order time
    # error stays below the third-order spatial error; no interaction
    errs = []
    w, x0, t_end = 0.08, 0.35, 0.1
    for n in (64, 128, 256):
        pb = W.Problem(name="ye_adv", dims=1, n=(n, 1, 1), x_lo=(0, 0, 0), x_hi=(1, 1, 1),
                       bc_lo=("outflow",) * 3, bc_hi=("outflow",) * 3, ngroups=1, gamma=1.4,
                       kappa0=0.0, kap_rho_exp=0.0, kap_T_exp=0.0, kap_eps_exp=0.0, c_light=2.0,
                       couple=0, species=3, xi0=0.0)
        f = np.linspace(0, 1, n + 1)
        avg = lambda sh: 0.3 + 0.1 * w * (np.log(np.cosh((f[1:] - sh) / w)) -  # noqa: E731
                                           np.log(np.cosh((f[:-1] - sh) / w))) * n
        s = np.concatenate([np.ones(n), np.ones(n), np.full(n, 1.0 / 0.4 + 0.5),
                            np.full(3 * n, 1e-6), np.zeros(3 * n), avg(x0)])
        dt0 = 0.3 * (1.0 / n) ** 1.5
        nst = int(math.ceil(t_end / dt0))
        out, st = oracle.run(pb, s, t_end / nst, nst)
        assert st == 0
        mid = slice(int(0.3 * n), int(0.7 * n))
        errs.append(np.abs(out[-n:][mid] - avg(x0 + t_end)[mid]).mean())
    order = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(order) > 2.6, (errs, order)


# ------------------------------------------------------------- three species with velocity terms
def species_vterms_problem(couple, dims=2):
    n = (14, 12, 1) if dims == 2 else (40, 1, 1)
    return W.Problem(name="nuvt", dims=dims, n=n, x_lo=(0, 0, 0), x_hi=(1, 1, 1),
                     bc_lo=("periodic",) * 3, bc_hi=("periodic",) * 3, ngroups=5, gamma=4 / 3,
                     kappa0=2.0, kap_rho_exp=1.0, kap_T_exp=-1.5, kap_eps_exp=-2.0, c_light=4.0,
                     couple=couple, species=3, xi0=0.002, vterms=1)


def species_vterms_state(pb, seed=21):
    """Random gas (velocities changing sign from cell to cell), random E and F (|F| up to
    0.6 cE) per channel, random Y_e."""
    rng = np.random.default_rng(seed)
    N, G, D = pb.ncell, pb.nchan, pb.dims
    one = W.Problem(**{**pb.__dict__, "species": 1, "ngroups": G})
    s = W.random_state(one, seed=seed, flux_frac=0.6)
    rho = s[:N]
    return np.concatenate([s, rho * rng.uniform(0.1, 0.45, N)])


@pytest.mark.parametrize("dims", [1, 2])
def test_species_evolve_independently_under_the_velocity_terms(dims):
    # Reading R35: each species' groups form their own frequency chain.  Without the interaction
    # the gas evolves by itself and every species exactly as a one-species run with its own E and
    # F (a flux between the last group of one species and the first of the next fails this);
    # rho Y_e is advected as without the terms.
    pb = species_vterms_problem(couple=0, dims=dims)
    s = species_vterms_state(pb)
    dt = 0.3 / max(pb.n[:dims]) / pb.c_light
    out, st = oracle.run(pb, s, dt, 4)
    assert st == 0
    N, G, Gs, D = pb.ncell, pb.nchan, pb.ngroups, pb.dims
    NG = 2 + D
    rad = s[NG * N:(NG + (1 + D) * G) * N].reshape(1 + D, N, G)
    rad_out = out[NG * N:(NG + (1 + D) * G) * N].reshape(1 + D, N, G)
    moved = 0.0
    for sp in range(3):
        one = W.Problem(**{**pb.__dict__, "species": 1, "xi0": 0.0})
        s1 = np.concatenate([s[:NG * N], rad[:, :, sp * Gs:(sp + 1) * Gs].reshape(-1)])
        o1, st1 = oracle.run(one, s1, dt, 4)
        assert st1 == 0
        np.testing.assert_array_equal(o1[:NG * N], out[:NG * N])
        np.testing.assert_allclose(o1[NG * N:], rad_out[:, :, sp * Gs:(sp + 1) * Gs].reshape(-1),
                                   rtol=1e-14, atol=1e-14 * np.abs(o1[NG * N:]).max())
        moved = max(moved, np.abs(o1[NG * N:] - s1[NG * N:]).max())
    assert moved > 1e-3
    pb0 = W.Problem(**{**pb.__dict__, "vterms": 0})
    out0, _ = oracle.run(pb0, s, dt, 4)
    np.testing.assert_array_equal(out0[-N:], out[-N:])  # rho Y_e: the terms leave it alone
    assert np.abs(out0[NG * N:-N] - out[NG * N:-N]).max() > 1e-3 * np.abs(out[NG * N:-N]).max()


def test_species_with_velocity_terms_close_the_energy_budget():
    # the interaction on: total energy changes only by the flux-absorption work, the E floor and
    # the radiation energy the velocity terms add (reading R13; periodic grid)
    pb = species_vterms_problem(couple=1)
    s = species_vterms_state(pb, seed=3)  # (some random states have cells the Newton cannot solve)
    dt = 0.3 / max(pb.n[:2]) / pb.c_light
    out, st, bud = oracle.run_budget(pb, s, dt, 4)
    assert st == 0
    t0, t1 = oracle.totals(pb, s), oracle.totals(pb, out)
    assert abs(bud[8]) > 1e-6 * abs(t0[4])
    assert abs(t0[4] - t1[4] - bud[6] + bud[7] + bud[8]) <= 1e-13 * abs(t0[4])
