"""Pins of the oracle's velocity-dependent radiation terms (Sec. 3.2, the group form of the moment
equations; Sec. 5.2, the volume-averaged velocity gradient and the upwind frequency fluxes;
Step 2 of Sec. 6; readings R23-R28).

Every test runs on the CPU and checks the oracle against something other than itself: exact
identities of the continuous terms (the frequency fluxes telescope, so only the work terms change
the group sums), spectra for which the discrete scheme is exact (spectral densities linear in
frequency), closed-form solutions of the frequency-advection equation (homologous compression
of a Planck spectrum, the flux spectrum in the diffusion limit), a linear velocity field, and the
Doppler-shift test of Sec. 9 with the error bounds the paper prints.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_07390_gb300 import workloads as W


def cell_problem(D, G, c=1.0, eps_min=1e-3, eps_max=60.0):
    n = (4, 4 if D > 1 else 1, 4 if D > 2 else 1)
    return W.Problem(name="vt", dims=D, n=n, x_lo=(0, 0, 0), x_hi=(1, 1, 1),
                     bc_lo=("outflow",) * 3, bc_hi=("outflow",) * 3, ngroups=G, gamma=5 / 3,
                     kappa0=0.0, kap_rho_exp=0.0, kap_T_exp=0.0, kap_eps_exp=0.0, c_light=c,
                     couple=0, vterms=1, eps_min=eps_min, eps_max=eps_max)


def log_edges(pb):
    return pb.eps_min * (pb.eps_max / pb.eps_min) ** (np.arange(pb.ngroups + 1) / pb.ngroups)


def planck_bands(pb, edges, T=1.0, scale=1.0):
    """B_g(T) over the band [scale*lo, scale*hi] (R14's group integral of the Planck spectrum)."""
    norm = pb.a_rad * 15.0 / math.pi ** 4 * T ** 4
    return np.array([norm * oracle.lib().orc_planck_band(scale * edges[g] / T, scale * edges[g + 1] / T)
                     for g in range(len(edges) - 1)])


def closure_P(D, c, E, F):
    """Full M1 pressure tensor from the pinned normal rows (R7)."""
    return np.array([oracle.m1_pressure_row(D, c, E, F, n) for n in range(D)])


# ------------------------------------------------------------------ identities of the terms
@pytest.mark.parametrize("D", [1, 2, 3])
def test_group_sums_change_only_by_the_work_terms(D):
    # The frequency fluxes of nu P and nu Q telescope over the groups (none through the range
    # ends), so summed over groups the E equation changes by -v^i_;j sum_g P^j_gi and the F_j
    # equation by -v^i_;j sum_g F_gi: exact for any field, any f and any (non-symmetric) V.
    G, c = 7, 3.0
    pb = cell_problem(D, G, c=c)
    rng = np.random.default_rng(5)
    V = rng.uniform(-1.0, 1.0, (D, D))
    rad = np.zeros((G, 1 + D))
    rad[:, 0] = rng.uniform(0.5, 2.0, G)
    for g in range(G):
        n = rng.standard_normal(D)
        rad[g, 1:] = rng.uniform(0.0, 0.95) * c * rad[g, 0] * n / np.linalg.norm(n)
    out, dEsum = oracle.vterms(pb, V, rad)
    Psum = sum(closure_P(D, c, rad[g, 0], rad[g, 1:]) for g in range(G))
    Fsum = rad[:, 1:].sum(axis=0)
    scale = np.abs(V).max() * rad[:, 0].sum()
    assert abs(out[:, 0].sum() + np.sum(V * Psum)) <= 1e-13 * scale
    assert abs(dEsum - out[:, 0].sum()) <= 1e-13 * scale
    # dF_j = -sum_i V_ij F_i: the transpose of V would fail this for D > 1
    np.testing.assert_allclose(out[:, 1:].sum(axis=0), -(V.T @ Fsum), rtol=0, atol=1e-13 * c * scale)


def test_zero_velocity_gradient_gives_zero():
    pb = cell_problem(3, 5)
    rad = np.abs(np.random.default_rng(1).standard_normal((5, 4)))
    out, s = oracle.vterms(pb, np.zeros((3, 3)), rad)
    assert np.all(out == 0.0) and s == 0.0


@pytest.mark.parametrize("D", [1, 2, 3])
def test_linear_spectral_densities_are_advected_exactly(D):
    # For spectral densities linear in nu, the limited linear reconstruction is exact on interior
    # groups (the three slopes agree), so a group whose two edges both lie between interior
    # groups gets exactly the group integral of
    # the continuous terms.  In the diffusion limit (f ~ 1e-5) P = E/3 delta + O(f^2) and, by R23,
    # Q_kji = (F_k d_ji + F_j d_ki + F_i d_kj)/5 + O(f^3), so with e(nu) = a + b nu, F(nu) =
    # (a' + b' nu) u:
    #   dE_g/dt = -(tr V / 3) E_g + (tr V / 3) [nu e(nu)]_{lo}^{hi}
    #   dF_gj/dt = -(V^T F_g)_j + [nu (M F(nu))_j]_{lo}^{hi},  M = (V + tr V I + V^T) / 5.
    G, c = 12, 2.0
    pb = cell_problem(D, G, c=c, eps_min=1.0, eps_max=5.0)
    e = log_edges(pb)
    rng = np.random.default_rng(7 + D)
    V = rng.uniform(-1.0, 1.0, (D, D))
    u = rng.standard_normal(D)
    u /= np.linalg.norm(u)
    a, b, af, bf = 3.0, -0.4, 2e-5, 1e-5
    dens_E = lambda nu: a + b * nu                 # noqa: E731
    dens_F = lambda nu: c * (af + bf * nu)         # noqa: E731
    integ = lambda f0, f1, lo, hi: f0 * (hi - lo) + 0.5 * f1 * (hi * hi - lo * lo)  # noqa: E731
    rad = np.zeros((G, 1 + D))
    for g in range(G):
        rad[g, 0] = integ(a, b, e[g], e[g + 1])
        rad[g, 1:] = c * integ(af, bf, e[g], e[g + 1]) * u
    out, _ = oracle.vterms(pb, V, rad)
    trV = np.trace(V)
    M = (V + trV * np.eye(D) + V.T) / 5.0
    for g in range(2, G - 2):  # both edges between two interior groups (end groups: zero slope)
        lo, hi = e[g], e[g + 1]
        dE = -(trV / 3) * rad[g, 0] + (trV / 3) * (hi * dens_E(hi) - lo * dens_E(lo))
        dF = -(V.T @ rad[g, 1:]) + (hi * dens_F(hi) - lo * dens_F(lo)) * (M @ u)
        assert abs(out[g, 0] - dE) <= 1e-7 * abs(rad[g, 0]), g
        np.testing.assert_allclose(out[g, 1:], dF, rtol=0, atol=1e-6 * np.abs(rad[g, 1:]).max())


# ------------------------------------------------------------------ closed-form spectra
def integrate_cell(pb, V, rad, t, nsteps):
    """SSP-RK2 in time of d rad/dt = (velocity terms), the scheme the step uses."""
    h = t / nsteps
    for _ in range(nsteps):
        k1, _ = oracle.vterms(pb, V, rad)
        r1 = rad + h * k1
        k2, _ = oracle.vterms(pb, V, r1)
        rad = 0.5 * rad + 0.5 * (r1 + h * k2)
    return rad


@pytest.mark.parametrize("lam", [-0.6, 0.6])
def test_homologous_flow_shifts_a_planck_spectrum(lam):
    # Isotropic radiation (F = 0, P = E/3) in a 1-d flow with dv/dx = lam: the E equation is
    # dE_nu/dt = (lam/3) nu dE_nu/dnu, solved by E_nu(t) = E_nu(0)(nu b), b = exp(lam t/3):
    # compression (lam < 0) shifts the spectrum up and adds energy, expansion the reverse.  Group
    # form: E_g(t) = B_[b lo, b hi] / b.  The total follows exp(-lam t/3) up to the RK2 error
    # alone; the groups converge to the closed form as the groups are refined.
    t = 1.0
    errs = []
    for G in (24, 48, 96):
        pb = cell_problem(1, G, eps_min=1e-2, eps_max=40.0)
        e = log_edges(pb)
        rad = np.zeros((G, 2))
        rad[:, 0] = planck_bands(pb, e)
        out = integrate_cell(pb, np.array([[lam]]), rad, t, 400)
        b = math.exp(lam * t / 3)
        ref = planck_bands(pb, e, scale=b) / b
        q = lam * t / 3 / 400
        assert abs(out[:, 0].sum() - rad[:, 0].sum() * (1 - q + 0.5 * q * q) ** 400) <= 1e-12 * rad[:, 0].sum()
        assert np.all(out[:, 1] == 0.0)
        errs.append(np.abs(out[:, 0] - ref).max() / ref.max())
    # first order at the spectrum's peak, where the limiter clips, second order elsewhere
    assert errs[2] < 5e-3, errs
    assert errs[0] / errs[1] > 2.0 and errs[1] / errs[2] > 2.0, errs


@pytest.mark.parametrize("lam", [-0.5, 0.5])
def test_flux_spectrum_in_the_diffusion_limit(lam):
    # With f << 1 (R23: Q = 3F/5 in 1-d) the F equation is dF_nu/dt = -lam F_nu + (3 lam/5)
    # d(nu F_nu)/dnu, solved by F_nu(t) = exp(-2 lam t/5) F_nu(0)(nu b), b = exp(3 lam t/5); the
    # total decays as exp(-lam t).  A closure with another diffusion-limit coefficient, or
    # without the heat-flux fluxes, fails the group comparison.
    t, f0, c = 1.0, 1e-5, 1.0
    errs = []
    for G in (24, 48, 96):
        pb = cell_problem(1, G, c=c, eps_min=1e-2, eps_max=40.0)
        e = log_edges(pb)
        rad = np.zeros((G, 2))
        rad[:, 0] = planck_bands(pb, e)
        rad[:, 1] = f0 * c * rad[:, 0]
        out = integrate_cell(pb, np.array([[lam]]), rad, t, 400)
        b = math.exp(3 * lam * t / 5)
        ref = math.exp(-2 * lam * t / 5) * f0 * c * planck_bands(pb, e, scale=b) / b
        assert abs(out[:, 1].sum() / rad[:, 1].sum() - math.exp(-lam * t)) < 1e-5
        errs.append(np.abs(out[:, 1] - ref).max() / ref.max())
    assert errs[2] < 1e-2, errs
    assert errs[0] / errs[1] > 2.0 and errs[1] / errs[2] > 2.0, errs


# ------------------------------------------------------------------ velocity gradient (R24-R25)
@pytest.mark.parametrize("D", [2, 3])
def test_velocity_gradient_of_a_linear_field(D):
    # Uniform rho and p with v = A x + v0: the parabolic reconstruction is exact on linear data,
    # HLLC of two equal states has v* = the normal velocity, and the upwind state carries the
    # transverse one, so every cell at least two cells from the boundary gets <v^i_,j> = A_ij.
    n = (9, 8, 7)[:D]
    pb = W.Problem(name="lin", dims=D, n=tuple(n) + (1,) * (3 - D), x_lo=(0, 0, 0), x_hi=(1, 1.2, 0.8),
                   bc_lo=("outflow",) * 3, bc_hi=("outflow",) * 3, ngroups=2, gamma=1.4,
                   kappa0=0.0, kap_rho_exp=0.0, kap_T_exp=0.0, kap_eps_exp=0.0, c_light=5.0,
                   couple=0, vterms=1)
    rng = np.random.default_rng(3)
    A = rng.uniform(-0.3, 0.3, (D, D))
    v0 = rng.uniform(-0.2, 0.2, D)
    xs = [pb.cell_centres(d) for d in range(D)]
    X = np.meshgrid(*xs[::-1], indexing="ij")[::-1]  # X[d] over (z, y, x) cell order
    vel = [v0[i] + sum(A[i, j] * X[j] for j in range(D)) for i in range(D)]
    N = pb.ncell
    s = np.zeros(pb.state_size())
    s[:N] = 1.3
    ke = 0
    for i in range(D):
        s[(1 + i) * N:(2 + i) * N] = 1.3 * vel[i].ravel()
        ke = ke + 0.5 * 1.3 * vel[i].ravel() ** 2
    s[(1 + D) * N:(2 + D) * N] = 2.0 / (pb.gamma - 1) + ke
    s[(2 + D) * N:(2 + D) * N + N * pb.ngroups] = 0.3
    vg = oracle.vgrad(pb, s).reshape(tuple(n[::-1]) + (3, 3))
    inner = tuple(slice(2, m - 2) for m in n[::-1])
    got = vg[inner][..., :D, :D]
    np.testing.assert_allclose(got, np.broadcast_to(A, got.shape), rtol=0, atol=1e-12)


@pytest.mark.parametrize("u0", [0.25, -0.25])
def test_transverse_face_velocity_is_the_upwind_one(u0):
    # A shear layer: uniform rho, p and v_x = u0, v_y jumping from a to b across x = 0.5.  The
    # x faces' Riemann problems are contacts moving with u0, and the HLLC face state carries the
    # transverse velocity of the side it is taken from: its y-momentum flux over its mass flux.
    # So <dv_y/dx> is (v_face - a)/dx in the cell left of the layer and (b - v_face)/dx right of
    # it, with v_face from the gas flux itself (left state for u0 > 0, right for u0 < 0).
    nx, ny, a, b = 10, 4, 0.1, -0.3
    pb = W.Problem(name="shear", dims=2, n=(nx, ny, 1), x_lo=(0, 0, 0), x_hi=(1, 1, 1),
                   bc_lo=("outflow", "periodic", "periodic"), bc_hi=("outflow", "periodic", "periodic"),
                   ngroups=2, gamma=1.4, kappa0=0.0, kap_rho_exp=0.0, kap_T_exp=0.0,
                   kap_eps_exp=0.0, c_light=5.0, couple=0, vterms=1)
    N = pb.ncell
    x = np.tile(pb.cell_centres(0), ny)
    vy = np.where(x < 0.5, a, b)
    s = np.zeros(pb.state_size())
    s[:N], s[N:2 * N], s[2 * N:3 * N] = 1.0, u0, vy
    s[3 * N:4 * N] = 1.0 / (pb.gamma - 1) + 0.5 * (u0 * u0 + vy * vy)
    s[4 * N:4 * N + 2 * N] = 0.2
    fl, vs = oracle.hllc(2, pb.gamma, [1.0, 1.0, u0, a], [1.0, 1.0, u0, b])
    v_face = fl[2] / fl[0]
    assert abs(vs - u0) <= 1e-15 and abs(v_face - (a if u0 > 0 else b)) <= 1e-15
    vg = oracle.vgrad(pb, s).reshape(ny, nx, 3, 3)
    dx = 1.0 / nx
    np.testing.assert_allclose(vg[:, nx // 2 - 1, 1, 0], (v_face - a) / dx, rtol=0, atol=1e-12)
    np.testing.assert_allclose(vg[:, nx // 2, 1, 0], (b - v_face) / dx, rtol=0, atol=1e-12)
    assert np.abs(vg[:, nx // 2 - 1, 0, :]).max() <= 1e-12  # v_x uniform


def test_uniform_velocity_leaves_the_operator_unchanged():
    # v and p uniform (density and radiation vary): every face's Riemann problem is a contact
    # moving with v, so every face carries the same velocity, <v^i_;j> = 0 to round-off and the
    # velocity terms vanish; the rest of the operator is the one without them.
    pb, _ = W.blobs_2d(shape=(12, 10), ngroups=4, precision="fp64")
    pb.c_light, pb.couple = 4.0, 0
    s = W.random_state(pb, seed=5, flux_frac=0.4)
    N = pb.ncell
    rho = s[:N]
    u = np.array([0.3, -0.2])
    ke = 0.5 * rho * (u ** 2).sum()
    s[N:2 * N], s[2 * N:3 * N] = rho * u[0], rho * u[1]
    s[3 * N:4 * N] = 1.7 / (pb.gamma - 1) + ke
    r0 = oracle.rhs(pb, s)
    pb.vterms = 1
    r1 = oracle.rhs(pb, s)
    assert np.abs(oracle.vgrad(pb, s)).max() <= 1e-13
    np.testing.assert_allclose(r1, r0, rtol=0, atol=1e-13 * np.abs(r0).max())


def test_energy_budget_closes_with_the_velocity_terms():
    # Reading R13 with R27: the radiation energy the velocity terms add (not conserved in the
    # comoving frame) enters the total-energy budget beside the outflow and the coupling work.
    pb, _ = W.sod_1d(n=32, ngroups=5)
    pb.c_light, pb.vterms = 8.0, 1
    pb.dt = 0.2 / pb.n[0] / pb.c_light
    s = W.random_state(pb, seed=19, flux_frac=0.5)
    t0 = oracle.totals(pb, s)
    out, st, bud = oracle.run_budget(pb, s, pb.dt, 5)
    assert st == 0
    t1 = oracle.totals(pb, out)
    assert abs(bud[8]) > 1e3 * 1e-14 * abs(t0[4])
    assert abs(t0[0] - t1[0] - bud[0]) <= 1e-14 * abs(t0[0])
    assert abs(t0[4] - t1[4] - bud[4] - bud[6] + bud[7] + bud[8]) <= 1e-14 * abs(t0[4])


# ------------------------------------------------------------------ spherical grid (R34)
def sph_problem(nr, nth, G=2, vterms=1, c=50.0):
    return W.Problem(name="sphv", dims=2, n=(nr, nth, 1), x_lo=(0.0, 0.3, 0), x_hi=(math.log(10.0), math.pi - 0.3, 1),
                     bc_lo=("outflow",) * 3, bc_hi=("outflow",) * 3, ngroups=G, gamma=4 / 3, kappa0=0.0,
                     kap_rho_exp=0.0, kap_T_exp=0.0, kap_eps_exp=0.0, c_light=c, couple=0, geom="sph",
                     map1="exp", vterms=vterms, eps_min=1e-2, eps_max=40.0)


def sph_state(pb, vr, vt):
    nr, nth = pb.n[0], pb.n[1]
    N = nr * nth
    prim = np.stack([np.ones(N), np.ones(N), np.ravel(vr), np.ravel(vt), np.ones(N)])
    return oracle.init_equilibrium(pb, prim)


def test_spherical_velocity_gradient():
    # Homologous flow v = H r: grad v = H I (rr, theta-theta and phi-phi entries), exact up to
    # the reconstruction of v*; a uniform Cartesian flow v = v0 z: grad v = 0, every component
    # converging at second order in L1 (the TVD clip at the extremum of v_theta at the equator is
    # a local first-order error there)
    H, v0 = 0.3, 0.4
    ehom, euni = [], []
    for nr, nth in ((32, 16), (64, 32), (128, 64)):
        pb = sph_problem(nr, nth)
        r = np.exp(pb.cell_centres(0))[None, :] * np.ones((nth, 1))
        th = pb.cell_centres(1)[:, None] * np.ones((1, nr))
        vg = oracle.vgrad(pb, sph_state(pb, H * r, 0 * r)).reshape(nth, nr, 3, 3)[3:-3, 3:-3]
        ehom.append(max(np.abs(vg[..., a, a] / H - 1).max() for a in range(3)))
        assert np.abs(vg[..., 0, 1]).max() == 0.0 and np.abs(vg[..., 1, 0]).max() == 0.0
        vg = oracle.vgrad(pb, sph_state(pb, v0 * np.cos(th), -v0 * np.sin(th))).reshape(nth, nr, 3, 3)[3:-3, 3:-3]
        euni.append(np.abs(vg).mean() / v0)
    assert ehom[-1] < 2e-4 and ehom[0] / ehom[1] > 3.5 and ehom[1] / ehom[2] > 3.5, ehom
    assert euni[0] / euni[1] > 3.0 and euni[1] / euni[2] > 3.0, euni


def test_spherical_homologous_expansion():
    # A uniform Planck field in homologous flow v = H r (frozen gas, no opacity): the comoving
    # field stays uniform, cools as exp(-4 H t) (the divergence of vE gives 3 H, the work term
    # v:P = H E) and redshifts as E_nu(t) = exp(-3 H t) E_nu(0)(nu exp(H t)).  Measured before
    # light from either boundary reaches the cells at 3 < r < 6.
    H, t_end = 0.5, 0.1
    etot, espec = [], []
    for nr, nth, G in ((32, 8, 24), (64, 16, 48)):
        pb = sph_problem(nr, nth, G=G, c=20.0)
        r = np.exp(pb.cell_centres(0))
        s = sph_state(pb, H * r[None, :] * np.ones((nth, 1)), np.zeros((nth, nr)))
        dt = 0.2 * min(math.log(10) / nr, 0.3 * (math.pi - 0.6) / nth) / pb.c_light
        nst = int(math.ceil(t_end / dt))
        out, st = oracle.run(pb, s, t_end / nst, nst, nthreads=8, frozen_gas=1)
        assert st == 0
        N = pb.ncell
        E0 = s[4 * N:4 * N + N * G].reshape(nth, nr, G)
        E1 = out[4 * N:4 * N + N * G].reshape(nth, nr, G)
        e = log_edges(pb)
        b = math.exp(H * t_end)
        ref = planck_bands(pb, e, scale=b) / b * math.exp(-3 * H * t_end)
        Em = E1[nth // 2][(r > 3.0) & (r < 6.0)]
        etot.append(np.abs(Em.sum(-1) / E0[0, 0].sum() / math.exp(-4 * H * t_end) - 1).max())
        espec.append((np.abs(Em - ref[None, :]).max(-1) / ref.max()).max())
    assert etot[1] < 1e-4 and etot[0] / etot[1] > 3.5, etot
    assert espec[1] < 3e-3 and espec[0] / espec[1] > 2.5, espec


def test_lab_frame_flux_continuity_at_a_transparent_shock():
    # Sec. 9's continuity test: a steady point source (a radial beam entering at the inner
    # boundary), no opacity, and the imposed core-collapse-like velocity field with a standing
    # shock at r_s = 1 (v = -0.1 v_s r / r_s inside, v = -v_s (sqrt(r_max/r) - 1)/(sqrt(r_max/r_s)
    # - 1) outside, v_s = 0.1 c, r_max = 10 r_s; frozen gas).  The comoving r^2 E jumps at the
    # shock; Lorentz-transformed to the lab frame (E_lab = gamma^2 (E + 2 beta F/c + beta^2 P_rr))
    # it is flat to the first zone's value, as a transparent medium requires.  Two light-crossing
    # times on a log-r grid from 0.3 to 10 (96 cells) and a 4-cell equatorial wedge.
    c, vs, r_in, nr, nth = 1.0, 0.1, 0.3, 96, 4
    x0, x1 = math.log(r_in), math.log(10.0)
    pb = W.Problem(name="labflux", dims=2, n=(nr, nth, 1), x_lo=(x0, math.pi / 2 - 0.4, 0),
                   x_hi=(x1, math.pi / 2 + 0.4, 1), bc_lo=("outflow", "reflect", "periodic"),
                   bc_hi=("outflow", "reflect", "periodic"), ngroups=1, gamma=4 / 3, kappa0=0.0,
                   kap_rho_exp=0.0, kap_T_exp=0.0, kap_eps_exp=0.0, c_light=c, couple=0, geom="sph",
                   map1="exp", vterms=1)
    N, dx = pb.ncell, (x1 - x0) / nr
    r = np.exp(pb.cell_centres(0))
    v = np.where(r < 1.0, -0.1 * vs * r, -vs * (np.sqrt(10.0 / r) - 1) / (math.sqrt(10.0) - 1))
    prim = np.stack([np.ones(N), np.full(N, 1e-3), np.tile(v, nth), np.zeros(N), np.full(N, 1e-3)])
    s = oracle.init_equilibrium(pb, prim)
    s[4 * N:] = 0.0
    s[4 * N:5 * N] = 1e-8
    # the inflow ghosts: E = 1 and a beam's covariant flux h_1 c E, h_1 of the ghost next to the
    # boundary (log map: h_1^2 = (3/5)(e^{5b} - e^{5a})/(e^{3b} - e^{3a}) on [a, b])
    a, b = x0 - dx, x0
    h1g = math.sqrt(0.6 * (math.exp(5 * b) - math.exp(5 * a)) / (math.exp(3 * b) - math.exp(3 * a)))
    dt0 = 0.15 * r_in * dx / c
    nst = int(math.ceil(20.0 / dt0))
    out, st = oracle.run(pb, s, 20.0 / nst, nst, nthreads=8, inflow=np.array([1.0, 0.999 * c * h1g]),
                         frozen_gas=1)
    assert st == 0
    unit = np.array(prim, copy=True)
    unit[0], unit[2], unit[3] = 1.0, 1.0, 1.0
    h1 = oracle.init_equilibrium(pb, unit)[N:2 * N].reshape(nth, nr)[nth // 2]
    E = out[4 * N:5 * N].reshape(nth, nr)[nth // 2]
    F = out[5 * N:6 * N].reshape(nth, nr)[nth // 2] / h1
    f = np.clip(F / (c * E), 0.0, 1.0)
    chi = (3 + 4 * f * f) / (5 + 2 * np.sqrt(4 - 3 * f * f))
    beta = v / c
    Elab = (E + 2 * beta * F / c + beta ** 2 * chi * E) / (1 - beta ** 2)
    y, yl = r ** 2 * E, r ** 2 * Elab
    k = int(np.searchsorted(r, 1.0))  # first cell outside the shock
    inside, outside = slice(k - 5, k - 2), slice(k + 2, k + 5)
    jump = y[outside].mean() / y[inside].mean() - 1
    jump_lab = yl[outside].mean() / yl[inside].mean() - 1
    away = np.r_[0:k - 2, k + 2:nr]  # the shock's two cells on each side smear the profile
    flat = np.abs(yl[away] / yl[0] - 1).max()
    assert jump > 0.15, jump
    assert abs(jump_lab) < 0.02, jump_lab
    assert flat < 0.035, flat


# ------------------------------------------------------------------ Doppler-shift test (Sec. 9)
def doppler_run(ng_lin):
    """Sec. 9's Doppler-shift test (reading R28): 50 cells on [0, 10] cm, rho = 1, no opacity,
    v = A sin^2(pi x / 10) (0 at the left edge, A = 5e7 cm/s at the centre), c = 3e10 cm/s, a
    Planck beam at T = 1000 K entering at the left, ng_lin equal groups over h nu / kT in [0,
    9.60] (2e14 Hz) plus two groups for the rest of the spectrum (one more of the same width,
    then everything above), 10 light-crossing times.  Returns the comoving spectrum of the
    centre cell, the analytic one, the incident one and the centre cell's flux factors."""
    n, L = 50, 10.0
    c = 1.0  # time in units of L/c; velocities in units of c
    beta_a = 5e7 / 2.99792458e10
    xmax = 6.62607015e-34 * 2e14 / (1.380649e-23 * 1000.0)
    w = xmax / ng_lin
    edges = np.concatenate([np.linspace(0.0, xmax, ng_lin + 1), [xmax + w, 60.0]])
    G = len(edges) - 1
    pb = W.Problem(name="doppler", dims=1, n=(n, 1, 1), x_lo=(0, 0, 0), x_hi=(L, 1, 1),
                   bc_lo=("outflow",) * 3, bc_hi=("outflow",) * 3, ngroups=G, gamma=5 / 3,
                   kappa0=0.0, kap_rho_exp=0.0, kap_T_exp=0.0, kap_eps_exp=0.0, c_light=c,
                   couple=0, vterms=1)
    B = planck_bands(pb, edges)
    x = (np.arange(n) + 0.5) * L / n
    v = beta_a * c * np.sin(np.pi * x / L) ** 2
    s = np.zeros(pb.state_size())
    s[:n] = 1.0
    s[n:2 * n] = v
    s[2 * n:3 * n] = 1.0 / (pb.gamma - 1) + 0.5 * v * v
    s[3 * n:3 * n + n * G] = np.tile(B, n)
    s[3 * n + n * G:] = np.tile(c * B, n)
    dt = 0.5 * (L / n) / c
    out, st = oracle.run(pb, s, dt, int(round(10 * L / c / dt)), edges=edges,
                         inflow=np.concatenate([B, c * B]), frozen_gas=1)
    assert st == 0
    ic = n // 2 - 1  # the cell whose centre is nearest the domain centre from the left
    E = out[3 * n:3 * n + n * G].reshape(n, G)[ic]
    F = out[3 * n + n * G:].reshape(n, G)[ic]
    beta = v[ic] / c
    Dop = math.sqrt((1 + beta) / (1 - beta))
    # analytic: E_nu = (4 pi / c) B_nu at comoving frequencies Dop * nu, divided by Dop
    Ean = planck_bands(pb, edges, scale=Dop) / Dop ** 2
    mid = 0.5 * (edges[:-1] + edges[1:])
    return E[:ng_lin], Ean[:ng_lin], B[:ng_lin], F[:ng_lin] / (c * E[:ng_lin]), mid[:ng_lin]


@pytest.mark.parametrize("ng_lin,away,near", [(20, 0.065, 0.23), (40, 0.0085, 0.056)])
def test_doppler_shift(ng_lin, away, near):
    # Sec. 9 prints, for the difference between the shifted spectrum at the centre and the
    # incident one, relative errors below 6.5 % (20 groups) and 0.85 % (40 groups) away from the
    # spectral peak (h nu ~ 2.82 kT), rising to 23 % and 5.6 % near it where the slope limiter
    # clips.  The error of each group is measured against the largest analytic difference (the
    # difference itself changes sign near h nu = 1.59 kT).  The last equal-width group is left
    # out: its upper neighbour's slope is clipped by the semi-infinite group above it.
    E, Ean, B, f, mid = doppler_run(ng_lin)
    dnum, dan = E - B, Ean - B
    err = np.abs(dnum - dan)[:-1] / np.abs(dan).max()
    nearpk = ((mid > 0.5 * 2.821) & (mid < 1.5 * 2.821))[:-1]
    print(f"{ng_lin} groups: away {err[~nearpk].max():.4f} near {err[nearpk].max():.4f}")
    assert err[~nearpk].max() <= away
    assert err[nearpk].max() <= near
    # a beam stays a beam: the heat-flux fluxes shift F exactly as the pressure fluxes shift E
    # when f = 1 (R23: q(1) = 1)
    assert np.abs(f - 1.0).max() <= 1e-9
