"""Pins of the oracle's boundary-outflow objective J (reading R19) and of its tangent.

J = sum over steps of dt (Phi(U^n) + Phi(U^(1)))/2, Phi = radiation energy flux through the
upper x boundary times the face area, summed over groups and faces: the outflow that the SSP-RK2
update itself applies (Sec. 4).  The pins below fix it by a closed form, by the radiation energy
budget of a conservative update, and its tangent (dual numbers) by central differences taken
only where no branch of the discrete map changes between the two runs.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1806_07390_gb300 import workloads as W
from tests import helpers as H


def _beam_problem(nx=12, ny=10, G=3):
    pb, prim = W.blobs_2d(shape=(nx, ny), ngroups=G, nsteps=3, precision="fp64")
    return pb, prim


def test_objective_of_a_uniform_beam_is_closed_form():
    # uniform gas at rest, uniform radiation with F = f c E along +x, no opacity: the state stays
    # uniform, every boundary face carries F (the HLL energy flux of identical states), v* = 0,
    # so J = nsteps dt (face area sum = L_y) sum_g F_g exactly
    pb, _ = _beam_problem()
    pb.kappa0 = 0.0
    pb.sigma0 = 0.0
    N, G = pb.ncell, pb.ngroups
    s = np.zeros(pb.state_size())
    s[:N] = 1.3
    s[3 * N:4 * N] = 0.8 / (pb.gamma - 1.0)
    E = np.array([0.7, 0.2, 0.05])
    rad = s[4 * N:].reshape(3, N, G)
    rad[0] = E
    rad[1] = 0.4 * pb.c_light * E
    nsteps = 4
    out, J, _, _, st = oracle.run_objective(pb, s, pb.dt, nsteps)
    assert st == 0
    Ly = pb.x_hi[1] - pb.x_lo[1]
    expect = nsteps * pb.dt * Ly * (0.4 * pb.c_light * E).sum()
    assert abs(J - expect) <= 1e-14 * expect
    assert np.max(np.abs(out - s)) <= 1e-13 * np.max(np.abs(s))


def test_objective_closes_the_radiation_energy_budget():
    # reflecting wall at x_lo (zero energy flux), outflow at x_hi, periodic y, no opacity and a
    # gas at rest: the conservative update changes the radiation energy only through the x_hi
    # faces, so E_rad(0) - E_rad(N) = J to round-off (a wrong RK weight, area or sign fails)
    pb, _ = _beam_problem(14, 9, 3)
    pb.kappa0 = 0.0
    pb.sigma0 = 0.0
    pb.bc_lo = ("reflect", "periodic", "periodic")
    N, G = pb.ncell, pb.ngroups
    rng = np.random.default_rng(7)
    s = np.zeros(pb.state_size())
    s[:N] = 1.0
    s[3 * N:4 * N] = 1.0 / (pb.gamma - 1.0)
    rad = s[4 * N:].reshape(3, N, G)
    rad[0] = rng.uniform(0.2, 1.0, (N, G))
    rad[1] = rng.uniform(-0.3, 0.6, (N, G)) * pb.c_light * rad[0]
    rad[2] = rng.uniform(-0.3, 0.3, (N, G)) * pb.c_light * rad[0]
    e0 = oracle.totals(pb, s)[5]
    out, J, _, _, st = oracle.run_objective(pb, s, pb.dt, 5)
    e1 = oracle.totals(pb, out)[5]
    assert st == 0
    assert abs(J) > 1e-3 * e0  # the budget is not trivially zero
    assert abs((e0 - e1) - J) <= 2e-14 * e0


def test_objective_is_zero_without_steps_and_matches_plain_run():
    pb, prim = _beam_problem()
    s = W.streaming_flux(pb, oracle.init_equilibrium(pb, prim), 0.5)
    out, J, dJ, _, _ = oracle.run_objective(pb, s, pb.dt, 0)
    assert J == 0.0 and dJ == 0.0 and np.array_equal(out, s)
    ref, _ = oracle.run(pb, s, pb.dt, 2)
    out, J, _, _, _ = oracle.run_objective(pb, s, pb.dt, 2)
    assert np.array_equal(out, ref) and J > 0.0


def _fd_and_tangent(pb, s, drho, dk, h, nsteps):
    t = H.rho_tangent(pb, s, drho)
    _, J, dJ, _, _ = oracle.run_objective(pb, s, pb.dt, nsteps, tangent=t, dkappa0=dk)
    N = pb.ncell
    rho = s[:N]
    sp = H.with_rho(pb, s, rho + h * drho)
    sm = H.with_rho(pb, s, rho - h * drho)
    k0 = pb.kappa0
    pb.kappa0 = k0 + h * dk
    _, Jp, _, sigp, _ = oracle.run_objective(pb, sp, pb.dt, nsteps, signature=True)
    pb.kappa0 = k0 - h * dk
    _, Jm, _, sigm, _ = oracle.run_objective(pb, sm, pb.dt, nsteps, signature=True)
    pb.kappa0 = k0
    return J, dJ, (Jp - Jm) / (2 * h), sigp == sigm


@pytest.mark.parametrize("direction", ["rho", "kappa0", "both"])
def test_objective_tangent_matches_central_differences(direction):
    # the dual-number tangent of J against (J(+h) - J(-h))/2h on a generic random state (no
    # degenerate stencils), taken only when both runs take identical branches, so that the
    # difference crosses no limiter, HLLC or Newton-fallback kink
    pb, _ = _beam_problem(12, 10, 3)
    s = W.random_state(pb, seed=5, flux_frac=0.5)
    N = pb.ncell
    rng = np.random.default_rng(11)
    drho = rng.uniform(-1.0, 1.0, N) * s[:N] if direction != "kappa0" else np.zeros(N)
    dk = pb.kappa0 if direction != "rho" else 0.0
    J, dJ, fd, same = _fd_and_tangent(pb, s, drho, dk, 1e-6, 3)
    assert same, "branch signature changed within +-h; pick another seed"
    assert abs(dJ) > 1e-6 * abs(J)
    assert abs(dJ - fd) <= 1e-6 * abs(dJ)


def test_objective_tangent_on_the_blob_screen():
    # the blob workload with a beam along +x: scaling the blob amplitudes (drho = rho - 1) keeps
    # every stencil of the uniform medium degenerate in the same way, so no branch flips
    pb, prim = _beam_problem(16, 12, 3)
    s = W.streaming_flux(pb, oracle.init_equilibrium(pb, prim), 0.5)
    N = pb.ncell
    drho = s[:N] - 1.0
    J, dJ, fd, same = _fd_and_tangent(pb, s, drho, 0.0, 1e-6, 4)
    assert same
    assert abs(dJ) > 1e-6 * abs(J)
    assert abs(dJ - fd) <= 1e-6 * abs(dJ)


@pytest.mark.parametrize("part", ["rho", "m", "rhoe", "E", "F"])
def test_objective_tangent_of_each_state_component(part):
    # the tangent along random perturbations of one block of conserved variables at a time
    pb, _ = _beam_problem(16, 12, 3)
    s = W.random_state(pb, seed=5, flux_frac=0.5)
    N, D, G = pb.ncell, pb.dims, pb.ngroups
    NG = 2 + D
    sl = {"rho": slice(0, N), "m": slice(N, (1 + D) * N), "rhoe": slice((1 + D) * N, NG * N),
          "E": slice(NG * N, NG * N + N * G), "F": slice(NG * N + N * G, None)}[part]
    t = np.zeros_like(s)
    rng = np.random.default_rng(1)
    t[sl] = rng.uniform(-1, 1, t[sl].size) * np.abs(s[sl]).mean()
    dJ = oracle.run_objective(pb, s, pb.dt, 3, tangent=t)[2]
    h = 1e-6
    Jp = oracle.run_objective(pb, s + h * t, pb.dt, 3, signature=True)
    Jm = oracle.run_objective(pb, s - h * t, pb.dt, 3, signature=True)
    assert Jp[3] == Jm[3]
    fd = (Jp[1] - Jm[1]) / (2 * h)
    assert abs(dJ - fd) <= 1e-7 * abs(fd)


def test_branch_signature_is_deterministic_and_sees_a_kink():
    pb, prim = _beam_problem(12, 10, 3)
    s = W.streaming_flux(pb, oracle.init_equilibrium(pb, prim), 0.5)
    a = oracle.run_objective(pb, s, pb.dt, 2, signature=True)[3]
    b = oracle.run_objective(pb, s, pb.dt, 2, signature=True)[3]
    assert a == b
    # turn a monotone density profile into a local extremum: the reconstruction branch changes
    N = pb.ncell
    s2 = np.array(s, copy=True)
    rho = s[:N].reshape(pb.shape)
    rho2 = rho.copy()
    rho2[5, 6] = 3.0 * rho.max()
    s2 = H.with_rho(pb, s, rho2.reshape(-1))
    c = oracle.run_objective(pb, s2, pb.dt, 2, signature=True)[3]
    assert c != a
