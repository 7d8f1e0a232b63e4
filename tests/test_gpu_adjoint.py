"""Objective and adjoint of the CUDA path against the FP64 oracle (through the C ABI).

Bars: J of the FP64 path within 1e-12 of the oracle's; gradients of the FP64 adjoint within
1e-6 (relative) of the oracle's tangent-linear (dual-number) run in a dot-product test, and within
1e-4 of central differences of the oracle taken where no branch flips within +-h.  The FP32
forms' gradients are held to the same bars (measured: 1e-8 to 1.2e-7 against the tangent-linear
run).
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


def beam_case(shape=(24, 20), G=4, precision="fp64"):
    pb, prim = W.blobs_2d(shape=shape, ngroups=G, nsteps=6, precision=precision)
    pb64, _ = W.blobs_2d(shape=shape, ngroups=G, nsteps=6, precision="fp64")
    s = W.streaming_flux(pb64, oracle.init_equilibrium(pb64, prim), 0.5)
    return pb, pb64, s


def gpu_adjoint(fxmod, pb, s, nsteps, k):
    g = fxmod.Grid(pb)
    g.upload(np.asarray(s, dtype=np.float64))
    J, gs, gr, dk = g.adjoint(pb.dt, nsteps, k)
    after = g.download()
    g.close()
    return J, gs.double().cpu().numpy(), gr.double().cpu().numpy(), dk, after


def test_objective_matches_oracle_fp64(fxmod):
    pb, pb64, s = beam_case()
    _, Jr, _, _, _ = oracle.run_objective(pb64, s, pb.dt, 6)
    g = fxmod.Grid(pb)
    g.upload(s)
    g.objective(True)
    g.step(pb.dt, 6)
    J = g.boundary_energy_out()
    assert g.launches_per_step() == 8  # per stage: gas faces, radiation/update, interaction, objective
    g.objective(False)
    g.close()
    assert Jr > 0
    assert abs(J - Jr) <= 1e-12 * abs(Jr)
    Ja, *_ = gpu_adjoint(fxmod, pb, s, 6, 4)
    assert abs(Ja - Jr) <= 1e-12 * abs(Jr)


def _random_tangent(pb, s, seed):
    rng = np.random.default_rng(seed)
    N, D, G = pb.ncell, pb.dims, pb.ngroups
    NG = 2 + D
    t = np.zeros_like(s)
    gas = np.abs(s[:NG * N]).reshape(NG, N).mean(1)
    t[:NG * N] = (rng.uniform(-1, 1, (NG, N)) * gas[:, None]).reshape(-1)
    rad = np.abs(s[NG * N:]).reshape(1 + D, N * G).mean(1)
    t[NG * N:] = (rng.uniform(-1, 1, (1 + D, N * G)) * rad[:, None]).reshape(-1)
    return t


def test_adjoint_matches_tangent_linear_fp64(fxmod):
    # dot-product test on a generic random state (no degenerate stencils, so the GPU and the
    # oracle take the same branches): <dJ/dU^0, dU> + dJ/dkappa0 dk against the oracle's
    # dual-number tangent for random full-state directions
    pb, _ = W.blobs_2d(shape=(24, 20), ngroups=4, nsteps=4, precision="fp64")
    s = W.random_state(pb, seed=9, flux_frac=0.5)
    J, gs, gr, dk, after = gpu_adjoint(fxmod, pb, s, 4, 3)
    assert np.array_equal(after, s)  # the handle's state is left unchanged
    for seed in (1, 2):
        t = _random_tangent(pb, s, seed)
        dkap = 0.3 * pb.kappa0
        _, Jr, dJ, _, _ = oracle.run_objective(pb, s, pb.dt, 4, tangent=t, dkappa0=dkap)
        assert abs(J - Jr) <= 1e-12 * abs(Jr)
        got = float(gs @ t) + dk * dkap
        assert abs(got - dJ) <= 1e-6 * abs(dJ), (got, dJ)
    N = pb.ncell
    drho = np.random.default_rng(3).uniform(-1, 1, N) * s[:N]
    _, _, dJ, _, _ = oracle.run_objective(pb, s, pb.dt, 4, tangent=H.rho_tangent(pb, s, drho))
    assert abs(float(gr @ drho) - dJ) <= 1e-6 * abs(dJ)


def test_adjoint_on_the_blob_screen_fp64(fxmod):
    # the blob workload with a beam along +x.  Its uniform medium makes every stencil there
    # degenerate (near-ties of the limiters), so only directions that keep that pattern have a
    # well-defined derivative: scaling the blob amplitudes (drho = rho - 1) and kappa0.
    pb, pb64, s = beam_case()
    J, gs, gr, dk, _ = gpu_adjoint(fxmod, pb, s, 6, 4)
    N = pb.ncell
    drho = s[:N] - 1.0
    dkap = 0.3 * pb.kappa0
    _, _, dJ, _, _ = oracle.run_objective(pb64, s, pb.dt, 6, tangent=H.rho_tangent(pb64, s, drho),
                                          dkappa0=dkap)
    got = float(gr @ drho) + dk * dkap
    assert abs(got - dJ) <= 1e-6 * abs(dJ), (got, dJ)


def test_adjoint_is_independent_of_the_checkpoint_interval(fxmod):
    pb, _, s = beam_case((20, 16), 3)
    ref = gpu_adjoint(fxmod, pb, s, 5, 5)
    for k in (1, 2, 3):
        J, gs, gr, dk, _ = gpu_adjoint(fxmod, pb, s, 5, k)
        assert J == ref[0]
        assert np.max(np.abs(gs - ref[1])) <= 1e-12 * np.max(np.abs(ref[1]))
        assert abs(dk - ref[3]) <= 1e-12 * abs(ref[3])


def test_adjoint_matches_central_differences_fp64(fxmod):
    # random generic state (no degenerate stencils); +-h runs must take identical branches
    pb, _ = W.blobs_2d(shape=(16, 12), ngroups=3, nsteps=3, precision="fp64")
    s = W.random_state(pb, seed=5, flux_frac=0.5)
    N = pb.ncell
    J, gs, gr, dk, _ = gpu_adjoint(fxmod, pb, s, 3, 2)
    drho = np.random.default_rng(11).uniform(-1, 1, N) * s[:N]
    h = 1e-6
    Jp = oracle.run_objective(pb, H.with_rho(pb, s, s[:N] + h * drho), pb.dt, 3, signature=True)
    Jm = oracle.run_objective(pb, H.with_rho(pb, s, s[:N] - h * drho), pb.dt, 3, signature=True)
    assert Jp[3] == Jm[3]
    fd = (Jp[1] - Jm[1]) / (2 * h)
    assert abs(float(gr @ drho) - fd) <= 1e-4 * abs(fd)
    k0 = pb.kappa0
    pb.kappa0 = k0 * (1 + h)
    Jp = oracle.run_objective(pb, s, pb.dt, 3, signature=True)
    pb.kappa0 = k0 * (1 - h)
    Jm = oracle.run_objective(pb, s, pb.dt, 3, signature=True)
    pb.kappa0 = k0
    assert Jp[3] == Jm[3]
    fd = (Jp[1] - Jm[1]) / (2 * h * k0)
    assert abs(dk - fd) <= 1e-4 * abs(fd)


@pytest.mark.parametrize("form", ["fp32", "fp32n64"])
def test_adjoint_fp32_form_matches_tangent_linear(fxmod, form):
    pb, pb64, s = beam_case(precision=form)
    J, gs, gr, dk, _ = gpu_adjoint(fxmod, pb, s, 6, 3)
    _, Jr, _, _, _ = oracle.run_objective(pb64, s, pb.dt, 6)
    assert abs(J - Jr) <= 1e-5 * abs(Jr)
    N = pb.ncell
    drho = s[:N] - 1.0
    dkap = 0.3 * pb.kappa0
    _, _, dJ, _, _ = oracle.run_objective(pb64, s, pb.dt, 6, tangent=H.rho_tangent(pb64, s, drho),
                                          dkappa0=dkap)
    got = float(gr @ drho) + dk * dkap
    assert abs(got - dJ) <= 1e-6 * abs(dJ), (got, dJ)
    # generic random state, full-state direction
    pb2, _ = W.blobs_2d(shape=(24, 20), ngroups=4, nsteps=4, precision=form)
    s2 = W.random_state(pb2, seed=9, flux_frac=0.5)
    J, gs, gr, dk, _ = gpu_adjoint(fxmod, pb2, s2, 4, 2)
    pb2.precision = "fp64"
    t = _random_tangent(pb2, s2, 1)
    _, _, dJ, _, _ = oracle.run_objective(pb2, s2, pb2.dt, 4, tangent=t, dkappa0=dkap)
    got = float(gs @ t) + dk * dkap
    assert abs(got - dJ) <= 1e-6 * abs(dJ), (got, dJ)


@pytest.mark.parametrize("form", ["fp32", "fp32n64"])
def test_adjoint_fp32_form_matches_central_differences(fxmod, form):
    # the FP32 form's gradients against central differences of the FP64 oracle (+-h runs with
    # identical branch signatures), density direction and kappa0
    pb, _ = W.blobs_2d(shape=(16, 12), ngroups=3, nsteps=3, precision=form)
    s = W.random_state(pb, seed=5, flux_frac=0.5)
    N = pb.ncell
    J, gs, gr, dk, _ = gpu_adjoint(fxmod, pb, s, 3, 2)
    pb.precision = "fp64"
    drho = np.random.default_rng(11).uniform(-1, 1, N) * s[:N]
    h = 1e-6
    Jp = oracle.run_objective(pb, H.with_rho(pb, s, s[:N] + h * drho), pb.dt, 3, signature=True)
    Jm = oracle.run_objective(pb, H.with_rho(pb, s, s[:N] - h * drho), pb.dt, 3, signature=True)
    assert Jp[3] == Jm[3]
    fd = (Jp[1] - Jm[1]) / (2 * h)
    assert abs(float(gr @ drho) - fd) <= 1e-4 * abs(fd)
    k0 = pb.kappa0
    pb.kappa0 = k0 * (1 + h)
    Jp = oracle.run_objective(pb, s, pb.dt, 3, signature=True)
    pb.kappa0 = k0 * (1 - h)
    Jm = oracle.run_objective(pb, s, pb.dt, 3, signature=True)
    pb.kappa0 = k0
    assert Jp[3] == Jm[3]
    fd = (Jp[1] - Jm[1]) / (2 * h * k0)
    assert abs(dk - fd) <= 1e-4 * abs(fd)


def test_autograd_function_matches_the_adjoint(fxmod):
    import torch

    from paper_1806_07390_gb300.autograd import boundary_outflow
    pb, pb64, s = beam_case((20, 16), 3)
    g = fxmod.Grid(pb)
    N = pb.ncell
    rho0 = torch.tensor(s[:N], dtype=torch.float64, device="cuda", requires_grad=True)
    k0 = torch.tensor(pb.kappa0, dtype=torch.float64, requires_grad=True)
    J = boundary_outflow(g, s, rho0, k0, pb.dt, 5, 2)
    (3.0 * J).backward()
    g2 = fxmod.Grid(pb)
    g2.upload(s)
    J2, gs, gr, dk = g2.adjoint(pb.dt, 5, 2)
    assert abs(float(J.detach()) - J2) <= 1e-14 * abs(J2)
    assert torch.allclose(rho0.grad, 3.0 * gr, rtol=1e-12, atol=0)
    assert abs(float(k0.grad) - 3.0 * dk) <= 1e-12 * abs(dk)
    # a different density through set_density reproduces a fresh upload
    rho1 = rho0.detach() * 1.01
    J3 = boundary_outflow(g, s, rho1, k0.detach(), pb.dt, 5, 2)
    _, J4, _, _, _ = oracle.run_objective(pb64, H.with_rho(pb64, s, s[:N] * 1.01), pb.dt, 5)
    assert abs(float(J3) - J4) <= 1e-12 * abs(J4)
    g.close()
    g2.close()
