"""fx_step's captured step graphs against direct launches.

fx_step replays one captured CUDA graph per step unless per-kernel timing or the objective is
on; with timing on it launches the kernels one by one.  Both must give the same state bit for
bit, on a grid with boundary layers (their time advances on the device), on the three-species
form with the velocity terms and the budgets, and across a change of dt (a new capture).
"""
import numpy as np
import pytest

from paper_1806_07390_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fxmod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07390_gb300 import build, fx
    build.build()
    return fx


def run(fxmod, pb, s0, steps, direct, layers=None, budgets=False):
    g = fxmod.Grid(pb)
    g.upload(s0)
    if layers:
        g.boundary_layers(layers)
    if budgets:
        g.budgets_enable(True)
    g.kernel_timing(direct)  # per-kernel timing launches the kernels one by one
    for dt, n in steps:
        g.step(dt, n)
    g.kernel_timing(False)
    st = g.status()
    out = g.download()
    bud = g.budgets() if budgets else None
    g.close()
    return out, st, bud


@pytest.mark.parametrize("precision", ["fp64", "fp32n64"])
def test_graph_replay_with_boundary_layers(fxmod, precision):
    import oracle
    pb, prim, layers = W.double_mach(nx=64, ny=20, t_end=0.01, precision=precision)
    s0 = oracle.init_equilibrium(pb, prim)
    steps = [(pb.dt, 3), (0.5 * pb.dt, 2), (pb.dt, 1)]
    a, sa, _ = run(fxmod, pb, s0, steps, direct=False, layers=layers)
    b, sb, _ = run(fxmod, pb, s0, steps, direct=True, layers=layers)
    assert sa == 0 and sb == 0
    assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_replay_three_species_with_budgets(fxmod, precision):
    from tests.test_oracle_ye import species_vterms_problem, species_vterms_state
    pb = species_vterms_problem(couple=1)
    pb.precision = precision
    s0 = species_vterms_state(pb, seed=3)
    dt = 0.3 / max(pb.n[:2]) / pb.c_light
    steps = [(dt, 2), (dt, 2)]
    a, sa, ba = run(fxmod, pb, s0, steps, direct=False, budgets=True)
    b, sb, bb = run(fxmod, pb, s0, steps, direct=True, budgets=True)
    assert sa == 0 and sb == 0
    assert np.array_equal(a, b)
    np.testing.assert_allclose(ba, bb, rtol=1e-12, atol=1e-300)  # (atomic sums: order may differ)
