"""GPU parity of the boundary layers (reading R29) and of the double Mach reflection (Sec. 8.4)
with the FP64 oracle, through the C ABI.

The double Mach reflection runs at 130 x 40 cells to t = 0.05 (HLLC with the carbuncle guard,
and without it), FP64 at 1e-10 / 1e-8 and both FP32 forms at 1e-4 against the natural scales.
A 3-d box with a mirror layer, a fixed-state layer and a moving front exercises the layer kernel
in another geometry.
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


def run_gpu(fxmod, pb, s0, layers, t0=0.0):
    g = fxmod.Grid(pb)
    g.upload(s0)
    g.boundary_layers(layers, t0)
    g.step(pb.dt, pb.nsteps)
    st = g.status()
    out = g.download()
    nl = g.launches_per_step()
    g.close()
    return out, st, nl


@pytest.mark.parametrize("guard", [0.5, 0.0])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4), ("fp32n64", 1e-4)])
def test_double_mach_reflection(fxmod, precision, tol, guard):
    pb, prim, layers = W.double_mach(nx=130, ny=40, t_end=0.05, shock_guard=guard, precision=precision)
    s0 = oracle.init_equilibrium(pb, prim)
    ref, rst = oracle.run(pb, s0, pb.dt, pb.nsteps, nthreads=8, layers=layers)
    got, st, nl = run_gpu(fxmod, pb, s0, layers)
    assert st == 0 and rst == 0
    # per step: two stages of faces, radiation/update (+ shock flags with the guard), three
    # layer launches and the layers' time advance
    assert nl == 2 * (2 + (guard > 0)) + 4
    if precision == "fp64":
        H.assert_parity(pb, got, ref, tol, 1e-8)
    else:
        H.assert_parity(pb, got, ref, tol, natural=True)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32n64", 1e-4)])
def test_layers_in_3d(fxmod, precision, tol):
    pb, _ = W.lognormal_3d(shape=(12, 10, 9), ngroups=4, nsteps=3, precision=precision)
    pb.bc_lo = ("outflow", "outflow", "outflow")
    pb.bc_hi = ("outflow", "outflow", "outflow")
    pb.c_light = 5.0
    pb.dt = 0.3 / 12 / pb.c_light
    s = W.random_state(pb, seed=41, flux_frac=0.5)
    layers = [
        dict(kind="mirror", d=2, m=2, lo=(0, 0, 0), hi=(12, 10, 2)),
        dict(kind="front", lo=(0, 0, 4), hi=(2, 10, 9), x0=1e30, y0=0.0, cot_alpha=0.0, speed=0.0,
             A=(1.3, 0.9, 0.2, -0.1, 0.05, 0.8), B=(1.3, 0.9, 0.2, -0.1, 0.05, 0.8)),
        dict(kind="front", lo=(2, 8, 4), hi=(12, 10, 9), x0=0.3, y0=0.5, cot_alpha=0.7, speed=2.0,
             A=(2.0, 1.5, 0.3, 0.0, 0.0, 1.1), B=(0.8, 0.6, 0.0, 0.1, 0.0, 0.7)),
    ]
    ref, rst = oracle.run(pb, s, pb.dt, pb.nsteps, nthreads=8, layers=layers, t0=0.05)
    got, st, _ = run_gpu(fxmod, pb, s, layers, t0=0.05)
    assert st == 0 and rst == 0
    if precision == "fp64":
        H.assert_parity(pb, got, ref, tol, 1e-8)
    else:
        H.assert_parity(pb, got, ref, tol, natural=True)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_host_primitives_staged_in_chunks(fxmod, precision):
    # one group in FP32: a cell's five FP64 primitives need more room than its state row, so the
    # host primitives go through the scratch buffer in several chunks; the state equals the one
    # built from device primitives, and the oracle's
    import torch
    pb, prim, _ = W.double_mach(nx=64, ny=20, precision=precision)
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    host = g.download()
    g.init_equilibrium(torch.from_numpy(np.ascontiguousarray(prim)).cuda())
    dev = g.download()
    g.close()
    assert np.array_equal(host, dev)
    ref = oracle.init_equilibrium(pb, prim)
    tol = 1e-14 if precision == "fp64" else 1e-6
    np.testing.assert_allclose(host, ref, rtol=tol, atol=1e-30 * pb.a_rad)


def test_layer_validation_and_adjoint(fxmod):
    pb, prim, layers = W.double_mach(nx=26, ny=8, t_end=0.01)
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    bad = [[dict(layers[0], hi=(2, pb.n[1] + 1, 1))],                      # box outside the grid
           [layers[0], dict(layers[1], lo=(1, 0, 0))],                       # boxes overlap
           [dict(kind="mirror", d=1, m=1, lo=(4, 0, 0), hi=(8, 2, 1))]]      # mirror reads its box
    for b in bad:
        with pytest.raises(fxmod.FxError) as ei:
            g.boundary_layers(b)
        assert ei.value.status == -1
        g.L.fx_clear_error(g.h)
    g.boundary_layers(layers)
    ws = g.adjoint_workspace(2, 1)
    with pytest.raises(fxmod.FxError) as ei:
        g.adjoint_forward(ws, pb.dt, 2, 1)
    assert ei.value.status == -7
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32n64"])
def test_layers_follow_the_handle_to_a_new_workspace(fxmod, precision):
    # a handle bound again, to zeroed memory, sets its boundary layers there at the handle's
    # time: two steps, the new workspace with the state uploaded again, two more steps equal four
    # steps in one workspace bit for bit (zeroed memory without the layers would hold n = 0
    # layers and leave the boundary cells alone)
    import ctypes
    import torch
    pb, prim, layers = W.double_mach(nx=130, ny=40, t_end=0.05, precision=precision)
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    g.boundary_layers(layers)
    g.step(pb.dt, 4)
    assert g.status() == 0
    ref = g.download()
    g.close()
    g = fxmod.Grid(pb)
    g.init_equilibrium(prim)
    g.boundary_layers(layers)
    g.step(pb.dt, 2)
    mid = g.download()
    old = g.workspace
    ws2 = torch.zeros(g.ws_bytes, dtype=torch.uint8, device=old.device)
    g._check(g.L.fx_bind_workspace(g.h, ctypes.c_void_p(ws2.data_ptr()), g.ws_bytes,
                                   ctypes.c_void_p(g.stream.cuda_stream)))
    g.workspace = ws2
    g.upload(mid)
    g.step(pb.dt, 2)
    st = g.status()
    got = g.download()
    g.close()
    del old
    assert st == 0
    assert np.array_equal(got, ref)
