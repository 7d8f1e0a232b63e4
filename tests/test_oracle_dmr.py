"""Pins of the oracle's boundary layers (reading R29) and of the double Mach reflection workload
(Sec. 8.4).

- The pre- and post-shock states the paper prints satisfy the Rankine-Hugoniot conditions of a
  shock moving at 10 (Mach 10 in the pre-shock gas) normal to itself.
- Mirror layers reproduce the oracle's own reflecting boundary (Sec. 7.5) cell for cell.
- In the double Mach reflection the incident shock, away from the wall, stays at its exact
  position x0 + y cot(alpha) + 10 t / sin(alpha): the moving front of the top layer and the
  solver agree on the shock speed.
- Ahead of the reflected structures, the fixed post-shock layers keep the inflow region exactly
  at the post-shock state.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_07390_gb300 import workloads as W


def test_double_mach_states_satisfy_rankine_hugoniot():
    # shock normal n = (sin a, -cos a) (pointing into the pre-shock gas), speed 10 along n: mass,
    # normal momentum, tangential velocity and energy fluxes across the moving shock agree
    pb, _, layers = W.double_mach(nx=26, ny=8)
    post, pre = layers[3]["A"], layers[3]["B"]
    g = pb.gamma
    a = math.pi / 3
    n = np.array([math.sin(a), -math.cos(a)])
    s = 10.0

    def fluxes(st):
        rho, p, vx, vy = st[:4]
        un = np.dot([vx, vy], n) - s
        ut = vx * (-n[1]) + vy * n[0]
        e = p / (g - 1) / rho + 0.5 * un * un
        return np.array([rho * un, rho * un * un + p, ut, rho * un * (e + p / rho)])

    f1, f2 = fluxes(pre), fluxes(post)
    assert np.all(np.abs(f1 - f2) <= 1e-9 * np.abs(f1).max()), (f1, f2)
    # Mach 10 in the pre-shock gas (sound speed 1)
    assert abs(s / math.sqrt(g * pre[1] / pre[0]) - 10.0) < 1e-12


def test_mirror_layers_reproduce_the_reflecting_boundary():
    # the same problem with a native reflecting lower-y boundary and on a grid two rows taller
    # whose two bottom rows are mirror layers: every physical cell agrees to round-off
    nx, ny = 18, 14
    base, _ = W.blobs_2d(shape=(nx, ny), ngroups=3, precision="fp64")
    base.c_light, base.couple = 5.0, 1
    base.bc_lo = ("outflow", "reflect", "periodic")
    base.bc_hi = ("outflow", "outflow", "periodic")
    dy = (base.x_hi[1] - base.x_lo[1]) / ny
    s = W.random_state(base, seed=31, flux_frac=0.5)
    ext = W.Problem(**{**base.__dict__, "n": (nx, ny + 2, 1),
                       "x_lo": (base.x_lo[0], base.x_lo[1] - 2 * dy, 0.0),
                       "bc_lo": ("outflow", "outflow", "periodic")})
    # extended state: the base state in rows 2.., the layer rows filled by the layer itself
    N0, N1 = base.ncell, ext.ncell
    D, G = 2, base.ngroups
    se = np.zeros(ext.state_size())
    for v in range(2 + D):
        se[v * N1:(v + 1) * N1].reshape(ny + 2, nx)[2:] = s[v * N0:(v + 1) * N0].reshape(ny, nx)
    for v in range(1 + D):
        dst = se[(2 + D) * N1 + v * N1 * G:(2 + D) * N1 + (v + 1) * N1 * G].reshape(ny + 2, nx, G)
        dst[2:] = s[(2 + D) * N0 + v * N0 * G:(2 + D) * N0 + (v + 1) * N0 * G].reshape(ny, nx, G)
        dst[:2] = 1.0  # overwritten by the mirror before the first stage
    layers = [dict(kind="mirror", d=1, m=2, lo=(0, 0, 0), hi=(nx, 2, 1))]
    a, sa = oracle.run(base, s, base.dt, 4)
    b, sb = oracle.run(ext, se, base.dt, 4, layers=layers)
    assert sa == 0 and sb == 0
    for v in range(2 + D):
        ga = a[v * N0:(v + 1) * N0].reshape(ny, nx)
        gb = b[v * N1:(v + 1) * N1].reshape(ny + 2, nx)[2:]
        np.testing.assert_allclose(gb, ga, rtol=0, atol=1e-13 * np.abs(ga).max())
    ra = a[(2 + D) * N0:].reshape(1 + D, ny, nx, G)
    rb = b[(2 + D) * N1:].reshape(1 + D, ny + 2, nx, G)[:, 2:]
    np.testing.assert_allclose(rb, ra, rtol=0, atol=1e-13 * np.abs(ra).max())


@pytest.fixture(scope="module")
def dmr_run():
    pb, prim, layers = W.double_mach(nx=130, ny=40, t_end=0.05)
    s0 = oracle.init_equilibrium(pb, prim)
    out, st = oracle.run(pb, s0, pb.dt, pb.nsteps, nthreads=8, layers=layers)
    assert st == 0
    return pb, layers, out


def test_double_mach_incident_shock_moves_at_its_exact_speed(dmr_run):
    pb, layers, out = dmr_run
    t = pb.nsteps * pb.dt
    top = layers[3]
    nx, ny = pb.n[0], pb.n[1]
    rho = out[:pb.ncell].reshape(ny, nx)
    xc, yc = pb.cell_centres(0), pb.cell_centres(1)
    dx = xc[1] - xc[0]
    for y in (0.6, 0.75, 0.9):
        j = int(np.argmin(np.abs(yc - y)))
        xs = top["x0"] + yc[j] * top["cot_alpha"] + top["speed"] * t
        # the shock is where rho crosses the middle of its two sides, approaching from the right
        mid = 0.5 * (1.4 + 8.0)
        i = nx - 1
        while i > 0 and rho[j, i] < mid:
            i -= 1
        xnum = xc[i] + dx * (mid - rho[j, i]) / (rho[j, i + 1] - rho[j, i])
        assert abs(xnum - xs) < 1.5 * dx, (y, xnum, xs)


def test_double_mach_inflow_region_stays_post_shock(dmr_run):
    # behind the shock and before any wave from the wall arrives (x < x0, y > 0.5) the flow is the
    # uniform post-shock state that the left and bottom-left layers hold fixed
    pb, layers, out = dmr_run
    nx, ny = pb.n[0], pb.n[1]
    N = pb.ncell
    xc, yc = pb.cell_centres(0), pb.cell_centres(1)
    A = layers[3]["A"]
    sel = (xc[None, :] < 1.0 / 6.0) & (xc[None, :] > 0.0) & (yc[:, None] > 0.5)
    rho = out[:N].reshape(ny, nx)[sel]
    mx = out[N:2 * N].reshape(ny, nx)[sel]
    assert np.all(np.abs(rho - A[0]) <= 1e-12 * A[0])
    assert np.all(np.abs(mx - A[0] * A[2]) <= 1e-12 * A[0] * abs(A[2]))
