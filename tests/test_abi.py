"""CPU tests of the C ABI boundary: the library loads, exports every declared symbol, validates
parameters, and its host-built reconstruction tables reproduce the oracle's reconstruction."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1806_07390_gb300 import fx
from paper_1806_07390_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(fx.LIB_PATH):
        from paper_1806_07390_gb300 import build
        build.build()
    return fx.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fx_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert set(names) == set(fx.EXPORTS), names
    for n in names:
        assert hasattr(L, n), n


def create(pb):
    P = fx.params(pb)
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    st = fx.lib().fx_grid_create(ctypes.byref(P), ctypes.byref(h), ctypes.byref(ws))
    return st, h, ws.value


def test_create_validates_parameters(L):
    pb, _ = W.kh_2d(nx=16, ny=12, ngroups=4)
    st, h, ws = create(pb)
    assert st == 0 and ws > 0
    assert L.fx_state_elems(h) == pb.state_size()
    assert L.fx_launches_per_step(h) == 6  # per stage: gas faces, radiation/update, interaction
    assert L.fx_march_chunk(h) == 12  # the march axis is shorter than the default 32 planes
    # workspace size covers two FP64 states
    assert ws >= 2 * pb.state_size() * 8
    L.fx_grid_destroy(h)
    bad = [dict(ngroups=0), dict(ngroups=33), dict(kap_T_exp=-1.25), dict(gamma=1.0),
           dict(c_light=0.0), dict(n=(3, 12, 1)), dict(newton_maxit=0)]
    for kw in bad:
        pb2, _ = W.kh_2d(nx=16, ny=12, ngroups=4)
        for k, v in kw.items():
            setattr(pb2, k, v)
        st, h, _ = create(pb2)
        assert st != 0 and not h.value, kw
    pb3, _ = W.kh_2d(nx=16, ny=12, ngroups=4)
    pb3.bc_lo = ("periodic", "outflow", "periodic")
    pb3.bc_hi = ("outflow", "outflow", "periodic")
    assert create(pb3)[0] == -1


def test_velocity_terms_parameters(L):
    # vterms: 0 or 1; Cartesian and spherical grids; one more kernel per stage; the face buffer
    # holds the transverse face velocities on top of the fluxes and contact speeds
    pb, _ = W.kh_2d(nx=16, ny=12, ngroups=4)
    st0, h0, ws0 = create(pb)
    pb.vterms = 1
    st1, h1, ws1 = create(pb)
    assert st0 == 0 and st1 == 0
    assert L.fx_launches_per_step(h1) == L.fx_launches_per_step(h0) + 2
    faces = (16 + 1) * 12 + 16 * (12 + 1)  # faces of the two directions
    assert ws1 - ws0 >= faces * 8 and ws1 - ws0 <= faces * 8 + 4 * 256
    L.fx_grid_destroy(h0)
    L.fx_grid_destroy(h1)
    pb.vterms = 2
    assert create(pb)[0] == -1
    pb2, _ = W.spherical_2d(nr=16, nth=8, ngroups=4)
    st2, h2, _ = create(pb2)
    pb2.vterms = 1
    st3, h3, _ = create(pb2)
    assert st2 == 0 and st3 == 0
    assert L.fx_launches_per_step(h3) == L.fx_launches_per_step(h2) + 2
    L.fx_grid_destroy(h2)
    L.fx_grid_destroy(h3)


def test_three_species_parameters(L):
    # species: 0/1 or 3; three species need at most 32 channels (the velocity terms are allowed);
    # the state gains a composition block; one more kernel per stage
    pb, _ = W.neutrino_2d(nx=16, ny=12, ngroups=8)
    st, h, ws = create(pb)
    assert st == 0
    assert L.fx_state_elems(h) == pb.state_size() == pb.ncell * (4 + 3 * 24 + 1)
    pb1, _ = W.kh_2d(nx=16, ny=12, ngroups=4)
    h1 = create(pb1)[1]
    assert L.fx_launches_per_step(h) == L.fx_launches_per_step(h1) + 2
    L.fx_grid_destroy(h)
    L.fx_grid_destroy(h1)
    for kw, code in ((dict(species=2), -1), (dict(ngroups=11), -7), (dict(vterms=1), 0),
                     (dict(xi0=-1.0), -1)):
        pb2, _ = W.neutrino_2d(nx=16, ny=12, ngroups=8)
        for k, v in kw.items():
            setattr(pb2, k, v)
        st2, h2, _ = create(pb2)
        assert st2 == code, kw
        if st2 == 0:
            L.fx_grid_destroy(h2)


def test_unbound_handle_reports_workspace_error(L):
    pb, _ = W.sod_1d(n=16, ngroups=3)
    st, h, _ = create(pb)
    assert st == 0
    assert L.fx_step(h, 1e-3, 1) == -3
    assert L.fx_sync(h) == -3
    assert b"workspace" in L.fx_last_error(h)
    L.fx_grid_destroy(h)


def _table_recon(T, ip, pm, p0, pp, kind):
    """Face values from one row of the host table (mirrors the device arithmetic in numpy)."""
    e = {n: i for i, n in enumerate(["WA0", "WA1", "WA2", "WB0", "WB1", "WB2", "SL2", "TL2", "SR2",
                                     "TR2", "AL0", "AL1", "AL2", "AR0", "AR1", "AR2", "RHL", "RHR",
                                     "IL", "IR", "IC", "DL", "DR", "FL", "FR", "ELL", "VOL"])}
    t = lambda n: T[e[n], ip]
    if kind == 1:
        sL, sR = (p0 - pm) * t("IL"), (pp - p0) * t("IR")
        s = 0.0
        if sL * sR > 0:
            sC = (pp - pm) * t("IC")
            m = min(2 * abs(sL), 2 * abs(sR), abs(sC))
            s = m if sC > 0 else -m
        return p0 + s * t("DL"), p0 + s * t("DR")
    dl, dr = p0 - pm, pp - p0
    if dl * dr <= 0:
        return p0, p0
    a = t("WA0") * pm + t("WA1") * p0 + t("WA2") * pp
    b = t("WB0") * pm + t("WB1") * p0 + t("WB2") * pp
    lo, hi = pm + dl * t("SL2"), p0 - dl * t("TL2")
    lo, hi = (hi, lo) if dl < 0 else (lo, hi)
    a = min(max(a, lo), hi)
    lo, hi = p0 + dr * t("SR2"), pp - dr * t("TR2")
    lo, hi = (hi, lo) if dr < 0 else (lo, hi)
    b = min(max(b, lo), hi)
    sl = t("AL0") * a + t("AL1") * p0 + t("AL2") * b
    sr = t("AR0") * a + t("AR1") * p0 + t("AR2") * b
    if sl * sr >= 0:
        return a, b
    if abs(sl) == abs(sr):
        return p0, p0
    if abs(sl) < abs(sr):
        b = a + (p0 - a) * t("RHL")
    else:
        a = b + (p0 - b) * t("RHR")
    return a, b


@pytest.mark.parametrize("maker", ["kh", "sph"])
def test_host_tables_reproduce_oracle_reconstruction(L, maker):
    if maker == "kh":
        pb, _ = W.kh_2d(nx=24, ny=20, ngroups=2)
    else:
        pb, _ = W.spherical_2d(nr=24, nth=20, ngroups=2)
    st, h, _ = create(pb)
    assert st == 0
    ntab = L.fx_debug_ntab()
    rng = np.random.default_rng(0)
    for d in range(2):
        n = pb.n[d] + 4
        T = np.zeros(ntab * n)
        assert L.fx_debug_table(h, d, T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), T.size) == T.size
        T = T.reshape(ntab, n)
        for _ in range(300):
            i = int(rng.integers(0, pb.n[d]))
            pm, p0, pp = rng.uniform(0, 1, 3)
            for kind in (1, 2):
                a, b = _table_recon(T, i + 2, pm, p0, pp, kind)
                ra, rb = oracle.recon_cell(pb, d, i, pm, p0, pp, kind=kind)
                assert abs(a - ra) < 1e-13 and abs(b - rb) < 1e-13, (d, i, kind, a, ra, b, rb)
    L.fx_grid_destroy(h)


def test_fp32_planck_tables_interpolate_the_band_integrals(L):
    # the host-built FP32 band tables, interpolated with the device's cubic Hermite formula,
    # reproduce the oracle's Planck band integrals to FP32 precision over the table's range
    pb, _ = W.kh_2d(nx=16, ny=16, ngroups=16)
    st, h, _ = create(pb)
    assert st == 0
    nu, u0 = ctypes.c_int(), ctypes.c_float()
    n = L.fx_debug_planck_table(h, None, 0, ctypes.byref(nu), ctypes.byref(u0))
    buf = np.zeros(n, dtype=np.float32)
    L.fx_debug_planck_table(h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n,
                            ctypes.byref(nu), ctypes.byref(u0))
    tab = buf.reshape(pb.ngroups, nu.value, 4).astype(np.float64)
    # the fourth entry is the exact FP32 power of two 2^floor(L), or 0 below the normal range
    want = np.where(tab[..., 2] >= -126, 2.0 ** tab[..., 2], 0.0)
    assert np.array_equal(tab[..., 3], want)
    edges = pb.eps_min * (pb.eps_max / pb.eps_min) ** (np.arange(pb.ngroups + 1) / pb.ngroups)
    rng = np.random.default_rng(3)
    worst = 0.0
    for T in np.exp(rng.uniform(np.log(0.02), np.log(50.0), 60)):
        s = (np.log2(T) - u0.value) * 32.0
        i = int(s)
        t = s - i
        for g in range(pb.ngroups):
            p0, p1 = tab[g, i], tab[g, i + 1]
            d1 = (p1[2] - p0[2]) + p1[0]
            Lg = p0[2] + ((2 * t ** 3 - 3 * t ** 2 + 1) * p0[0] + (t ** 3 - 2 * t ** 2 + t) * p0[1] +
                          (3 * t ** 2 - 2 * t ** 3) * d1 + (t ** 3 - t ** 2) * p1[1])
            ref = oracle.lib().orc_planck_band(edges[g] / T, edges[g + 1] / T)
            if ref < 1e-30:
                continue
            worst = max(worst, abs(2.0 ** Lg / ref - 1.0))
    L.fx_grid_destroy(h)
    assert worst < 3e-7, worst


@pytest.mark.parametrize("map1", ["exp", "sinh"])
def test_spherical_tables_match_oracle_geometry(L, map1):
    # volumes, connection coefficients and face factors of the library's host tables against
    # the oracle's independently integrated geometry (Appendices A-D), log-r and sinh radial maps
    pb, _ = W.spherical_2d(nr=20, nth=12, ngroups=2, map1=map1)
    st, h, _ = create(pb)
    assert st == 0
    ntab = L.fx_debug_ntab()
    T = []
    for d in range(2):
        n = pb.n[d] + 4
        buf = np.zeros(ntab * n)
        L.fx_debug_table(h, d, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), buf.size)
        T.append(buf.reshape(ntab, n)[:, 2:-2])
    names = ["WA0", "WA1", "WA2", "WB0", "WB1", "WB2", "SL2", "TL2", "SR2", "TR2", "AL0", "AL1",
             "AL2", "AR0", "AR1", "AR2", "RHL", "RHR", "IL", "IR", "IC", "DL", "DR", "FL", "FR",
             "ELL", "VOL", "FL1", "FR1", "FL2", "FR2", "XS", "X1", "X2", "XH", "HA", "HB", "GA",
             "GB", "GC", "QI", "RI"]
    e = {nm: i for i, nm in enumerate(names)}
    assert ntab == len(names)
    vol_r, _, _ = oracle.geometry(pb, 0)
    vol_t, _, _ = oracle.geometry(pb, 1)
    np.testing.assert_allclose(T[0][e["VOL"]], vol_r, rtol=1e-13)
    np.testing.assert_allclose(T[1][e["VOL"]], vol_t, rtol=1e-13)
    G = oracle.christoffel(pb)
    np.testing.assert_allclose(T[0][e["GA"]], G["G111"], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(T[0][e["GB"]], G["G221"], rtol=1e-12)
    np.testing.assert_allclose(T[0][e["GC"]], G["G122"], rtol=1e-12)
    np.testing.assert_allclose(T[1][e["GA"]], G["G222"], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(T[1][e["GB"]], G["G332"], rtol=1e-12, atol=1e-14)
    # radial faces: r^2 / V_r and r^3 / V_r from the map
    xf = np.linspace(pb.x_lo[0], pb.x_hi[0], pb.n[0] + 1)
    rf = np.exp(xf) if map1 == "exp" else pb.map_rt * np.sinh(xf / pb.map_rt)
    np.testing.assert_allclose(T[0][e["FL"]], rf[:-1] ** 2 / vol_r, rtol=1e-13)
    np.testing.assert_allclose(T[0][e["FR2"]], rf[1:] ** 3 / vol_r, rtol=1e-13)
    # the radial map at the lower faces for the velocity gradient: 1 / (dr/dx1) and 1 / r
    qf = np.exp(xf) if map1 == "exp" else np.cosh(xf / pb.map_rt)
    np.testing.assert_allclose(T[0][e["QI"]], 1.0 / qf[:-1], rtol=1e-14)
    np.testing.assert_allclose(T[0][e["RI"]], 1.0 / rf[:-1], rtol=1e-14)
    assert np.all(T[1][e["QI"]] == 1.0) and np.all(T[1][e["RI"]] == 1.0)
    L.fx_grid_destroy(h)
