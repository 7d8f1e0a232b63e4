"""Exact solution of the 1-d Riemann problem for the ideal-gas Euler equations.

Written from the textbook method (Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", ch. 4): Newton iteration for the star pressure on the pressure function
f_L(p) + f_R(p) + (u_R - u_L) = 0, then sampling of the self-similar wave pattern.
Used as an independent pin for the oracle's hydrodynamics (Sec. 8.3, Sod shock tube).
"""
import math

import numpy as np


def _f_and_df(p, rho, pk, a, gam):
    if p > pk:  # shock
        A = 2.0 / ((gam + 1.0) * rho)
        B = (gam - 1.0) / (gam + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (B + p))
    pr = p / pk  # rarefaction
    f = 2.0 * a / (gam - 1.0) * (pr ** ((gam - 1.0) / (2.0 * gam)) - 1.0)
    df = 1.0 / (rho * a) * pr ** (-(gam + 1.0) / (2.0 * gam))
    return f, df


def star_state(rl, ul, pl, rr, ur, pr, gam):
    al, ar = math.sqrt(gam * pl / rl), math.sqrt(gam * pr / rr)
    p = max(1e-10, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dfl = _f_and_df(p, rl, pl, al, gam)
        fr, dfr = _f_and_df(p, rr, pr, ar, gam)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(1e-12, p - dp)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, pl, al, gam)
    fr, _ = _f_and_df(p, rr, pr, ar, gam)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(xi, rl, ul, pl, rr, ur, pr, gam):
    """(rho, u, p) at similarity coordinate xi = (x - x0)/t."""
    ps, us = star_state(rl, ul, pl, rr, ur, pr, gam)
    g1 = (gam - 1.0) / (gam + 1.0)
    if xi <= us:  # left of the contact
        a = math.sqrt(gam * pl / rl)
        if ps > pl:  # left shock
            S = ul - a * math.sqrt((gam + 1.0) / (2.0 * gam) * ps / pl + (gam - 1.0) / (2.0 * gam))
            if xi <= S:
                return rl, ul, pl
            return rl * (ps / pl + g1) / (g1 * ps / pl + 1.0), us, ps
        ash = a * (ps / pl) ** ((gam - 1.0) / (2.0 * gam))
        if xi <= ul - a:
            return rl, ul, pl
        if xi >= us - ash:
            return rl * (ps / pl) ** (1.0 / gam), us, ps
        u = 2.0 / (gam + 1.0) * (a + 0.5 * (gam - 1.0) * ul + xi)
        c = 2.0 / (gam + 1.0) * (a + 0.5 * (gam - 1.0) * (ul - xi))
        rho = rl * (c / a) ** (2.0 / (gam - 1.0))
        return rho, u, pl * (c / a) ** (2.0 * gam / (gam - 1.0))
    a = math.sqrt(gam * pr / rr)
    if ps > pr:  # right shock
        S = ur + a * math.sqrt((gam + 1.0) / (2.0 * gam) * ps / pr + (gam - 1.0) / (2.0 * gam))
        if xi >= S:
            return rr, ur, pr
        return rr * (ps / pr + g1) / (g1 * ps / pr + 1.0), us, ps
    ash = a * (ps / pr) ** ((gam - 1.0) / (2.0 * gam))
    if xi >= ur + a:
        return rr, ur, pr
    if xi <= us + ash:
        return rr * (ps / pr) ** (1.0 / gam), us, ps
    u = 2.0 / (gam + 1.0) * (-a + 0.5 * (gam - 1.0) * ur + xi)
    c = 2.0 / (gam + 1.0) * (a - 0.5 * (gam - 1.0) * (ur - xi))
    rho = rr * (c / a) ** (2.0 / (gam - 1.0))
    return rho, u, pr * (c / a) ** (2.0 * gam / (gam - 1.0))


def cell_averages(x_faces, t, x0, left, right, gam, sub=16):
    """Cell averages of (rho, u, p) by midpoint sub-sampling of each cell."""
    n = len(x_faces) - 1
    out = np.zeros((3, n))
    for i in range(n):
        xs = x_faces[i] + (np.arange(sub) + 0.5) * (x_faces[i + 1] - x_faces[i]) / sub
        vals = np.array([sample((x - x0) / t, *left, *right, gam) for x in xs])
        out[:, i] = vals.mean(0)
    return out
