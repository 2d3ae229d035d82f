"""Exact solution of the Riemann problem for the 1D Euler equations (ideal gas).

Written from the mathematics of the Riemann problem (E. Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", Ch. 4, the reference the paper cites for it):
the star pressure is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the
shock (Rankine-Hugoniot) or rarefaction (isentropic) velocity change across wave K.
Used by the tests only, to pin the oracle's Sod-tube solution.
"""
from __future__ import annotations

import math

import numpy as np


def _f_and_df(p, rho, pk, ck, g):
    if p > pk:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        f = (p - pk) * s
        df = s * (1.0 - 0.5 * (p - pk) / (B + p))
    else:        # rarefaction
        pr = p / pk
        f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _f_and_df(p, rl, pl, cl, g)
        fr, dfr = _f_and_df(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(1e-12, p - dp)
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, pl, cl, g)
    fr, _ = _f_and_df(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(xi, left, right, g=1.4):
    """Primitive state (rho, u, p) at similarity coordinate xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    if xi <= us:   # left of contact
        if ps > pl:
            rs = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
            sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
            return (rl, ul, pl) if xi <= sl else (rs, us, ps)
        rs = rl * (ps / pl) ** (1 / g)
        cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
        sh, st = ul - cl, us - cs
        if xi <= sh:
            return rl, ul, pl
        if xi >= st:
            return rs, us, ps
        u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + xi)
        c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - xi))
        rho = rl * (c / cl) ** (2 / (g - 1))
        return rho, u, pl * (c / cl) ** (2 * g / (g - 1))
    if ps > pr:
        rs = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
        sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
        return (rr, ur, pr) if xi >= sr else (rs, us, ps)
    rs = rr * (ps / pr) ** (1 / g)
    cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
    sh, st = ur + cr, us + cs
    if xi >= sh:
        return rr, ur, pr
    if xi <= st:
        return rs, us, ps
    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + xi)
    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - xi))
    rho = rr * (c / cr) ** (2 / (g - 1))
    return rho, u, pr * (c / cr) ** (2 * g / (g - 1))


def cell_average_density(N, x0, x1, xjump, t, left, right, g=1.4, nsub=64):
    """Cell averages of the exact density (midpoint sub-sampling of each cell)."""
    dx = (x1 - x0) / N
    out = np.zeros(N)
    for i in range(N):
        xs = x0 + dx * (i + (np.arange(nsub) + 0.5) / nsub)
        out[i] = np.mean([sample((x - xjump) / t, left, right, g)[0] for x in xs])
    return out
