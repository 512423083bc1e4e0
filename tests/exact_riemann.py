"""Exact solution of the 1D Riemann problem for the ideal-gas Euler equations.

Written from the textbook construction (Toro, "Riemann Solvers and Numerical
Methods for Fluid Dynamics", Ch. 4): the star-region pressure is the root of
f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock (Rankine-Hugoniot) or
rarefaction (isentropic) relation across the K-wave; the star velocity follows,
and the solution at x/t is sampled from the wave pattern.  Used only as an
independent pin of the oracle's finite-volume step.
"""
from __future__ import annotations

import math

import numpy as np


def _f_and_df(p, rho, u, pk, g):
    a = math.sqrt(g * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        f = (p - pk) * s
        df = s * (1.0 - 0.5 * (p - pk) / (p + B))
    else:  # rarefaction
        f = 2.0 * a / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * a) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dfl = _f_and_df(p, rl, ul, pl, g)
        fr, dfr = _f_and_df(p, rr, ur, pr, g)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-12)
        if abs(pn - p) <= 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, ul, pl, g)
    fr, _ = _f_and_df(p, rr, ur, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, g=1.4):
    """(rho, u, p) at similarity coordinate xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, g)
    if xi <= us:  # left of contact
        al = math.sqrt(g * pl / rl)
        if ps > pl:
            sl = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
            if xi <= sl:
                return rl, ul, pl
            r = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
            return r, us, ps
        ash = al * (ps / pl) ** ((g - 1) / (2 * g))
        shl, stl = ul - al, us - ash
        if xi <= shl:
            return rl, ul, pl
        if xi >= stl:
            return rl * (ps / pl) ** (1 / g), us, ps
        c = 2 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - xi)
        return rl * c ** (2 / (g - 1)), 2 / (g + 1) * (al + (g - 1) / 2 * ul + xi), pl * c ** (2 * g / (g - 1))
    ar = math.sqrt(g * pr / rr)
    if ps > pr:
        sr = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
        if xi >= sr:
            return rr, ur, pr
        r = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
        return r, us, ps
    ash = ar * (ps / pr) ** ((g - 1) / (2 * g))
    shr, str_ = ur + ar, us + ash
    if xi >= shr:
        return rr, ur, pr
    if xi <= str_:
        return rr * (ps / pr) ** (1 / g), us, ps
    c = 2 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - xi)
    return rr * c ** (2 / (g - 1)), 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + xi), pr * c ** (2 * g / (g - 1))


def cell_average_density(left, right, x0, t, edges, g=1.4, sub=64):
    """Cell averages of the exact density on cells [edges[i], edges[i+1]] (midpoint rule, ``sub`` points)."""
    out = np.empty(len(edges) - 1)
    for i in range(len(edges) - 1):
        xs = edges[i] + (np.arange(sub) + 0.5) * (edges[i + 1] - edges[i]) / sub
        out[i] = np.mean([sample(left, right, (x - x0) / t, g)[0] for x in xs])
    return out
