"""ORACLE -- test infrastructure only.

Exact solution of the Riemann problem of the 1D Euler equations for an ideal gas, from
the textbook derivation (the pressure function of a shock or a rarefaction on each side,
Newton iteration for the star pressure, then sampling the self-similar wave pattern).
Used to pin the oracle's shock-tube results.
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np


def _f_side(p: float, rho: float, pk: float, ck: float, g: float) -> Tuple[float, float]:
    """Pressure function f_K(p) and its derivative for one side K."""
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        sq = math.sqrt(A / (p + B))
        return (p - pk) * sq, sq * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    pr = p / pk
    f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g: float = 1.4):
    """(p*, u*) of the Riemann problem with primitive states left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("vacuum is generated")
    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(200):
        fl, dfl = _f_side(p, rl, pl, cl, g)
        fr, dfr = _f_side(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-12)
        if abs(pn - p) <= 1e-15 * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_side(p, rl, pl, cl, g)
    fr, _ = _f_side(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, s: float, g: float = 1.4):
    """Primitive state (rho, u, p) on the ray x/t = s."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, g)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    gm = (g - 1.0) / (g + 1.0)
    if s <= us:  # left of the contact
        if ps > pl:  # left shock
            sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
            if s <= sl:
                return rl, ul, pl
            return rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps
        cs = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
        if s <= ul - cl:
            return rl, ul, pl
        if s >= us - cs:
            return rl * (ps / pl) ** (1.0 / g), us, ps
        u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
        c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
        rho = rl * (c / cl) ** (2.0 / (g - 1.0))
        return rho, u, pl * (c / cl) ** (2.0 * g / (g - 1.0))
    if ps > pr:  # right shock
        sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
        if s >= sr:
            return rr, ur, pr
        return rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps
    cs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
    if s >= ur + cr:
        return rr, ur, pr
    if s <= us + cs:
        return rr * (ps / pr) ** (1.0 / g), us, ps
    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
    rho = rr * (c / cr) ** (2.0 / (g - 1.0))
    return rho, u, pr * (c / cr) ** (2.0 * g / (g - 1.0))


def cell_averages(left, right, x0: float, x1: float, n: int, xd: float, t: float,
                  g: float = 1.4, sub: int = 64) -> np.ndarray:
    """Cell averages of the primitive exact solution [(rho, u, p), n] at time t, by
    midpoint sub-sampling of each cell."""
    dx = (x1 - x0) / n
    out = np.zeros((3, n))
    for i in range(n):
        acc = np.zeros(3)
        for q in range(sub):
            x = x0 + (i + (q + 0.5) / sub) * dx
            acc += sample(left, right, (x - xd) / t, g)
        out[:, i] = acc / sub
    return out
