"""Exact solution of the 1-D Riemann problem for an ideal gas.

Used only as a pin for the Euler oracle (shock capturing on the Sod tube).
Standard construction (Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", Ch. 4): the star pressure p* is the root of
    f_L(p) + f_R(p) + (u_R - u_L) = 0,
with f_K the shock (Rankine-Hugoniot) branch for p > p_K and the rarefaction
(isentropic) branch otherwise; u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2.
The self-similar solution is then sampled at xi = (x - x0)/t.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, g):
    c = math.sqrt(g * pk / rho)
    if p > pk:
        a = 2.0 / ((g + 1.0) * rho)
        b = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(a / (p + b))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (b + p))
    r = p / pk
    f = 2.0 * c / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * c) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(L, R, g=1.4):
    """(p*, u*) for primitive states L = (rho, u, p), R = (rho, u, p)."""
    rl, ul, pl = L
    rr, ur, pr = R
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _fk(p, rl, pl, g)
        fr, dfr = _fk(p, rr, pr, g)
        f = fl + fr + (ur - ul)
        pn = p - f / (dfl + dfr)
        if pn <= 0:
            pn = 0.5 * p
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, g)
    fr, _ = _fk(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(L, R, xi, g=1.4):
    """Primitive (rho, u, p) at similarity coordinate xi = (x - x0)/t."""
    rl, ul, pl = L
    rr, ur, pr = R
    ps, us = star_state(L, R, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    gm = (g - 1.0) / (g + 1.0)
    if xi <= us:
        if ps > pl:  # left shock
            sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
            if xi <= sl:
                return rl, ul, pl
            return rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps
        # left rarefaction
        head = ul - cl
        cls = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
        tail = us - cls
        if xi <= head:
            return rl, ul, pl
        if xi >= tail:
            return rl * (ps / pl) ** (1.0 / g), us, ps
        u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + xi)
        c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - xi))
        return rl * (c / cl) ** (2.0 / (g - 1.0)), u, pl * (c / cl) ** (2.0 * g / (g - 1.0))
    if ps > pr:  # right shock
        sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
        if xi >= sr:
            return rr, ur, pr
        return rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps
    head = ur + cr
    crs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
    tail = us + crs
    if xi >= head:
        return rr, ur, pr
    if xi <= tail:
        return rr * (ps / pr) ** (1.0 / g), us, ps
    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + xi)
    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - xi))
    return rr * (c / cr) ** (2.0 / (g - 1.0)), u, pr * (c / cr) ** (2.0 * g / (g - 1.0))


def profile(L, R, x, x0, t, g=1.4):
    out = np.array([sample(L, R, (xx - x0) / t, g) for xx in x])
    return out[:, 0], out[:, 1], out[:, 2]
