"""Exact solution of the 1-D Euler Riemann problem for an ideal gas.

Textbook construction (Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", ch. 4): Newton iteration on the pressure function for the star
pressure, then sampling of the self-similar wave fan.  Used by the tests as an
independent pin of the oracle (Sod problem, Sec. 5.2 (b) of the paper).
"""
from __future__ import annotations

import math

import numpy as np


def _f_side(p, rho, pk, gamma):
    a = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    r = (p / pk) ** ((gamma - 1.0) / (2.0 * gamma))
    return 2.0 * a / (gamma - 1.0) * (r - 1.0), 1.0 / (rho * a) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))


def star_state(left, right, gamma=1.4, tol=1e-15):
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(0.5 * (pl + pr), 1e-12)
    for _ in range(200):
        fl, dl = _f_side(p, rl, pl, gamma)
        fr, dr = _f_side(p, rr, pr, gamma)
        f = fl + fr + (ur - ul)
        pn = p - f / (dl + dr)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_side(p, rl, pl, gamma)
    fr, _ = _f_side(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, x, t, x0=0.5, gamma=1.4):
    """Point values (rho, u, p) of the exact solution at positions x, time t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    al = math.sqrt(gamma * pl / rl)
    ar = math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((3, len(x)))
    for k, xx in enumerate(np.asarray(x, dtype=float)):
        s = (xx - x0) / t
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                sl = ul - al * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
                if s <= sl:
                    st = (rl, ul, pl)
                else:
                    st = (rl * (ps / pl + g1) / (g1 * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                als = al * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                if s <= ul - al:
                    st = (rl, ul, pl)
                elif s >= us - als:
                    st = (rl * (ps / pl) ** (1 / gamma), us, ps)
                else:
                    c = 2 / (gamma + 1) + g1 / al * (ul - s)
                    st = (rl * c ** (2 / (gamma - 1)), 2 / (gamma + 1) * (al + (gamma - 1) / 2 * ul + s),
                          pl * c ** (2 * gamma / (gamma - 1)))
        else:
            if ps > pr:  # right shock
                sr = ur + ar * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
                if s >= sr:
                    st = (rr, ur, pr)
                else:
                    st = (rr * (ps / pr + g1) / (g1 * ps / pr + 1.0), us, ps)
            else:
                ars = ar * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                if s >= ur + ar:
                    st = (rr, ur, pr)
                elif s <= us + ars:
                    st = (rr * (ps / pr) ** (1 / gamma), us, ps)
                else:
                    c = 2 / (gamma + 1) - g1 / ar * (ur - s)
                    st = (rr * c ** (2 / (gamma - 1)), 2 / (gamma + 1) * (-ar + (gamma - 1) / 2 * ur + s),
                          pr * c ** (2 * gamma / (gamma - 1)))
        out[:, k] = st
    return out


def cell_averages(left, right, n, t, x0=0.5, gamma=1.4, length=1.0, sub=16):
    """Cell averages of (rho, rho u, E) by sub-sampling each cell (midpoint rule)."""
    edges = np.linspace(0.0, length, n + 1)
    h = length / n
    xs = (edges[:-1, None] + (np.arange(sub)[None, :] + 0.5) * h / sub).ravel()
    r, u, p = sample(left, right, xs, t, x0, gamma)
    W = np.stack([r, r * u, p / (gamma - 1) + 0.5 * r * u * u]).reshape(3, n, sub)
    return W.mean(axis=2)
