"""Exact solution of the one-dimensional Riemann problem for a polytropic gas.

TEST INFRASTRUCTURE ONLY (part of the oracle).  Textbook Godunov exact solver
(pressure function with shock / rarefaction branches, Newton iteration for the
star pressure, self-similar sampling); the exact solution the Sod shock tubes of
Sec. III.C are checked against, where the single-population D2V37 model has
gamma = (D+2)/D = 2.
"""
from __future__ import annotations

import numpy as np


def _pressure_function(p, rho_k, p_k, a_k, gamma):
    """f_K(p) and its derivative for one side K of the contact."""
    if p > p_k:  # shock
        A = 2.0 / ((gamma + 1.0) * rho_k)
        B = (gamma - 1.0) / (gamma + 1.0) * p_k
        q = np.sqrt(A / (p + B))
        return (p - p_k) * q, q * (1.0 - 0.5 * (p - p_k) / (B + p))
    # rarefaction
    r = (p / p_k) ** ((gamma - 1.0) / (2.0 * gamma))
    f = 2.0 * a_k / (gamma - 1.0) * (r - 1.0)
    df = (1.0 / (rho_k * a_k)) * (p / p_k) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma):
    """(p*, u*) for left/right states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _pressure_function(p, rl, pl, al, gamma)
        fr, dfr = _pressure_function(p, rr, pr, ar, gamma)
        g = fl + fr + (ur - ul)
        p_new = max(1e-14, p - g / (dfl + dfr))
        if abs(p_new - p) <= 1e-15 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _pressure_function(p, rl, pl, al, gamma)
    fr, _ = _pressure_function(p, rr, pr, ar, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, gamma, xi):
    """(rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    ps, us = star_state(left, right, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((3, len(xi)))
    for k, s in enumerate(np.asarray(xi, dtype=float)):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                rs = rl * ((ps / pl + g1) / (g1 * ps / pl + 1.0))
                sl = ul - al * np.sqrt((gamma + 1.0) / (2 * gamma) * ps / pl + (gamma - 1.0) / (2 * gamma))
                out[:, k] = (rl, ul, pl) if s <= sl else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / gamma)
                ash = al * (ps / pl) ** ((gamma - 1.0) / (2 * gamma))
                head, tail = ul - al, us - ash
                if s <= head:
                    out[:, k] = (rl, ul, pl)
                elif s >= tail:
                    out[:, k] = (rs, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) + (gamma - 1.0) / ((gamma + 1.0) * al) * (ul - s)
                    out[:, k] = (rl * c ** (2.0 / (gamma - 1.0)),
                                 2.0 / (gamma + 1.0) * (al + (gamma - 1.0) / 2.0 * ul + s),
                                 pl * c ** (2.0 * gamma / (gamma - 1.0)))
        else:  # right of contact
            if ps > pr:  # right shock
                rs = rr * ((ps / pr + g1) / (g1 * ps / pr + 1.0))
                sr = ur + ar * np.sqrt((gamma + 1.0) / (2 * gamma) * ps / pr + (gamma - 1.0) / (2 * gamma))
                out[:, k] = (rr, ur, pr) if s >= sr else (rs, us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / gamma)
                ash = ar * (ps / pr) ** ((gamma - 1.0) / (2 * gamma))
                head, tail = ur + ar, us + ash
                if s >= head:
                    out[:, k] = (rr, ur, pr)
                elif s <= tail:
                    out[:, k] = (rs, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) - (gamma - 1.0) / ((gamma + 1.0) * ar) * (ur - s)
                    out[:, k] = (rr * c ** (2.0 / (gamma - 1.0)),
                                 2.0 / (gamma + 1.0) * (-ar + (gamma - 1.0) / 2.0 * ur + s),
                                 pr * c ** (2.0 * gamma / (gamma - 1.0)))
    return out
