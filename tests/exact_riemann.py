"""Exact solution of the 1D Riemann problem of the Euler equations for an ideal gas.

Test infrastructure: it pins the oracle's Sod run to the exact self-similar solution.  It is
written from the classical wave analysis (shock: Rankine-Hugoniot; rarefaction: isentropic
fan with constant Riemann invariant), not from the oracle, and shares nothing with it.

    p*  solves  f_L(p) + f_R(p) + (u_R - u_L) = 0,
    f_K(p) = (p - p_K) sqrt(A_K / (p + B_K))                     if p > p_K  (shock)
           = 2 a_K/(g-1) ((p/p_K)^((g-1)/(2g)) - 1)               otherwise   (rarefaction)
    A_K = 2 / ((g+1) rho_K),  B_K = (g-1)/(g+1) p_K,  u* = (u_L + u_R + f_R(p*) - f_L(p*)) / 2
"""
from __future__ import annotations

import math

import numpy as np


def _f(p, rho, pk, g):
    a = math.sqrt(g * pk / rho)
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (B + p))
    r = p / pk
    return (2.0 * a / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0),
            1.0 / (rho * a) * r ** (-(g + 1.0) / (2.0 * g)))


def star_state(left, right, g):
    """(p*, u*, rho*_L, rho*_R) for primitive states left=(rho, u, p), right=(rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    if 2.0 * (al + ar) / (g - 1.0) <= ur - ul:
        raise ValueError("vacuum is generated")
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dl = _f(p, rl, pl, g)
        fr, dr = _f(p, rr, pr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(1e-14, p - dp)
        if abs(pn - p) <= 1e-15 * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, g)
    fr, _ = _f(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    gm = (g - 1.0) / (g + 1.0)

    def rho_star(rho, pk):
        if p > pk:  # shock
            return rho * (p / pk + gm) / (gm * p / pk + 1.0)
        return rho * (p / pk) ** (1.0 / g)  # rarefaction: isentropic

    return p, u, rho_star(rl, pl), rho_star(rr, pr)


def sample(left, right, g, xi):
    """Primitive state (rho, u, p) at similarity coordinate xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us, rsl, rsr = star_state(left, right, g)
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    if xi <= us:  # left of the contact
        if ps > pl:  # left shock
            s = ul - al * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
            return (rl, ul, pl) if xi <= s else (rsl, us, ps)
        head = ul - al
        asl = al * (ps / pl) ** ((g - 1.0) / (2.0 * g))
        tail = us - asl
        if xi <= head:
            return (rl, ul, pl)
        if xi >= tail:
            return (rsl, us, ps)
        c = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * al) * (ul - xi)
        return (rl * c ** (2.0 / (g - 1.0)),
                2.0 / (g + 1.0) * (al + 0.5 * (g - 1.0) * ul + xi),
                pl * c ** (2.0 * g / (g - 1.0)))
    if ps > pr:  # right shock
        s = ur + ar * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
        return (rsr, us, ps) if xi <= s else (rr, ur, pr)
    head = ur + ar
    asr = ar * (ps / pr) ** ((g - 1.0) / (2.0 * g))
    tail = us + asr
    if xi >= head:
        return (rr, ur, pr)
    if xi <= tail:
        return (rsr, us, ps)
    c = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * ar) * (ur - xi)
    return (rr * c ** (2.0 / (g - 1.0)),
            2.0 / (g + 1.0) * (-ar + 0.5 * (g - 1.0) * ur + xi),
            pr * c ** (2.0 * g / (g - 1.0)))


def cell_averages(left, right, g, n, t, x0=0.5, sub=16):
    """Exact cell averages of (rho, u, p) on n cells of [0, 1] at time t (sub-sampled midpoint rule)."""
    out = np.zeros((3, n))
    for i in range(n):
        acc = np.zeros(3)
        for s in range(sub):
            x = (i + (s + 0.5) / sub) / n
            acc += sample(left, right, g, (x - x0) / t)
        out[:, i] = acc / sub
    return out
