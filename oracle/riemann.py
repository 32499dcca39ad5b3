"""Exact solution of the Riemann problem of the 1D Euler equations (ideal gas),
for the classical tests of Sec. 2 (Table classical_tests_1d).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Written from the mathematics of the problem: the star pressure p* is the root
of f(p) = f_L(p) + f_R(p) + (u_R - u_L), where for side K with state
(rho_K, u_K, p_K) and sound speed c_K
    f_K(p) = (p - p_K) sqrt(A_K / (p + B_K)),   A_K = 2 / ((g+1) rho_K),
                                               B_K = (g-1)/(g+1) p_K        (p > p_K, shock)
    f_K(p) = 2 c_K / (g-1) ((p/p_K)^((g-1)/(2g)) - 1)                      (p <= p_K, rarefaction)
(the Rankine-Hugoniot and isentropic relations across the nonlinear waves),
solved by Newton's method; u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2; the
solution is self-similar in x/t and is sampled wave by wave.
"""
from __future__ import annotations

import numpy as np


def _fk(p, rho, pk, ck, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    r = (p / pk) ** ((g - 1.0) / (2.0 * g))
    return 2.0 * ck / (g - 1.0) * (r - 1.0), 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def star_state(left, right, g=1.4, tol=1e-14, max_iter=100):
    """(p*, u*) of the Riemann problem with primitive states left, right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("the initial data generate vacuum")
    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(max_iter):
        fl, dl = _fk(p, rl, pl, cl, g)
        fr, dr = _fk(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dl + dr)
        if pn < 0:
            pn = 1e-8
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, xi, g=1.4):
    """Primitive (rho, u, p) of the exact solution at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    xi = np.asarray(xi, dtype=np.float64)
    rho, u, p = np.empty_like(xi), np.empty_like(xi), np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for idx, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                sl = ul - cl * np.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                st = (rl, ul, pl) if s <= sl else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / g)
                cs = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                head, tail = ul - cl, us - cs
                if s <= head:
                    st = (rl, ul, pl)
                elif s >= tail:
                    st = (rs, us, ps)
                else:
                    uf = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    cf = uf - s
                    rf = rl * (cf / cl) ** (2.0 / (g - 1.0))
                    st = (rf, uf, pl * (cf / cl) ** (2.0 * g / (g - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                sr = ur + cr * np.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                st = (rr, ur, pr) if s >= sr else (rs, us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / g)
                cs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                head, tail = ur + cr, us + cs
                if s >= head:
                    st = (rr, ur, pr)
                elif s <= tail:
                    st = (rs, us, ps)
                else:
                    uf = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    cf = s - uf
                    rf = rr * (cf / cr) ** (2.0 / (g - 1.0))
                    st = (rf, uf, pr * (cf / cr) ** (2.0 * g / (g - 1.0)))
        rho[idx], u[idx], p[idx] = st
    return rho, u, p


def solution(left, right, x, t, x0=0.5, g=1.4):
    """Exact (rho, u, p) at points x and time t > 0 for an initial jump at x0."""
    return sample(left, right, (np.asarray(x, dtype=np.float64) - x0) / t, g)
