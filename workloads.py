"""Seeded synthetic inputs for the 1D Euler ADER workloads.

This module only draws random numbers and evaluates closed-form initial
fields; it holds none of the scheme's arithmetic (no basis, no quadrature
nodes, no fluxes).  Both the CUDA path (tests, bench) and the CPU oracle take
their inputs from here: each side supplies its own node coordinates.

Workloads (1D stand-ins for the paper's sine-wave advection of Sec. 2.1:
constant velocity and pressure, a density perturbation that is advected
unchanged, exact solution rho0(x - u t) on the periodic unit interval):

* ``sine``     rho = 1 + 0.2 sin(2 pi x), u = 1, p = 1 (DG N=2, 100 cells, t_end = 1)
* ``modes4``   rho = 1 + sum_{k=1..4} a_k sin(2 pi k x + phi_k), a_k ~ U(0, 0.05),
               phi_k ~ U(0, 2 pi), u = 1, p = 1 (DG N=5 10^5 cells; WENO5 10^6; DG N=7 10^6)
* ``serving``  independent requests: cells log-uniform in [64, 65536], N ~ U{1..7},
               rho, p = 1 + sum_{j=1..3} a_j sin(2 pi j x + phi_j), a_j ~ U(0, 0.1/3), u = 0.5,
               t_end = 0.5, Poisson arrivals.
* ``riemann``  the classical Riemann problems of Sec. 2 (Table classical_tests_1d: Sod,
               Lax, two shocks, two rarefactions; jump at x = 0.5, t_final = 0.15) and
               their exact solution (star state by Newton's method on the pressure
               function, then the self-similar waves), the reference for the errors.
* ``reacting`` the two-component reacting flow of Sec. 2 (eq. pdes_2_comps) in 1D:
               (rho, rho u, E, rho c1, rho c2) with rho, p = 1 + three seeded modes,
               u = 0.5, c1 = 0.5 + 0.3 sin 2 pi x, c2 = 0.2 cos 2 pi x; and the uniform
               state of the ODE test of Sec. 2.1 (eq. harm_osc): rho = u = p = 1,
               c1 = 1, c2 = 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 12483
GAMMA = 1.4
TWO_PI = 2.0 * np.pi


@dataclass
class Field1D:
    """rho(x) = rho0 + sum a_k sin(2 pi k x + phi_k); same form for p; constant u."""
    rho0: float = 1.0
    rho_amp: np.ndarray = field(default_factory=lambda: np.zeros(0))
    rho_phase: np.ndarray = field(default_factory=lambda: np.zeros(0))
    rho_k: np.ndarray = field(default_factory=lambda: np.zeros(0))
    u: float = 1.0
    p0: float = 1.0
    p_amp: np.ndarray = field(default_factory=lambda: np.zeros(0))
    p_phase: np.ndarray = field(default_factory=lambda: np.zeros(0))
    p_k: np.ndarray = field(default_factory=lambda: np.zeros(0))

    # -- point values --
    @staticmethod
    def _modes(x, base, amp, phase, k):
        x = np.asarray(x, dtype=np.float64)
        out = np.full(x.shape, base, dtype=np.float64)
        for a, ph, kk in zip(amp, phase, k):
            out = out + a * np.sin(TWO_PI * kk * x + ph)
        return out

    def rho(self, x, t: float = 0.0):
        """Density at x; for constant p the exact solution is rho0(x - u t)."""
        return self._modes(np.asarray(x) - self.u * t, self.rho0, self.rho_amp, self.rho_phase,
                           self.rho_k)

    def p(self, x, t: float = 0.0):
        return self._modes(np.asarray(x) - self.u * t, self.p0, self.p_amp, self.p_phase, self.p_k)

    # -- exact cell averages over [xa, xb] --
    @staticmethod
    def _avg(xa, xb, base, amp, phase, k):
        xa = np.asarray(xa, dtype=np.float64)
        xb = np.asarray(xb, dtype=np.float64)
        out = np.full(xa.shape, base, dtype=np.float64)
        h = xb - xa
        for a, ph, kk in zip(amp, phase, k):
            w = TWO_PI * kk
            out = out + a * (np.cos(w * xa + ph) - np.cos(w * xb + ph)) / (w * h)
        return out

    def rho_avg(self, xa, xb, t: float = 0.0):
        s = self.u * t
        return self._avg(np.asarray(xa) - s, np.asarray(xb) - s, self.rho0, self.rho_amp,
                         self.rho_phase, self.rho_k)

    def p_avg(self, xa, xb, t: float = 0.0):
        s = self.u * t
        return self._avg(np.asarray(xa) - s, np.asarray(xb) - s, self.p0, self.p_amp,
                         self.p_phase, self.p_k)

    @property
    def pressure_is_constant(self) -> bool:
        return len(self.p_amp) == 0 or not np.any(self.p_amp)


def conserved(rho, u, p, gamma: float = GAMMA):
    """(rho, rho u, E = p/(gamma-1) + rho u^2 / 2) stacked on a new last axis."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), rho.shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape)
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u], axis=-1)


def nodal_state(f: Field1D, x_nodes, gamma: float = GAMMA):
    """Conserved variables at the given node coordinates (any shape) -> [..., 3]."""
    x = np.asarray(x_nodes, dtype=np.float64)
    return conserved(f.rho(x), f.u, f.p(x), gamma)


def cell_average_state(f: Field1D, ncells: int, x0: float = 0.0, x1: float = 1.0,
                       gamma: float = GAMMA):
    """Exact cell averages [ncells, 3]; exact because rho u and E are linear in rho and p."""
    edges = x0 + (x1 - x0) * np.arange(ncells + 1) / ncells
    ra = f.rho_avg(edges[:-1], edges[1:])
    pa = f.p_avg(edges[:-1], edges[1:])
    return np.stack([ra, ra * f.u, pa / (gamma - 1.0) + 0.5 * ra * f.u * f.u], axis=-1)


# ---------------------------------------------------------------------------
# the named workloads
# ---------------------------------------------------------------------------

def sine() -> Field1D:
    return Field1D(rho_amp=np.array([0.2]), rho_phase=np.array([0.0]), rho_k=np.array([1.0]))


def modes4(seed: int = DEFAULT_SEED) -> Field1D:
    g = np.random.Generator(np.random.PCG64(seed))
    a = g.uniform(0.0, 0.05, size=4)
    ph = g.uniform(0.0, TWO_PI, size=4)
    return Field1D(rho_amp=a, rho_phase=ph, rho_k=np.arange(1, 5, dtype=np.float64))


def random_state(rng: np.random.Generator, shape, rho=(0.5, 2.0), u=(-1.0, 1.0), p=(0.5, 2.0),
                 gamma: float = GAMMA):
    """Independent random positive states (for predictor / Riemann unit cases)."""
    r = rng.uniform(*rho, size=shape)
    v = rng.uniform(*u, size=shape)
    pp = rng.uniform(*p, size=shape)
    return conserved(r, v, pp, gamma)


@dataclass
class Request:
    rid: int
    arrival: float
    cells: int
    degree: int
    field: Field1D
    t_end: float = 0.5


def serving_requests(count: int = 4096, seed: int = DEFAULT_SEED, rate: float = 1.0,
                     min_cells: int = 64, max_cells: int = 65536, degrees=(1, 7),
                     t_end: float = 0.5):
    """Poisson stream of independent solves (arrival times in seconds for the given rate)."""
    g = np.random.Generator(np.random.PCG64(seed))
    gaps = g.exponential(1.0 / rate, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    cells = np.rint(np.exp(g.uniform(np.log(min_cells), np.log(max_cells), size=count))).astype(int)
    degs = g.integers(degrees[0], degrees[1] + 1, size=count)
    out = []
    for i in range(count):
        a_r = g.uniform(0.0, 0.1 / 3.0, size=3)
        ph_r = g.uniform(0.0, TWO_PI, size=3)
        a_p = g.uniform(0.0, 0.1 / 3.0, size=3)
        ph_p = g.uniform(0.0, TWO_PI, size=3)
        k = np.arange(1, 4, dtype=np.float64)
        f = Field1D(rho_amp=a_r, rho_phase=ph_r, rho_k=k, u=0.5, p_amp=a_p, p_phase=ph_p, p_k=k)
        out.append(Request(i, float(arrivals[i]), int(cells[i]), int(degs[i]), f, t_end))
    return out


def reacting_state(x, seed: int = 1, u0: float = 0.5, gamma: float = GAMMA):
    """(rho, rho u, E, rho c1, rho c2) at points x (any shape) for the 1D
    two-component reacting flow: rho = 1 + sum_{k=1..3} a_k sin(2 pi k x + phi_k),
    p = 1 + 0.5 sum_k a_k cos(2 pi k x + phi_k), a_k ~ U(0, 0.1), phi_k ~ U(0, 2 pi),
    velocity u0, c1 = 0.5 + 0.3 sin 2 pi x, c2 = 0.2 cos 2 pi x."""
    g = np.random.default_rng(seed)
    a, ph = g.uniform(0, 0.1, 3), g.uniform(0, TWO_PI, 3)
    x = np.asarray(x, dtype=np.float64)
    k = np.arange(1, 4).reshape((3,) + (1,) * x.ndim)
    arg = TWO_PI * k * x + ph.reshape(k.shape)
    rho = 1 + (a.reshape(k.shape) * np.sin(arg)).sum(0)
    p = 1 + 0.5 * (a.reshape(k.shape) * np.cos(arg)).sum(0)
    c1 = 0.5 + 0.3 * np.sin(TWO_PI * x)
    c2 = 0.2 * np.cos(TWO_PI * x)
    return np.stack([rho, rho * u0, p / (gamma - 1) + 0.5 * rho * u0 ** 2, rho * c1, rho * c2], -1)


def ode_state(npts: int, c1: float = 1.0, c2: float = 0.0, gamma: float = GAMMA):
    """The uniform state of the ODE initial-value problem of Sec. 2.1: rho = 1,
    u = 1, p = 1, species (c1, c2), repeated at npts points."""
    U = np.array([1.0, 1.0, 1.0 / (gamma - 1) + 0.5, c1, c2])
    return np.tile(U, (npts, 1))


# Table classical_tests_1d: primitive (rho, u, p) left / right of x = 0.5, t_final = 0.15
RIEMANN_TESTS = {1: ((1.000, 0.000, 1.000), (0.125, 0.000, 0.100)),
                 2: ((0.445, 0.698, 3.528), (0.500, 0.000, 0.571)),
                 3: ((1.000, 1.000, 1.000), (1.000, -1.000, 1.000)),
                 4: ((1.000, -1.000, 1.000), (1.000, 1.000, 1.000))}


def riemann_initial(x, test: int, gamma: float = GAMMA):
    """Conserved (rho, rho u, E) of Riemann problem `test` at points x (jump at 0.5)."""
    L, R = RIEMANN_TESTS[test]
    x = np.asarray(x, dtype=np.float64)
    prim = np.where(x[..., None] < 0.5, np.array(L), np.array(R))
    rho, u, p = prim[..., 0], prim[..., 1], prim[..., 2]
    return np.stack([rho, rho * u, p / (gamma - 1) + 0.5 * rho * u * u], -1)


# Exact solution of the Riemann problem of the 1D Euler equations (ideal gas),
# written from the mathematics of the problem: the star pressure p* is the root
# of f(p) = f_L(p) + f_R(p) + (u_R - u_L), where for side K with state
# (rho_K, u_K, p_K) and sound speed c_K
#     f_K(p) = (p - p_K) sqrt(A_K / (p + B_K)),  A_K = 2 / ((g+1) rho_K),
#                                               B_K = (g-1)/(g+1) p_K        (p > p_K: shock)
#     f_K(p) = 2 c_K / (g-1) ((p/p_K)^((g-1)/(2g)) - 1)                     (p <= p_K: rarefaction)
# (the Rankine-Hugoniot and isentropic relations across the nonlinear waves),
# solved by Newton's method; u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2; the
# solution is self-similar in x/t and is sampled wave by wave.

def _riemann_fk(p, rho, pk, ck, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    r = (p / pk) ** ((g - 1.0) / (2.0 * g))
    return 2.0 * ck / (g - 1.0) * (r - 1.0), 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def riemann_star_state(left, right, g=1.4, tol=1e-14, max_iter=100):
    """(p*, u*) of the Riemann problem with primitive states left, right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("the initial data generate vacuum")
    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(max_iter):
        fl, dl = _riemann_fk(p, rl, pl, cl, g)
        fr, dr = _riemann_fk(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dl + dr)
        if pn < 0:
            pn = 1e-8
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _riemann_fk(p, rl, pl, cl, g)
    fr, _ = _riemann_fk(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def riemann_sample(left, right, xi, g=1.4):
    """Primitive (rho, u, p) of the exact solution at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = riemann_star_state(left, right, g)
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


def riemann_solution(left, right, x, t, x0=0.5, g=1.4):
    """Exact (rho, u, p) at points x and time t > 0 for an initial jump at x0."""
    return riemann_sample(left, right, (np.asarray(x, dtype=np.float64) - x0) / t, g)
