"""Exact solution of the 1D Riemann problem between two stiffened gases.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each side K obeys the stiffened-gas EOS of arXiv 2305.09163 Sec. 2.1 (Eq. "soe"),
rho e = (p + gamma pinf)/(gamma - 1).  With P = p + pinf the side behaves as an
ideal gas in P, so the classical exact solver (Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", Ch. 4) applies per side with p replaced
by P: the star pressure solves f_L(p) + f_R(p) + u_R - u_L = 0, where f_K is the
shock (Rankine-Hugoniot) branch for p > p_K and the isentropic rarefaction
branch otherwise.  Only the material on each side enters its branch, so the two
sides may have different (gamma, pinf).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Side:
    rho: float
    u: float
    p: float
    gamma: float
    pinf: float = 0.0

    @property
    def P(self) -> float:
        return self.p + self.pinf

    @property
    def c(self) -> float:
        return math.sqrt(self.gamma * self.P / self.rho)


def _f_and_df(s: Side, p: float):
    """Velocity jump function f_K(p) and its derivative (Toro Eqs. 4.6-4.7 in P)."""
    g = s.gamma
    P = p + s.pinf
    PK = s.P
    if P > PK:  # shock
        A = 2.0 / ((g + 1.0) * s.rho)
        B = (g - 1.0) / (g + 1.0) * PK
        sq = math.sqrt(A / (P + B))
        f = (P - PK) * sq
        df = sq * (1.0 - 0.5 * (P - PK) / (B + P))
    else:  # rarefaction
        c = s.c
        e = (g - 1.0) / (2.0 * g)
        f = 2.0 * c / (g - 1.0) * ((P / PK) ** e - 1.0)
        df = (1.0 / (s.rho * c)) * (P / PK) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(L: Side, R: Side, tol: float = 1e-14, max_iter: int = 200):
    """Star-region pressure p* and velocity u* (Newton with bisection safeguard)."""
    du = R.u - L.u
    # admissible pressures: P > 0 on both sides
    p_min = max(-L.pinf, -R.pinf)
    lo = p_min + 1e-14 * max(1.0, abs(p_min))
    hi = max(L.p, R.p) + 1.0
    def g(p):
        return _f_and_df(L, p)[0] + _f_and_df(R, p)[0] + du
    while g(hi) < 0.0:
        hi = 2.0 * hi + 1.0
    if g(lo) > 0.0:
        raise ValueError("vacuum generated: no positive star pressure")
    p = 0.5 * (L.p + R.p)
    if not (lo < p < hi):
        p = 0.5 * (lo + hi)
    for _ in range(max_iter):
        fL, dL = _f_and_df(L, p)
        fR, dR = _f_and_df(R, p)
        gv = fL + fR + du
        if gv > 0.0:
            hi = p
        else:
            lo = p
        pn = p - gv / (dL + dR)
        if not (lo < pn < hi):
            pn = 0.5 * (lo + hi)
        if abs(pn - p) <= tol * max(abs(pn + L.pinf), abs(pn + R.pinf), 1e-300):
            p = pn
            break
        p = pn
    fL, _ = _f_and_df(L, p)
    fR, _ = _f_and_df(R, p)
    u = 0.5 * (L.u + R.u) + 0.5 * (fR - fL)
    return p, u


def star_densities(L: Side, R: Side, p: float):
    """Densities on each side of the contact in the star region."""
    out = []
    for s in (L, R):
        g = s.gamma
        P, PK = p + s.pinf, s.P
        if P > PK:
            r = (g - 1.0) / (g + 1.0)
            out.append(s.rho * (P / PK + r) / (r * P / PK + 1.0))
        else:
            out.append(s.rho * (P / PK) ** (1.0 / g))
    return tuple(out)


def wave_speeds(L: Side, R: Side, p: float, u: float):
    """(left head, left tail, right tail, right head) speeds; head == tail for a shock."""
    res = []
    for s, sign in ((L, -1.0), (R, 1.0)):
        g = s.gamma
        P, PK = p + s.pinf, s.P
        if P > PK:
            S = s.u + sign * s.c * math.sqrt((g + 1.0) / (2.0 * g) * P / PK + (g - 1.0) / (2.0 * g))
            res.append((S, S))
        else:
            cs = s.c * (P / PK) ** ((g - 1.0) / (2.0 * g))
            res.append((s.u + sign * s.c, u + sign * cs))
    (hL, tL), (hR, tR) = res
    return hL, tL, tR, hR


def sample(L: Side, R: Side, xi):
    """Density, velocity, pressure and material (0 = left, 1 = right) at x/t = xi."""
    p_s, u_s = star_state(L, R)
    rL_s, rR_s = star_densities(L, R, p_s)
    hL, tL, tR, hR = wave_speeds(L, R, p_s, u_s)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    mat = np.where(xi < u_s, 0, 1)
    for n, x in enumerate(xi):
        if x < u_s:
            s, sign, rs, head, tail = L, -1.0, rL_s, hL, tL
        else:
            s, sign, rs, head, tail = R, 1.0, rR_s, hR, tR
        beyond = (x < head) if sign < 0 else (x > head)
        inside_star = (x > tail) if sign < 0 else (x < tail)
        if beyond:
            rho[n], u[n], p[n] = s.rho, s.u, s.p
        elif inside_star:
            rho[n], u[n], p[n] = rs, u_s, p_s
        else:  # inside a rarefaction fan
            g = s.gamma
            c = 2.0 / (g + 1.0) * (s.c - sign * 0.5 * (g - 1.0) * (s.u - x))
            uu = 2.0 / (g + 1.0) * (-sign * s.c + 0.5 * (g - 1.0) * s.u + x)
            rho[n] = s.rho * (c / s.c) ** (2.0 / (g - 1.0))
            u[n] = uu
            p[n] = s.P * (c / s.c) ** (2.0 * g / (g - 1.0)) - s.pinf
    return rho, u, p, mat


def shocked_state(pre: Side, p_post: float):
    """State behind a right-running shock that raises pre.p to p_post in a material
    at rest ahead of it (pre.u may be nonzero): density, velocity and shock speed,
    from the Rankine-Hugoniot relations in P = p + pinf."""
    g = pre.gamma
    P, PK = p_post + pre.pinf, pre.P
    r = (g - 1.0) / (g + 1.0)
    rho = pre.rho * (P / PK + r) / (r * P / PK + 1.0)
    f, _ = _f_and_df(pre, p_post)
    u = pre.u + f  # velocity jump across a left-facing (right-running into pre) shock
    S = pre.u + pre.c * math.sqrt((g + 1.0) / (2.0 * g) * P / PK + (g - 1.0) / (2.0 * g))
    return rho, u, S
