"""Exact solution of the one-dimensional Riemann problem for the Euler equations of an
ideal gas with constant adiabatic exponent gamma.

TEST INFRASTRUCTURE ONLY (part of the oracle package): it pins the whole PonD step on
Sod-type shock tubes.  Written from the gas-dynamics textbook mathematics: the star
pressure p* solves f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock
(Rankine-Hugoniot) branch for p > p_K and the rarefaction (isentropic, Riemann
invariant) branch for p <= p_K; the solution is self-similar in xi = x / t.
"""
from __future__ import annotations

import math

import numpy as np


def _f_branch(p, rho, pK, a, gamma):
    if p > pK:                                  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pK
        return (p - pK) * math.sqrt(A / (p + B))
    # rarefaction
    return 2.0 * a / (gamma - 1.0) * ((p / pK) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


class RiemannSolution:
    def __init__(self, left, right, gamma):
        rl, ul, pl = map(float, left)
        rr, ur, pr = map(float, right)
        self.gamma = g = float(gamma)
        self.L, self.R = (rl, ul, pl), (rr, ur, pr)
        self.aL = math.sqrt(g * pl / rl)
        self.aR = math.sqrt(g * pr / rr)
        if 2.0 * (self.aL + self.aR) / (g - 1.0) <= ur - ul:
            raise ValueError("vacuum is generated; not handled")

        def F(p):
            return (_f_branch(p, rl, pl, self.aL, g) + _f_branch(p, rr, pr, self.aR, g) + ur - ul)

        lo, hi = 1e-14, max(pl, pr)
        while F(hi) < 0.0:
            hi *= 2.0
        for _ in range(200):                    # bisection to round-off
            mid = 0.5 * (lo + hi)
            if F(mid) > 0.0:
                hi = mid
            else:
                lo = mid
        self.p_star = p = 0.5 * (lo + hi)
        fl = _f_branch(p, rl, pl, self.aL, g)
        fr = _f_branch(p, rr, pr, self.aR, g)
        self.u_star = 0.5 * (ul + ur) + 0.5 * (fr - fl)
        gm = (g - 1.0) / (g + 1.0)
        if p > pl:
            self.rho_star_L = rl * (p / pl + gm) / (gm * p / pl + 1.0)
        else:
            self.rho_star_L = rl * (p / pl) ** (1.0 / g)
        if p > pr:
            self.rho_star_R = rr * (p / pr + gm) / (gm * p / pr + 1.0)
        else:
            self.rho_star_R = rr * (p / pr) ** (1.0 / g)

    def wave_speeds(self):
        """(left-most, right-most) signal speeds."""
        g, p = self.gamma, self.p_star
        rl, ul, pl = self.L
        rr, ur, pr = self.R
        if p > pl:
            sl = ul - self.aL * math.sqrt((g + 1) / (2 * g) * p / pl + (g - 1) / (2 * g))
        else:
            sl = ul - self.aL
        if p > pr:
            sr = ur + self.aR * math.sqrt((g + 1) / (2 * g) * p / pr + (g - 1) / (2 * g))
        else:
            sr = ur + self.aR
        return sl, sr

    def sample(self, xi):
        """(rho, u, p) at similarity coordinates xi = (x - x0) / t (array)."""
        xi = np.asarray(xi, dtype=np.float64)
        out = np.zeros((3,) + xi.shape)
        for idx, s in np.ndenumerate(xi):
            out[(slice(None),) + idx] = self._sample1(float(s))
        return out[0], out[1], out[2]

    def _sample1(self, s):
        g, p, us = self.gamma, self.p_star, self.u_star
        rl, ul, pl = self.L
        rr, ur, pr = self.R
        if s <= us:
            if p > pl:
                SL = ul - self.aL * math.sqrt((g + 1) / (2 * g) * p / pl + (g - 1) / (2 * g))
                return (rl, ul, pl) if s <= SL else (self.rho_star_L, us, p)
            SHL = ul - self.aL
            aSL = self.aL * (p / pl) ** ((g - 1) / (2 * g))
            STL = us - aSL
            if s <= SHL:
                return (rl, ul, pl)
            if s >= STL:
                return (self.rho_star_L, us, p)
            u = 2.0 / (g + 1) * (self.aL + 0.5 * (g - 1) * ul + s)
            a = 2.0 / (g + 1) * (self.aL + 0.5 * (g - 1) * (ul - s))
            return (rl * (a / self.aL) ** (2 / (g - 1)), u, pl * (a / self.aL) ** (2 * g / (g - 1)))
        if p > pr:
            SR = ur + self.aR * math.sqrt((g + 1) / (2 * g) * p / pr + (g - 1) / (2 * g))
            return (rr, ur, pr) if s >= SR else (self.rho_star_R, us, p)
        SHR = ur + self.aR
        aSR = self.aR * (p / pr) ** ((g - 1) / (2 * g))
        STR = us + aSR
        if s >= SHR:
            return (rr, ur, pr)
        if s <= STR:
            return (self.rho_star_R, us, p)
        u = 2.0 / (g + 1) * (-self.aR + 0.5 * (g - 1) * ur + s)
        a = 2.0 / (g + 1) * (self.aR - 0.5 * (g - 1) * (ur - s))
        return (rr * (a / self.aR) ** (2 / (g - 1)), u, pr * (a / self.aR) ** (2 * g / (g - 1)))
