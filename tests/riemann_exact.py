"""Exact solution of the 1D Euler Riemann problem (textbook: Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", ch. 4).  Test helper: an independent source of
maximum wave speeds (for the lambda_max upper bound) and of the Sod solution.
"""
import numpy as np
from scipy.optimize import brentq


def _fK(p, rho, pK, a, g):
    if p > pK:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        return (p - pK) * np.sqrt(A / (p + B))
    return 2.0 * a / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(WL, WR, g=1.4):
    """(p*, u*) for primitive states W = (rho, u, p); None if the data generate vacuum."""
    rL, uL, pL = WL
    rR, uR, pR = WR
    aL, aR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    if 2.0 * (aL + aR) / (g - 1.0) <= uR - uL:
        return None
    f = lambda p: _fK(p, rL, pL, aL, g) + _fK(p, rR, pR, aR, g) + (uR - uL)
    lo, hi = 1e-300, max(pL, pR)
    while f(hi) < 0:
        hi *= 2.0
    ps = brentq(f, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
    us = 0.5 * (uL + uR) + 0.5 * (_fK(ps, rR, pR, aR, g) - _fK(ps, rL, pL, aL, g))
    return ps, us


def max_wave_speed(WL, WR, g=1.4):
    """lambda_max of Eq. (riemann-problem): the smallest lambda with u = u^- for x/t <= -lambda
    and u = u^+ for x/t >= lambda, i.e. max(-S_left, S_right, 0)."""
    rL, uL, pL = WL
    rR, uR, pR = WR
    aL, aR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    st = star_state(WL, WR, g)
    if st is None:
        SL, SR = uL - aL, uR + aR
    else:
        ps, _ = st
        SL = uL - aL * np.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g)) if ps > pL else uL - aL
        SR = uR + aR * np.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g)) if ps > pR else uR + aR
    return max(-SL, SR, 0.0)


def sample(WL, WR, s, g=1.4):
    """Primitive solution (rho, u, p) at similarity coordinate s = x/t (Toro's sampling)."""
    rL, uL, pL = WL
    rR, uR, pR = WR
    aL, aR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    ps, us = star_state(WL, WR, g)
    if s <= us:  # left of contact
        if ps > pL:
            SL = uL - aL * np.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
            if s <= SL:
                return rL, uL, pL
            r = rL * ((ps / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pL + 1))
            return r, us, ps
        SHL = uL - aL
        if s <= SHL:
            return rL, uL, pL
        aSL = aL * (ps / pL) ** ((g - 1) / (2 * g))
        STL = us - aSL
        if s > STL:
            return rL * (ps / pL) ** (1 / g), us, ps
        c = 2 / (g + 1) + (g - 1) / ((g + 1) * aL) * (uL - s)
        return rL * c ** (2 / (g - 1)), 2 / (g + 1) * (aL + (g - 1) / 2 * uL + s), pL * c ** (2 * g / (g - 1))
    if ps > pR:
        SR = uR + aR * np.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
        if s >= SR:
            return rR, uR, pR
        r = rR * ((ps / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pR + 1))
        return r, us, ps
    SHR = uR + aR
    if s >= SHR:
        return rR, uR, pR
    aSR = aR * (ps / pR) ** ((g - 1) / (2 * g))
    STR = us + aSR
    if s <= STR:
        return rR * (ps / pR) ** (1 / g), us, ps
    c = 2 / (g + 1) - (g - 1) / ((g + 1) * aR) * (uR - s)
    return rR * c ** (2 / (g - 1)), 2 / (g + 1) * (-aR + (g - 1) / 2 * uR + s), pR * c ** (2 * g / (g - 1))
