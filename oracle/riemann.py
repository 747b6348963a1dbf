"""Exact Riemann solver for the one-dimensional Euler equations of an ideal gas.

TEST INFRASTRUCTURE ONLY.  Used to pin the oracle's Sod shock tube run
(Sec. III.B of the paper) against the exact solution.

The model's energy equation (Sec. II.B, Eq. 27) carries the energy flux
rho u (2T + u^2/2) with P = rho T (Eq. 10), i.e. internal energy per unit mass
T = P/rho: an ideal gas with gamma = 2 (two translational degrees of freedom).
The solver is the standard two-rarefaction / two-shock construction: the star
pressure p* is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0 with the shock
(Rankine-Hugoniot) and rarefaction (isentropic) branches of f_K, solved with
scipy's brentq; the self-similar solution is then sampled at x/t.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq


def _fK(p, rho, pK, gamma):
    c = np.sqrt(gamma * pK / rho)
    if p > pK:  # shock branch
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pK
        return (p - pK) * np.sqrt(A / (p + B))
    # rarefaction branch
    return 2.0 * c / (gamma - 1.0) * ((p / pK) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(left, right, gamma=2.0):
    """(p*, u*, rho*_L, rho*_R) for left/right = (rho, u, p)."""
    rL, uL, pL = left
    rR, uR, pR = right
    g = lambda p: _fK(p, rL, pL, gamma) + _fK(p, rR, pR, gamma) + (uR - uL)
    p_star = brentq(g, 1e-12, 100.0 * max(pL, pR), xtol=1e-15, rtol=1e-15, maxiter=500)
    u_star = 0.5 * (uL + uR) + 0.5 * (_fK(p_star, rR, pR, gamma) - _fK(p_star, rL, pL, gamma))
    gm = (gamma - 1.0) / (gamma + 1.0)

    def rho_star(rK, pK):
        if p_star > pK:
            return rK * (p_star / pK + gm) / (gm * p_star / pK + 1.0)
        return rK * (p_star / pK) ** (1.0 / gamma)

    return p_star, u_star, rho_star(rL, pL), rho_star(rR, pR)


def wave_speeds(left, right, gamma=2.0):
    """Positions/speeds: (rarefaction head, rarefaction tail, contact, shock) for a
    left rarefaction + right shock (Sod-type) problem."""
    rL, uL, pL = left
    rR, uR, pR = right
    p_s, u_s, rsL, rsR = star_state(left, right, gamma)
    cL = np.sqrt(gamma * pL / rL)
    csL = cL * (p_s / pL) ** ((gamma - 1.0) / (2.0 * gamma))
    cR = np.sqrt(gamma * pR / rR)
    S_shock = uR + cR * np.sqrt((gamma + 1.0) / (2.0 * gamma) * p_s / pR + (gamma - 1.0) / (2.0 * gamma))
    return uL - cL, u_s - csL, u_s, S_shock


def sample(x, t, x0, left, right, gamma=2.0):
    """Exact (rho, u, p) at positions x and time t for a Sod-type problem
    (left rarefaction, contact, right shock) with the jump at x0."""
    rL, uL, pL = left
    rR, uR, pR = right
    p_s, u_s, rsL, rsR = star_state(left, right, gamma)
    head, tail, contact, shock = wave_speeds(left, right, gamma)
    if not (p_s <= pL and p_s > pR):
        raise ValueError("sample() covers the left-rarefaction / right-shock pattern only")
    cL = np.sqrt(gamma * pL / rL)
    s = (np.asarray(x, dtype=np.float64) - x0) / t
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    for n, si in enumerate(s):
        if si < head:
            rho[n], u[n], p[n] = rL, uL, pL
        elif si < tail:  # inside the left rarefaction fan
            uu = 2.0 / (gamma + 1.0) * (cL + (gamma - 1.0) / 2.0 * uL + si)
            cc = 2.0 / (gamma + 1.0) * (cL + (gamma - 1.0) / 2.0 * (uL - si))
            rho[n] = rL * (cc / cL) ** (2.0 / (gamma - 1.0))
            u[n] = uu
            p[n] = pL * (cc / cL) ** (2.0 * gamma / (gamma - 1.0))
        elif si < contact:
            rho[n], u[n], p[n] = rsL, u_s, p_s
        elif si < shock:
            rho[n], u[n], p[n] = rsR, u_s, p_s
        else:
            rho[n], u[n], p[n] = rR, uR, pR
    return rho, u, p
