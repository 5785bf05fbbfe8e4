"""Two-body closed form for the oracle's pins.

Kepler's equation M = E - e sin E is solved the way the paper's Kepler solver does it
(Sect. 3.11): a cubic first approximation in s = sin(E/3), then Newton-Raphson, with
bisection as the fallback that always converges.  The cubic start here is the exact real
root of the cubic obtained by expanding arcsin(s) to third order,
    (1 - e) s + (1/6 + 4e/3) s^3 = M/3,
written with a hyperbolic sine (the paper prints this start in a garbled form; only its
role as a first guess matters, the iteration fixes the rest).

The orbit is propagated with Lagrange's f and g functions of the eccentric-anomaly
change, so the orbit's orientation never has to be computed.
"""
from __future__ import annotations

import math

import numpy as np


def kepler_E(M: float, e: float, tol: float = 1e-15) -> float:
    """Eccentric anomaly E for mean anomaly M (any real) and 0 <= e < 1."""
    twopi = 2.0 * math.pi
    k = math.floor((M + math.pi) / twopi)
    Mr = M - k * twopi                      # in [-pi, pi)
    sgn = 1.0 if Mr >= 0 else -1.0
    Ma = abs(Mr)                            # in [0, pi]
    # cubic start: s^3 + p s - q = 0
    c3 = 1.0 / 6.0 + 4.0 * e / 3.0
    p = (1.0 - e) / c3
    q = (Ma / 3.0) / c3
    alpha = 2.0 * math.sqrt(p / 3.0)
    s = alpha * math.sinh(math.asinh(4.0 * q / alpha ** 3) / 3.0) if alpha > 0 else q ** (1 / 3)
    s = max(-1.0, min(1.0, s))
    E = 3.0 * math.asin(s)
    # Newton-Raphson, bracketed so that a step leaving [0, pi] falls back to bisection
    lo, hi = 0.0, math.pi
    for _ in range(200):
        f = E - e * math.sin(E) - Ma
        if f > 0:
            hi = min(hi, E)
        else:
            lo = max(lo, E)
        fp = 1.0 - e * math.cos(E)
        En = E - f / fp
        if not (lo <= En <= hi):
            En = 0.5 * (lo + hi)
        if abs(En - E) < tol:
            E = En
            break
        E = En
    return sgn * E + k * twopi


def two_body_propagate(x1, v1, m1, x2, v2, m2, t):
    """Exact Newtonian two-body state at time t (G = 1, bound orbit)."""
    x1, v1, x2, v2 = (np.asarray(a, dtype=float) for a in (x1, v1, x2, v2))
    M = m1 + m2
    X = (m1 * x1 + m2 * x2) / M
    V = (m1 * v1 + m2 * v2) / M
    r0v = x2 - x1
    v0v = v2 - v1
    r0 = np.linalg.norm(r0v)
    v02 = v0v @ v0v
    a = 1.0 / (2.0 / r0 - v02 / M)
    if a <= 0:
        raise ValueError("unbound orbit")
    n = math.sqrt(M / a ** 3)
    ecosE = 1.0 - r0 / a
    esinE = (r0v @ v0v) / math.sqrt(M * a)
    e = math.hypot(ecosE, esinE)
    E0 = math.atan2(esinE, ecosE)
    M0 = E0 - esinE
    E = kepler_E(M0 + n * t, e)
    dE = E - E0
    r = a * (1.0 - e * math.cos(E))
    f = 1.0 - (a / r0) * (1.0 - math.cos(dE))
    g = t - (dE - math.sin(dE)) / n
    fdot = -a * a * n * math.sin(dE) / (r * r0)
    gdot = 1.0 - (a / r) * (1.0 - math.cos(dE))
    rv = f * r0v + g * v0v
    vv = fdot * r0v + gdot * v0v
    Xt = X + V * t
    return (Xt - m2 / M * rv, V - m2 / M * vv, Xt + m1 / M * rv, V + m1 / M * vv)


def binary(m1, m2, a, e, phase_at_apo=True):
    """Positions/velocities (3, 2) of a two-body orbit in its COM frame, at apoapsis."""
    M = m1 + m2
    r = a * (1 + e)
    v = math.sqrt(M * (2.0 / r - 1.0 / a))
    rel_x = np.array([r, 0.0, 0.0])
    rel_v = np.array([0.0, v, 0.0])
    pos = np.stack([-m2 / M * rel_x, m1 / M * rel_x], axis=1)
    vel = np.stack([-m2 / M * rel_v, m1 / M * rel_v], axis=1)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel)


def period(m1, m2, a):
    return 2.0 * math.pi * math.sqrt(a ** 3 / (m1 + m2))
