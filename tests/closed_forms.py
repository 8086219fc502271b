"""Closed-form two-body results used to pin the oracle (independent of its code).

Classical Kepler equations solved by plain bisection:
  elliptic    M = E - e sin E
  hyperbolic  M = e sinh F - F
with the standard position formulas (Murray & Dermott 2000, Ch. 2).
"""
import math

import numpy as np


def bisect(f, lo, hi, iters=200):
    flo = f(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def elliptic_state(mu, a, e, E):
    """In-plane relative position/velocity (orbit in the xy plane, pericentre on +x)."""
    b = a * math.sqrt(1 - e * e)
    edot = math.sqrt(mu / a ** 3) / (1 - e * math.cos(E))
    r = np.array([a * (math.cos(E) - e), b * math.sin(E), 0.0])
    v = np.array([-a * math.sin(E) * edot, b * math.cos(E) * edot, 0.0])
    return r, v


def elliptic_at(mu, a, e, E0, t):
    """Relative state at time t of an orbit that is at eccentric anomaly E0 at t = 0."""
    n = math.sqrt(mu / a ** 3)
    M = (E0 - e * math.sin(E0)) + n * t
    k = math.floor(M / (2 * math.pi))
    Mr = M - 2 * math.pi * k
    E = bisect(lambda E: E - e * math.sin(E) - Mr, -1e-12, 2 * math.pi + 1e-12) + 2 * math.pi * k
    return elliptic_state(mu, a, e, E)


def hyperbolic_state(mu, a, e, F):
    """a < 0 for hyperbolae; in-plane state at hyperbolic anomaly F."""
    aa = -a
    b = aa * math.sqrt(e * e - 1)
    fdot = math.sqrt(mu / aa ** 3) / (e * math.cosh(F) - 1)
    r = np.array([aa * (e - math.cosh(F)), b * math.sinh(F), 0.0])
    v = np.array([-aa * math.sinh(F) * fdot, b * math.cosh(F) * fdot, 0.0])
    return r, v


def hyperbolic_at(mu, a, e, F0, t):
    aa = -a
    n = math.sqrt(mu / aa ** 3)
    M = (e * math.sinh(F0) - F0) + n * t
    F = bisect(lambda F: e * math.sinh(F) - F - M, -50.0, 50.0)
    return hyperbolic_state(mu, a, e, F)


def period(mu, a):
    return 2 * math.pi * math.sqrt(a ** 3 / mu)
