"""FP64 CPU oracle of the spectral-bound sources -- TEST INFRASTRUCTURE ONLY.

The paper asks for a rescaling before the sign iteration so that the spectrum lies where the
Newton-Schulz map converges (Sec. "Linear-Scaling Electronic Structure Calculations", after Eq. NS2)
and names no norm. Three interval sources for A = T_J(S)^-1 T_J(H0) (real spectrum: A is similar to
the symmetric L^-1 T_J(H0) L^-T) are defined here the way the library defines them:

  gershgorin(A)            [min_i a_ii - r_i, max_i a_ii + r_i], r_i = sum_{j != i} |a_ij|
  power_bounds(A, lo, hi)  k steps of the power iteration on (A - lo I) and on (hi I - A) from the
                           start vector 1 + (i mod 7)/7, each normalised after every step; the last norm
                           estimates hi_true - lo and hi - lo_true; the estimates are widened by 5 % of
                           their width on each side and clipped to [lo, hi]
  learned_interval(y, ..)  the network's (lo, hi) ordered, widened by 1 % of the width (the network is
                           trained on the power interval, which is already widened), clipped to the
                           Gershgorin interval; step budget ceil(1.5 * max(16 y2, 1)) + 3 in [4, max_iter]

and the scale the sign iteration uses for an interval at mu:

  scale_alpha(lam, lam_g, mu) = max(alpha(lam), alpha(lam_g) / 1.7),  alpha([l, h]) = max(h - mu, mu - l)

Since the Gershgorin interval contains the spectrum, every eigenvalue of X_0 = (A - mu I)/alpha lies in
[-1.7, 1.7], inside (-sqrt(3), sqrt(3)) where x -> x (3 - x^2)/2 keeps its sign and converges.
"""
from __future__ import annotations

import math

import numpy as np


def gershgorin(A: np.ndarray):
    d = np.diag(A)
    r = np.sum(np.abs(A), axis=1) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


def power_bounds(A: np.ndarray, lo: float, hi: float, iters: int = 30):
    """Power-iteration interval (see the module docstring), FP64."""
    n = A.shape[0]
    x0 = 1.0 + (np.arange(n) % 7) / 7.0
    u = x0 / np.linalg.norm(x0)
    v = u.copy()
    eu = ev = 0.0
    for _ in range(iters):
        u2 = A @ u - lo * u
        v2 = hi * v - A @ v
        eu = float(np.linalg.norm(u2))
        ev = float(np.linalg.norm(v2))
        u = u2 / eu if eu > 0 else u2
        v = v2 / ev if ev > 0 else v2
    ehi, elo = lo + eu, hi - ev
    w = max(ehi - elo, 1e-12)
    plo, phi = max(elo - 0.05 * w, lo), min(ehi + 0.05 * w, hi)
    if not (plo < phi) or not (math.isfinite(plo) and math.isfinite(phi)):
        plo, phi = lo, hi
    return plo, phi


def learned_interval(y, lam_g, max_iter: int):
    """Interval and step budget from the network outputs y = (lo, hi, steps / 16)."""
    a, b = float(y[0]), float(y[1])
    if a > b:
        a, b = b, a
    w = max(b - a, 1e-6)
    lo, hi = max(a - 0.01 * w, lam_g[0]), min(b + 0.01 * w, lam_g[1])
    if not (lo < hi) or not (math.isfinite(lo) and math.isfinite(hi)):
        lo, hi = lam_g
    k = 16.0 * float(y[2])
    bud = int(math.ceil(1.5 * max(k, 1.0))) + 3 if math.isfinite(k) else max_iter
    return (lo, hi), min(max(bud, 4), max_iter)


def alpha(lam, mu: float) -> float:
    return max(lam[1] - mu, mu - lam[0])


def scale_alpha(lam, lam_g, mu: float) -> float:
    return max(alpha(lam, mu), alpha(lam_g, mu) / 1.7)
