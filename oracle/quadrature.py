"""Quadrature rules for the oracle (Sec. 5.1: "quadrature rules of order four").

Reference triangle: {(s, t) : s >= 0, t >= 0, s + t <= 1}, area 1/2, with
barycentric coordinates (1 - s - t, s, t).

The regular-pair rule is the 6-point fully symmetric rule exact for polynomials of
total degree 4: two orbits of points with barycentric coordinates (a, a, 1 - 2a)
and permutations.  Its four unknowns (a1, w1, a2, w2) are obtained here by
Gauss-Newton on the exact monomial moments, so no tabulated digits are trusted.
"""
from __future__ import annotations

from functools import lru_cache
from math import factorial

import numpy as np


def monomial_moment(i: int, j: int) -> float:
    """Exact integral of s^i t^j over the reference triangle: i! j! / (i+j+2)!."""
    return factorial(i) * factorial(j) / factorial(i + j + 2)


def _orbit_points(a: float):
    b = 1.0 - 2.0 * a
    # barycentric (l0, l1, l2) permutations of (a, a, b); (s, t) = (l1, l2)
    return np.array([[a, a], [a, b], [b, a]])


def _rule_from_params(p):
    a1, w1, a2, w2 = p
    pts = np.vstack([_orbit_points(a1), _orbit_points(a2)])
    w = np.array([w1] * 3 + [w2] * 3)
    return pts, w


@lru_cache(maxsize=None)
def triangle_rule_degree4():
    """6-point symmetric rule exact to degree 4.  Returns (pts [6,2], w [6]) with
    sum(w) = 1/2 (the reference area)."""
    mons = [(i, j) for i in range(5) for j in range(5 - i)]
    target = np.array([monomial_moment(i, j) for i, j in mons])

    def resid(p):
        pts, w = _rule_from_params(p)
        return np.array([np.sum(w * pts[:, 0] ** i * pts[:, 1] ** j) for i, j in mons]) - target

    p = np.array([0.44, 0.11, 0.09, 0.055])
    for _ in range(60):
        r = resid(p)
        Jm = np.empty((len(mons), 4))
        for k in range(4):
            dp = np.zeros(4)
            dp[k] = 1e-7
            Jm[:, k] = (resid(p + dp) - resid(p - dp)) / 2e-7
        step = np.linalg.lstsq(Jm, -r, rcond=None)[0]
        p = p + step
        if np.max(np.abs(step)) < 1e-16:
            break
    pts, w = _rule_from_params(p)
    return pts, w


def gauss_legendre_01(n: int):
    """n-point Gauss-Legendre rule on [0, 1] (nodes, weights)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def triangle_rule_collapsed(n: int):
    """Conical-product (collapsed Gauss) rule on the reference triangle with n^2
    points, exact to total degree 2n - 2 (the map (u, v) -> (u, v (1 - u)) adds
    one degree in u through its Jacobian 1 - u).  Used for brute-force references."""
    u, wu = gauss_legendre_01(n)
    S, V = np.meshgrid(u, u, indexing="ij")
    s = S.ravel()
    t = (V * (1.0 - S)).ravel()
    W = (np.outer(wu, wu) * (1.0 - S)).ravel()
    return np.stack([s, t], axis=1), W
