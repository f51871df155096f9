"""Pins of the oracle's quadrature rules and Sauter-Schwab maps (Sec. 5.1)."""
import numpy as np
import pytest

from oracle.quadrature import (gauss_legendre_01, monomial_moment, triangle_rule_degree4,
                               triangle_rule_collapsed)
from oracle.helmholtz import ss_coincident, ss_edge, ss_vertex


def test_degree4_rule_exact_to_degree_4():
    pts, w = triangle_rule_degree4()
    assert len(w) == 6 and abs(w.sum() - 0.5) < 1e-15
    for i in range(5):
        for j in range(5 - i):
            q = np.sum(w * pts[:, 0] ** i * pts[:, 1] ** j)
            assert abs(q - monomial_moment(i, j)) < 1e-15, (i, j)
    # and genuinely degree 4: some degree-5 monomial is not integrated exactly
    errs = [abs(np.sum(w * pts[:, 0] ** i * pts[:, 1] ** (5 - i)) - monomial_moment(i, 5 - i)) for i in range(6)]
    assert max(errs) > 1e-6


def test_degree4_rule_is_symmetric_and_interior():
    pts, w = triangle_rule_degree4()
    bary = np.stack([1 - pts[:, 0] - pts[:, 1], pts[:, 0], pts[:, 1]], 1)
    assert (bary > 0).all() and (w > 0).all()
    # invariance under the vertex permutations
    for perm in ([1, 2, 0], [0, 2, 1]):
        p2 = bary[:, perm]
        for q in p2:
            assert np.min(np.linalg.norm(bary - q, axis=1)) < 1e-14


def test_monomial_moment_closed_form():
    # brute force of the moment formula with a high-order conical rule
    P, W = triangle_rule_collapsed(8)
    for i in range(6):
        for j in range(6 - i):
            assert abs(np.sum(W * P[:, 0] ** i * P[:, 1] ** j) - monomial_moment(i, j)) < 1e-15


@pytest.mark.parametrize("n", [1, 3, 6])
def test_gauss_legendre_exactness(n):
    x, w = gauss_legendre_01(n)
    for m in range(2 * n):
        assert abs(np.sum(w * x ** m) - 1.0 / (m + 1)) < 1e-15
    assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-8


def _direct(f, n=12):
    # product rule on {0 <= x2 <= x1 <= 1} x {0 <= y2 <= y1 <= 1}
    u, wu = gauss_legendre_01(n)
    a1 = np.repeat(u, n)
    a2 = (u[:, None] * u[None, :]).ravel()
    aw = (wu[:, None] * wu[None, :] * u[:, None]).ravel()
    X1, Y1 = np.meshgrid(a1, a1, indexing="ij")
    X2, Y2 = np.meshgrid(a2, a2, indexing="ij")
    return np.sum(np.outer(aw, aw) * f(X1, X2, Y1, Y2))


def _smooth(x1, x2, y1, y2):
    return np.exp(0.3 * x1 - 0.7 * x2 + 0.5 * y1 + 1.1 * y2) * np.cos(x1 * y2 + 2 * x2 * y1)


@pytest.mark.parametrize("rule", [ss_coincident, ss_edge, ss_vertex])
def test_sauter_schwab_maps_are_exact_changes_of_variables(rule):
    """For a smooth integrand every transformed rule must reproduce the plain 4D
    integral over T^ x T^: a wrong map, Jacobian or missing region fails this."""
    X, Y, W = rule(12)
    got = np.sum(W * _smooth(X[:, 0], X[:, 1], Y[:, 0], Y[:, 1]))
    assert abs(got - _direct(_smooth)) < 1e-13
    assert abs(W.sum() - 0.25) < 1e-14  # |T^|^2
    for P in (X, Y):  # points inside T^
        assert (P[:, 1] >= -1e-15).all() and (P[:, 1] <= P[:, 0] + 1e-15).all() and (P[:, 0] <= 1 + 1e-15).all()


@pytest.mark.parametrize("rule", [ss_coincident, ss_edge, ss_vertex])
def test_sauter_schwab_swap_symmetry(rule):
    """The point sets are symmetric under exchanging the two triangles."""
    X, Y, W = rule(3)
    A = np.concatenate([X, Y, W[:, None]], 1)
    B = np.concatenate([Y, X, W[:, None]], 1)
    A = A[np.lexsort(A.T[::-1])]
    B = B[np.lexsort(B.T[::-1])]
    assert np.abs(A - B).max() < 1e-15
