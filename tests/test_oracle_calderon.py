"""Calderon-projector pins of the oracle's four operators together (Sec. 2.2, the
Calderon systems eq. calderon:potentials and the operator matrix they define).

For A = [[-K, V], [D, T]] the interior projector is 1/2 I - A and the exterior one
-1/2 I - A; both are projectors exactly when A^2 = I/4.  So, with the oracle's
Galerkin matrices on the unit sphere (exact normals x / |x| at the vertices):

* Cauchy data of a field that solves the Helmholtz equation inside (a plane wave):
  (1/2 M + K) u - V du = 0 and -D u + (1/2 M - T) du = 0, tested against P1
  interpolants of u and du = du/dn; the residual falls at O(h^2).
* Cauchy data of a field radiating outside (a point source inside the sphere):
  (1/2 M - K) g + V dg = 0 and D g + (1/2 M + T) dg = 0 (the exterior relation with
  no incident field), also O(h^2).
* (S A)^2 v = v / 4 with S = blockdiag(M^-1, M^-1) for smooth v, up to
  discretisation error.

A sign error in any of K, T, D, or a dropped identity term, makes a residual of order
one; the last test plants such mistakes and checks that the pins see them."""
import numpy as np
import pytest

import bem_inputs as bi
from oracle.helmholtz import assemble
from oracle.mass import mass_matrix

K_INT = 2.0
DIRECTION = np.array([0.3, -0.5, 0.81]) / np.linalg.norm([0.3, -0.5, 0.81])
SOURCE = np.array([0.1, 0.2, -0.15])  # inside the unit sphere


@pytest.fixture(scope="module")
def ops():
    out = {}
    for L in (1, 2):
        v, t = bi.icosphere(L)
        out[L] = (v, assemble(v, t, K_INT), mass_matrix(v, t))
    return out


def _dual(M, r):
    """Norm of a tested residual r (entries <r_h, theta_i>): sqrt(r^H M^-1 r)."""
    return np.sqrt(abs(np.vdot(r, np.linalg.solve(M, r))))


def _energy(M, *fs):
    return np.sqrt(sum(abs(np.vdot(f, M @ f)) for f in fs))


def _plane_wave(v):
    n = v / np.linalg.norm(v, axis=1)[:, None]
    u = np.exp(1j * K_INT * v @ DIRECTION)
    return u, 1j * K_INT * (n @ DIRECTION) * u


def _point_source(v):
    n = v / np.linalg.norm(v, axis=1)[:, None]
    rv = v - SOURCE
    r = np.linalg.norm(rv, axis=1)
    g = np.exp(1j * K_INT * r) / (4 * np.pi * r)
    return g, g * (1j * K_INT - 1.0 / r) * np.einsum("ij,ij->i", rv, n) / r


def interior_residual(A, M, u, du, sK=1.0, sT=1.0, sD=1.0, half=0.5):
    r1 = (half * M + sK * A["K"]) @ u - A["V"] @ du
    r2 = -sD * A["D"] @ u + (half * M - sT * A["T"]) @ du
    return np.hypot(_dual(M, r1), _dual(M, r2)) / _energy(M, u, du)


def exterior_residual(A, M, g, dg, sK=1.0, sT=1.0, sD=1.0, half=0.5):
    r1 = (half * M - sK * A["K"]) @ g + A["V"] @ dg
    r2 = sD * A["D"] @ g + (half * M + sT * A["T"]) @ dg
    return np.hypot(_dual(M, r1), _dual(M, r2)) / _energy(M, g, dg)


def square_residual(A, M, w, sK=1.0, sT=1.0, sD=1.0):
    Mi = np.linalg.inv(M)
    SA = np.block([[-sK * Mi @ A["K"], Mi @ A["V"]], [sD * Mi @ A["D"], sT * Mi @ A["T"]]])
    z = SA @ (SA @ w) - 0.25 * w
    MM = np.kron(np.eye(2), M)
    return np.sqrt(abs(np.vdot(z, MM @ z)) / abs(np.vdot(w, MM @ w)))


def _smooth_pair(v):
    return np.concatenate([np.exp(1.3j * v[:, 0]) * (1 + v[:, 2]), np.cos(2 * v[:, 0]) + 1j * v[:, 1] ** 2])


def test_interior_calderon_relation_of_a_plane_wave(ops):
    e = {L: interior_residual(A, M, *_plane_wave(v)) for L, (v, A, M) in ops.items()}
    assert e[2] < 0.03, e
    assert e[1] / e[2] > 3.2, e  # O(h^2): the mesh size halves per level


def test_exterior_calderon_relation_of_a_point_source_inside(ops):
    e = {L: exterior_residual(A, M, *_point_source(v)) for L, (v, A, M) in ops.items()}
    assert e[2] < 0.006, e
    assert e[1] / e[2] > 3.2, e


def test_calderon_operator_squares_to_a_quarter(ops):
    for L, (v, A, M) in ops.items():
        assert square_residual(A, M, _smooth_pair(v)) < 3e-3, L


def test_pins_detect_planted_sign_and_identity_mistakes(ops):
    """Mistakes planted in the oracle's matrices (on the CPU): each one raises one of
    the residuals above by more than an order of magnitude."""
    v, A, M = ops[2]
    u, du = _plane_wave(v)
    g, dg = _point_source(v)
    w = _smooth_pair(v)
    good = (interior_residual(A, M, u, du), exterior_residual(A, M, g, dg), square_residual(A, M, w))
    for planted in (dict(sK=-1.0), dict(sT=-1.0), dict(sD=-1.0)):
        bad = (interior_residual(A, M, u, du, **planted), exterior_residual(A, M, g, dg, **planted),
               square_residual(A, M, w, **planted))
        assert max(b / a for a, b in zip(good, bad)) > 10.0, planted
    assert interior_residual(A, M, u, du, half=0.0) > 10 * good[0]
    assert exterior_residual(A, M, g, dg, half=0.0) > 10 * good[1]
