"""The mass inverse of the multiple-traces system is a left preconditioner only
(S A x = S b in Sec. 5.1's mass-preconditioned GMRES; no inverse inside A, whose
transmission blocks are the mortar's Gram matrices), so a fixed approximation S' of it
applied to both sides leaves the solution unchanged and moves the iteration count by
the change of the preconditioned spectrum.  The mixed-precision solver's FP32 inner
solves rely on this with S' = 6 Chebyshev steps on the Jacobi-scaled mass matrices
(error <= 2 * 3^-6).  Checked here on the oracle's own matrices: the solution matches
the exact-inverse solve to the GMRES tolerance, the iteration count is within a few of
it, and a one-step (Jacobi) S' is visibly worse, so the check discriminates."""
import numpy as np
import pytest

import bem_inputs as bi
from oracle import mtf


def _chebyshev_inverse(M, z, steps, lo=0.5, hi=2.0):
    """k steps of the Chebyshev iteration for M y = z on the spectrum [lo, hi] of
    D^-1 M (D = diag M), from y = 0: the Chebyshev semi-iteration of Golub and Varga
    (1961) in its three-term form."""
    dinv = 1.0 / np.diag(M)
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = theta / delta
    y = np.zeros_like(z)
    r = z.copy()
    d = dinv * r / theta
    rho = 1.0 / sigma
    for _ in range(steps):
        y = y + d
        r = r - M @ d
        rho_next = 1.0 / (2.0 * sigma - rho)
        d = rho_next * rho * d + (2.0 * rho_next / delta) * dinv * r
        rho = rho_next
    return y


@pytest.fixture(scope="module")
def system():
    ve, te, vi, ti = bi.transmission_pair(2, 2, 2)
    blocks = mtf.mtf_blocks(ve, te, vi, ti, 3.0, 4.5)
    A = mtf.mtf_matrix(blocks, 2.0)
    f, g = mtf.plane_wave_data(ve, te, 3.0, np.array([0.0, 0.0, 1.0]))
    Ne, Ni = len(ve), len(vi)
    b = np.concatenate([-f, -g, np.zeros(2 * Ni, dtype=np.complex128)])
    cuts = [0, Ne, 2 * Ne, 2 * Ne + Ni, 2 * Ne + 2 * Ni]
    masses = (blocks["Me"], blocks["Me"], blocks["Mi"], blocks["Mi"])
    return A, b, cuts, masses


def _left(cuts, masses, z, steps):
    out = np.empty_like(z)
    for blk, M in enumerate(masses):
        sl = slice(cuts[blk], cuts[blk + 1])
        out[sl] = np.linalg.solve(M, z[sl]) if steps is None else _chebyshev_inverse(M, z[sl], steps)
    return out


def test_chebyshev_mass_inverse_error_bound(system):
    _, _, cuts, masses = system
    rng = np.random.default_rng(5)
    M = masses[0]
    z = rng.standard_normal(len(M)) + 1j * rng.standard_normal(len(M))
    exact = np.linalg.solve(M, z)
    for steps in (2, 6, 17):
        err = np.linalg.norm(_chebyshev_inverse(M, z, steps) - exact) / np.linalg.norm(exact)
        # the Chebyshev error polynomial on [1/2, 2] is bounded by 2 * 3^-k; the 2-norm of
        # the error grows by at most the square root of the condition of D (mesh-regular)
        assert err < 4 * 2 * 3.0 ** -steps


def test_six_step_left_preconditioner_keeps_solution_and_iterations(system):
    A, b, cuts, masses = system
    xref = np.linalg.solve(A, b)
    x0, it0, _ = mtf.gmres(lambda z: _left(cuts, masses, A @ z, None), _left(cuts, masses, b, None), 1e-8, 2000)
    x6, it6, _ = mtf.gmres(lambda z: _left(cuts, masses, A @ z, 6), _left(cuts, masses, b, 6), 1e-8, 2000)
    x1, it1, _ = mtf.gmres(lambda z: _left(cuts, masses, A @ z, 1), _left(cuts, masses, b, 1), 1e-8, 2000)
    for x in (x0, x6, x1):
        assert np.linalg.norm(x - xref) / np.linalg.norm(xref) < 1e-6
    assert abs(it6 - it0) <= max(3, it0 // 50)
    assert it1 > 1.5 * it0
