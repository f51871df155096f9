"""Pins of the oracle's right-hand side, GMRES, MTF system and Mie series, and of
the whole solve against the Mie closed form (Sec. 2.2, Sec. 3.3, Sec. 5.1)."""
import numpy as np
import pytest
from scipy.special import spherical_jn, spherical_yn

import bem_inputs as bi
from oracle.mass import mass_matrix
from oracle.mie import mie_coefficients, mie_traces, mie_potentials
from oracle.mtf import gmres, plane_wave_data, solve_transmission, mtf_blocks
from oracle.quadrature import triangle_rule_collapsed


def test_plane_wave_data_small_k_limits():
    v, t = bi.icosphere(2)
    v = bi.ellipsoid(v, [1.2, 0.8, 1.0])
    d = np.array([0.3, -0.4, np.sqrt(0.75)])
    k = 1e-9
    f, g = plane_wave_data(v, t, k, d)
    M = mass_matrix(v, t)
    assert np.abs(f - M.sum(1)).max() < 1e-8
    gk = g / (1j * k)
    # int_Gamma d . n = 0 on a closed surface (divergence of a constant field); the
    # O(k) remainder is i k int (d.x)(d.n) = i k |Omega|, which is imaginary
    assert abs(gk.sum().real) < 1e-12
    # int (d.n) theta_j: one third of each incident triangle's (d . n) area
    from oracle.geometry import triangle_geometry
    geo = triangle_geometry(v, t)
    ref = np.zeros(len(v))
    np.add.at(ref, t, np.repeat((geo["J"] / 6.0 * (geo["n"] @ d))[:, None], 3, 1))
    assert np.abs(gk - ref).max() < 1e-8


def test_plane_wave_data_against_high_order_rule():
    v, t = bi.icosphere(2)
    d = np.array([0.0, 0.0, 1.0])
    f, g = plane_wave_data(v, t, 2.0, d)
    import oracle.mtf as m
    import oracle.quadrature as q
    orig = q.triangle_rule_degree4
    try:
        m.triangle_rule_degree4 = lambda: triangle_rule_collapsed(10)
        fh, gh = plane_wave_data(v, t, 2.0, d)
    finally:
        m.triangle_rule_degree4 = orig
    assert np.abs(f - fh).max() < 1e-5 * np.abs(fh).max()
    assert np.abs(g - gh).max() < 1e-5 * np.abs(gh).max()


def test_gmres_solves_dense_system_and_residuals_do_not_increase():
    rng = np.random.default_rng(3)
    n = 60
    A = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, hist = gmres(lambda z: A @ z, b, 1e-12, 500)
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-10
    assert np.linalg.norm(A @ x - b) <= 1.01e-12 * np.linalg.norm(b) * 10
    assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(hist, hist[1:]))
    # the recursive residual estimate equals the true residual at every step
    x5, it5, h5 = gmres(lambda z: A @ z, b, 0.0, 5)
    assert it5 == 5 and abs(np.linalg.norm(A @ x5 - b) - h5[-1]) < 1e-10 * h5[0]
    # exact in n steps for a generic matrix
    C = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    xc, itc, _ = gmres(lambda z: C @ z, b[:8], 0.0, 100)
    assert itc == 8 and np.linalg.norm(C @ xc - b[:8]) < 1e-10 * np.linalg.norm(b[:8])


def test_mie_interface_conditions_and_wronskian():
    k_e, k_i, rr = 3.0, 4.5, 2.0
    x = bi.icosphere(2)[0]
    gDp, gNp, gDm, gNm = mie_traces(x, [0, 0, 1], k_e, k_i, rr)
    assert np.abs(gDp - gDm).max() < 1e-12 * np.abs(gDp).max()
    assert np.abs(gNp / 1.0 - gNm / rr).max() < 1e-12 * np.abs(gNp).max()
    for n in range(8):
        for z in (0.7, 3.0, 11.0):
            w = spherical_jn(n, z) * spherical_yn(n, z, True) - spherical_jn(n, z, True) * spherical_yn(n, z)
            assert abs(w - 1.0 / z ** 2) < 1e-12


def test_mie_without_scatterer_is_the_incident_wave():
    x = bi.icosphere(2)[0]
    a, c = mie_coefficients(2.0, 2.0, 1.0)
    assert np.abs(a).max() < 1e-13 and np.abs(c - 1).max() < 1e-12
    gDp, gNp, _, _ = mie_traces(x, [0, 0, 1], 2.0, 2.0, 1.0)
    u = np.exp(2j * x[:, 2])
    assert np.abs(gDp - u).max() < 1e-12
    assert np.abs(gNp - 2j * x[:, 2] * u).max() < 1e-11  # radial derivative on r = 1


def _merr(x, y, M):
    d = x - y
    return np.sqrt(np.real(np.conj(d) @ M @ d) / np.real(np.conj(y) @ M @ y))


@pytest.mark.parametrize("k_e,k_i,rr", [(1.0, 2.0, 1.0), (1.0, 1.5, 2.0)])
def test_bem_converges_to_mie(k_e, k_i, rr):
    d = [0.0, 0.0, 1.0]
    errs = []
    for L in (1, 2):
        ve, te, vi, ti = bi.transmission_pair(L, L, seed=1)
        r = solve_transmission(ve, te, vi, ti, k_e, k_i, rr, d, tol=1e-10)
        ref = mie_potentials(ve, vi, d, k_e, k_i, rr)
        B = r["blocks"]
        errs.append([_merr(r[key], ref[i], B[M]) for i, (key, M) in enumerate(
            [("v_ext", "Me"), ("w_ext", "Me"), ("v_int", "Mi"), ("w_int", "Mi")])])
    errs = np.array(errs)
    assert (errs[1] < 0.05).all(), errs
    assert (errs[0] / errs[1] > 3.0).all(), errs  # O(h^2)


def test_printed_sign_variant_negates_interior_potentials():
    ve, te, vi, ti = bi.transmission_pair(1, 1, seed=2)
    B = mtf_blocks(ve, te, vi, ti, 1.0, 2.0)
    a = solve_transmission(ve, te, vi, ti, 1.0, 2.0, 2.0, [0, 1, 0], tol=1e-12, blocks=B)
    b = solve_transmission(ve, te, vi, ti, 1.0, 2.0, 2.0, [0, 1, 0], tol=1e-12, blocks=B, variant="printed")
    assert a["iters"] == b["iters"]
    for key, s in (("v_ext", 1), ("w_ext", 1), ("v_int", -1), ("w_int", -1)):
        assert np.abs(a[key] - s * b[key]).max() < 1e-9 * np.abs(a[key]).max()
