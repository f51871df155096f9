"""Pins of the oracle's geometry, mass matrices and Helmholtz operators (Sec. 2.1,
Sec. 2.4, Sec. 3.1), against closed forms, invariants and the spherical-harmonic
eigenvalues of the operators on the unit sphere."""
import numpy as np
import pytest
from scipy.special import spherical_jn, spherical_yn, sph_harm_y

import bem_inputs as bi
from oracle.geometry import triangle_geometry
from oracle.helmholtz import assemble, singular_pairs, classify_pairs, regular_pairs
from oracle.mass import mass_matrix


def _tri_area_heron(p, q, r):
    a, b, c = np.linalg.norm(q - r), np.linalg.norm(p - r), np.linalg.norm(p - q)
    s = 0.5 * (a + b + c)
    return np.sqrt(max(s * (s - a) * (s - b) * (s - c), 0.0))


def test_geometry_jacobian_normals_gradients():
    v, t = bi.icosphere(2)
    v = bi.ellipsoid(v, [1.3, 0.7, 1.1])
    g = triangle_geometry(v, t)
    for i in (0, 17, 200):
        assert abs(g["J"][i] / 2 - _tri_area_heron(*v[t[i]])) < 1e-14
    cen = v[t].mean(1)
    assert (np.einsum("ij,ij->i", g["n"], cen) > 0).all()  # outward on a convex body
    # grad lambda_a . (v_b - v_0) = delta_ab - delta_a0 ; tangential; sum zero
    for i in (3, 99):
        P = v[t[i]]
        for a in range(3):
            for b in range(3):
                assert abs(g["grad"][i, a] @ (P[b] - P[0]) - ((a == b) - (a == 0))) < 1e-12
        assert np.abs(g["grad"][i] @ g["n"][i]).max() < 1e-13
        assert np.abs(g["grad"][i].sum(0)).max() < 1e-13
        assert np.abs(np.cross(g["n"][i], g["grad"][i]) - g["curl"][i]).max() < 1e-15


def test_mass_matrix_sums_and_closed_form():
    v, t = bi.icosphere(2)
    v = bi.ellipsoid(v, [1.2, 0.8, 1.0])
    M = mass_matrix(v, t)
    areas = np.array([_tri_area_heron(*v[tt]) for tt in t])
    rows = np.zeros(len(v))
    np.add.at(rows, t, np.repeat(areas[:, None] / 3.0, 3, 1))
    assert np.abs(M.sum(1) - rows).max() < 1e-15
    assert abs(M.sum() - areas.sum()) < 1e-13
    # element matrix (|tau|/12) [[2,1,1],[1,2,1],[1,1,2]]
    Mc = np.zeros_like(M)
    loc = (np.ones((3, 3)) + np.eye(3)) / 12.0
    for tt, ar in zip(t, areas):
        Mc[np.ix_(tt, tt)] += ar * loc
    assert np.abs(M - Mc).max() < 1e-16
    assert np.allclose(M, M.T, atol=0) and np.linalg.eigvalsh(M).min() > 0


def test_symmetry_and_transpose_relation():
    v, t = bi.icosphere(1)
    v = bi.ellipsoid(v, [1.2, 0.9, 1.0])
    A = assemble(v, t, 1.7 + 0.2j)
    scale = {op: np.abs(A[op]).max() for op in "VKTD"}
    assert np.abs(A["V"] - A["V"].T).max() < 1e-14 * scale["V"]
    assert np.abs(A["D"] - A["D"].T).max() < 1e-14 * scale["D"]
    assert np.abs(A["T"] - A["K"].T).max() < 1e-14 * scale["K"]


def test_double_layer_vanishes_on_flat_coincident_pairs():
    v, t = bi.icosphere(1)
    g = triangle_geometry(v, t)
    idx = np.arange(len(t))
    nsh, pt, ps = classify_pairs(t.astype(np.int64), idx, idx)
    assert (nsh == 3).all()
    V, K, T, D = singular_pairs(2.0, v, t.astype(np.int64), g, idx, idx, pt, ps, "coincident")
    assert np.abs(K).max() < 1e-17 and np.abs(T).max() < 1e-17
    assert np.abs(V).min() > 0


def _split4(P):
    a, b, c = P
    mab, mbc, mca = (a + b) / 2, (b + c) / 2, (c + a) / 2
    v = np.array([a, b, c, mab, mbc, mca])
    t = np.array([[0, 3, 5], [3, 1, 4], [5, 4, 2], [3, 4, 5]], dtype=np.int32)
    return v, t


@pytest.mark.parametrize("n", [10])
def test_self_similarity_ties_coincident_to_edge_and_vertex_rules(n):
    """Laplace kernel (k = 0), constant density: a midpoint 4-split gives children
    congruent to tau/2 and 1/r is homogeneous of degree -1, so
    I(tau, tau) = 2 * sum over the 12 ordered non-coincident child pairs
    (6 edge-adjacent, 6 vertex-adjacent)."""
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.3, 0.8, 0.0]])
    A1 = assemble(P, np.array([[0, 1, 2]], dtype=np.int32), 0.0, n_singular=n)
    I_tau = A1["V"].sum().real
    v4, t4 = _split4(P)
    A4 = assemble(v4, t4, 0.0, n_singular=n)
    S_all = A4["V"].sum().real
    g = triangle_geometry(v4, t4)
    idx = np.arange(4)
    nsh, pt, ps = classify_pairs(t4.astype(np.int64), idx, idx)
    Vc = singular_pairs(0.0, v4, t4.astype(np.int64), g, idx, idx, pt, ps, "coincident", n)[0]
    S_off = S_all - Vc.sum().real
    assert abs(I_tau - 2.0 * S_off) < 1e-9 * I_tau
    # the coarse rule is visibly worse: the identity really exercises the rules
    A1c = assemble(P, np.array([[0, 1, 2]], dtype=np.int32), 0.0, n_singular=2)
    A4c = assemble(v4, t4, 0.0, n_singular=2)
    Vcc = singular_pairs(0.0, v4, t4.astype(np.int64), g, idx, idx, pt, ps, "coincident", 2)[0]
    bad = abs(A1c["V"].sum().real - 2.0 * (A4c["V"].sum().real - Vcc.sum().real))
    assert bad > 10 * abs(I_tau - 2.0 * S_off)


def test_singular_rules_converge_in_n():
    v, t = bi.icosphere(1)
    v = bi.ellipsoid(v, [1.2, 0.9, 1.0])
    A = {n: assemble(v, t, 2.0, n_singular=n) for n in (3, 5, 9)}
    for op in "VKD":
        e35 = np.abs(A[3][op] - A[9][op]).max()
        e59 = np.abs(A[5][op] - A[9][op]).max()
        assert e59 < 0.2 * e35, op


def test_regular_pairs_match_brute_force_high_order():
    """Well separated pairs: the degree-4 tensor rule agrees with a 100-point
    conical rule to its expected accuracy."""
    from oracle.quadrature import triangle_rule_collapsed
    v, t = bi.icosphere(2)
    g = triangle_geometry(v, t)
    ti = np.array([0, 5, 9])
    si = np.array([200, 311, 150])
    lo = regular_pairs(3.0, g, ti, si)
    hi = regular_pairs(3.0, g, ti, si, rule=triangle_rule_collapsed(10))
    for a, b in zip(lo, hi):
        assert np.abs(a - b).max() < 1e-4 * np.abs(b).max()


def _hn(n, x, d=False):
    return spherical_jn(n, x, d) + 1j * spherical_yn(n, x, d)


def _eigs(n, k):
    lv = 1j * k * spherical_jn(n, k) * _hn(n, k)
    lk = 1j * k * k * spherical_jn(n, k) * _hn(n, k, True) + 0.5
    ld = -1j * k ** 3 * spherical_jn(n, k, True) * _hn(n, k, True)
    return lv, lk, ld


def test_sphere_eigenvalue_formulas_calderon_identity():
    # lambda_K^2 + lambda_V lambda_D = 1/4 (Calderon projector identity on the sphere)
    for n in range(5):
        for k in (0.5, 1.0, 3.0):
            lv, lk, ld = _eigs(n, k)
            assert abs(lk * lk + lv * ld - 0.25) < 1e-12
    # Laplace limits 1/(2n+1), -1/(2(2n+1)), n(n+1)/(2n+1)
    for n in range(4):
        lv, lk, ld = _eigs(n, 1e-7)
        assert abs(lv - 1 / (2 * n + 1)) < 1e-6
        assert abs(lk + 0.5 / (2 * n + 1)) < 1e-6
        assert abs(ld - n * (n + 1) / (2 * n + 1)) < 1e-6


def test_rayleigh_quotients_converge_to_sphere_eigenvalues():
    k = 1.0
    errs = {}
    for L in (1, 2):
        v, t = bi.icosphere(L)
        A = assemble(v, t, k)
        M = mass_matrix(v, t)
        th = np.arccos(np.clip(v[:, 2], -1, 1))
        ph = np.arctan2(v[:, 1], v[:, 0])
        for n in (0, 1, 2):
            u = np.real(sph_harm_y(n, 0, th, ph))
            den = u @ M @ u
            for op, lam in zip("VKD", _eigs(n, k)):
                errs[(L, n, op)] = abs(u @ A[op] @ u / den - lam) / max(abs(lam), 1e-3)
    for n in (0, 1, 2):
        for op in "VKD":
            assert errs[(2, n, op)] < 0.025, (n, op, errs[(2, n, op)])
            assert errs[(1, n, op)] / errs[(2, n, op)] > 3.0, (n, op)  # O(h^2)
