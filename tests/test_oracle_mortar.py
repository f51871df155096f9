"""Pins of the oracle mortar matrix P_int,ext (Sec. 3.1) and the projection
errors E_int, E_ext (eq. error:projection, Sec. 5.2)."""
import numpy as np
import pytest

import bem_inputs as bi
from oracle.mass import mass_matrix
from oracle.mortar import mortar_matrix


def refine4(v, t):
    """Midpoint 4-split of every triangle (midpoints not moved), with the P1
    prolongation matrix I [N_fine, N_coarse]: coarse functions = I-combinations
    of fine functions."""
    v = np.asarray(v)
    t = np.asarray(t, dtype=np.int64)
    mids = {}
    vl = list(v)
    Irows = [(i, i, 1.0) for i in range(len(v))]

    def mid(a, b):
        key = (min(a, b), max(a, b))
        if key not in mids:
            vl.append((v[a] + v[b]) / 2)
            m = len(vl) - 1
            mids[key] = m
            Irows.extend([(m, a, 0.5), (m, b, 0.5)])
        return mids[key]

    nt = []
    for a, b, c in t:
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        nt += [[a, ab, ca], [ab, b, bc], [ca, bc, c], [ab, bc, ca]]
    I = np.zeros((len(vl), len(v)))
    for r, c, w in Irows:
        I[r, c] += w
    return np.array(vl), np.array(nt, dtype=np.int32), I


def proj_errors(P, Mi, Me):
    Ni, Ne = P.shape
    Eint = np.eye(Ni) - np.linalg.solve(Mi, P) @ np.linalg.solve(Me, P.T)
    Eext = np.eye(Ne) - np.linalg.solve(Me, P.T) @ np.linalg.solve(Mi, P)
    return np.linalg.norm(Eint), np.linalg.norm(Eext), np.abs(Eint).max(), np.abs(Eext).max()


def test_constant_transfer_and_total_area_on_nonconforming_spheres():
    ve, te, vi, ti = bi.transmission_pair(2, 1, seed=1)
    P = mortar_matrix(vi, ti, ve, te)
    Mi = mass_matrix(vi, ti)
    assert np.abs(np.linalg.solve(Mi, P.sum(1)) - 1.0).max() < 1e-13
    assert abs(P.sum() - Mi.sum()) < 1e-12  # area of the interior polyhedron
    assert (P >= -1e-15).all()


def test_identical_grids_give_mass_matrix_and_zero_projection_error():
    v, t = bi.icosphere(2)
    v = bi.ellipsoid(v, [1.3, 0.8, 1.0])
    P = mortar_matrix(v, t, v, t)
    M = mass_matrix(v, t)
    assert np.abs(P - M).max() < 1e-15
    assert max(proj_errors(P, M, M)) < 1e-12


@pytest.mark.parametrize("level", [0, 1])
def test_nested_refinement_matches_prolongation_identity(level):
    """Exterior grid = 4-split of the interior grid (same polyhedron): the coarse
    basis is an exact combination of fine ones, so P_int,ext = I^T M_ext."""
    vc, tc = bi.icosphere(level)
    vc = bi.ellipsoid(vc, [1.2, 0.9, 1.0])
    vf, tf, I = refine4(vc, tc)
    P = mortar_matrix(vc, tc, vf, tf)
    Mf = mass_matrix(vf, tf)
    assert np.abs(P - I.T @ Mf).max() < 1e-15 * 50


def test_nested_refinement_on_the_unit_square():
    vc, tc = bi.unit_square_grid(3)
    vf, tf, I = refine4(vc, tc)
    vf2, tf2, I2 = refine4(vf, tf)
    c0 = (0.5, 0.5, 1.0)
    P = mortar_matrix(vc, tc, vf2, tf2, center=c0)
    assert np.abs(P - (I2 @ I).T @ mass_matrix(vf2, tf2)).max() < 1e-15 * 50


def test_projection_error_decays_with_node_perturbation():
    """Sec. 5.2: the projection error between a fixed grid and a randomly
    perturbed copy decays with the perturbation size."""
    vi, ti = bi.unit_square_grid(6)
    Mi = mass_matrix(vi, ti)
    c0 = (0.5, 0.5, 1.0)
    errs = []
    for sigma in (3e-2, 3e-3, 3e-4, 0.0):
        ve = bi.perturb_square_grid(vi, sigma, seed=7)
        P = mortar_matrix(vi, ti, ve, ti, center=c0)
        Me = mass_matrix(ve, ti)
        errs.append(proj_errors(P, Mi, Me))
    fro_int = [e[0] for e in errs]
    assert fro_int[0] > fro_int[1] > fro_int[2] > fro_int[3]
    assert max(errs[-1]) < 1e-12
    assert fro_int[1] < 0.3 * fro_int[0]


def test_projection_error_with_refined_exterior():
    """Sec. 5.2: fixed coarse interior grid, increasingly fine exterior grids:
    E_int decreases while E_ext increases."""
    vi, ti = bi.unit_square_grid(2)
    Mi = mass_matrix(vi, ti)
    c0 = (0.5, 0.5, 1.0)
    out = []
    for n in (2, 3, 5, 9):
        ve, te = bi.unit_square_grid(n)
        P = mortar_matrix(vi, ti, ve, te, center=c0)
        out.append(proj_errors(P, Mi, mass_matrix(ve, te)))
    assert out[0][0] < 1e-12  # equal grids
    Eint = [o[0] for o in out[1:]]
    Eext = [o[1] for o in out[1:]]
    assert Eint[0] > Eint[-1]
    assert Eext[-1] > Eext[0]
