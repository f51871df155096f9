"""The unit-cube workload of Sec. 5.3-5.5 (synthetic structured face grids from
bem_inputs.cube_grid standing in for the paper's Gmsh meshes): the grids themselves
and the mortar matrix between two independent cube grids.

On a polyhedron both grids lie on the same planar faces, so the projection reading
of the mortar (central projection onto the interior triangle's plane) is the plain
coplanar overlap on each face: P1 spaces on both grids contain every globally linear
function, and M_i^-1 P_ie must reproduce them exactly (to rounding), in both
directions -- a stronger property than the constant transfer that holds on curved
surfaces."""
import numpy as np
import pytest

import bem_inputs as bi
from oracle.mass import mass_matrix
from oracle.mortar import mortar_matrix


@pytest.mark.parametrize("n", [1, 3, 7])
def test_cube_grid_is_a_closed_outward_surface(n):
    v, t = bi.cube_grid(n, jitter=0.3, seed=4)
    assert len(v) == 6 * n * n + 2 and len(t) == 12 * n * n
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    cr = np.cross(b - a, c - a)
    assert abs(0.5 * np.linalg.norm(cr, axis=1).sum() - 6.0) < 1e-12  # faces stay planar
    assert abs(np.einsum("ij,ij->i", a, cr).sum() / 6.0 - 1.0) < 1e-12  # outward, volume 1
    e = np.sort(np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    assert np.all(cnt == 2)  # every edge shared by exactly two triangles


@pytest.mark.parametrize("ne,ni", [(4, 3), (5, 2)])
def test_mortar_on_cube_faces_transfers_linear_functions_exactly(ne, ni):
    ve, te = bi.cube_grid(ne, jitter=0.3, seed=1)
    vi, ti = bi.cube_grid(ni, jitter=0.3, seed=2)
    P = mortar_matrix(vi, ti, ve, te, (0.5, 0.5, 0.5))
    P = np.asarray(P.todense()) if hasattr(P, "todense") else np.asarray(P)
    Mi, Me = mass_matrix(vi, ti), mass_matrix(ve, te)
    assert abs(P.sum() - 6.0) < 1e-12
    for f_e, f_i in ((np.ones(len(ve)), np.ones(len(vi))),) + tuple((ve[:, a], vi[:, a]) for a in range(3)):
        assert np.abs(np.linalg.solve(Mi, P @ f_e) - f_i).max() < 1e-12
        assert np.abs(np.linalg.solve(Me, P.T @ f_i) - f_e).max() < 1e-12
