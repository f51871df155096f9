"""P1 mass matrix M_ij = <phi_j, theta_i> on one grid (Sec. 3.1).

Computed with the degree-4 triangle rule, which is exact for the quadratic
products of P1 shape functions.  Returned dense (the grids of the oracle are small).
"""
from __future__ import annotations

import numpy as np

from .geometry import triangle_geometry, shape_values
from .quadrature import triangle_rule_degree4


def mass_matrix(v, tri):
    tri = np.asarray(tri, dtype=np.int64)
    geo = triangle_geometry(v, tri)
    pts, w = triangle_rule_degree4()
    L = shape_values(pts)  # [q,3]
    local = np.einsum("q,qa,qb->ab", w, L, L)[None] * geo["J"][:, None, None]  # [T,3,3]
    N = len(v)
    M = np.zeros((N, N))
    np.add.at(M, (tri[:, :, None].repeat(3, 2), tri[:, None, :].repeat(3, 1)), local)
    return M
