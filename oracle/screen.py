"""Neumann screen with opposite-order operator preconditioning on a nonconforming
coarse grid (Sec. 4.2, eq. neumannscreen, and the benchmark of Sec. 5.7).

Test infrastructure only: the FP64 reference the CUDA path is checked against.

A sound-hard open screen S: the scattered field is the double-layer potential of the
jump phi of the total field across S, and gamma_N of the total field vanishes on S, so
D phi = gamma_N u_inc with the hypersingular operator D of Sec. 2.1 (whose definition
carries the minus sign: D = -gamma_N K).  phi lies in the space of functions vanishing
on the boundary of S: P1 functions of the interior nodes of the fine grid (the nodes
not on an edge used by a single triangle); the weak form is D_II phi_I = g_I with
g_i = <i k (d . n) exp(i k x . d), theta_i> (the second plane-wave data vector).

Preconditioners (left, strong form):
  mass:  M_II^-1 D_II phi = M_II^-1 g
  opposite order, single layer on a coarse grid c (all its nodes):
         M_II^-1 V^_c M_II^-1 D_II phi = M_II^-1 V^_c M_II^-1 g,
         V^_c = P_cI^T M_c^-1 V_c M_c^-1 P_cI,
with P_cI the mortar matrix between the coarse grid and the fine interior nodes (the
coarse grid's test functions against the fine grid's; the grids are coplanar, so the
projection is the identity on the plane) and V_c the single layer on the coarse grid
at the same wavenumber.
"""
from __future__ import annotations

import numpy as np

from .helmholtz import assemble
from .mass import mass_matrix
from .mortar import mortar_matrix
from .mtf import gmres, plane_wave_data


def boundary_nodes(tri, nv):
    """Boolean [nv]: nodes on an edge that belongs to a single triangle."""
    tri = np.asarray(tri, dtype=np.int64)
    e = np.sort(np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
    u, cnt = np.unique(e, axis=0, return_counts=True)
    out = np.zeros(nv, dtype=bool)
    out[u[cnt == 1].ravel()] = True
    return out


def screen_center(v):
    """A point off the screen's plane on its normal through the centroid (centre of the
    central projection; on coplanar grids the projection does not depend on it)."""
    v = np.asarray(v, dtype=np.float64)
    c = v.mean(axis=0)
    _, _, vt = np.linalg.svd(v - c)
    return tuple(c + vt[2])


def solve_screen(v, tri, k, d, precond="mass", vc=None, tc=None, tol=1e-8, maxiter=2000, n_singular=4):
    """Returns dict(phi [nv] (zero on the boundary), iters, hist)."""
    nv = len(v)
    bnd = boundary_nodes(tri, nv)
    I = np.flatnonzero(~bnd)
    D = assemble(v, tri, k, n_singular=n_singular)["D"][np.ix_(I, I)]
    M = mass_matrix(v, tri)[np.ix_(I, I)]
    _, g = plane_wave_data(v, tri, k, d)
    g = g[I]
    if precond == "mass":
        SA = np.linalg.solve(M, D)
        Sb = np.linalg.solve(M, g)
    elif precond == "oo":
        Vc = assemble(vc, tc, k, n_singular=n_singular)["V"]
        Mc = mass_matrix(vc, tc)
        P = mortar_matrix(vc, tc, v, tri, screen_center(v))
        P = np.asarray(P.todense()) if hasattr(P, "todense") else np.asarray(P)
        R = np.linalg.solve(Mc, P[:, I])  # M_c^-1 P_cI
        Vh = R.T @ Vc @ R
        SA = np.linalg.solve(M, Vh @ np.linalg.solve(M, D))
        Sb = np.linalg.solve(M, Vh @ np.linalg.solve(M, g))
    else:
        raise ValueError(precond)
    x, it, hist = gmres(lambda z: SA @ z, Sb, tol, maxiter)
    phi = np.zeros(nv, dtype=np.complex128)
    phi[I] = x
    return dict(phi=phi, iters=it, hist=hist)
