"""Mortar (mixed mass) matrix between nonconforming grids (Sec. 3.1).

P_int,ext[i, j] = <phi_j^ext, theta_i^int>, the L2 product of interior test
function i and exterior basis function j over the common surface; the exterior
mortar is its transpose, P_ext,int = P_int,ext^T (Sec. 3.1 and Sec. 5.4).

The paper assumes both grids cover one polyhedral surface.  Two grids of a curved
surface (rotated, jittered icospheres) are different polyhedra, so the common
surface is read through central projection from a centre point c0 (the origin by
default; both surfaces are star-shaped about it): every exterior triangle sigma is
projected onto the plane of each interior triangle tau along rays from c0, which
gives a triangle sigma' in that plane, and on tau the exterior basis function is
the linear barycentric function of sigma'.  Then

  P_int,ext[i, j] = sum_tau sum_sigma  int_{tau cap sigma'} lambda_i^tau lambda_j^sigma' dS,

a polynomial integral that is exact under any triangulation of tau cap sigma'.
For coplanar grids the projection is the identity and this is the plain mortar
matrix of the paper; for identical grids P = M.

The oracle tests every (tau, sigma) pair against a conservative angular bound seen
from c0 (two triangles can only overlap in projection if their angular discs
meet), then clips the survivors exactly (Sutherland-Hodgman against the three edges
of tau) and integrates on a fan triangulation of the clipped polygon with the
degree-4 rule.
"""
from __future__ import annotations

import numpy as np

from .geometry import triangle_geometry
from .quadrature import triangle_rule_degree4


def _angular_discs(v, tri, c0):
    P = v[tri] - c0  # [T,3,3]
    u = P / np.linalg.norm(P, axis=2, keepdims=True)
    cen = u.mean(axis=1)
    cen /= np.linalg.norm(cen, axis=1, keepdims=True)
    ang = np.arccos(np.clip(np.einsum("tkd,td->tk", u, cen), -1.0, 1.0)).max(axis=1)
    return cen, ang


def _clip(poly, s_min_edges):
    """Sutherland-Hodgman clip of a 2D polygon by half-planes f(p) >= 0."""
    for f in s_min_edges:
        if not poly:
            return poly
        out = []
        n = len(poly)
        for k in range(n):
            p, q = poly[k], poly[(k + 1) % n]
            fp, fq = f(p), f(q)
            if fp >= 0:
                out.append(p)
            if (fp >= 0) != (fq >= 0):
                t = fp / (fp - fq)
                out.append(p + t * (q - p))
        poly = out
    return poly


_HALF_PLANES = (lambda p: p[0], lambda p: p[1], lambda p: 1.0 - p[0] - p[1])


def _bary2(tri2, p):
    """Barycentric coordinates of 2D points p [...,2] in the 2D triangle tri2 [3,2]."""
    a, b, c = tri2
    Mx = np.array([[b[0] - a[0], c[0] - a[0]], [b[1] - a[1], c[1] - a[1]]])
    st = np.linalg.solve(Mx, (p - a).T).T
    return np.stack([1.0 - st[..., 0] - st[..., 1], st[..., 0], st[..., 1]], axis=-1)


def mortar_matrix(v_int, t_int, v_ext, t_ext, center=(0.0, 0.0, 0.0)):
    """Dense P_int,ext [N_int, N_ext] (float64)."""
    v_int = np.asarray(v_int, dtype=np.float64)
    v_ext = np.asarray(v_ext, dtype=np.float64)
    t_int = np.asarray(t_int, dtype=np.int64)
    t_ext = np.asarray(t_ext, dtype=np.int64)
    c0 = np.asarray(center, dtype=np.float64)
    gi = triangle_geometry(v_int, t_int)
    ci, ai = _angular_discs(v_int, t_int, c0)
    ce, ae = _angular_discs(v_ext, t_ext, c0)
    pts, w = triangle_rule_degree4()
    P = np.zeros((len(v_int), len(v_ext)))
    for tau in range(len(t_int)):
        cosang = np.clip(ce @ ci[tau], -1.0, 1.0)
        cand = np.nonzero(np.arccos(cosang) <= ai[tau] + ae + 1e-9)[0]
        a, e1, e2, n = gi["a"][tau], gi["e1"][tau], gi["e2"][tau], gi["n"][tau]
        G = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
        Ginv = np.linalg.inv(G)
        for sig in cand:
            X = v_ext[t_ext[sig]] - c0  # [3,3]
            den = X @ n
            if np.any(den == 0.0):
                continue
            scale = ((a - c0) @ n) / den
            if np.any(scale <= 0.0):  # the ray from c0 must meet tau's plane ahead of it
                continue
            Xp = c0 + X * scale[:, None]  # projection onto tau's plane
            rel = Xp - a
            q = (Ginv @ np.stack([rel @ e1, rel @ e2])).T  # [3,2] reference coords in tau
            poly = _clip([q[0], q[1], q[2]], _HALF_PLANES)
            if len(poly) < 3:
                continue
            for m in range(1, len(poly) - 1):
                p0, p1, p2 = poly[0], poly[m], poly[m + 1]
                area2 = (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0])
                if area2 == 0.0:
                    continue
                sp = p0[None, :] + pts[:, 0:1] * (p1 - p0)[None, :] + pts[:, 1:2] * (p2 - p0)[None, :]
                lt = np.stack([1.0 - sp[:, 0] - sp[:, 1], sp[:, 0], sp[:, 1]], axis=-1)
                ls = _bary2(q, sp)
                wq = w * abs(area2) * gi["J"][tau]
                loc = np.einsum("q,qa,qb->ab", wq, lt, ls)
                P[np.ix_(t_int[tau], t_ext[sig])] += loc
    return P
