"""Triangle geometry for P1 Galerkin discretisation (Sec. 2.4).

A triangle tau = (a, b, c) is parametrised over the reference triangle by
x(s, t) = a + s (b - a) + t (c - a); the P1 shape functions are the barycentric
coordinates (1 - s - t, s, t).  The surface element is J ds dt with
J = |(b - a) x (c - a)|, and the unit normal (b - a) x (c - a) / J points outward
because triangles are counter-clockwise seen from outside (Sec. 2: the normal is
always the outward one).
"""
from __future__ import annotations

import numpy as np


def triangle_geometry(v, tri):
    """Per-triangle geometry.

    Returns a dict of arrays:
      a, b, c  [T,3]  vertices;  e1 = b - a, e2 = c - a
      J        [T]    |e1 x e2| (twice the area)
      n        [T,3]  outward unit normal
      grad     [T,3,3] surface gradients of the three shape functions
      curl     [T,3,3] surface curls n x grad of the three shape functions
    The gradients use the inverse metric tensor of the parametrisation: for
    phi(s, t), grad_G phi = (g^{-1})_{ij} d_j phi  e_i with g_ij = e_i . e_j.
    """
    v = np.asarray(v, dtype=np.float64)
    tri = np.asarray(tri)
    a, b, c = v[tri[:, 0]], v[tri[:, 1]], v[tri[:, 2]]
    e1, e2 = b - a, c - a
    cr = np.cross(e1, e2)
    J = np.linalg.norm(cr, axis=1)
    n = cr / J[:, None]
    g = np.empty((len(tri), 2, 2))
    g[:, 0, 0] = np.einsum("ij,ij->i", e1, e1)
    g[:, 0, 1] = g[:, 1, 0] = np.einsum("ij,ij->i", e1, e2)
    g[:, 1, 1] = np.einsum("ij,ij->i", e2, e2)
    ginv = np.linalg.inv(g)
    # derivatives of (l0, l1, l2) with respect to (s, t)
    dref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    E = np.stack([e1, e2], axis=1)  # [T, 2, 3]
    grad = np.einsum("kj,tij,tid->tkd", dref, ginv, E)
    curl = np.cross(n[:, None, :], grad)
    return dict(a=a, b=b, c=c, e1=e1, e2=e2, J=J, n=n, grad=grad, curl=curl)


def map_reference(geo, idx, st):
    """Physical points of reference coordinates st [..., 2] on triangles idx."""
    a, e1, e2 = geo["a"][idx], geo["e1"][idx], geo["e2"][idx]
    return a[..., None, :] + st[..., 0:1] * e1[..., None, :] + st[..., 1:2] * e2[..., None, :]


def shape_values(st):
    """P1 shape functions (1 - s - t, s, t) at reference points st [..., 2] -> [..., 3]."""
    s, t = st[..., 0], st[..., 1]
    return np.stack([1.0 - s - t, s, t], axis=-1)
