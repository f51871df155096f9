"""Galerkin P1 matrices of the Helmholtz boundary integral operators (Sec. 2.1).

Green's function  G(x, y) = exp(i k r) / (4 pi r),  r = |x - y|.
For test functions theta_i and trial functions phi_j (P1 on the same grid):

  V_ij = int int G(x,y) phi_j(y) theta_i(x)                     single layer
  K_ij = int int dG/dn(y) phi_j(y) theta_i(x)                   double layer
  T_ij = int int dG/dn(x) phi_j(y) theta_i(x)                   adjoint double layer
  D_ij = int int G(x,y) [curl theta_i(x) . curl phi_j(y)
                         - k^2 (n(x) . n(y)) theta_i(x) phi_j(y)]  hypersingular

D is the weak form of -d/dn(x) int dG/dn(y) (the sign of Sec. 2.1) written by
Maue's integration by parts, the standard reading for P1 elements.  Differentiating
G gives

  dG/dn(y) = exp(ikr) (1 - ikr) ((x - y) . n(y)) / (4 pi r^3)
  dG/dn(x) = exp(ikr) (1 - ikr) ((y - x) . n(x)) / (4 pi r^3).

Quadrature (Sec. 5.1: rules of order four with semi-analytical transformations for
singularities, after Sauter and Schwab):
  * triangle pairs sharing no vertex: tensor product of the 6-point degree-4 rule;
  * coincident, edge-adjacent and vertex-adjacent pairs: the regularising
    transformations of the 4D integral to [0,1]^4, Gauss-Legendre with n points per
    axis.  Coincident pairs use 6 regions and vertex-adjacent pairs 2 regions.
    Edge-adjacent pairs use a 4-region split derived here: the half x1 >= y1 is cut
    by the plane x2 = x1 - y1 + y2 into two Duffy-collapsible regions, and the half
    y1 > x1 is its mirror image.

Sauter-Schwab reference element: T^ = {0 <= x2 <= x1 <= 1} with
chi(x^) = A + x1 (B - A) + x2 (C - B), barycentric (1 - x1, x1 - x2, x2).  Shared
vertices are mapped to A (vertex case) or to A, B (edge case) on both triangles.
"""
from __future__ import annotations

import numpy as np

from .geometry import triangle_geometry, shape_values
from .quadrature import triangle_rule_degree4, gauss_legendre_01

FOUR_PI = 4.0 * np.pi


def helmholtz_kernels(k, x, y, nx, ny):
    """G, dG/dn(y), dG/dn(x) at point pairs (x, y) [..., 3] with normals [..., 3]."""
    d = x - y
    r = np.sqrt(np.sum(d * d, axis=-1))
    e = np.exp(1j * k * r) / (FOUR_PI * r)
    F = e * (1.0 - 1j * k * r) / (r * r)
    dGdny = F * np.sum(d * ny, axis=-1)
    dGdnx = -F * np.sum(d * nx, axis=-1)
    return e, dGdny, dGdnx


def _local_matrices(k, x, y, w, Lx, Ly, nx, ny, cx, cy):
    """Local 3x3 V, K, T, D for P pairs from M point pairs each.

    x, y [P,M,3]; w [P,M] (all Jacobians included); Lx, Ly [P,M,3] shape values;
    nx, ny [P,3]; cx, cy [P,3,3] surface curls of the test / trial shape functions.
    """
    G, dny, dnx = helmholtz_kernels(k, x, y, nx[:, None, :], ny[:, None, :])
    wl = w[..., None] * Lx  # [P,M,3]
    V = np.einsum("pma,pm,pmb->pab", wl, G, Ly)
    K = np.einsum("pma,pm,pmb->pab", wl, dny, Ly)
    T = np.einsum("pma,pm,pmb->pab", wl, dnx, Ly)
    I0 = np.sum(w * G, axis=1)  # int int G
    cc = np.einsum("pad,pbd->pab", cx, cy)
    nn = np.sum(nx * ny, axis=-1)
    D = cc * I0[:, None, None] - (k * k) * nn[:, None, None] * V
    return V, K, T, D


def regular_pairs(k, geo, ti, si, rule=None):
    """Local matrices of pairs (ti[p], si[p]) with the tensor triangle rule."""
    pts, wts = rule if rule is not None else triangle_rule_degree4()
    q = len(wts)
    L = shape_values(pts)  # [q,3]
    a, e1, e2 = geo["a"], geo["e1"], geo["e2"]
    X = a[ti][:, None, :] + pts[None, :, 0:1] * e1[ti][:, None, :] + pts[None, :, 1:2] * e2[ti][:, None, :]
    Y = a[si][:, None, :] + pts[None, :, 0:1] * e1[si][:, None, :] + pts[None, :, 1:2] * e2[si][:, None, :]
    P = len(ti)
    x = np.repeat(X, q, axis=1)  # [P, q*q, 3]  index = i*q + j
    y = np.tile(Y, (1, q, 1))
    w = (np.outer(wts, wts).ravel()[None, :] * (geo["J"][ti] * geo["J"][si])[:, None])
    Lx = np.broadcast_to(np.repeat(L, q, axis=0)[None], (P, q * q, 3))
    Ly = np.broadcast_to(np.tile(L, (q, 1))[None], (P, q * q, 3))
    return _local_matrices(k, x, y, w, Lx, Ly, geo["n"][ti], geo["n"][si], geo["curl"][ti], geo["curl"][si])


# ---------------------------------------------------------------- Sauter-Schwab

def _grid4(n):
    g, gw = gauss_legendre_01(n)
    xi, e1, e2, e3 = [a.ravel() for a in np.meshgrid(g, g, g, g, indexing="ij")]
    w = np.einsum("i,j,k,l->ijkl", gw, gw, gw, gw).ravel()
    return xi, e1, e2, e3, w


def ss_coincident(n):
    """Points (x^, y^) in T^ x T^ and weights for identical triangles: 6 regions,
    Jacobian xi^3 eta1^2 eta2."""
    xi, e1, e2, e3, w = _grid4(n)
    jac = w * xi ** 3 * e1 ** 2 * e2
    maps = [
        ((xi, xi * (1 - e1 + e1 * e2)), (xi * (1 - e1 * e2 * e3), xi * (1 - e1))),
        ((xi * (1 - e1 * e2 * e3), xi * (1 - e1)), (xi, xi * (1 - e1 + e1 * e2))),
        ((xi, xi * e1 * (1 - e2 + e2 * e3)), (xi * (1 - e1 * e2), xi * e1 * (1 - e2))),
        ((xi * (1 - e1 * e2), xi * e1 * (1 - e2)), (xi, xi * e1 * (1 - e2 + e2 * e3))),
        ((xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), (xi, xi * e1 * (1 - e2))),
        ((xi, xi * e1 * (1 - e2)), (xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3))),
    ]
    X = np.concatenate([np.stack(m[0], -1) for m in maps])
    Y = np.concatenate([np.stack(m[1], -1) for m in maps])
    W = np.concatenate([jac] * 6)
    return X, Y, W


def ss_edge(n):
    """Triangles sharing the edge x2 = 0 <-> y2 = 0 (with x1 = y1 on it): 4 regions."""
    xi, e1, e2, e3, w = _grid4(n)
    j1 = w * xi ** 3 * e1 ** 2
    j2 = j1 * e2
    r1 = ((xi, xi * e1 * e3), (xi * (1 - e1 * e2), xi * e1 * (1 - e2)))
    r2 = ((xi, xi * e1), (xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)))
    maps = [r1, r2, (r1[1], r1[0]), (r2[1], r2[0])]
    X = np.concatenate([np.stack(m[0], -1) for m in maps])
    Y = np.concatenate([np.stack(m[1], -1) for m in maps])
    W = np.concatenate([j1, j2, j1, j2])
    return X, Y, W


def ss_vertex(n):
    """Triangles sharing the vertex x^ = 0 <-> y^ = 0: 2 regions, Jacobian xi^3 eta2."""
    xi, e1, e2, e3, w = _grid4(n)
    jac = w * xi ** 3 * e2
    X = np.concatenate([np.stack((xi, xi * e1), -1), np.stack((xi * e2, xi * e2 * e1), -1)])
    Y = np.concatenate([np.stack((xi * e2, xi * e2 * e3), -1), np.stack((xi, xi * e3), -1)])
    W = np.concatenate([jac, jac])
    return X, Y, W


def _ss_bary(xh):
    return np.stack([1.0 - xh[:, 0], xh[:, 0] - xh[:, 1], xh[:, 1]], axis=-1)


def singular_pairs(k, v, tri, geo, ti, si, perm_t, perm_s, kind, n=4):
    """Local matrices of singular pairs of one kind ('coincident'|'edge'|'vertex').

    perm_t[p, m] is the local index (0..2) of triangle ti[p] placed at Sauter-Schwab
    reference vertex m (A, B, C); likewise perm_s for si[p]."""
    X, Y, W = {"coincident": ss_coincident, "edge": ss_edge, "vertex": ss_vertex}[kind](n)
    Bx, By = _ss_bary(X), _ss_bary(Y)  # [M,3] in reordered vertex order
    P = len(ti)
    vt = v[tri[ti][np.arange(P)[:, None], perm_t]]  # [P,3,3] reordered vertex coords
    vs = v[tri[si][np.arange(P)[:, None], perm_s]]
    x = np.einsum("mk,pkd->pmd", Bx, vt)
    y = np.einsum("mk,pkd->pmd", By, vs)
    w = W[None, :] * (geo["J"][ti] * geo["J"][si])[:, None]
    # shape values in the original local order: L[..., perm[m]] = B[..., m]
    Lx = np.zeros((P, len(W), 3))
    Ly = np.zeros((P, len(W), 3))
    for m in range(3):
        Lx[np.arange(P), :, perm_t[:, m]] = Bx[None, :, m]
        Ly[np.arange(P), :, perm_s[:, m]] = By[None, :, m]
    return _local_matrices(k, x, y, w, Lx, Ly, geo["n"][ti], geo["n"][si], geo["curl"][ti], geo["curl"][si])


def classify_pairs(tri, ti, si):
    """Number of shared vertices (0..3) of pairs (ti, si) and the Sauter-Schwab
    vertex permutations of both triangles.

    Canonical placement (it fixes the quadrature points, so both orders of a pair
    see the same points and V, D come out symmetric and T = K^T):
      * edge-adjacent: A = the shared vertex with the smaller global index,
        B = the other shared vertex, C = the remaining vertex of each triangle;
      * vertex-adjacent: A = the shared vertex, then B, C follow the triangle's
        own cyclic vertex order;
      * coincident: the triangle's own vertex order.
    """
    A = tri[ti]  # [P,3]
    B = tri[si]
    eq = A[:, :, None] == B[:, None, :]  # [P,3,3]
    nshared = eq.sum(axis=(1, 2))
    P = len(ti)
    perm_t = np.tile(np.arange(3), (P, 1))
    perm_s = np.tile(np.arange(3), (P, 1))
    for p in np.nonzero(nshared == 2)[0]:
        shared = sorted(set(A[p].tolist()) & set(B[p].tolist()))
        for row, perm in ((A[p], perm_t), (B[p], perm_s)):
            la = int(np.nonzero(row == shared[0])[0][0])
            lb = int(np.nonzero(row == shared[1])[0][0])
            perm[p] = [la, lb, 3 - la - lb]
    for p in np.nonzero(nshared == 1)[0]:
        shared = (set(A[p].tolist()) & set(B[p].tolist())).pop()
        for row, perm in ((A[p], perm_t), (B[p], perm_s)):
            la = int(np.nonzero(row == shared)[0][0])
            perm[p] = [la, (la + 1) % 3, (la + 2) % 3]
    return nshared, perm_t, perm_s


def assemble(v, tri, k, rows=None, n_singular=4, rule=None, chunk=20000):
    """Galerkin V, K, T, D on one grid for wavenumber k (complex allowed).

    rows=None: full [N,N] matrices.  Otherwise rows is an array of test DOFs and the
    result holds only those rows, [len(rows), N], in the given order.
    Returns dict(V=..., K=..., T=..., D=...), complex128.
    """
    v = np.asarray(v, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    N, Tn = len(v), len(tri)
    geo = triangle_geometry(v, tri)
    if rows is None:
        row_of = np.arange(N)
        nrows = N
        test_tris = np.arange(Tn)
    else:
        rows = np.asarray(rows, dtype=np.int64)
        row_of = np.full(N, -1)
        row_of[rows] = np.arange(len(rows))
        nrows = len(rows)
        test_tris = np.nonzero((row_of[tri] >= 0).any(axis=1))[0]
    out = {op: np.zeros(nrows * N, dtype=np.complex128) for op in "VKTD"}

    def scatter(ti, si, mats):
        r = row_of[tri[ti]]  # [P,3]
        c = tri[si]  # [P,3]
        R = np.repeat(r[:, :, None], 3, axis=2)
        C = np.repeat(c[:, None, :], 3, axis=1)
        ok = R >= 0
        flat = (R * N + C)[ok]
        for op, m in zip("VKTD", mats):
            vals = m[ok]
            out[op] += np.bincount(flat, weights=vals.real, minlength=nrows * N) + 1j * np.bincount(
                flat, weights=vals.imag, minlength=nrows * N)

    all_s = np.arange(Tn)
    step = max(1, chunk // Tn)
    for c0 in range(0, len(test_tris), step):
        tt = test_tris[c0:c0 + step]
        ti = np.repeat(tt, Tn)
        si = np.tile(all_s, len(tt))
        nsh, pt, ps = classify_pairs(tri, ti, si)
        reg = nsh == 0
        if reg.any():
            scatter(ti[reg], si[reg], regular_pairs(k, geo, ti[reg], si[reg], rule))
        for kind, cnt in (("coincident", 3), ("edge", 2), ("vertex", 1)):
            sel = nsh == cnt
            if sel.any():
                scatter(ti[sel], si[sel], singular_pairs(k, v, tri, geo, ti[sel], si[sel], pt[sel], ps[sel], kind, n_singular))
    return {op: out[op].reshape(nrows, N) for op in "VKTD"}
