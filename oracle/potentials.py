"""Field evaluation with the potential operators (Sec. 2.1, eq. representation).

Test infrastructure only: the FP64 reference that the CUDA path is checked against.

For P1 densities phi, psi (vertex values) on a grid and a point x off the surface,

    u(x) = [V psi](x) - [K phi](x)
         = int G(x, y) psi(y) dy - int dG/dn(y)(x, y) phi(y) dy,

with the Green's function and normal derivative of the Galerkin operators
(G = exp(ikr) / (4 pi r), dG/dn(y) = exp(ikr) (1 - ikr) ((x - y) . n(y)) / (4 pi r^3)),
integrated triangle by triangle with the 6-point degree-4 rule of the regular pairs.
With the interior traces this is the interior field u_int of eq. representation:int,
with the exterior traces the scattered field u_ext of eq. representation:ext.
"""
from __future__ import annotations

import numpy as np

from .geometry import triangle_geometry, shape_values
from .helmholtz import helmholtz_kernels
from .quadrature import triangle_rule_degree4


def representation(v, tri, k, points, phi=None, psi=None, chunk=256):
    """u [M] at points [M, 3]; phi or psi may be None (its term is left out)."""
    tri = np.asarray(tri, dtype=np.int64)
    geo = triangle_geometry(v, tri)
    pts, w = triangle_rule_degree4()
    L = shape_values(pts)  # [6, 3]
    Y = geo["a"][:, None, :] + pts[None, :, 0:1] * geo["e1"][:, None, :] + pts[None, :, 1:2] * geo["e2"][:, None, :]
    wj = w[None, :] * geo["J"][:, None]  # [T, 6]
    ny = np.broadcast_to(geo["n"][:, None, :], Y.shape)
    dens_psi = None if psi is None else np.einsum("qa,ta->tq", L, np.asarray(psi, dtype=np.complex128)[tri])
    dens_phi = None if phi is None else np.einsum("qa,ta->tq", L, np.asarray(phi, dtype=np.complex128)[tri])
    Yf, nyf, wf = Y.reshape(-1, 3), ny.reshape(-1, 3), wj.reshape(-1)
    points = np.asarray(points, dtype=np.float64)
    u = np.zeros(len(points), dtype=np.complex128)
    for m0 in range(0, len(points), chunk):
        x = points[m0:m0 + chunk, None, :]
        G, dny, _ = helmholtz_kernels(k, x, Yf[None, :, :], nyf[None, :, :], nyf[None, :, :])
        acc = np.zeros(x.shape[0], dtype=np.complex128)
        if dens_psi is not None:
            acc += G @ (wf * dens_psi.reshape(-1))
        if dens_phi is not None:
            acc -= dny @ (wf * dens_phi.reshape(-1))
        u[m0:m0 + chunk] = acc
    return u
