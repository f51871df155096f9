"""Discrete multiple-traces formulation and its solution (Sec. 2.2, Sec. 3.3, Sec. 5.1).

Unknowns (Sec. 2.2): v_ext, w_ext on the exterior grid (phi_ext = -gamma_D^+ p,
psi_ext = -gamma_N^+ p) and v_int, w_int on the interior grid (phi_int = gamma_D^- p,
psi_int = gamma_N^- p).

Sign reading.  Substituting the transmission conditions -phi_ext = phi_int and
-(1/rho_ext) psi_ext = (1/rho_int) psi_int into the identity terms of the two
Calderon systems of Sec. 2.2 gives

  [ -K_e   V_e   -1/2 P_ei          0                ] [v_e]   [-f]
  [  D_e   T_e    0                -1/2 (re/ri) P_ei ] [w_e] = [-g]
  [ 1/2 P_ie  0   -K_i              V_i              ] [v_i]   [ 0]
  [  0  1/2 (ri/re) P_ie   D_i      T_i              ] [w_i]   [ 0]

("derived").  The matrix printed in eq. (mtf:discrete) carries the opposite sign on
all four transfer blocks ("printed"); it equals S A S with S = diag(I, I, -I, -I),
so its solution is the derived one with the interior potentials negated.  The
derived variant is the default, so that v_int, w_int are phi_int, psi_int.

Data (Sec. 2.2 and eq. planewave): f_j = <u_inc, theta_j>, g_j = <d u_inc/dn, theta_j>
on the exterior grid with u_inc = exp(i k_ext x . d), d u_inc/dn = i k_ext (d . n) u_inc;
the same tests of a point source's field (the fundamental solution with its pole in
the exterior medium), or data given by the caller.

Mass-matrix preconditioning (Sec. 3.3): left multiplication by
blockdiag(M_ext^-1, M_ext^-1, M_int^-1, M_int^-1).  GMRES (Sec. 5.1): no restart,
x0 = 0, stopping when the 2-norm of the preconditioned residual is at most
tol times the 2-norm of the preconditioned right-hand side.
"""
from __future__ import annotations

import numpy as np

from .geometry import triangle_geometry, shape_values
from .helmholtz import assemble
from .mass import mass_matrix
from .mortar import mortar_matrix
from .quadrature import triangle_rule_degree4


def plane_wave_data(v, tri, k, d, amp=1.0):
    """f, g [N] of the plane wave amp * exp(i k x . d) tested with P1 functions."""
    tri = np.asarray(tri, dtype=np.int64)
    geo = triangle_geometry(v, tri)
    pts, w = triangle_rule_degree4()
    L = shape_values(pts)
    X = geo["a"][:, None, :] + pts[None, :, 0:1] * geo["e1"][:, None, :] + pts[None, :, 1:2] * geo["e2"][:, None, :]
    d = np.asarray(d, dtype=np.float64)
    u = amp * np.exp(1j * k * (X @ d))  # [T,q]
    dn = 1j * k * (geo["n"] @ d)[:, None] * u
    wj = w[None, :] * geo["J"][:, None]
    fl = np.einsum("tq,tq,qa->ta", wj, u, L)
    gl = np.einsum("tq,tq,qa->ta", wj, dn, L)
    N = len(v)
    f = np.zeros(N, dtype=np.complex128)
    g = np.zeros(N, dtype=np.complex128)
    np.add.at(f, tri, fl)
    np.add.at(g, tri, gl)
    return f, g


def point_source_data(v, tri, k, src, amp=1.0):
    """f, g [N] of the point-source field u = amp exp(i k r) / (4 pi r), r = |x - src|
    (the fundamental solution with its pole at src), tested with P1 functions:
    du/dn = u (i k - 1/r) ((x - src) . n) / r."""
    tri = np.asarray(tri, dtype=np.int64)
    geo = triangle_geometry(v, tri)
    pts, w = triangle_rule_degree4()
    L = shape_values(pts)
    X = geo["a"][:, None, :] + pts[None, :, 0:1] * geo["e1"][:, None, :] + pts[None, :, 1:2] * geo["e2"][:, None, :]
    R = X - np.asarray(src, dtype=np.float64)
    r = np.linalg.norm(R, axis=-1)  # [T,q]
    u = amp * np.exp(1j * k * r) / (4.0 * np.pi * r)
    dn = u * (1j * k - 1.0 / r) * np.einsum("tqd,td->tq", R, geo["n"]) / r
    wj = w[None, :] * geo["J"][:, None]
    fl = np.einsum("tq,tq,qa->ta", wj, u, L)
    gl = np.einsum("tq,tq,qa->ta", wj, dn, L)
    N = len(v)
    f = np.zeros(N, dtype=np.complex128)
    g = np.zeros(N, dtype=np.complex128)
    np.add.at(f, tri, fl)
    np.add.at(g, tri, gl)
    return f, g


def mtf_blocks(v_ext, t_ext, v_int, t_int, k_ext, k_int, n_singular=4, center=(0.0, 0.0, 0.0)):
    """All matrices of the discrete MTF: operators on both grids, masses, mortar."""
    Ae = assemble(v_ext, t_ext, k_ext, n_singular=n_singular)
    Ai = assemble(v_int, t_int, k_int, n_singular=n_singular)
    Me = mass_matrix(v_ext, t_ext)
    Mi = mass_matrix(v_int, t_int)
    Pie = mortar_matrix(v_int, t_int, v_ext, t_ext, center)
    return dict(ext=Ae, int=Ai, Me=Me, Mi=Mi, Pie=Pie)


def mtf_matrix(blocks, rho_int_over_rho_ext, variant="derived"):
    """Weak-form MTF matrix (dense) in the unknown order (v_e, w_e, v_i, w_i)."""
    Ae, Ai, Pie = blocks["ext"], blocks["int"], blocks["Pie"]
    Pei = Pie.T
    ri_re = rho_int_over_rho_ext
    re_ri = 1.0 / rho_int_over_rho_ext
    s = 1.0 if variant == "derived" else -1.0
    Ne, Ni = Pei.shape
    Z = lambda a, b: np.zeros((a, b))
    return np.block([
        [-Ae["K"], Ae["V"], -0.5 * s * Pei, Z(Ne, Ni)],
        [Ae["D"], Ae["T"], Z(Ne, Ni), -0.5 * s * re_ri * Pei],
        [0.5 * s * Pie, Z(Ni, Ne), -Ai["K"], Ai["V"]],
        [Z(Ni, Ne), 0.5 * s * ri_re * Pie, Ai["D"], Ai["T"]],
    ])


def strong_form(A, b, Me, Mi):
    """Left mass-matrix preconditioning: S A, S b with S = blockdiag(Me^-1, Me^-1, Mi^-1, Mi^-1)."""
    Ne, Ni = len(Me), len(Mi)
    cuts = [0, Ne, 2 * Ne, 2 * Ne + Ni, 2 * Ne + 2 * Ni]
    SA = np.empty_like(A)
    Sb = np.empty_like(b)
    for blk, M in enumerate((Me, Me, Mi, Mi)):
        r = slice(cuts[blk], cuts[blk + 1])
        SA[r] = np.linalg.solve(M, A[r])
        Sb[r] = np.linalg.solve(M, b[r])
    return SA, Sb


def gmres(matvec, b, tol, maxiter):
    """Unrestarted GMRES (Saad-Schultz) from x0 = 0 with modified Gram-Schmidt and
    complex Givens rotations.  Returns (x, iterations, residual history)."""
    n = len(b)
    beta = np.linalg.norm(b)
    hist = [beta]
    if beta == 0.0:
        return np.zeros_like(b), 0, hist
    m = min(maxiter, n)
    Vb = np.zeros((m + 1, n), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    cs = np.zeros(m, dtype=np.float64)
    sn = np.zeros(m, dtype=np.complex128)
    g = np.zeros(m + 1, dtype=np.complex128)
    g[0] = beta
    Vb[0] = b / beta
    j = 0
    for j in range(m):
        w = matvec(Vb[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(Vb[i], w)
            w = w - H[i, j] * Vb[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] != 0.0:
            Vb[j + 1] = w / H[j + 1, j]
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        a, bb = H[j, j], H[j + 1, j]
        if a == 0.0:
            cs[j], sn[j], r = 0.0, 1.0, bb
        else:
            t = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = abs(a) / t
            sn[j] = (a / abs(a)) * np.conj(bb) / t
            r = (a / abs(a)) * t
        H[j, j] = r
        H[j + 1, j] = 0.0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        hist.append(abs(g[j + 1]))
        if abs(g[j + 1]) <= tol * beta:
            j += 1
            break
    else:
        j = m
    y = np.linalg.solve(np.triu(H[:j, :j]), g[:j]) if j > 0 else np.zeros(0)
    x = Vb[:j].T @ y
    return x, j, hist


def solve_transmission(v_ext, t_ext, v_int, t_int, k_ext, k_int, rho_int_over_rho_ext, d,
                       tol=1e-8, maxiter=2000, variant="derived", n_singular=4, blocks=None,
                       center=(0.0, 0.0, 0.0), data=None):
    """Full oracle solve for the plane wave along d, or for the weak-form data
    data = (f, g) on the exterior grid (any incident field) when given.
    Returns dict(v_ext, w_ext, v_int, w_int, iters, hist, blocks)."""
    if blocks is None:
        blocks = mtf_blocks(v_ext, t_ext, v_int, t_int, k_ext, k_int, n_singular, center)
    A = mtf_matrix(blocks, rho_int_over_rho_ext, variant)
    f, g = plane_wave_data(v_ext, t_ext, k_ext, d) if data is None else data
    Ne, Ni = len(v_ext), len(v_int)
    b = np.concatenate([-f, -g, np.zeros(2 * Ni, dtype=np.complex128)])
    SA, Sb = strong_form(A, b, blocks["Me"], blocks["Mi"])
    x, it, hist = gmres(lambda z: SA @ z, Sb, tol, maxiter)
    return dict(v_ext=x[:Ne], w_ext=x[Ne:2 * Ne], v_int=x[2 * Ne:2 * Ne + Ni], w_int=x[2 * Ne + Ni:],
                iters=it, hist=hist, blocks=blocks, f=f, g=g)
