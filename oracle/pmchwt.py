"""Single-trace formulations (Sec. 2.2): the exterior PMCHWT (eq. pmchwt:ext and eq.
pmchwt:discrete) on nonconforming grids, and below it the exterior Mueller and the
interior PMCHWT and Mueller systems discretised the same way.

Test infrastructure only: the FP64 reference the CUDA path is checked against.

Reading.  The formulation is obtained from the discrete multiple-traces system of
oracle/mtf.py (derived signs) by eliminating the interior potentials with the tested
transmission conditions, M_i v_i = -P_ie v_e and M_i w_i = -(rho_i / rho_e) P_ie w_e,
mapping the interior rows to the exterior grid with P_ei M_i^-1 and subtracting them
from the exterior rows: the identity terms cancel and

  [ -K_e - K^_i              V_e + (rho_i/rho_e) V^_i ] [v_e]   [-f]
  [  D_e + (rho_e/rho_i) D^_i   T_e + T^_i            ] [w_e] = [-g],

  X^_i = P_ei M_i^-1 X_i M_i^-1 P_ie   (the hat transformation of eq. pmchwt:discrete),

with the density ratios of the scaled interior Calderon operator of eq.
(pmchwt:ext).  The unknowns are the exterior potentials of the MTF (v_e = phi_ext =
-gamma_D^+ p; the paper's phi = -phi_ext, hence its right-hand side +f, +g), and the
interior potentials follow from the two transmission conditions above.  Left mass
preconditioning blockdiag(M_e^-1, M_e^-1) and unrestarted GMRES as for the MTF.
"""
from __future__ import annotations

import numpy as np

from .mtf import gmres, mtf_blocks, plane_wave_data


def pmchwt_matrix(blocks, rho_int_over_rho_ext):
    """Weak-form exterior PMCHWT matrix (dense) in the unknown order (v_e, w_e)."""
    Ae, Ai, Pie, Mi = blocks["ext"], blocks["int"], blocks["Pie"], blocks["Mi"]
    R = np.linalg.solve(Mi, Pie)  # M_i^-1 P_ie [Ni, Ne]
    hat = lambda X: R.T @ X @ R  # P_ei M_i^-1 X M_i^-1 P_ie (M_i symmetric)
    ri_re = rho_int_over_rho_ext
    return np.block([
        [-Ae["K"] - hat(Ai["K"]), Ae["V"] + ri_re * hat(Ai["V"])],
        [Ae["D"] + hat(Ai["D"]) / ri_re, Ae["T"] + hat(Ai["T"])],
    ])


def solve_pmchwt(v_ext, t_ext, v_int, t_int, k_ext, k_int, rho_int_over_rho_ext, d, tol=1e-8, maxiter=2000,
                 n_singular=4, blocks=None, center=(0.0, 0.0, 0.0)):
    """Full oracle solve.  Returns dict(v_ext, w_ext, v_int, w_int, iters, hist, blocks)
    with the potentials in the conventions of the MTF solve."""
    if blocks is None:
        blocks = mtf_blocks(v_ext, t_ext, v_int, t_int, k_ext, k_int, n_singular, center)
    A = pmchwt_matrix(blocks, rho_int_over_rho_ext)
    f, g = plane_wave_data(v_ext, t_ext, k_ext, d)
    Me, Mi, Pie = blocks["Me"], blocks["Mi"], blocks["Pie"]
    Ne = len(v_ext)
    SA = np.vstack([np.linalg.solve(Me, A[:Ne]), np.linalg.solve(Me, A[Ne:])])
    Sb = np.concatenate([np.linalg.solve(Me, -f), np.linalg.solve(Me, -g)])
    x, it, hist = gmres(lambda z: SA @ z, Sb, tol, maxiter)
    ve, we = x[:Ne], x[Ne:]
    vi = -np.linalg.solve(Mi, Pie @ ve)
    wi = -rho_int_over_rho_ext * np.linalg.solve(Mi, Pie @ we)
    return dict(v_ext=ve, w_ext=we, v_int=vi, w_int=wi, iters=it, hist=hist, blocks=blocks)


# ---------------------------------------------------------------------------------
# All four single-trace systems of Sec. 2.2 (eq. pmchwt:ext, muller:ext, pmchwt:int,
# muller:int), discretised as eq. pmchwt:discrete ("all other formulations can be
# discretised similarly").
#
# Exterior variants: unknowns v_e, w_e (the MTF's exterior potentials, phi = -v_e),
# the interior Calderon operator scaled by the densities, A_i^rho = [[-K_i, r V_i],
# [D_i / r, T_i]] (r = rho_i / rho_e), mapped to the exterior grid by
# X^ = P_ei M_i^-1 X M_i^-1 P_ie:
#   PMCHWT:  (A_e + A_i^rho^) x = [-f; -g]
#   Mueller: (M_e + A_e - A_i^rho^) x = [-f; -g]
# (the paper's I + (A_e - A_i^rho^) acting on phi = -x; the identity discretised by
# the exterior mass matrix, the "exact projection of the identity").
#
# Interior variants: unknowns v_i, w_i (phi = phi_int, psi = psi_int), the exterior
# operator scaled the other way, A_e^rho = [[-K_e, V_e / r], [r D_e, T_e]], mapped to
# the interior grid by X^ = P_ie M_e^-1 X M_e^-1 P_ei, and the data mapped likewise:
#   PMCHWT:  (A_e^rho^ + A_i) x = [P_ie M_e^-1 f; r P_ie M_e^-1 g]
#   Mueller: (M_i + A_e^rho^ - A_i) x = [P_ie M_e^-1 f; r P_ie M_e^-1 g]
#
# The potentials not solved for follow from the transmission conditions tested on
# the other grid: M_i v_i = -P_ie v_e, M_i w_i = -r P_ie w_e (exterior variants);
# M_e v_e = -P_ei v_i, M_e w_e = -(1/r) P_ei w_i (interior variants).
# Left mass preconditioning with the mass matrix of the unknowns' grid.

SINGLE_TRACE = ("pmchwt_ext", "muller_ext", "pmchwt_int", "muller_int")


def _calderon(A, c_v, c_d):
    """[[-K, c_v V], [c_d D, T]] of one grid's operators."""
    return np.block([[-A["K"], c_v * A["V"]], [c_d * A["D"], A["T"]]])


def single_trace_matrix(blocks, rho_int_over_rho_ext, formulation):
    """Weak-form matrix of one of SINGLE_TRACE (dense, 2N x 2N on the unknowns' grid)."""
    Ae, Ai, Pie, Me, Mi = blocks["ext"], blocks["int"], blocks["Pie"], blocks["Me"], blocks["Mi"]
    r = rho_int_over_rho_ext
    if formulation.endswith("_ext"):
        own = _calderon(Ae, 1.0, 1.0)
        other = _calderon(Ai, r, 1.0 / r)
        Rm = np.linalg.solve(Mi, Pie)  # M_i^-1 P_ie [Ni, Ne]
        M = Me
    else:
        own = _calderon(Ai, 1.0, 1.0)
        other = _calderon(Ae, 1.0 / r, r)
        Rm = np.linalg.solve(Me, Pie.T)  # M_e^-1 P_ei [Ne, Ni]
        M = Mi
    Z = np.zeros_like(Rm)
    R2 = np.block([[Rm, Z], [Z, Rm]])  # the map on both potentials
    hat = R2.T @ other @ R2  # P M^-1 X M^-1 P (mass matrices symmetric)
    M2 = np.block([[M, np.zeros_like(M)], [np.zeros_like(M), M]])
    if formulation == "pmchwt_ext":
        return own + hat
    if formulation == "muller_ext":
        return M2 + own - hat
    if formulation == "pmchwt_int":
        return hat + own
    if formulation == "muller_int":
        return M2 + hat - own
    raise ValueError(formulation)


def single_trace_rhs(blocks, rho_int_over_rho_ext, formulation, f, g):
    """Weak-form right-hand side of one of SINGLE_TRACE from the exterior data f, g."""
    if formulation.endswith("_ext"):
        return np.concatenate([-f, -g])
    Me, Pie = blocks["Me"], blocks["Pie"]
    r = rho_int_over_rho_ext
    return np.concatenate([Pie @ np.linalg.solve(Me, f), r * (Pie @ np.linalg.solve(Me, g))])


def solve_single_trace(v_ext, t_ext, v_int, t_int, k_ext, k_int, rho_int_over_rho_ext, d, formulation,
                       tol=1e-8, maxiter=2000, n_singular=4, blocks=None, center=(0.0, 0.0, 0.0), data=None):
    """Full oracle solve of one of SINGLE_TRACE for the plane wave along d, or for the
    exterior-grid data data = (f, g) when given.  Returns dict(v_ext, w_ext, v_int,
    w_int, iters, hist, blocks) with the potentials in the conventions of the MTF solve."""
    if blocks is None:
        blocks = mtf_blocks(v_ext, t_ext, v_int, t_int, k_ext, k_int, n_singular, center)
    r = rho_int_over_rho_ext
    A = single_trace_matrix(blocks, r, formulation)
    f, g = plane_wave_data(v_ext, t_ext, k_ext, d) if data is None else data
    b = single_trace_rhs(blocks, r, formulation, f, g)
    Me, Mi, Pie = blocks["Me"], blocks["Mi"], blocks["Pie"]
    ext = formulation.endswith("_ext")
    M = Me if ext else Mi
    N = len(M)
    SA = np.vstack([np.linalg.solve(M, A[:N]), np.linalg.solve(M, A[N:])])
    Sb = np.concatenate([np.linalg.solve(M, b[:N]), np.linalg.solve(M, b[N:])])
    x, it, hist = gmres(lambda z: SA @ z, Sb, tol, maxiter)
    if ext:
        ve, we = x[:N], x[N:]
        vi = -np.linalg.solve(Mi, Pie @ ve)
        wi = -r * np.linalg.solve(Mi, Pie @ we)
    else:
        vi, wi = x[:N], x[N:]
        ve = -np.linalg.solve(Me, Pie.T @ vi)
        we = -(1.0 / r) * np.linalg.solve(Me, Pie.T @ wi)
    return dict(v_ext=ve, w_ext=we, v_int=vi, w_int=wi, iters=it, hist=hist, blocks=blocks)
