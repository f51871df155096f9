"""Exterior PMCHWT single-trace formulation (Sec. 2.2, eq. pmchwt:ext and eq.
pmchwt:discrete) on nonconforming grids.

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
