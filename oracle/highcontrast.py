"""High-contrast formulations (Sec. 2.3, eq. highcontrast:ext:neu, highcontrast:ext:dir,
highcontrast:int:neu, highcontrast:int:dir) on nonconforming grids.

Test infrastructure only: the FP64 reference the CUDA path is checked against.

Each formulation represents one field indirectly (a single-layer density mu or a
double-layer density nu) and the other directly, and couples them through operators
"passed through the opposite mesh" (X o = Z^-1 Z X Z^-1 Z).  Discretised as the paper
does for the exterior Neumann variant (after eq. pmchwt:discrete), with the weak-form
matrices of oracle/helmholtz.py, r = rho_int / rho_ext and

  X^_i = P_ei M_i^-1 X_i M_i^-1 P_ie  (an interior operator on the exterior grid),
  X^_e = P_ie M_e^-1 X_e M_e^-1 P_ei  (an exterior operator on the interior grid);

a product of two operators gets the inverse mass matrix of the grid between them, and
a weak-form data vector that an operator acts on is first made a coefficient vector
by the mass inverse of its grid (the paper's right-hand side D^_i f reads D^_i M_e^-1 f).

  exterior Neumann (unknowns a = gamma_N^+ p, mu on the exterior grid):
    [ M_e/2 - T^_i   -(1/r) D^_i M_e^-1 V_e ] [a ]   [ (1/r) D^_i M_e^-1 f ]
    [ M_e            M_e/2 - T_e           ] [mu] = [ g                   ]
  exterior Dirichlet (unknowns nu, b = gamma_D^+ p on the exterior grid):
    [ M_e/2 + K_e             M_e          ] [nu]   [ f                  ]
    [ -r V^_i M_e^-1 D_e      M_e/2 + K^_i ] [b ] = [ r V^_i M_e^-1 g    ]
  interior Neumann (unknowns a = gamma_N^- p, mu on the interior grid):
    [ M_i/2 + T^_e   r D^_e M_i^-1 V_i ] [a ]   [ r P_ie M_e^-1 (D_e M_e^-1 f + g/2 + T_e M_e^-1 g) ]
    [ -M_i           M_i/2 + T_i       ] [mu] = [ 0                                                ]
  interior Dirichlet (unknowns nu, b = gamma_D^- p on the interior grid):
    [ M_i/2 - K_i               -M_i         ] [nu]   [ 0                                              ]
    [ (1/r) V^_e M_i^-1 D_i     M_i/2 - K^_e ] [b ] = [ P_ie M_e^-1 (V_e M_e^-1 g + f/2 - K_e M_e^-1 f) ]

Left preconditioning with the mass inverse of the unknowns' grid (Sec. 3.3); GMRES as
for the MTF.  The four trace potentials of the MTF follow from the representations:
  exterior Neumann:   w_e = -a, v_e = -M_e^-1 (f + V_e mu)       (u_s = V mu)
  exterior Dirichlet: v_e = -b, w_e = -M_e^-1 (g + D_e nu)       (u_s = -K nu)
  interior Neumann:   w_i = a,  v_i = M_i^-1 V_i mu              (u_int = V mu)
  interior Dirichlet: v_i = b,  w_i = M_i^-1 D_i nu              (u_int = -K nu)
and the other grid's from the transmission conditions tested on it, as for the
single-trace systems.
"""
from __future__ import annotations

import numpy as np

from .mtf import gmres, mtf_blocks, plane_wave_data

HIGH_CONTRAST = ("hc_ext_neu", "hc_ext_dir", "hc_int_neu", "hc_int_dir")


def _inv(M, X):
    return np.linalg.solve(M, X)


def high_contrast_system(blocks, rho_int_over_rho_ext, formulation, f, g):
    """(A, b): weak-form matrix and right-hand side of one of HIGH_CONTRAST."""
    Ae, Ai, Pie, Me, Mi = blocks["ext"], blocks["int"], blocks["Pie"], blocks["Me"], blocks["Mi"]
    Pei = Pie.T
    r = rho_int_over_rho_ext
    hat_i = lambda X: Pei @ _inv(Mi, X) @ _inv(Mi, Pie)  # interior operator on the exterior grid
    hat_e = lambda X: Pie @ _inv(Me, X) @ _inv(Me, Pei)  # exterior operator on the interior grid
    if formulation == "hc_ext_neu":
        A = np.block([[0.5 * Me - hat_i(Ai["T"]), -(1.0 / r) * hat_i(Ai["D"]) @ _inv(Me, Ae["V"])],
                      [Me, 0.5 * Me - Ae["T"]]])
        b = np.concatenate([(1.0 / r) * hat_i(Ai["D"]) @ _inv(Me, f), g])
    elif formulation == "hc_ext_dir":
        A = np.block([[0.5 * Me + Ae["K"], Me],
                      [-r * hat_i(Ai["V"]) @ _inv(Me, Ae["D"]), 0.5 * Me + hat_i(Ai["K"])]])
        b = np.concatenate([f, r * hat_i(Ai["V"]) @ _inv(Me, g)])
    elif formulation == "hc_int_neu":
        A = np.block([[0.5 * Mi + hat_e(Ae["T"]), r * hat_e(Ae["D"]) @ _inv(Mi, Ai["V"])],
                      [-Mi, 0.5 * Mi + Ai["T"]]])
        data = Ae["D"] @ _inv(Me, f) + 0.5 * g + Ae["T"] @ _inv(Me, g)
        b = np.concatenate([r * (Pie @ _inv(Me, data)), np.zeros(len(Mi), dtype=np.complex128)])
    elif formulation == "hc_int_dir":
        A = np.block([[0.5 * Mi - Ai["K"], -Mi],
                      [(1.0 / r) * hat_e(Ae["V"]) @ _inv(Mi, Ai["D"]), 0.5 * Mi - hat_e(Ae["K"])]])
        data = Ae["V"] @ _inv(Me, g) + 0.5 * f - Ae["K"] @ _inv(Me, f)
        b = np.concatenate([np.zeros(len(Mi), dtype=np.complex128), Pie @ _inv(Me, data)])
    else:
        raise ValueError(formulation)
    return A, b


def solve_high_contrast(v_ext, t_ext, v_int, t_int, k_ext, k_int, rho_int_over_rho_ext, d, formulation,
                        tol=1e-8, maxiter=2000, n_singular=4, blocks=None, center=(0.0, 0.0, 0.0)):
    """Full oracle solve of one of HIGH_CONTRAST.  Returns dict(v_ext, w_ext, v_int, w_int,
    iters, hist, blocks, x) with the potentials in the conventions of the MTF solve and
    x the formulation's own unknowns."""
    if blocks is None:
        blocks = mtf_blocks(v_ext, t_ext, v_int, t_int, k_ext, k_int, n_singular, center)
    r = rho_int_over_rho_ext
    f, g = plane_wave_data(v_ext, t_ext, k_ext, d)
    A, b = high_contrast_system(blocks, r, formulation, f, g)
    Ae, Ai, Pie, Me, Mi = blocks["ext"], blocks["int"], blocks["Pie"], blocks["Me"], blocks["Mi"]
    ext = formulation.startswith("hc_ext")
    M = Me if ext else Mi
    N = len(M)
    SA = np.vstack([_inv(M, A[:N]), _inv(M, A[N:])])
    Sb = np.concatenate([_inv(M, b[:N]), _inv(M, b[N:])])
    x, it, hist = gmres(lambda z: SA @ z, Sb, tol, maxiter)
    x1, x2 = x[:N], x[N:]
    if formulation == "hc_ext_neu":
        we = -x1
        ve = -_inv(Me, f + Ae["V"] @ x2)
    elif formulation == "hc_ext_dir":
        ve = -x2
        we = -_inv(Me, g + Ae["D"] @ x1)
    elif formulation == "hc_int_neu":
        wi = x1
        vi = _inv(Mi, Ai["V"] @ x2)
    else:
        vi = x2
        wi = _inv(Mi, Ai["D"] @ x1)
    if ext:
        vi = -_inv(Mi, Pie @ ve)
        wi = -r * _inv(Mi, Pie @ we)
    else:
        ve = -_inv(Me, Pie.T @ vi)
        we = -(1.0 / r) * _inv(Me, Pie.T @ wi)
    return dict(v_ext=ve, w_ext=we, v_int=vi, w_int=wi, iters=it, hist=hist, blocks=blocks, x=x)
