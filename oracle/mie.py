"""Mie series for plane-wave transmission through a homogeneous sphere.

The closed form the whole oracle solve is pinned to.  Time convention
exp(-i omega t) (Sec. 2), incident field exp(i k_e x . d) with the Rayleigh
expansion  sum_n i^n (2n+1) j_n(k_e r) P_n(cos theta),  cos theta = x^ . d.
Outside: total field sum_n i^n (2n+1) [j_n(k_e r) + a_n h_n(k_e r)] P_n;
inside: sum_n i^n (2n+1) c_n j_n(k_i r) P_n, with h_n = j_n + i y_n.
For each n the two interface conditions of eq. (helmholtz),
  p^+ = p^-   and   (1/rho_e) dp^+/dr = (1/rho_i) dp^-/dr   at r = R,
form a 2x2 linear system for (a_n, c_n), solved directly.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn, eval_legendre


def _h(n, x, deriv=False):
    return spherical_jn(n, x, deriv) + 1j * spherical_yn(n, x, deriv)


def mie_coefficients(k_e, k_i, rho_int_over_rho_ext, R=1.0, n_max=None):
    kmax = max(abs(k_e), abs(k_i)) * R
    if n_max is None:
        n_max = int(np.ceil(kmax + 4.0 * kmax ** (1.0 / 3.0))) + 10
    rho_e, rho_i = 1.0, rho_int_over_rho_ext
    a = np.zeros(n_max + 1, dtype=np.complex128)
    c = np.zeros(n_max + 1, dtype=np.complex128)
    xe, xi = k_e * R, k_i * R
    for n in range(n_max + 1):
        Mx = np.array([
            [_h(n, xe), -spherical_jn(n, xi)],
            [k_e / rho_e * _h(n, xe, True), -k_i / rho_i * spherical_jn(n, xi, True)],
        ], dtype=np.complex128)
        rhs = -np.array([spherical_jn(n, xe), k_e / rho_e * spherical_jn(n, xe, True)], dtype=np.complex128)
        a[n], c[n] = np.linalg.solve(Mx, rhs)
    return a, c


def mie_traces(x, d, k_e, k_i, rho_int_over_rho_ext, R=1.0, n_max=None):
    """Exterior and interior traces at points x [M,3] on the sphere |x| = R.

    Returns (gD_plus, gN_plus, gD_minus, gN_minus): Dirichlet and Neumann (radial
    derivative) traces of the total field from outside and inside."""
    a, c = mie_coefficients(k_e, k_i, rho_int_over_rho_ext, R, n_max)
    x = np.asarray(x, dtype=np.float64)
    r = np.linalg.norm(x, axis=1)
    ct = np.clip((x @ np.asarray(d, dtype=np.float64)) / r, -1.0, 1.0)
    gDp = np.zeros(len(x), dtype=np.complex128)
    gNp = np.zeros(len(x), dtype=np.complex128)
    gDm = np.zeros(len(x), dtype=np.complex128)
    gNm = np.zeros(len(x), dtype=np.complex128)
    xe, xi = k_e * R, k_i * R
    for n in range(len(a)):
        Pn = eval_legendre(n, ct)
        f = (1j ** n) * (2 * n + 1)
        gDp += f * (spherical_jn(n, xe) + a[n] * _h(n, xe)) * Pn
        gNp += f * k_e * (spherical_jn(n, xe, True) + a[n] * _h(n, xe, True)) * Pn
        gDm += f * c[n] * spherical_jn(n, xi) * Pn
        gNm += f * c[n] * k_i * spherical_jn(n, xi, True) * Pn
    return gDp, gNp, gDm, gNm


def mie_potentials(v_ext, v_int, d, k_e, k_i, rho_int_over_rho_ext, R=1.0):
    """Vertex values of the four MTF potentials on both grids (unit sphere grids):
    phi_ext = -gamma_D^+ p, psi_ext = -gamma_N^+ p, phi_int = gamma_D^- p,
    psi_int = gamma_N^- p (Sec. 2.2)."""
    gDp, gNp, _, _ = mie_traces(v_ext, d, k_e, k_i, rho_int_over_rho_ext, R)
    _, _, gDm, gNm = mie_traces(v_int, d, k_e, k_i, rho_int_over_rho_ext, R)
    return -gDp, -gNp, gDm, gNm


def mie_field(x, d, k_e, k_i, rho_int_over_rho_ext, R=1.0, n_max=None):
    """Total field at points x [M, 3] off the sphere |x| = R: inside sum c_n j_n(k_i r) P_n,
    outside sum (j_n(k_e r) + a_n h_n(k_e r)) P_n, each term times i^n (2n + 1); returns
    (total, incident) so that the scattered field outside is total - incident."""
    a, c = mie_coefficients(k_e, k_i, rho_int_over_rho_ext, R, n_max)
    x = np.asarray(x, dtype=np.float64)
    r = np.linalg.norm(x, axis=1)
    rs = np.where(r > 0, r, 1.0)  # at the centre only n = 0 contributes (j_n(0) = 0 for n > 0)
    ct = np.clip((x @ np.asarray(d, dtype=np.float64)) / rs, -1.0, 1.0)
    inside = r < R
    tot = np.zeros(len(x), dtype=np.complex128)
    for n in range(len(a)):
        Pn = eval_legendre(n, ct)
        f = (1j ** n) * (2 * n + 1)
        term_in = c[n] * spherical_jn(n, k_i * r)
        term_out = spherical_jn(n, k_e * r) + a[n] * _h(n, k_e * np.where(inside, R, r))
        tot += f * np.where(inside, term_in, term_out) * Pn
    inc = np.exp(1j * k_e * (x @ np.asarray(d, dtype=np.float64)))
    return tot, inc
