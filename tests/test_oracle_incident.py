"""Pins of the oracle's point-source data and of a solve driven by it (Sec. 2: the
incident field u_inc of the exterior medium enters only through f = <u_inc, theta>
and g = <du_inc/dn, theta> on the exterior grid).

u = exp(i k r) / (4 pi r) is the fundamental solution, so at k -> 0:
* Gauss's law on any closed surface: the flux int du/dn is -1 when the pole is
  inside and 0 when it is outside (sum_j g_j = int du/dn, the P1 functions sum to 1);
* on the unit sphere, int 1/(4 pi |x - s|) dS = 1 for |s| < 1 and 1/|s| for |s| > 1
  (the potential of a uniform layer), reached at O(h^2) on the inscribed polyhedra.
Without contrast (k_int = k_ext, equal densities) the total field is the incident
field in both media, so the computed potentials converge to its traces."""
import numpy as np
import pytest

import bem_inputs as bi
from oracle.mtf import point_source_data, plane_wave_data, solve_transmission
from oracle.quadrature import triangle_rule_collapsed

INSIDE = np.array([0.1, 0.2, -0.15])
OUTSIDE = np.array([0.3, -0.4, 2.2])


def test_point_source_flux_is_gauss_law():
    v, t = bi.icosphere(2)
    v = bi.ellipsoid(v, [1.2, 0.9, 1.1])  # any closed surface
    for src, flux in ((INSIDE, -1.0), (OUTSIDE, 0.0)):
        f, g = point_source_data(v, t, 1e-9, src)
        assert abs(g.sum() - flux) < 1e-5, (src, g.sum())


def test_point_source_layer_potential_on_the_sphere():
    err_in, err_out = [], []
    for L in (1, 2, 3):
        v, t = bi.icosphere(L)
        f_in, _ = point_source_data(v, t, 1e-9, INSIDE)
        f_out, _ = point_source_data(v, t, 1e-9, OUTSIDE)
        err_in.append(abs(f_in.sum() - 1.0))
        err_out.append(abs(f_out.sum() - 1.0 / np.linalg.norm(OUTSIDE)))
    assert err_in[-1] < 0.01 and err_out[-1] < 0.01, (err_in, err_out)
    for e in (err_in, err_out):
        assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0, e  # O(h^2): the polyhedra approach the sphere


def test_point_source_data_against_high_order_rule():
    v, t = bi.icosphere(2)
    f, g = point_source_data(v, t, 2.0 + 0.3j, OUTSIDE, amp=0.7 - 0.2j)
    import oracle.mtf as m
    orig = m.triangle_rule_degree4
    try:
        m.triangle_rule_degree4 = lambda: triangle_rule_collapsed(10)
        fh, gh = point_source_data(v, t, 2.0 + 0.3j, OUTSIDE, amp=0.7 - 0.2j)
    finally:
        m.triangle_rule_degree4 = orig
    assert np.abs(f - fh).max() < 1e-5 * np.abs(fh).max()
    assert np.abs(g - gh).max() < 1e-5 * np.abs(gh).max()


def test_solve_with_given_data_equals_the_plane_wave_solve():
    ve, te, vi, ti = bi.transmission_pair(1, 1, seed=3)
    d = np.array([0.0, 0.6, 0.8])
    a = solve_transmission(ve, te, vi, ti, 1.5, 2.5, 1.7, d, tol=1e-12)
    b = solve_transmission(ve, te, vi, ti, 1.5, 2.5, 1.7, None, tol=1e-12, blocks=a["blocks"],
                           data=plane_wave_data(ve, te, 1.5, d))
    for key in ("v_ext", "w_ext", "v_int", "w_int"):
        assert np.abs(a[key] - b[key]).max() <= 1e-14 * np.abs(a[key]).max()


def _traces(v, k, src):
    n = v / np.linalg.norm(v, axis=1)[:, None]
    R = v - src
    r = np.linalg.norm(R, axis=1)
    u = np.exp(1j * k * r) / (4 * np.pi * r)
    return u, u * (1j * k - 1.0 / r) * np.einsum("ij,ij->i", R, n) / r


def _merr(x, y, M):
    d = x - y
    return np.sqrt(np.real(np.conj(d) @ M @ d) / np.real(np.conj(y) @ M @ y))


def test_point_source_without_contrast_gives_the_incident_traces():
    k = 1.5
    errs = []
    for L in (1, 2):
        ve, te, vi, ti = bi.transmission_pair(L, L, seed=5)
        r = solve_transmission(ve, te, vi, ti, k, k, 1.0, None, tol=1e-11,
                               data=point_source_data(ve, te, k, OUTSIDE))
        B = r["blocks"]
        ue, due = _traces(ve, k, OUTSIDE)
        ui, dui = _traces(vi, k, OUTSIDE)
        errs.append([_merr(r["v_ext"], -ue, B["Me"]), _merr(r["w_ext"], -due, B["Me"]),
                     _merr(r["v_int"], ui, B["Mi"]), _merr(r["w_int"], dui, B["Mi"])])
    errs = np.array(errs)
    assert (errs[1] < 0.05).all(), errs
    assert (errs[0] / errs[1] > 3.0).all(), errs
