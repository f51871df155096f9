"""Pins of the oracle's field evaluation (oracle/potentials.py, eq. representation)
against closed forms that do not use it: Gauss's solid-angle law, the single-layer
potential of a uniform density on the sphere, Green's representation of a plane wave
and of a point source, and the Mie series for the transmission problem."""
import numpy as np

import bem_inputs as bi
from oracle.mie import mie_field
from oracle.potentials import representation

INSIDE = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1], [-0.1, 0.4, -0.3]])
OUTSIDE = np.array([[2.0, 1.0, 0.0], [0.0, -2.5, 0.5], [1.2, 1.2, 1.2]])


def test_double_layer_of_one_is_the_solid_angle():
    """-K[1](x) = 1 inside a closed surface and 0 outside (Laplace limit); exact for
    the polyhedron, so only the quadrature error of points away from the surface
    remains."""
    v, t = bi.icosphere(3)
    one = np.ones(len(v))
    for x, ref in ((INSIDE, 1.0), (OUTSIDE, 0.0)):
        u = representation(v, t, 1e-9, x, phi=one)
        assert np.max(np.abs(u - ref)) < 1e-7, u


def test_single_layer_of_one_on_the_sphere_converges():
    """V[1](x) = R^2 / |x| outside the sphere of radius R (k -> 0): the icosphere
    error falls at O(h^2)."""
    errs = []
    for L in (2, 3, 4):
        v, t = bi.icosphere(L)
        u = representation(v, t, 1e-9, OUTSIDE, psi=np.ones(len(v)))
        errs.append(np.max(np.abs(u - 1.0 / np.linalg.norm(OUTSIDE, axis=1))))
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs


def _plane_wave_traces(v, k, d):
    u = np.exp(1j * k * (v @ d))
    n = v / np.linalg.norm(v, axis=1)[:, None]  # sphere: the vertex normal
    return u, 1j * k * (n @ d) * u


def test_green_representation_of_a_plane_wave():
    """V[du/dn] - K[u] = u inside and 0 outside for u = exp(i k x.d) (an entire
    solution); the P1 interpolation error falls at O(h^2)."""
    d = np.array([0.0, 0.6, 0.8])
    k = 2.0
    errs = []
    for L in (2, 3, 4):
        v, t = bi.icosphere(L)
        phi, psi = _plane_wave_traces(v, k, d)
        ui = representation(v, t, k, INSIDE, phi=phi, psi=psi)
        uo = representation(v, t, k, OUTSIDE, phi=phi, psi=psi)
        errs.append(max(np.max(np.abs(ui - np.exp(1j * k * (INSIDE @ d)))), np.max(np.abs(uo))))
    assert errs[2] < 5e-3
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs


def test_green_representation_of_a_point_source():
    """For the radiating w = exp(ikr) / (4 pi r) with the source inside, V[psi] - K[phi]
    with phi = -w, psi = -dw/dn on the surface (the exterior convention of Sec. 2.2)
    is w outside."""
    k = 1.5
    v, t = bi.icosphere(4)
    r = np.linalg.norm(v, axis=1)
    w = np.exp(1j * k * r) / (4 * np.pi * r)
    dw = w * (1j * k - 1.0 / r)  # radial derivative = normal derivative on the sphere
    u = representation(v, t, k, OUTSIDE, phi=-w, psi=-dw)
    ro = np.linalg.norm(OUTSIDE, axis=1)
    ref = np.exp(1j * k * ro) / (4 * np.pi * ro)
    assert np.max(np.abs(u - ref) / np.abs(ref)) < 5e-3


def test_fields_of_the_mie_traces():
    """With the exact (Mie) traces interpolated at the vertices, the interior and the
    scattered representations give the Mie fields inside and outside; the error falls
    at O(h^2) with the grid."""
    from oracle.mie import mie_traces
    k_e, k_i, rho = 1.0, 2.0, 1.5
    d = np.array([0.0, 0.0, 1.0])
    ti, _ = mie_field(INSIDE, d, k_e, k_i, rho)
    to, io = mie_field(OUTSIDE, d, k_e, k_i, rho)
    errs = []
    for L in (2, 3, 4):
        v, t = bi.icosphere(L)
        gDp, gNp, gDm, gNm = mie_traces(v, d, k_e, k_i, rho)
        inc = np.exp(1j * k_e * (v @ d))
        dinc = 1j * k_e * ((v / np.linalg.norm(v, axis=1)[:, None]) @ d) * inc
        # interior: phi_int = gD^-, psi_int = gN^-; scattered: phi_ext, psi_ext = -(traces of p - p_inc)
        ui = representation(v, t, k_i, INSIDE, phi=gDm, psi=gNm)
        us = representation(v, t, k_e, OUTSIDE, phi=-(gDp - inc), psi=-(gNp - dinc))
        errs.append(max(np.max(np.abs(ui - ti)), np.max(np.abs(us - (to - io)))))
    assert errs[2] < 5e-3
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs
