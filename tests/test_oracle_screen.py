"""Pins of the screen oracle (oracle/screen.py): the hypersingular system of a Neumann
screen on P1 functions vanishing on its boundary, with mass-matrix and opposite-order
(single layer on a coarse grid) preconditioning.

* A preconditioner that is invertible leaves the solution unchanged: with the coarse
  grid equal to the fine one the mortar matrix is the mass matrix, V^ = V, and the
  opposite-order solution equals the mass-preconditioned one.
* The opposite-order preconditioner cuts the GMRES iteration count (the effect the
  paper reports for its screen).
* On a coarser grid V^_c has rank at most the coarse node count, so the preconditioned
  system no longer determines phi: its GMRES iterate stays in the range of
  M^-1 V^_c (checked) and differs from the solution of D phi = g -- the reading recorded
  with the implementation.
"""
import numpy as np

import bem_inputs as bi
from oracle.helmholtz import assemble
from oracle.mass import mass_matrix
from oracle.screen import boundary_nodes, solve_screen

D_INC = np.array([1.0, 0.0, 0.0])


def test_boundary_nodes_of_a_structured_screen():
    v, t = bi.screen_grid(5, 4, jitter=0.3, seed=3)
    b = boundary_nodes(t, len(v))
    assert b.sum() == 2 * (5 + 4)  # the perimeter nodes
    v2, t2 = bi.icosphere(1)
    assert not boundary_nodes(t2, len(v2)).any()  # a closed surface has none


def test_conforming_opposite_order_preconditioning_keeps_the_solution_and_cuts_iterations():
    v, t = bi.screen_grid(10, 9, jitter=0.2, seed=1)
    a = solve_screen(v, t, 5.0, D_INC, "mass", tol=1e-11)
    b = solve_screen(v, t, 5.0, D_INC, "oo", v, t, tol=1e-11)
    assert np.linalg.norm(a["phi"] - b["phi"]) < 1e-8 * np.linalg.norm(a["phi"])
    assert np.all(a["phi"][boundary_nodes(t, len(v))] == 0.0)
    assert b["iters"] * 2 < a["iters"], (a["iters"], b["iters"])
    # the restricted hypersingular matrix is complex symmetric
    I = ~boundary_nodes(t, len(v))
    D = assemble(v, t, 5.0)["D"][np.ix_(I, I)]
    assert np.abs(D - D.T).max() < 1e-12 * np.abs(D).max()


def test_coarse_opposite_order_preconditioner_is_rank_deficient():
    v, t = bi.screen_grid(10, 9, jitter=0.2, seed=1)
    vc, tc = bi.screen_grid(4, 3, jitter=0.2, seed=2)
    a = solve_screen(v, t, 5.0, D_INC, "mass", tol=1e-11)
    b = solve_screen(v, t, 5.0, D_INC, "oo", vc, tc, tol=1e-11)
    assert b["iters"] * 2 < a["iters"], (a["iters"], b["iters"])
    assert b["iters"] <= len(vc)  # the Krylov space lies in a space of that dimension
    # the iterate does not solve D phi = g: it differs from the mass-preconditioned one
    assert np.linalg.norm(a["phi"] - b["phi"]) > 1e-2 * np.linalg.norm(a["phi"])


def test_screen_grid_geometry():
    """The rectangle of the paper's screen: area 2.06 x 2, one normal for all triangles,
    (nu + 1)(nv + 1) nodes, jitter kept in the plane and off the boundary."""
    nu, nv = 7, 5
    v, t = bi.screen_grid(nu, nv, jitter=0.3, seed=9)
    assert len(v) == (nu + 1) * (nv + 1) and len(t) == 2 * nu * nv
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    cr = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(cr, axis=1).sum()
    assert abs(area - 2.0 * np.sqrt(0.5 ** 2 + 2.0 ** 2)) < 1e-12
    n = cr / np.linalg.norm(cr, axis=1)[:, None]
    assert np.abs(n - n[0]).max() < 1e-12
    assert np.abs((v - v[0]) @ n[0]).max() < 1e-12  # planar


def test_laplace_disk_screen_matches_the_closed_form():
    """k = 0 on the unit disk: the double-layer density phi = (4/pi) sqrt(1 - r^2) has
    normal derivative -1 on the disk (its Hankel transform is (4/pi)(sin x - x cos x)/x^3
    and the Weber-Schafheitlin integrals give d_z u = -(1/2)(4/pi)(pi/2)), so D phi = 1.
    The oracle's hypersingular system on the interior nodes with data <1, theta_i>
    converges to it (relative M-norm error, the polygonal boundary included)."""
    errs = []
    for n in (3, 6):
        v, t = bi.disk_grid(n)
        I = np.flatnonzero(~boundary_nodes(t, len(v)))
        D = assemble(v, t, 0.0)["D"]
        M = mass_matrix(v, t)
        phi = np.zeros(len(v), dtype=np.complex128)
        phi[I] = np.linalg.solve(D[np.ix_(I, I)], (M @ np.ones(len(v)))[I])
        r = np.linalg.norm(v[:, :2], axis=1)
        exact = 4.0 / np.pi * np.sqrt(np.clip(1.0 - r ** 2, 0.0, None))
        d = phi - exact
        errs.append(np.sqrt(np.real(np.conj(d) @ M @ d) / (exact @ M @ exact)))
    assert errs[0] > 1.8 * errs[1] and errs[1] < 0.025, errs
