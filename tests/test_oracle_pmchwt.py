"""Pins of the exterior PMCHWT oracle (oracle/pmchwt.py): convergence to the Mie
series at O(h^2), agreement with the multiple-traces solution up to the
discretisation error (the two formulations discretise the same problem), the
transmission conditions satisfied by its interior potentials, and Table 1's
structure (8 dense operators, 2 unknown potentials)."""
import numpy as np

import bem_inputs as bi
from oracle.mie import mie_potentials
from oracle.mtf import solve_transmission
from oracle.pmchwt import pmchwt_matrix, solve_pmchwt


def _merr(x, y, M):
    d = x - y
    return np.sqrt(np.real(np.conj(d) @ M @ d) / np.real(np.conj(y) @ M @ y))


def test_pmchwt_converges_to_mie():
    d = [0.0, 0.0, 1.0]
    k_e, k_i, rr = 1.0, 2.0, 1.5
    errs = []
    for L in (1, 2):
        ve, te, vi, ti = bi.transmission_pair(L, L, seed=1)
        r = solve_pmchwt(ve, te, vi, ti, k_e, k_i, rr, d, tol=1e-10)
        ref = mie_potentials(ve, vi, d, k_e, k_i, rr)
        B = r["blocks"]
        errs.append([_merr(r[key], ref[i], B[M]) for i, (key, M) in enumerate(
            [("v_ext", "Me"), ("w_ext", "Me"), ("v_int", "Mi"), ("w_int", "Mi")])])
    errs = np.array(errs)
    assert np.all(errs[0] / errs[1] > 3.0), errs  # O(h^2)
    assert errs[1].max() < 0.05, errs


def test_pmchwt_agrees_with_mtf_to_discretisation_error():
    d = np.array([0.0, 0.6, 0.8])
    diffs = []
    for L in (1, 2):
        ve, te, vi, ti = bi.transmission_pair(L, L, seed=3, axes=[1.2, 0.9, 1.0])
        p = solve_pmchwt(ve, te, vi, ti, 1.5, 2.5, 0.5, d, tol=1e-11)
        m = solve_transmission(ve, te, vi, ti, 1.5, 2.5, 0.5, d, tol=1e-11, blocks=p["blocks"])
        diffs.append(max(np.linalg.norm(p[k] - m[k]) / np.linalg.norm(m[k]) for k in ("v_ext", "w_ext")))
    assert diffs[1] < diffs[0] and diffs[1] < 2e-2, diffs


def test_pmchwt_interior_potentials_satisfy_the_transmission_conditions():
    ve, te, vi, ti = bi.transmission_pair(2, 1, seed=5)
    rho = 3.0
    p = solve_pmchwt(ve, te, vi, ti, 1.0, 1.7, rho, [1.0, 0.0, 0.0], tol=1e-11)
    B = p["blocks"]
    assert np.allclose(B["Mi"] @ p["v_int"], -B["Pie"] @ p["v_ext"], rtol=0, atol=1e-12)
    assert np.allclose(B["Mi"] @ p["w_int"], -rho * (B["Pie"] @ p["w_ext"]), rtol=0, atol=1e-12)


def test_pmchwt_identical_grids_reduce_to_the_conforming_operator():
    """With the interior grid equal to the exterior one, P_ie = M and the hat
    transformation is the identity: the matrix is the conforming PMCHWT."""
    from oracle.mtf import mtf_blocks
    v, t = bi.icosphere(1)
    B = mtf_blocks(v, t, v, t, 1.0, 2.0)
    A = pmchwt_matrix(B, 2.0)
    Ae, Ai = B["ext"], B["int"]
    ref = np.block([[-Ae["K"] - Ai["K"], Ae["V"] + 2.0 * Ai["V"]], [Ae["D"] + Ai["D"] / 2.0, Ae["T"] + Ai["T"]]])
    assert np.abs(A - ref).max() < 1e-12 * np.abs(ref).max()


def test_single_trace_exterior_pmchwt_is_the_pmchwt_matrix():
    from oracle.mtf import mtf_blocks
    from oracle.pmchwt import single_trace_matrix
    ve, te, vi, ti = bi.transmission_pair(1, 1, seed=4)
    B = mtf_blocks(ve, te, vi, ti, 1.0, 2.0)
    A = single_trace_matrix(B, 0.7, "pmchwt_ext")
    assert np.abs(A - pmchwt_matrix(B, 0.7)).max() < 1e-13 * np.abs(A).max()


def test_single_trace_variants_converge_to_mie():
    """Exterior Mueller, interior PMCHWT and interior Mueller on nonconforming sphere
    pairs: all four potentials converge to the Mie series at O(h^2)."""
    from oracle.mtf import mtf_blocks
    from oracle.pmchwt import solve_single_trace
    d = [0.0, 0.0, 1.0]
    k_e, k_i, rr = 1.0, 2.0, 1.5
    forms = ("muller_ext", "pmchwt_int", "muller_int")
    errs = {f: [] for f in forms}
    for L in (1, 2):
        ve, te, vi, ti = bi.transmission_pair(L, L, seed=1)
        B = mtf_blocks(ve, te, vi, ti, k_e, k_i)
        ref = mie_potentials(ve, vi, d, k_e, k_i, rr)
        for f in forms:
            r = solve_single_trace(ve, te, vi, ti, k_e, k_i, rr, d, f, tol=1e-10, blocks=B)
            errs[f].append([_merr(r[key], ref[i], B[M]) for i, (key, M) in enumerate(
                [("v_ext", "Me"), ("w_ext", "Me"), ("v_int", "Mi"), ("w_int", "Mi")])])
    for f in forms:
        e = np.array(errs[f])
        assert np.all(e[0] / e[1] > 3.0), (f, e)
        assert e[1].max() < 0.05, (f, e)


def test_interior_and_exterior_variants_coincide_on_identical_grids():
    """With one grid for both sides (P_ie = M) the interior system is the exterior one
    with v_i = -v_e, w_i = -(rho_i/rho_e) w_e substituted and rows rescaled, so the two
    variants of each formulation give the same four potentials."""
    from oracle.mtf import mtf_blocks
    from oracle.pmchwt import solve_single_trace
    v, t = bi.icosphere(2)
    rho, d = 2.5, np.array([0.6, 0.0, 0.8])
    B = mtf_blocks(v, t, v, t, 1.3, 2.1 + 0.1j)
    for kind in ("pmchwt", "muller"):
        a = solve_single_trace(v, t, v, t, 1.3, 2.1 + 0.1j, rho, d, kind + "_ext", tol=1e-12, blocks=B)
        b = solve_single_trace(v, t, v, t, 1.3, 2.1 + 0.1j, rho, d, kind + "_int", tol=1e-12, blocks=B)
        for key in ("v_ext", "w_ext", "v_int", "w_int"):
            assert np.linalg.norm(a[key] - b[key]) < 1e-9 * np.linalg.norm(a[key]), (kind, key)


def test_muller_without_contrast_returns_the_incident_traces():
    """Same medium inside and out, same grid: the exterior Mueller operator is
    M + A - A^ = M exactly (the hat is the identity map), so its solution is the L2
    projection of the incident traces (phi_ext = -u_inc, psi_ext = -du_inc/dn); the
    interior variant gives the interior traces +u_inc, +du_inc/dn."""
    from oracle.mass import mass_matrix
    from oracle.mtf import mtf_blocks, plane_wave_data
    from oracle.pmchwt import solve_single_trace
    v, t = bi.icosphere(2)
    d = np.array([0.0, 1.0, 0.0])
    B = mtf_blocks(v, t, v, t, 2.0, 2.0)
    f, g = plane_wave_data(v, t, 2.0, d)
    M = mass_matrix(v, t)
    pf, pg = np.linalg.solve(M, f), np.linalg.solve(M, g)
    e = solve_single_trace(v, t, v, t, 2.0, 2.0, 1.0, d, "muller_ext", tol=1e-13, blocks=B)
    i = solve_single_trace(v, t, v, t, 2.0, 2.0, 1.0, d, "muller_int", tol=1e-13, blocks=B)
    for got, want in ((e["v_ext"], -pf), (e["w_ext"], -pg), (i["v_int"], pf), (i["w_int"], pg)):
        assert np.linalg.norm(got - want) < 1e-10 * np.linalg.norm(want)
    assert e["iters"] <= 2 and i["iters"] <= 2


def test_single_trace_variants_at_high_contrast():
    """The paper's high-contrast densities (rho_int / rho_ext = 2 / 0.11): every
    single-trace system still converges to the Mie series (a misplaced density ratio
    would show here first)."""
    from oracle.mtf import mtf_blocks
    from oracle.pmchwt import SINGLE_TRACE, solve_single_trace
    d = [0.0, 0.0, 1.0]
    k_e, k_i, rr = 1.0, 0.5, 2.0 / 0.11
    errs = {f: [] for f in SINGLE_TRACE}
    for L in (1, 2):
        ve, te, vi, ti = bi.transmission_pair(L, L, seed=1)
        B = mtf_blocks(ve, te, vi, ti, k_e, k_i)
        ref = mie_potentials(ve, vi, d, k_e, k_i, rr)
        for f in SINGLE_TRACE:
            r = solve_single_trace(ve, te, vi, ti, k_e, k_i, rr, d, f, tol=1e-10, blocks=B)
            errs[f].append([_merr(r[key], ref[i], B[M]) for i, (key, M) in enumerate(
                [("v_ext", "Me"), ("w_ext", "Me"), ("v_int", "Mi"), ("w_int", "Mi")])])
    for f in SINGLE_TRACE:
        e = np.array(errs[f])
        assert np.all(e[0] / e[1] > 2.0), (f, e)
        assert e[1].max() < 0.1, (f, e)
