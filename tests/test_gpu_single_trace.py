"""Parity of the single-trace solves (bem_solve_transmission with formulation =
BEM_FORM_PMCHWT, BEM_FORM_MULLER, BEM_FORM_PMCHWT_INT, BEM_FORM_MULLER_INT: Sec. 2.2,
eq. pmchwt:ext, muller:ext, pmchwt:int, muller:int, discretised as eq.
pmchwt:discrete) with the FP64 oracle of oracle/pmchwt.py.

Tolerances: relative L2 <= 1e-10 in FP64 mode (same operators, same GMRES, rounding
only: the GPU applies M^-1 by 34 Chebyshev steps, whose error ~1e-16 enters the
operator itself here, not only the preconditioner); <= 1e-6 in the mixed mode,
whose refinement converges to the complex64-stored system (1e-7 relative per entry).
"""
import numpy as np
import pytest

import bem_inputs as bi

pytestmark = pytest.mark.gpu

TOL = 1e-10
MIXED_TOL = 1e-6
KEYS = ("v_ext", "w_ext", "v_int", "w_int")
FORMS = ("pmchwt_ext", "muller_ext", "pmchwt_int", "muller_int")


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2206_00708_gb300 as bem
    ctx = bem.bem_context_create(0)
    yield bem, ctx
    bem.bem_context_destroy(ctx)


def code(bem, form):
    return {"pmchwt_ext": bem.BEM_FORM_PMCHWT, "muller_ext": bem.BEM_FORM_MULLER,
            "pmchwt_int": bem.BEM_FORM_PMCHWT_INT, "muller_int": bem.BEM_FORM_MULLER_INT}[form]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _solve(bem, ctx, form, ve, te, vi, ti, k_int, k_ext, rho, dirs, amps=None, **opts):
    ge = bem.bem_grid_create(ctx, ve, te)
    gi = bem.bem_grid_create(ctx, vi, ti)
    try:
        return bem.bem_solve_transmission(ctx, ge, gi, k_int, k_ext, rho, dirs, amps=amps,
                                          opts={"formulation": code(bem, form), **opts})
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)


@pytest.fixture(scope="module")
def ellipsoid_case():
    """Ellipsoid, exterior level 2 / interior level 1 (nonconforming, the interior grid
    rotated and jittered), density ratio 2, complex interior wavenumber."""
    from oracle.mtf import mtf_blocks
    ve, te, vi, ti = bi.transmission_pair(2, 1, seed=6, axes=[1.2, 0.9, 1.0])
    k_ext, k_int, rho = 2.0, 3.0 + 0.2j, 2.0
    return dict(grids=(ve, te, vi, ti), k_ext=k_ext, k_int=k_int, rho=rho,
                blocks=mtf_blocks(ve, te, vi, ti, k_ext, k_int))


@pytest.mark.parametrize("form", FORMS)
def test_single_trace_fp64_matches_oracle_nonconforming(env, ellipsoid_case, form):
    """All four potentials within 1e-10 of the oracle at GMRES tol 1e-12, and the
    iteration count at tol 1e-8 within one of the oracle's."""
    from oracle.pmchwt import solve_single_trace
    bem, ctx = env
    c = ellipsoid_case
    ve, te, vi, ti = c["grids"]
    d = np.array([[0.0, 0.6, 0.8]])
    out, rep = _solve(bem, ctx, form, ve, te, vi, ti, c["k_int"], c["k_ext"], c["rho"], d, gmres_tol=1e-12)
    ref = solve_single_trace(ve, te, vi, ti, c["k_ext"], c["k_int"], c["rho"], d[0], form, tol=1e-12,
                             blocks=c["blocks"])
    for key in KEYS:
        e = rel(out[key][0], ref[key])
        assert e < TOL, (form, key, e)
    assert rep["converged"] == 1
    _, rep8 = _solve(bem, ctx, form, ve, te, vi, ti, c["k_int"], c["k_ext"], c["rho"], d)
    ref8 = solve_single_trace(ve, te, vi, ti, c["k_ext"], c["k_int"], c["rho"], d[0], form, tol=1e-8,
                              blocks=c["blocks"])
    assert abs(rep8["iterations"] - ref8["iters"]) <= 1, (form, rep8["iterations"], ref8["iters"])


@pytest.mark.parametrize("form", ["pmchwt_ext", "muller_int"])
def test_single_trace_fp64_multi_rhs_and_interior_finer(env, form):
    """Interior grid finer than the exterior one (level 2 inside level 1), three plane
    waves with complex amplitudes in one call (a batch of 3 at kernel width 4): each
    column is amp_r times the oracle solution for a unit wave."""
    from oracle.mtf import mtf_blocks
    from oracle.pmchwt import solve_single_trace
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(1, 2, seed=8)
    dirs = bi.plane_wave_directions(3, seed=40)
    amps = [1.0, 0.5 - 0.25j, 2.0j]
    k_ext, k_int, rho = 1.5, 2.5, 0.5
    out, rep = _solve(bem, ctx, form, ve, te, vi, ti, k_int, k_ext, rho, dirs, amps=amps, gmres_tol=1e-12)
    B = mtf_blocks(ve, te, vi, ti, k_ext, k_int)
    for r in range(3):
        ref = solve_single_trace(ve, te, vi, ti, k_ext, k_int, rho, dirs[r], form, tol=1e-12, blocks=B)
        for key in KEYS:
            e = rel(out[key][r], amps[r] * ref[key])
            assert e < TOL, (form, r, key, e)


def test_single_trace_transmission_conditions_hold_on_the_gpu_solution(env):
    """The potentials not solved for are M^-1 P applied to the solved ones (eliminated
    transmission conditions): checked with the oracle's mass and mortar matrices for
    an exterior and an interior variant."""
    from oracle.mtf import mtf_blocks
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(2, 2, seed=5)
    rho = 3.0
    B = mtf_blocks(ve, te, vi, ti, 1.0, 1.7)
    d = np.array([[1.0, 0.0, 0.0]])
    out, _ = _solve(bem, ctx, "pmchwt_ext", ve, te, vi, ti, 1.7, 1.0, rho, d, gmres_tol=1e-11)
    assert rel(B["Mi"] @ out["v_int"][0], -B["Pie"] @ out["v_ext"][0]) < 1e-12
    assert rel(B["Mi"] @ out["w_int"][0], -rho * (B["Pie"] @ out["w_ext"][0])) < 1e-12
    out, _ = _solve(bem, ctx, "muller_int", ve, te, vi, ti, 1.7, 1.0, rho, d, gmres_tol=1e-11)
    assert rel(B["Me"] @ out["v_ext"][0], -B["Pie"].T @ out["v_int"][0]) < 1e-12
    assert rel(B["Me"] @ out["w_ext"][0], -(B["Pie"].T @ out["w_int"][0]) / rho) < 1e-12


@pytest.mark.parametrize("form,tensor_cores,n_rhs", [("pmchwt_ext", 0, 1), ("pmchwt_ext", 0, 5),
                                                     ("pmchwt_ext", 1, 12), ("muller_ext", 0, 1),
                                                     ("pmchwt_int", 1, 12), ("muller_int", 0, 3),
                                                     ("muller_ext", 2, 10)])
def test_single_trace_mixed_matches_oracle(env, form, tensor_cores, n_rhs):
    """Mixed precision (complex64 operators, refinement with FP64 residuals): one
    column (double-float then FP32 products), three or five columns on the CUDA cores,
    twelve on the tensor cores (TF32 split), ten on the tensor cores with the FP16
    split (two operator copies: the own grid's and the other grid's blocks, two of the
    four block rows empty); every column within 1e-6 of the FP64 oracle."""
    from oracle.mtf import mtf_blocks
    from oracle.pmchwt import solve_single_trace
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(2, 2, seed=11, axes=[1.1, 1.0, 0.9])
    dirs = bi.plane_wave_directions(n_rhs, seed=45)
    k_ext, k_int, rho = 2.5, 4.0, 1.5
    out, rep = _solve(bem, ctx, form, ve, te, vi, ti, k_int, k_ext, rho, dirs, gmres_tol=1e-10,
                      precision=bem.BEM_PREC_MIXED, tensor_cores=tensor_cores)
    assert rep["converged"] == 1
    B = mtf_blocks(ve, te, vi, ti, k_ext, k_int)
    for r in range(n_rhs):
        ref = solve_single_trace(ve, te, vi, ti, k_ext, k_int, rho, dirs[r], form, tol=1e-12, blocks=B)
        for key in KEYS:
            e = rel(out[key][r], ref[key])
            assert e < MIXED_TOL, (form, r, key, e)


def test_single_trace_and_mtf_agree_to_discretisation_error_at_level4(env):
    """At level 4 (2562 vertices per grid, k 10 / 15, density ratio 2) every
    formulation discretises the same transmission problem: the exterior potentials of
    each single-trace solve lie within the discretisation error of the
    multiple-traces ones, and the PMCHWT needs fewer GMRES iterations than the
    multiple-traces system."""
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(4, 4, seed=2)
    d = np.array([[0.0, 0.0, 1.0]])
    ge = bem.bem_grid_create(ctx, ve, te)
    gi = bem.bem_grid_create(ctx, vi, ti)
    res = {}
    try:
        for form in ("mtf",) + FORMS:
            opts = {"precision": bem.BEM_PREC_MIXED}
            if form != "mtf":
                opts["formulation"] = code(bem, form)
            res[form] = bem.bem_solve_transmission(ctx, ge, gi, 15.0, 10.0, 2.0, d, opts=opts)
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
    m, rm = res["mtf"]
    print({f: r[1]["iterations"] for f, r in res.items()})
    for form in FORMS:
        p, rp = res[form]
        assert rp["converged"] == 1, form
        for key in ("v_ext", "w_ext"):
            assert rel(p[key][0], m[key][0]) < 0.1, (form, key)
    assert res["pmchwt_ext"][1]["iterations"] < rm["iterations"]


def test_single_trace_rejected_where_not_supported(env):
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(1, 1, seed=2)
    ge = bem.bem_grid_create(ctx, ve, te)
    gi = bem.bem_grid_create(ctx, vi, ti)
    try:
        inst = [dict(ext=ge, intr=gi, k_ext=1.0, k_int=2.0, rho=1.0, dir=[0.0, 0.0, 1.0])]
        with pytest.raises(bem.BemError) as e:
            bem.bem_solve_many(ctx, inst, opts={"formulation": bem.BEM_FORM_PMCHWT})
        assert e.value.status == bem.BEM_E_INVALID_ARG
        with pytest.raises(bem.BemError) as e:
            bem.bem_solve_transmission(ctx, ge, gi, 2.0, 1.0, 1.0, np.array([[0.0, 0.0, 1.0]]),
                                       opts={"formulation": 99})
        assert e.value.status == bem.BEM_E_INVALID_ARG
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
