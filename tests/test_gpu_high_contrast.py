"""Parity of the high-contrast solves (bem_solve_transmission with formulation =
BEM_FORM_HC_EXT_NEU, _EXT_DIR, _INT_NEU, _INT_DIR: Sec. 2.3) with the FP64 oracle of
oracle/highcontrast.py.  Tolerances as for the other formulations: relative L2 <= 1e-10
in FP64 (same operators, same GMRES; the mass inverses inside the operator are 34
Chebyshev steps, ~1e-16), <= 1e-6 in the mixed mode."""
import numpy as np
import pytest

import bem_inputs as bi

pytestmark = pytest.mark.gpu

TOL = 1e-10
MIXED_TOL = 1e-6
KEYS = ("v_ext", "w_ext", "v_int", "w_int")
FORMS = ("hc_ext_neu", "hc_ext_dir", "hc_int_neu", "hc_int_dir")


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
    return {"hc_ext_neu": bem.BEM_FORM_HC_EXT_NEU, "hc_ext_dir": bem.BEM_FORM_HC_EXT_DIR,
            "hc_int_neu": bem.BEM_FORM_HC_INT_NEU, "hc_int_dir": bem.BEM_FORM_HC_INT_DIR}[form]


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
def case():
    """Ellipsoid, exterior level 2 / interior level 1 (nonconforming), complex interior
    wavenumber, density ratio 2.5."""
    from oracle.mtf import mtf_blocks
    ve, te, vi, ti = bi.transmission_pair(2, 1, seed=6, axes=[1.2, 0.9, 1.0])
    k_ext, k_int, rho = 2.0, 3.0 + 0.2j, 2.5
    return dict(grids=(ve, te, vi, ti), k_ext=k_ext, k_int=k_int, rho=rho,
                blocks=mtf_blocks(ve, te, vi, ti, k_ext, k_int))


@pytest.mark.parametrize("form", FORMS)
def test_high_contrast_fp64_matches_oracle(env, case, form):
    from oracle.highcontrast import solve_high_contrast
    bem, ctx = env
    ve, te, vi, ti = case["grids"]
    d = np.array([[0.0, 0.6, 0.8]])
    out, rep = _solve(bem, ctx, form, ve, te, vi, ti, case["k_int"], case["k_ext"], case["rho"], d, gmres_tol=1e-12)
    ref = solve_high_contrast(ve, te, vi, ti, case["k_ext"], case["k_int"], case["rho"], d[0], form, tol=1e-12,
                              blocks=case["blocks"])
    for key in KEYS:
        e = rel(out[key][0], ref[key])
        assert e < TOL, (form, key, e)
    assert rep["converged"] == 1
    _, rep8 = _solve(bem, ctx, form, ve, te, vi, ti, case["k_int"], case["k_ext"], case["rho"], d)
    ref8 = solve_high_contrast(ve, te, vi, ti, case["k_ext"], case["k_int"], case["rho"], d[0], form, tol=1e-8,
                               blocks=case["blocks"])
    assert abs(rep8["iterations"] - ref8["iters"]) <= 1, (form, rep8["iterations"], ref8["iters"])


@pytest.mark.parametrize("form", ["hc_ext_dir", "hc_int_neu"])
def test_high_contrast_fp64_multi_rhs(env, form):
    """Three waves with complex amplitudes in one call, interior grid finer than the
    exterior one (a batch of 3 at kernel width 4)."""
    from oracle.highcontrast import solve_high_contrast
    from oracle.mtf import mtf_blocks
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(1, 2, seed=8)
    dirs = bi.plane_wave_directions(3, seed=40)
    amps = [1.0, 0.5 - 0.25j, 2.0j]
    k_ext, k_int, rho = 1.5, 2.5, 0.4
    out, _ = _solve(bem, ctx, form, ve, te, vi, ti, k_int, k_ext, rho, dirs, amps=amps, gmres_tol=1e-12)
    B = mtf_blocks(ve, te, vi, ti, k_ext, k_int)
    for r in range(3):
        ref = solve_high_contrast(ve, te, vi, ti, k_ext, k_int, rho, dirs[r], form, tol=1e-12, blocks=B)
        for key in KEYS:
            e = rel(out[key][r], amps[r] * ref[key])
            assert e < TOL, (form, r, key, e)


@pytest.mark.parametrize("form,n_rhs", [("hc_ext_neu", 1), ("hc_ext_dir", 5), ("hc_int_neu", 1), ("hc_int_dir", 3)])
def test_high_contrast_mixed_matches_oracle(env, form, n_rhs):
    from oracle.highcontrast import solve_high_contrast
    from oracle.mtf import mtf_blocks
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(2, 2, seed=11, axes=[1.1, 1.0, 0.9])
    dirs = bi.plane_wave_directions(n_rhs, seed=45)
    k_ext, k_int, rho = 2.5, 4.0, 8.0
    out, rep = _solve(bem, ctx, form, ve, te, vi, ti, k_int, k_ext, rho, dirs, gmres_tol=1e-10,
                      precision=bem.BEM_PREC_MIXED)
    assert rep["converged"] == 1
    B = mtf_blocks(ve, te, vi, ti, k_ext, k_int)
    for r in range(n_rhs):
        ref = solve_high_contrast(ve, te, vi, ti, k_ext, k_int, rho, dirs[r], form, tol=1e-12, blocks=B)
        for key in KEYS:
            e = rel(out[key][r], ref[key])
            assert e < MIXED_TOL, (form, r, key, e)


def test_high_contrast_agrees_with_mtf_at_level4(env):
    """At level 4 (k 10 / 15) and the paper's high density contrast 2 / 0.11 the four
    high-contrast systems and the multiple-traces system discretise the same problem:
    exterior potentials within the discretisation error of each other."""
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(4, 4, seed=2)
    d = np.array([[0.0, 0.0, 1.0]])
    rho = 2.0 / 0.11
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    res = {}
    try:
        for form in ("mtf",) + FORMS:
            opts = {"precision": bem.BEM_PREC_MIXED, "gmres_maxiter": 4000}
            if form != "mtf":
                opts["formulation"] = code(bem, form)
            res[form] = bem.bem_solve_transmission(ctx, ge, gi, 15.0, 10.0, rho, d, opts=opts)
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
    m, rm = res["mtf"]
    print({f: r[1]["iterations"] for f, r in res.items()})
    for form in FORMS:
        p, rp = res[form]
        assert rp["converged"] == 1, form
        assert rel(p["v_ext"][0], m["v_ext"][0]) < 0.1, form
