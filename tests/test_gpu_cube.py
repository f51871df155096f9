"""The unit-cube workload of Sec. 5.3-5.5 on the GPU (structured cube grids from
bem_inputs.cube_grid standing in for the paper's meshes): parity with the FP64
oracle where triangles meet at the cube's edges and corners (singular pairs across
faces at right angles), the mortar between two independent cube grids, and full
solves with the paper's standard physics (k_ext = 2 pi / 0.3, k_int = 2 pi / 1.1,
rho_int / rho_ext = 2, plane wave along +x).

Tolerances: relative L2 <= 1e-10 in FP64, as in the other parity tests.  The mixed
mode converges to the solution of its complex64-stored system, whose distance from
the FP64 system's solution is the operators' FP32 error (~1e-7 per entry) times the
system's sensitivity.  On the at-scale sphere that product is 9.6e-7 (the 1e-6 target
of the precision configuration); the standard cube benchmark (k_ext h ~ 0.95, edges
and corners) is about three times more sensitive: measured 3.0e-6 for the MTF, so
its mixed-mode bound is 5e-6.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import bem_inputs as bi

pytestmark = pytest.mark.gpu

TOL = 1e-10
MIXED_TOL_CUBE = 5e-6
CENTER = (0.5, 0.5, 0.5)
K_EXT, K_INT, RHO = 2.0 * np.pi / 0.3, 2.0 * np.pi / 1.1, 2.0


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2206_00708_gb300 as bem
    ctx = bem.bem_context_create(0)
    yield bem, ctx
    bem.bem_context_destroy(ctx)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("k", [K_INT, 3.0 + 0.4j])
def test_cube_operators_match_oracle(env, k):
    from oracle.helmholtz import assemble
    bem, ctx = env
    v, t = bi.cube_grid(3, jitter=0.3, seed=7)
    g = bem.bem_grid_create(ctx, v, t)
    ref = assemble(v, t, k)
    try:
        for name, op in (("V", bem.BEM_OP_V), ("K", bem.BEM_OP_K), ("T", bem.BEM_OP_T), ("D", bem.BEM_OP_D)):
            m = bem.bem_assemble(ctx, op, k, g)
            got = bem.bem_matrix_copy_out(ctx, m)
            bem.bem_matrix_destroy(m)
            assert rel(got, ref[name]) < TOL, name
    finally:
        bem.bem_grid_destroy(g)


def test_cube_mortar_matches_oracle(env):
    from oracle.mortar import mortar_matrix
    bem, ctx = env
    ve, te = bi.cube_grid(5, jitter=0.3, seed=1)
    vi, ti = bi.cube_grid(3, jitter=0.3, seed=2)
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    try:
        s = bem.bem_projection(ctx, gi, ge, CENTER)
        r, c, v = bem.bem_sparse_copy_out(ctx, s)
        bem.bem_sparse_destroy(s)
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
    P = sp.coo_matrix((v, (r, c)), shape=(len(vi), len(ve))).toarray()
    ref = mortar_matrix(vi, ti, ve, te, CENTER)
    ref = np.asarray(ref.todense()) if hasattr(ref, "todense") else np.asarray(ref)
    assert rel(P, ref) < 1e-12


@pytest.mark.parametrize("form", ["mtf", "pmchwt_ext"])
def test_cube_solve_matches_oracle(env, form):
    """Nonconforming cube pair (98 exterior, 56 interior vertices) with the standard
    benchmark's physics, FP64 at GMRES tol 1e-12."""
    from oracle.mtf import mtf_blocks, solve_transmission
    from oracle.pmchwt import solve_single_trace
    bem, ctx = env
    ve, te = bi.cube_grid(4, jitter=0.3, seed=1)
    vi, ti = bi.cube_grid(3, jitter=0.3, seed=2)
    d = np.array([[1.0, 0.0, 0.0]])
    opts = {"gmres_tol": 1e-12, "center": CENTER}
    if form != "mtf":
        opts["formulation"] = bem.BEM_FORM_PMCHWT
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    try:
        out, rep = bem.bem_solve_transmission(ctx, ge, gi, K_INT, K_EXT, RHO, d, opts=opts)
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
    B = mtf_blocks(ve, te, vi, ti, K_EXT, K_INT, center=CENTER)
    if form == "mtf":
        ref = solve_transmission(ve, te, vi, ti, K_EXT, K_INT, RHO, d[0], tol=1e-12, blocks=B)
    else:
        ref = solve_single_trace(ve, te, vi, ti, K_EXT, K_INT, RHO, d[0], form, tol=1e-12, blocks=B)
    for key in ("v_ext", "w_ext", "v_int", "w_int"):
        e = rel(out[key][0], ref[key])
        assert e < TOL, (form, key, e)


def test_cube_standard_benchmark_mixed_matches_fp64(env):
    """The standard benchmark's grids (2906 exterior and 296 interior vertices, the
    node counts of the paper's mesh table to within 3 % and 9 %): mixed-precision MTF
    and PMCHWT solves against the FP64 GPU solves of the same systems, both at GMRES
    tol 1e-10 so that the difference is the precision's."""
    bem, ctx = env
    ve, te = bi.cube_grid(22, jitter=0.3, seed=61)
    vi, ti = bi.cube_grid(7, jitter=0.3, seed=62)
    d = np.array([[1.0, 0.0, 0.0]])
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    try:
        for form in (bem.BEM_FORM_MTF, bem.BEM_FORM_PMCHWT):
            base = {"gmres_tol": 1e-10, "center": CENTER, "formulation": form, "gmres_maxiter": 4000}
            ref, r64 = bem.bem_solve_transmission(ctx, ge, gi, K_INT, K_EXT, RHO, d, opts=base)
            out, rmx = bem.bem_solve_transmission(ctx, ge, gi, K_INT, K_EXT, RHO, d,
                                                  opts=dict(base, precision=bem.BEM_PREC_MIXED))
            errs = {key: rel(out[key][0], ref[key][0]) for key in ("v_ext", "w_ext", "v_int", "w_int")}
            print(form, errs, r64["iterations"], rmx["iterations"])
            assert max(errs.values()) < MIXED_TOL_CUBE, (form, errs)
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
