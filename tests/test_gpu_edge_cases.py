"""Degenerate and boundary cases of the method on the GPU, against the FP64 oracle
(relative L2 <= 1e-10 in FP64, <= 1e-6 in the mixed mode):

* a single triangle (only the coincident Sauter-Schwab pair, no regular pair, one
  ragged 64 x 64 tile) and two triangles sharing an edge (edge-adjacent pair only);
* wavenumbers near the Laplace limit (k = 1e-3, real and complex), where the phase
  k r vanishes and the kernels are those of the Laplace operators;
* identical interior and exterior grids (conforming: the mortar is the mass matrix);
* a zero incident field: the solution is zero after zero iterations, and a zero
  column among nonzero ones stays zero without slowing the others."""
import numpy as np
import pytest

import bem_inputs as bi

pytestmark = pytest.mark.gpu


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
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / n if n > 0 else np.linalg.norm(a)


def _ops(bem, ctx, v, t, k, precision):
    g = bem.bem_grid_create(ctx, v, t)
    out = {}
    for name, op in (("V", bem.BEM_OP_V), ("K", bem.BEM_OP_K), ("T", bem.BEM_OP_T), ("D", bem.BEM_OP_D)):
        m = bem.bem_assemble(ctx, op, k, g, precision=precision)
        out[name] = bem.bem_matrix_copy_out(ctx, m).astype(np.complex128)
        bem.bem_matrix_destroy(m)
    bem.bem_grid_destroy(g)
    return out


def _tiny_surfaces():
    one_v = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.1]])
    one_t = np.array([[0, 1, 2]])
    two_v = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.1, 1.0, 0.0], [1.1, 0.9, 0.3]])
    two_t = np.array([[0, 1, 2], [1, 3, 2]])
    return {"one-triangle": (one_v, one_t), "two-triangles": (two_v, two_t)}


@pytest.mark.parametrize("case", ["one-triangle", "two-triangles"])
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_tiny_surfaces_match_oracle(env, case, precision, tol):
    from oracle.helmholtz import assemble
    bem, ctx = env
    v, t = _tiny_surfaces()[case]
    got = _ops(bem, ctx, v, t, 2.5 + 0.3j, precision)
    ref = assemble(v, t, 2.5 + 0.3j)
    for op in "VKTD":
        # K and T of a flat triangle vanish ((x - y).n = 0): both sides hold rounding noise
        # there, measured against the operators' scale (the single layer's norm)
        scale = max(np.linalg.norm(ref[op]), np.linalg.norm(ref["V"]))
        err = np.linalg.norm(got[op] - ref[op]) / scale
        assert err < tol, (case, op, err)


@pytest.mark.parametrize("k", [1e-3, 1e-3 + 1e-3j])
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_near_laplace_wavenumbers_match_oracle(env, k, precision, tol):
    from oracle.helmholtz import assemble
    bem, ctx = env
    v, t = bi.icosphere(2)
    got = _ops(bem, ctx, v, t, k, precision)
    ref = assemble(v, t, k)
    for op in "VKTD":
        assert rel(got[op], ref[op]) < tol, (k, op, rel(got[op], ref[op]))


def test_identical_grids_solve_matches_oracle(env):
    from oracle.mtf import solve_transmission
    bem, ctx = env
    v, t = bi.icosphere(2)
    g = bem.bem_grid_create(ctx, v, t)
    try:
        d = np.array([[0.0, 0.6, 0.8]])
        out, rep = bem.bem_solve_transmission(ctx, g, g, 3.0, 2.0, 1.7, d, opts={"gmres_tol": 1e-12})
    finally:
        bem.bem_grid_destroy(g)
    ref = solve_transmission(v, t, v, t, 2.0, 3.0, 1.7, d[0], tol=1e-12)
    assert rep["converged"] == 1
    for key in ("v_ext", "w_ext", "v_int", "w_int"):
        assert rel(out[key][0], ref[key]) < 1e-10, key


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_incident_field(env, precision):
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(2, 2, seed=5)
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    try:
        d = bi.plane_wave_directions(3, seed=6)
        out0, rep0 = bem.bem_solve_transmission(ctx, ge, gi, 3.0, 2.0, 1.5, d[:1], amps=[0.0],
                                                opts={"precision": precision})
        assert rep0["converged"] == 1 and rep0["iterations"] == 0
        for key in ("v_ext", "w_ext", "v_int", "w_int"):
            assert np.all(out0[key] == 0), key
        # a zero column among nonzero ones
        out, rep = bem.bem_solve_transmission(ctx, ge, gi, 3.0, 2.0, 1.5, d, amps=[1.0, 0.0, 0.5j],
                                              opts={"precision": precision})
        solo, _ = bem.bem_solve_transmission(ctx, ge, gi, 3.0, 2.0, 1.5, d[2:], amps=[0.5j],
                                             opts={"precision": precision})
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
    assert rep["converged"] == 1
    tol = 1e-10 if precision == 0 else 1e-6
    for key in ("v_ext", "w_ext", "v_int", "w_int"):
        assert np.all(out[key][1] == 0), key
        assert rel(out[key][2], solo[key][0]) < tol, key
