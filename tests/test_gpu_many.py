"""Many uneven instances in one call (bem_solve_many): every instance's traces equal
the same problem solved alone with bem_solve_transmission in mixed precision, within
that mode's tolerance 1e-6 (the FP32 assemblies of two calls differ at FP32 rounding
level), and a small instance matches the FP64 oracle within 1e-6."""
import numpy as np
import pytest

import bem_inputs as bi

pytestmark = pytest.mark.gpu

TOL = 1e-6


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


def _instances(bem, ctx):
    rng = np.random.default_rng(7)
    specs = [(1, 1), (2, 1), (1, 2), (2, 2), (3, 2), (2, 3)]
    probs, grids = [], []
    for n, (le, li) in enumerate(specs):
        axes = rng.uniform(0.5, 1.5, 3)
        ve, te, vi, ti = bi.transmission_pair(le, li, seed=100 + n, axes=axes)
        ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
        grids += [ge, gi]
        k_ext = rng.uniform(1.0, 5.0)
        d = bi.plane_wave_directions(1, seed=200 + n)[0]
        probs.append(dict(ext=ge, intr=gi, k_ext=k_ext, k_int=k_ext * rng.uniform(1.2, 2.0),
                          rho=float(np.exp(rng.uniform(np.log(0.2), np.log(5.0)))), dir=d,
                          amp=complex(rng.uniform(0.5, 1.5), rng.uniform(-0.5, 0.5)), pair=(ve, te, vi, ti)))
    # a seventh instance on the grids of the first, another wavenumber
    p0 = dict(probs[0])
    p0["k_ext"], p0["k_int"] = 2.5, 4.0
    probs.append(p0)
    return probs, grids


def test_many_instances_equal_solo_solves(env):
    bem, ctx = env
    probs, grids = _instances(bem, ctx)
    try:
        outs, reps = bem.bem_solve_many(ctx, probs)
        for p, out, rep in zip(probs, outs, reps):
            assert rep["converged"] == 1
            solo, _ = bem.bem_solve_transmission(ctx, p["ext"], p["intr"], p["k_int"], p["k_ext"], p["rho"],
                                                 np.array([p["dir"]]), amps=[p["amp"]],
                                                 opts={"precision": bem.BEM_PREC_MIXED})
            for key in ("v_ext", "w_ext", "v_int", "w_int"):
                assert rel(out[key], solo[key][0]) < TOL, key
    finally:
        for g in grids:
            bem.bem_grid_destroy(g)


def test_many_instances_small_one_matches_oracle(env):
    from oracle.mtf import solve_transmission
    bem, ctx = env
    probs, grids = _instances(bem, ctx)
    try:
        outs, _ = bem.bem_solve_many(ctx, probs[:3])
        ve, te, vi, ti = probs[0]["pair"]
        p = probs[0]
        ref = solve_transmission(ve, te, vi, ti, p["k_ext"], p["k_int"], p["rho"], p["dir"], tol=1e-12)
        for key in ("v_ext", "w_ext", "v_int", "w_int"):
            assert rel(outs[0][key], p["amp"] * ref[key]) < TOL, key
    finally:
        for g in grids:
            bem.bem_grid_destroy(g)


def test_many_rejects_fp64_and_bad_input(env):
    bem, ctx = env
    v, t = bi.icosphere(1)
    g = bem.bem_grid_create(ctx, v, t)
    try:
        p = dict(ext=g, intr=g, k_ext=1.0, k_int=2.0, rho=1.0, dir=[0.0, 0.0, 1.0])
        with pytest.raises(bem.BemError) as e:
            bem.bem_solve_many(ctx, [p], opts={"precision": bem.BEM_PREC_FP64})
        assert e.value.status == bem.BEM_E_INVALID_ARG
        with pytest.raises(bem.BemError) as e:
            bem.bem_solve_many(ctx, [dict(p, dir=[0.0, 0.0, 2.0])])
        assert e.value.status == bem.BEM_E_INVALID_ARG
    finally:
        bem.bem_grid_destroy(g)


def test_instances_of_one_problem_share_operators_and_equal_solo_solves(env):
    """Instances with the same grids and wavenumbers (several waves, amplitudes and
    density ratios of one problem) share one copy of the operators; each still equals
    its solo solve, with the default switch from double-float to FP32 products, with
    double-float products throughout (dd_switch 0) and with FP32 throughout (1)."""
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(2, 3, seed=31, axes=(1.2, 0.8, 1.0))
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    try:
        dirs = bi.plane_wave_directions(4, seed=32)
        probs = [dict(ext=ge, intr=gi, k_ext=3.0, k_int=4.5, rho=[0.5, 1.0, 2.0, 7.0][i], dir=dirs[i],
                      amp=complex(1.0 + 0.2 * i, -0.1 * i)) for i in range(4)]
        for sw in (1e-3, 0.0, 1.0):
            outs, reps = bem.bem_solve_many(ctx, probs, opts={"dd_switch": sw})
            for p, out, rep in zip(probs, outs, reps):
                assert rep["converged"] == 1
                solo, _ = bem.bem_solve_transmission(ctx, ge, gi, p["k_int"], p["k_ext"], p["rho"],
                                                     np.array([p["dir"]]), amps=[p["amp"]],
                                                     opts={"precision": bem.BEM_PREC_MIXED})
                for key in ("v_ext", "w_ext", "v_int", "w_int"):
                    assert rel(out[key], solo[key][0]) < TOL, (sw, key)
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
