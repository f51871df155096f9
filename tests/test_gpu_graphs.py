"""CUDA-graph replay of the fixed launch sequences of the iteration (the Chebyshev mass
inverses, captured once per solve): the same kernels with the same arguments run
either way, so results agree with graphs on and off to the run-to-run rounding of
each mode (the assemblies add tile contributions with atomics whose order varies:
FP64 to ~1e-15, the mixed mode to FP32 rounding), and the library's launch counter
counts the kernels a graph launch runs."""
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


def _pair(bem, ctx, le, li, seed):
    ve, te, vi, ti = bi.transmission_pair(le, li, seed=seed, axes=[1.1, 0.9, 1.0])
    return bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)


@pytest.mark.parametrize("form", [0, 1])
def test_graphs_on_and_off_give_identical_fp64_solutions(env, form):
    bem, ctx = env
    ge, gi = _pair(bem, ctx, 2, 2, 3)
    dirs = bi.plane_wave_directions(3, seed=5)
    try:
        res = []
        for g in (0, 1):
            l0 = bem.bem_launch_count()
            out, rep = bem.bem_solve_transmission(ctx, ge, gi, 3.0, 2.0, 1.5, dirs,
                                                  opts={"cuda_graphs": g, "formulation": form})
            res.append((out, rep, bem.bem_launch_count() - l0))
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
    (a, ra, la), (b, rb, lb) = res
    assert abs(ra["iterations"] - rb["iterations"]) <= 1
    for key in a:
        e = np.linalg.norm(a[key] - b[key]) / np.linalg.norm(a[key])
        assert e < 1e-12, (key, e)
    if ra["iterations"] == rb["iterations"]:
        assert la == lb  # a graph launch counts the kernels it runs


def test_graphs_on_and_off_agree_in_mixed_precision_and_many_instances(env):
    bem, ctx = env
    ge, gi = _pair(bem, ctx, 3, 2, 4)
    g2e, g2i = _pair(bem, ctx, 2, 3, 6)
    try:
        d = np.array([[0.0, 0.0, 1.0]])
        out = [bem.bem_solve_transmission(ctx, ge, gi, 4.0, 2.5, 2.0, d,
                                          opts={"precision": bem.BEM_PREC_MIXED, "cuda_graphs": g})[0]
               for g in (0, 1)]
        for key in out[0]:
            e = np.linalg.norm(out[0][key] - out[1][key]) / np.linalg.norm(out[0][key])
            assert e < 1e-6, key
        probs = [dict(ext=ge, intr=gi, k_ext=2.5, k_int=4.0, rho=2.0, dir=[0.0, 0.0, 1.0]),
                 dict(ext=g2e, intr=g2i, k_ext=3.0, k_int=4.5, rho=0.5, dir=[1.0, 0.0, 0.0])]
        many = [bem.bem_solve_many(ctx, probs, opts={"cuda_graphs": g})[0] for g in (0, 1)]
        for i in range(2):
            for key in many[0][i]:
                e = np.linalg.norm(many[0][i][key] - many[1][i][key]) / np.linalg.norm(many[0][i][key])
                assert e < 1e-6, (i, key)
    finally:
        for g in (ge, gi, g2e, g2i):
            bem.bem_grid_destroy(g)


def test_grid_barrier_wait_is_bounded(env):
    """The fused mass inverse synchronises its blocks with a grid barrier whose waits
    give up after about a second: a barrier that can never complete (its count starts
    past the grid size) is flagged, and the launch returns."""
    bem, ctx = env
    r = bem.bem_selftest(ctx, 3)
    assert 1000.0 <= r < 1010.0, r


def test_fused_mass_inverse_matches_the_servers_step_launches(env):
    """Solves on an exclusive context run each mass inverse as one cooperative launch;
    the server's contexts (whose solves overlap) launch one kernel per step.  The
    arithmetic is the same item by item, so the traces agree to the run-to-run rounding
    of the FP64 assembly's atomics."""
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(2, 2, seed=3, axes=[1.1, 0.9, 1.0])
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    d = np.array([[0.0, 0.0, 1.0]])
    bem.bem_context_set_exclusive(ctx, True)
    try:
        a, ra = bem.bem_solve_transmission(ctx, ge, gi, 3.0, 2.0, 1.5, d)
    finally:
        bem.bem_context_set_exclusive(ctx, False)
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
    srv = bem.bem_serve_create(max_inflight=1)
    try:
        t = bem.bem_serve_submit(srv, ve, te, vi, ti, 2.0, 3.0, 1.5, d, precision=bem.BEM_PREC_FP64)
        assert bem.bem_serve_wait(srv, t, 120000.0)
        out, info = bem.bem_serve_take(srv, t, 1, len(ve), len(vi))
    finally:
        bem.bem_serve_destroy(srv)
    assert info["iterations"] == ra["iterations"]
    for key in a:
        e = np.linalg.norm(a[key][0] - out[key][0]) / np.linalg.norm(a[key][0])
        assert e < 1e-12, (key, e)
