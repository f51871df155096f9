"""The autotuner on the GPU: bem_autotune fills the launch-shape table for the grids'
sizes (every tuned kernel family and width, with the time it measured), the chosen
shapes are among the candidates, and solves that use them give the results of
solves with the built-in shapes (FP64 to rounding, mixed within the mode's 1e-6,
tensor-core batches included)."""
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
    bem.bem_tune_clear()
    bem.bem_context_destroy(ctx)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_autotune_fills_the_table_and_keeps_results(env, tmp_path):
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(3, 2, seed=7)
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    n = 2 * (len(ve) + len(vi))
    dirs = bi.plane_wave_directions(12, seed=8)
    try:
        bem.bem_tune_clear()
        ref64 = bem.bem_solve_transmission(ctx, ge, gi, 3.0, 2.0, 1.5, dirs[:3])[0]
        refmx = bem.bem_solve_transmission(ctx, ge, gi, 3.0, 2.0, 1.5, dirs, opts={"precision": 1})[0]
        bem.bem_autotune(ctx, ge, gi, 12)
        assert bem.bem_tune_count() == 2 + 1
        for w in (1, 8):
            assert bem.bem_tune_get("cheb", w, n)[0] in (64, 128, 256)
        b, v, ms = bem.bem_tune_get("gemm_tc", 16, n)
        assert b == 0 and v in (1, 2) and ms > 0.0
        out64 = bem.bem_solve_transmission(ctx, ge, gi, 3.0, 2.0, 1.5, dirs[:3])[0]
        outmx = bem.bem_solve_transmission(ctx, ge, gi, 3.0, 2.0, 1.5, dirs, opts={"precision": 1})[0]
        for key in ref64:
            assert rel(out64[key], ref64[key]) < 1e-12, key
            assert rel(outmx[key], refmx[key]) < 1e-6, key
        p = tmp_path / "tune.json"
        bem.bem_tune_save(str(p))
        bem.bem_tune_clear()
        bem.bem_tune_load(str(p))
        assert bem.bem_tune_count() == 3
    finally:
        bem.bem_tune_clear()
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
