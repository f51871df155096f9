"""Parity of the Neumann-screen solve (bem_solve_screen: Sec. 4.2 with mass-matrix and
opposite-order preconditioning) with the FP64 oracle of oracle/screen.py.  Tolerances:
relative L2 <= 1e-10 in FP64, <= 1e-6 in the mixed mode (whose refinement converges to
the complex64-stored system).  With a coarse opposite-order preconditioner the
preconditioned system is rank-deficient and its solution is not unique; the mixed
mode is checked there through the preconditioned residual only."""
import numpy as np
import pytest

import bem_inputs as bi

pytestmark = pytest.mark.gpu

TOL = 1e-10
MIXED_TOL = 1e-6
K = 5.0
D_INC = np.array([[1.0, 0.0, 0.0]])


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2206_00708_gb300 as bem
    ctx = bem.bem_context_create(0)
    v, t = bi.screen_grid(10, 9, jitter=0.2, seed=1)
    vc, tc = bi.screen_grid(4, 3, jitter=0.2, seed=2)
    gf, gc = bem.bem_grid_create(ctx, v, t), bem.bem_grid_create(ctx, vc, tc)
    yield bem, ctx, (v, t, gf), (vc, tc, gc)
    bem.bem_grid_destroy(gf)
    bem.bem_grid_destroy(gc)
    bem.bem_context_destroy(ctx)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("pre", ["mass", "oo", "oo_conforming"])
def test_screen_fp64_matches_oracle(env, pre):
    from oracle.screen import boundary_nodes, solve_screen
    bem, ctx, (v, t, gf), (vc, tc, gc) = env
    code = bem.BEM_SCREEN_MASS if pre == "mass" else bem.BEM_SCREEN_OO
    coarse = gc if pre == "oo" else (gf if pre == "oo_conforming" else None)
    cv, ct = (vc, tc) if pre == "oo" else (v, t)
    phi, rep = bem.bem_solve_screen(ctx, gf, K, D_INC, coarse=coarse, precond=code, opts={"gmres_tol": 1e-12})
    ref = solve_screen(v, t, K, D_INC[0], "mass" if pre == "mass" else "oo", cv, ct, tol=1e-12)
    e = rel(phi[0], ref["phi"])
    assert e < TOL, (pre, e)
    assert np.all(phi[0][boundary_nodes(t, len(v))] == 0.0)
    _, rep8 = bem.bem_solve_screen(ctx, gf, K, D_INC, coarse=coarse, precond=code)
    ref8 = solve_screen(v, t, K, D_INC[0], "mass" if pre == "mass" else "oo", cv, ct, tol=1e-8)
    assert abs(rep8["iterations"] - ref8["iters"]) <= 1, (pre, rep8["iterations"], ref8["iters"])


def test_screen_fp64_multi_rhs_with_amplitudes(env):
    from oracle.screen import solve_screen
    bem, ctx, (v, t, gf), _ = env
    dirs = bi.plane_wave_directions(3, seed=40)
    amps = [1.0, 0.5 - 0.25j, 2.0j]
    phi, _ = bem.bem_solve_screen(ctx, gf, K, dirs, amps=amps, opts={"gmres_tol": 1e-12})
    for r in range(3):
        ref = solve_screen(v, t, K, dirs[r], "mass", tol=1e-12)
        assert rel(phi[r], amps[r] * ref["phi"]) < TOL, r


def test_screen_conforming_preconditioner_keeps_the_solution(env):
    bem, ctx, (v, t, gf), _ = env
    a, ra = bem.bem_solve_screen(ctx, gf, K, D_INC, opts={"gmres_tol": 1e-11})
    b, rb = bem.bem_solve_screen(ctx, gf, K, D_INC, coarse=gf, precond=bem.BEM_SCREEN_OO, opts={"gmres_tol": 1e-11})
    assert rel(b[0], a[0]) < 1e-9
    assert 2 * rb["iterations"] < ra["iterations"]


@pytest.mark.parametrize("pre", ["mass", "oo_conforming"])
def test_screen_mixed_matches_oracle(env, pre):
    from oracle.screen import solve_screen
    bem, ctx, (v, t, gf), _ = env
    code = bem.BEM_SCREEN_MASS if pre == "mass" else bem.BEM_SCREEN_OO
    phi, rep = bem.bem_solve_screen(ctx, gf, K, D_INC, coarse=gf if pre != "mass" else None, precond=code,
                                    opts={"gmres_tol": 1e-10, "precision": bem.BEM_PREC_MIXED})
    ref = solve_screen(v, t, K, D_INC[0], "mass", tol=1e-12)
    assert rep["converged"] == 1
    assert rel(phi[0], ref["phi"]) < MIXED_TOL


def test_screen_mixed_coarse_preconditioner_converges(env):
    bem, ctx, (v, t, gf), (vc, tc, gc) = env
    phi, rep = bem.bem_solve_screen(ctx, gf, K, D_INC, coarse=gc, precond=bem.BEM_SCREEN_OO,
                                    opts={"gmres_tol": 1e-8, "precision": bem.BEM_PREC_MIXED})
    assert rep["converged"] == 1 and rep["residual"] <= 1e-8
    assert np.isfinite(phi).all()


def test_screen_invalid_arguments(env):
    bem, ctx, (v, t, gf), _ = env
    with pytest.raises(bem.BemError) as e:
        bem.bem_solve_screen(ctx, gf, K, D_INC, precond=bem.BEM_SCREEN_OO)  # no coarse grid
    assert e.value.status == bem.BEM_E_INVALID_ARG
    with pytest.raises(bem.BemError) as e:
        bem.bem_solve_screen(ctx, gf, K, D_INC, precond=5)
    assert e.value.status == bem.BEM_E_INVALID_ARG
