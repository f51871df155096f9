"""Mixed-precision accuracy of every formulation at a size where the storage error
shows (icosphere L4/L4 pair, 2 x 2562 vertices, k_ext 10, k_int 15, density ratio 2,
one plane wave), against the same formulation's FP64 GPU solve (which matches the
oracle to 1e-10, test_gpu_parity.py and the formulation tests).  The multiple-traces
system and the PMCHWT systems meet the mode's 1e-6; the Mueller systems and two of
the high-contrast systems, whose operators subtract or multiply stored operators,
do not, and their bounds here are the measured errors with a margin, so that a
regression is seen (the reasons are in the design notes on mixed precision)."""
import numpy as np
import pytest

import bem_inputs as bi

pytestmark = pytest.mark.gpu

KEYS = ("v_ext", "w_ext", "v_int", "w_int")
# formulation -> bound on the largest relative L2 error of the four traces
# (measured at L4: MTF 6.0e-7, PMCHWT 4.4e-7 / 4.3e-7, Mueller 1.01e-6 / 8.3e-7, high-contrast
# 4.5e-7 / 6.2e-6 / 2.3e-6 / 4.8e-7; at L5 the bench reports 9.6e-7 for the MTF)
BOUNDS = {"mtf": 1e-6, "pmchwt_ext": 1e-6, "pmchwt_int": 1e-6, "muller_ext": 2e-6, "muller_int": 2e-6,
          "hc_ext_neu": 1e-6, "hc_ext_dir": 1.5e-5, "hc_int_neu": 5e-6, "hc_int_dir": 1e-6}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2206_00708_gb300 as bem
    ctx = bem.bem_context_create(0)
    ve, te, vi, ti = bi.transmission_pair(4, 4, seed=2)
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    yield bem, ctx, ge, gi
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)
    bem.bem_context_destroy(ctx)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("form", list(BOUNDS))
def test_mixed_error_at_level4(env, form):
    bem, ctx, ge, gi = env
    code = {"mtf": bem.BEM_FORM_MTF, "pmchwt_ext": bem.BEM_FORM_PMCHWT, "pmchwt_int": bem.BEM_FORM_PMCHWT_INT,
            "muller_ext": bem.BEM_FORM_MULLER, "muller_int": bem.BEM_FORM_MULLER_INT,
            "hc_ext_neu": bem.BEM_FORM_HC_EXT_NEU, "hc_ext_dir": bem.BEM_FORM_HC_EXT_DIR,
            "hc_int_neu": bem.BEM_FORM_HC_INT_NEU, "hc_int_dir": bem.BEM_FORM_HC_INT_DIR}[form]
    d = np.array([[0.0, 0.0, 1.0]])
    ref, rr = bem.bem_solve_transmission(ctx, ge, gi, 15.0, 10.0, 2.0, d,
                                         opts={"precision": bem.BEM_PREC_FP64, "formulation": code,
                                               "gmres_tol": 1e-12})
    mix, rm = bem.bem_solve_transmission(ctx, ge, gi, 15.0, 10.0, 2.0, d,
                                         opts={"precision": bem.BEM_PREC_MIXED, "formulation": code,
                                               "gmres_tol": 1e-8})
    assert rr["converged"] == 1 and rm["converged"] == 1
    err = max(rel(mix[k][0], ref[k][0]) for k in KEYS)
    print(form, "mixed vs FP64 at L4:", err)
    assert err < BOUNDS[form], (form, err)
