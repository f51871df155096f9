"""bem_field (eq. representation) through the C ABI against the FP64 oracle
(oracle/potentials.py): relative L2 <= 1e-10, the FP64 tolerance of the path; and
the fields of a GPU transmission solve against the Mie series."""
import numpy as np
import pytest

import bem_inputs as bi

pytestmark = pytest.mark.gpu

TOL = 1e-10


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


def _points(seed, n):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = np.concatenate([rng.uniform(0.0, 0.6, n // 2), rng.uniform(1.6, 3.0, n - n // 2)])
    return d * r[:, None]


@pytest.mark.parametrize("k", [1.5, 4.0 + 0.3j])
def test_field_matches_oracle(env, k):
    from oracle.potentials import representation
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(3, 2, seed=4, axes=[1.2, 0.9, 1.0])
    rng = np.random.default_rng(11)
    phi = rng.normal(size=len(ve)) + 1j * rng.normal(size=len(ve))
    psi = rng.normal(size=len(ve)) + 1j * rng.normal(size=len(ve))
    x = _points(3, 301)  # ragged against every tile and slice size
    g = bem.bem_grid_create(ctx, ve, te)
    try:
        for a, b in ((phi, psi), (phi, None), (None, psi)):
            got = bem.bem_field(ctx, g, k, x, phi=a, psi=b)
            ref = representation(ve, te, k, x, phi=a, psi=b)
            assert rel(got, ref) < TOL
        assert len(bem.bem_field(ctx, g, k, np.zeros((0, 3)), phi=phi)) == 0
    finally:
        bem.bem_grid_destroy(g)


def test_fields_of_a_solve_converge_to_the_mie_series(env):
    """Sphere, icosphere L2 and L3 on both grids: the interior field and the scattered
    field from the FP64 GPU traces approach the Mie series at O(h^2) (L2: 5.7e-2 and
    1.6e-2 with the oracle's traces)."""
    from oracle.mie import mie_field
    bem, ctx = env
    k_e, k_i, rho = 1.0, 2.0, 1.5
    d = np.array([0.0, 0.0, 1.0])
    xin = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1], [-0.1, 0.4, -0.3]])
    xout = np.array([[2.0, 1.0, 0.0], [0.0, -2.5, 0.5], [1.2, 1.2, 1.2]])
    ti, _ = mie_field(xin, d, k_e, k_i, rho)
    to, io = mie_field(xout, d, k_e, k_i, rho)
    errs = []
    for L in (2, 3):
        ve, te, vi, ti_ = bi.transmission_pair(L, L, seed=1)
        ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti_)
        try:
            out, _ = bem.bem_solve_transmission(ctx, ge, gi, k_i, k_e, rho, d[None, :], opts={"gmres_tol": 1e-10})
            ui = bem.bem_field(ctx, gi, k_i, xin, phi=out["v_int"][0], psi=out["w_int"][0])
            us = bem.bem_field(ctx, ge, k_e, xout, phi=out["v_ext"][0], psi=out["w_ext"][0])
        finally:
            bem.bem_grid_destroy(ge)
            bem.bem_grid_destroy(gi)
        errs.append((np.max(np.abs(ui - ti)), np.max(np.abs(us - (to - io)))))
    print("field errors vs Mie", errs)
    assert errs[0][0] < 0.08 and errs[0][1] < 0.03
    assert errs[1][0] < errs[0][0] / 2.5 and errs[1][1] < errs[0][1] / 2.5
