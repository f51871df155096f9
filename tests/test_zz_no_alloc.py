"""bem_projection_noalloc: the mortar matrix for callers that must not have the
library allocate device memory (a host program that hands out all HBM from its own
budgeted pool, or a loop that cannot pay for an allocation).  Its output must equal
bem_projection's, call after call, although every call reuses the same fixed
scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest
import scipy.sparse as sp

import bem_inputs as bi

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the mortar tolerance of the parity tests


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2206_00708_gb300 as bem
    ctx = bem.bem_context_create(0)
    yield bem, ctx, torch
    bem.bem_context_destroy(ctx)


def _dense(r, c, v, shape):
    return sp.coo_matrix((v, (r, c)), shape=shape).toarray()


def _reference(bem, ctx, a, b, shape, center=None):
    s = bem.bem_projection(ctx, a, b, center)
    r, c, v = bem.bem_sparse_copy_out(ctx, s)
    bem.bem_sparse_destroy(s)
    return _dense(r, c, v, shape)


def _noalloc(bem, ctx, torch, a, b, shape, cap, center=None):
    row = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    col = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    val = torch.full((cap,), np.nan, dtype=torch.float64, device="cuda")
    n = bem.bem_projection_noalloc(ctx, a, b, row, col, val, center)
    bem.bem_context_synchronize(ctx)
    return _dense(row[:n].cpu().numpy(), col[:n].cpu().numpy(), val[:n].cpu().numpy(), shape)


@pytest.mark.parametrize("le,li,axes", [(2, 2, None), (3, 2, [1.3, 0.8, 1.1])])
def test_noalloc_matches_projection_on_two_calls_in_a_row(env, le, li, axes):
    bem, ctx, torch = env
    ve, te, vi, ti = bi.transmission_pair(le, li, seed=4, axes=axes)
    ge = bem.bem_grid_create(ctx, ve, te)
    gi = bem.bem_grid_create(ctx, vi, ti)
    shape = (len(vi), len(ve))
    ref = _reference(bem, ctx, gi, ge, shape)
    cap = 9 * len(ti) * 64
    for _ in range(2):  # the second call reuses the scratch left by the first
        got = _noalloc(bem, ctx, torch, gi, ge, shape, cap)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)


def test_noalloc_after_a_larger_call_and_with_a_centre(env):
    """A small call after a large one must not see the large call's candidates."""
    bem, ctx, torch = env
    big_e, big_te, big_i, big_ti = bi.transmission_pair(4, 4, seed=1)
    a = bem.bem_grid_create(ctx, big_i, big_ti)
    b = bem.bem_grid_create(ctx, big_e, big_te)
    _noalloc(bem, ctx, torch, a, b, (len(big_i), len(big_e)), 9 * len(big_ti) * 64)
    bem.bem_grid_destroy(a)
    bem.bem_grid_destroy(b)
    vi, ti = bi.unit_square_grid(5)
    ve = bi.perturb_square_grid(vi, 0.02, seed=3)
    a = bem.bem_grid_create(ctx, vi, ti)
    b = bem.bem_grid_create(ctx, ve, ti)
    c0 = (0.5, 0.5, 1.0)
    ref = _reference(bem, ctx, a, b, (len(vi), len(ve)), c0)
    got = _noalloc(bem, ctx, torch, a, b, (len(vi), len(ve)), 9 * len(ti) * 64, c0)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL
    bem.bem_grid_destroy(a)
    bem.bem_grid_destroy(b)


def test_noalloc_rejects_sizes_beyond_its_limits(env):
    bem, ctx, torch = env
    v, t = bi.icosphere(2)
    g = bem.bem_grid_create(ctx, v, t)
    tiny = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(bem.BemError) as e:  # output capacity too small
        bem.bem_projection_noalloc(ctx, g, g, tiny, tiny.clone(), torch.zeros(8, dtype=torch.float64, device="cuda"))
    assert e.value.status == bem.BEM_E_INVALID_ARG and "capacity" in str(e.value)
    v6, t6 = bi.icosphere(6)  # 81920 triangles: above the 32768 limit
    g6 = bem.bem_grid_create(ctx, v6, t6)
    with pytest.raises(bem.BemError) as e:
        bem.bem_projection_noalloc(ctx, g6, g, tiny, tiny.clone(), torch.zeros(8, dtype=torch.float64, device="cuda"))
    assert e.value.status == bem.BEM_E_INVALID_ARG and "32768" in str(e.value)
    bem.bem_grid_destroy(g6)
    bem.bem_grid_destroy(g)


def test_noalloc_rejects_unsuitable_device_outputs(env):
    """Wrong dtypes and strided views are refused by the binding before the call."""
    bem, ctx, torch = env
    v, t = bi.icosphere(1)
    g = bem.bem_grid_create(ctx, v, t)
    i32 = torch.zeros(4096, dtype=torch.int32, device="cuda")
    f64 = torch.zeros(4096, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError, match="dtype"):
        bem.bem_projection_noalloc(ctx, g, g, i32.long(), i32, f64)
    with pytest.raises(ValueError, match="dtype"):
        bem.bem_projection_noalloc(ctx, g, g, i32, i32, f64.float())
    with pytest.raises(ValueError, match="contiguous"):
        bem.bem_projection_noalloc(ctx, g, g, i32[::2], i32[::2], f64[::2])
    bem.bem_grid_destroy(g)
