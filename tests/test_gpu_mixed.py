"""Mixed-precision mode (BEM_PREC_MIXED): FP32 regular-pair assembly into complex64
operators, FP64 singular pairs / mass / mortar, FP32-matvec GMRES inside FP64
iterative refinement.

Stated tolerances: operator blocks within relative Frobenius 1e-6 of the FP64
oracle (the FP32 storage rounding is 6e-8); traces within relative L2 1e-6 of the
FP64 oracle, or of the FP64 GPU path where the oracle is too slow (that path matches
the oracle to 1e-10 in test_gpu_parity.py)."""
import numpy as np
import pytest

import bem_inputs as bi

pytestmark = pytest.mark.gpu

OP_TOL = 1e-6
TRACE_TOL = 1e-6


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


def test_fp32_kernel_sincos_matches_cuda_sincosf(env):
    """The FP32 assembly kernel's own sin/cos agrees with CUDA's sincosf to a few
    FP32 units in the last place over [-64, 64]."""
    bem, ctx = env
    err = bem.bem_selftest(ctx, 0)
    print("sincos max abs diff", err)
    assert err < 4.8e-7  # 4 ulp of 1.0


def mixed_ops(bem, ctx, v, t, k):
    g = bem.bem_grid_create(ctx, v, t)
    out = {}
    for name, op in (("V", bem.BEM_OP_V), ("K", bem.BEM_OP_K), ("T", bem.BEM_OP_T), ("D", bem.BEM_OP_D)):
        m = bem.bem_assemble(ctx, op, k, g, precision=bem.BEM_PREC_MIXED)
        assert bem.bem_matrix_entry_bytes(m) == 8
        out[name] = bem.bem_matrix_copy_out(ctx, m).astype(np.complex128)
        bem.bem_matrix_destroy(m)
    bem.bem_grid_destroy(g)
    return out


# The kernel takes a shorter sin/cos (no argument reduction) on tile pairs where every
# phase offset |k delta| <= |k| (rho_test + rho_trial) is below pi/4: the L2 cases with
# k near 1 and the full-size rows below run that form, the others the reduced one.
@pytest.mark.parametrize("case", ["sphere-L1", "ellipsoid-L2-complex-k", "sphere-L3-k8", "sphere-L2-k1-small-phase",
                                  "ellipsoid-L2-complex-k-small-phase"])
def test_mixed_operators_match_oracle(env, case):
    from oracle.helmholtz import assemble
    bem, ctx = env
    if case == "sphere-L1":
        v, t = bi.icosphere(1)
        k = 1.0
    elif case == "sphere-L2-k1-small-phase":
        v, t = bi.icosphere(2)
        k = 1.0
    elif case == "ellipsoid-L2-complex-k-small-phase":
        _, _, v, t = bi.transmission_pair(2, 2, seed=5, axes=[1.1, 0.9, 1.0])
        k = 1.2 + 0.3j
    elif case == "ellipsoid-L2-complex-k":
        _, _, v, t = bi.transmission_pair(2, 2, seed=3, axes=[1.3, 0.8, 1.1])
        k = 3.0 + 0.5j
    else:
        v, t = bi.icosphere(3)
        k = 8.0
    rows = None if len(v) < 200 else np.random.default_rng(0).choice(len(v), 24, replace=False)
    got = mixed_ops(bem, ctx, v, t, k)
    ref = assemble(v, t, k, rows=rows)
    for op in "VKTD":
        g = got[op] if rows is None else got[op][rows]
        e = rel(g, ref[op])
        print(case, op, e)
        assert e < OP_TOL, (case, op, e)


@pytest.mark.parametrize("k", [10.0, 15.0])
def test_mixed_operators_full_size_sampled_rows(env, k):
    from oracle.helmholtz import assemble
    bem, ctx = env
    v, t = bi.icosphere(5)
    if k == 15.0:
        v = bi.rotate_and_jitter(v, t, seed=2)
    rows = np.random.default_rng(1).choice(len(v), 4, replace=False)
    ref = assemble(v, t, k, rows=rows)
    g = bem.bem_grid_create(ctx, v, t)
    for name, op in (("V", bem.BEM_OP_V), ("K", bem.BEM_OP_K), ("D", bem.BEM_OP_D)):
        m = bem.bem_assemble(ctx, op, k, g, precision=bem.BEM_PREC_MIXED)
        full = bem.bem_matrix_copy_out(ctx, m)
        bem.bem_matrix_destroy(m)
        e = rel(full[rows].astype(np.complex128), ref[name])
        print("L5", k, name, e)
        assert e < OP_TOL, (name, e)
        del full
    bem.bem_grid_destroy(g)


def _solve(bem, ctx, ve, te, vi, ti, k_int, k_ext, rho, dirs, **opts):
    ge = bem.bem_grid_create(ctx, ve, te)
    gi = bem.bem_grid_create(ctx, vi, ti)
    try:
        return bem.bem_solve_transmission(ctx, ge, gi, k_int, k_ext, rho, dirs, opts=opts)
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)


def test_mixed_solve_matches_fp64_oracle_small(env):
    from oracle.mtf import solve_transmission
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(2, 2, seed=1)
    d = np.array([[0.0, 0.0, 1.0]])
    out, rep = _solve(bem, ctx, ve, te, vi, ti, 2.0, 1.0, 1.0, d, gmres_tol=1e-10, precision=bem.BEM_PREC_MIXED)
    ref = solve_transmission(ve, te, vi, ti, 1.0, 2.0, 1.0, d[0], tol=1e-12)
    for key in ("v_ext", "w_ext", "v_int", "w_int"):
        e = rel(out[key][0], ref[key])
        print(key, e, rep)
        assert e < TRACE_TOL, (key, e)
    assert rep["converged"] == 1 and rep["outer_iterations"] >= 1


def test_mixed_solve_matches_fp64_gpu_at_level4(env):
    """Level-4 grids, k 10 / 15, density ratio 2 (the at-scale wavenumbers)."""
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(4, 4, seed=2)
    d = np.array([[0.0, 0.0, 1.0]])
    ref, r64 = _solve(bem, ctx, ve, te, vi, ti, 15.0, 10.0, 2.0, d, gmres_tol=1e-10)
    out, rmx = _solve(bem, ctx, ve, te, vi, ti, 15.0, 10.0, 2.0, d, gmres_tol=1e-10, precision=bem.BEM_PREC_MIXED)
    errs = {key: rel(out[key][0], ref[key][0]) for key in ("v_ext", "w_ext", "v_int", "w_int")}
    print(errs, r64, rmx)
    assert max(errs.values()) < TRACE_TOL, errs


def test_tensor_core_product_matches_cuda_core_product(env):
    """The tcgen05 product (TF32, three-term split, FP32 accumulation in 8 TMEM
    accumulators, summed at the end) against the compensated FP32 CUDA-core product on
    seeded random blocks, 24 columns (three groups of 8 on the CUDA cores) and 8
    columns.  The split drops terms below 2^-22 of each product; the tensor cores'
    FP32 accumulation is biased (one accumulator over K = 1200 gave 1.04e-5 here),
    eight shorter chains keep it near 1e-6."""
    bem, ctx = env
    for which in (1, 2):
        err = bem.bem_selftest(ctx, which)
        print("tensor-core vs CUDA-core product, rel. L2", which, err)
        assert err < 1e-5


def test_fp16_split_tensor_core_product_matches_cuda_core_product(env):
    """The TMA-fed tcgen05 product with the FP16 two-term split of both operands
    (powers of two per block row and per column keep the parts in FP16's range;
    Ah Bh + Ah Bl + Al Bh, FP32 accumulation in 2-8 TMEM accumulators, summed at the end)
    against the FP32 CUDA-core product on the same seeded blocks: 24 columns (four
    ring stages) and 128 columns (MMA N = 256, two stages).  The split keeps 22
    significant bits of each operand, as the TF32 three-term split does."""
    bem, ctx = env
    for which in (10, 11):
        err = bem.bem_selftest(ctx, which)
        print("FP16-split tensor-core vs CUDA-core product, rel. L2", which, err)
        assert err < 1e-5


def test_bf16_split_tensor_core_product_is_coarser(env):
    """The same kernel with a BF16 two-term split (8 + 8 significant bits per operand:
    each split entry within 2^-17 of its value, against FP16's 2^-23): on these seeded
    blocks the rounding errors of the 1200-term dot products average out to ~3e-7; the
    bound allows the per-entry level."""
    bem, ctx = env
    err = bem.bem_selftest(ctx, 12)
    print("BF16-split tensor-core vs CUDA-core product, rel. L2", err)
    assert 1e-7 < err < 1e-4


@pytest.mark.parametrize("tc", [1, 2, 3])
def test_tensor_core_batches_equal_cuda_core_batches(env, tc):
    """Twenty plane waves in one mixed-precision call, products on the tensor cores
    (one batch of 20; TF32 three-term split, FP16 or BF16 two-term split) or on the
    CUDA cores (groups of 8): all refine to the same complex64 system, so the traces
    agree within the mode's tolerance."""
    bem, ctx = env
    ve, te, vi, ti = bi.transmission_pair(2, 2, seed=12)
    dirs = bi.plane_wave_directions(20, seed=44)
    ge = bem.bem_grid_create(ctx, ve, te)
    gi = bem.bem_grid_create(ctx, vi, ti)
    try:
        a, ra = bem.bem_solve_transmission(ctx, ge, gi, 4.5, 3.0, 1.3, dirs,
                                           opts={"precision": bem.BEM_PREC_MIXED, "tensor_cores": tc})
        b, rb = bem.bem_solve_transmission(ctx, ge, gi, 4.5, 3.0, 1.3, dirs,
                                           opts={"precision": bem.BEM_PREC_MIXED, "tensor_cores": 0})
    finally:
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
    assert ra["converged"] == 1 and rb["converged"] == 1
    for key in ("v_ext", "w_ext", "v_int", "w_int"):
        assert rel(a[key], b[key]) < TRACE_TOL, key
