"""The tiled operator product (symmetry-packed V and D, K applied as K and K^T, the
dense blocks of eq. mtf:discrete) against an FP64 product with dense copies of the
same seeded random operators, through bem_selftest: two grids of 300 and 170
vertices (ragged last tiles), coefficients other than +-1, 1 to 8 columns.

Tolerances: FP32 products on complex64 (the inputs rounded to complex64 on both
sides): 1e-6 (sums of up to ~300 FP32 products per row and column, then partial sums
added in double-float); double-float products (complex64 or complex128 operators):
1e-13 (each entry split into 24 + 24 bits, exact two-products, two-sums)."""
import pytest

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


@pytest.mark.parametrize("which,tol", [(4, 1e-6), (5, 1e-6), (6, 1e-13), (7, 1e-13), (8, 1e-13), (9, 1e-13)])
def test_tile_product_matches_fp64_dense_product(env, which, tol):
    bem, ctx = env
    err = bem.bem_selftest(ctx, which)
    print("tile product self-test", which, "rel. L2", err)
    assert err < tol
