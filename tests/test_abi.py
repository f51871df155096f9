"""The C ABI library builds, loads and exports every entry point declared in
include/bem.h (CPU only: no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    return sorted(set(re.findall(r"^BEM_API\s+[\w\s\*]+?\b(bem_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def bem():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2206_00708_gb300 as b
    return b


def test_header_declares_the_boundary_calls():
    names = _declared()
    for required in ("bem_grid_create", "bem_assemble", "bem_projection", "bem_solve_transmission",
                     "bem_mass", "bem_context_create", "bem_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(bem):
    lib = bem.library()
    for name in _declared():
        assert hasattr(lib, name), name
    # the binding types every declared call
    from paper_2206_00708_gb300 import _SIGNATURES
    assert set(_declared()) <= set(_SIGNATURES)


def test_library_hides_internal_symbols(bem):
    out = os.popen(f"nm -D --defined-only {bem.library_path()}").read()
    exported = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert exported and all(n.startswith("bem_") for n in exported), exported


def test_host_side_errors_without_gpu(bem):
    assert "sm_103a" in bem.bem_version()
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    with pytest.raises(bem.BemError) as ei:
        bem.bem_context_create(0)
    assert ei.value.status in (bem.BEM_E_CUDA, bem.BEM_E_INVALID_ARG)
    assert isinstance(bem.library().bem_last_error(), bytes)


def test_noalloc_wrapper_rejects_unsuitable_outputs_before_calling(bem):
    """bem_projection_noalloc writes with device stores into the caller's arrays: the
    binding must refuse host tensors, wrong dtypes and strided views before the call."""
    import ctypes
    import torch
    fake_ctx = ctypes.c_void_p(0x1000)
    i32 = torch.zeros(16, dtype=torch.int32)
    f64 = torch.zeros(16, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        bem.bem_projection_noalloc(fake_ctx, None, None, i32, i32, f64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        bem.bem_projection_noalloc(fake_ctx, None, None, i32.numpy(), i32, f64)


def test_solve_option_defaults(bem):
    """Defaults of bem_solve_opts that the solver's refinement depends on: FP32 inner
    products throughout (dd_switch 1), the inner tolerance 0 selecting its per-solve
    rule (1e-5 there, 1e-8 with a double-float phase), tensor cores on the FP16 split."""
    o = bem.bem_solve_opts_default()
    assert o.ir_inner_tol == 0.0
    assert o.tensor_cores == 2
    assert o.dd_switch == 1.0
    assert o.gmres_tol == pytest.approx(1e-8)
