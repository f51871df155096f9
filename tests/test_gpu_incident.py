"""Incident-field kinds of bem_incident through the C ABI: point sources and the
caller's own weak-form data (Sec. 2: the data f, g of eq. mtf:discrete), against the
FP64 oracle (relative L2 <= 1e-10 in FP64, <= 1e-6 in mixed precision) and against
the plane-wave path."""
import numpy as np
import pytest

import bem_inputs as bi

pytestmark = pytest.mark.gpu

TOL = 1e-10
TOL_MIXED = 1e-6
SOURCES = np.array([[0.3, -0.4, 2.2], [-1.9, 0.5, 0.8]])  # outside the ellipsoid
AMPS = np.array([1.0, 0.4 - 0.7j])


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2206_00708_gb300 as bem
    ctx = bem.bem_context_create(0)
    yield bem, ctx, torch
    bem.bem_context_destroy(ctx)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def problem():
    from oracle.mtf import mtf_blocks, point_source_data
    ve, te, vi, ti = bi.transmission_pair(2, 2, seed=7, axes=[1.2, 0.9, 1.05])
    k_ext, k_int, rho = 2.0 + 0.1j, 3.1, 1.8
    B = mtf_blocks(ve, te, vi, ti, k_ext, k_int)
    data = [tuple(a * x for x in point_source_data(ve, te, k_ext, s)) for s, a in zip(SOURCES, AMPS)]
    return dict(ve=ve, te=te, vi=vi, ti=ti, k_ext=k_ext, k_int=k_int, rho=rho, B=B, data=data)


def _oracle(p, r):
    from oracle.mtf import solve_transmission
    return solve_transmission(p["ve"], p["te"], p["vi"], p["ti"], p["k_ext"], p["k_int"], p["rho"], None,
                              tol=1e-12, blocks=p["B"], data=p["data"][r])


@pytest.mark.parametrize("precision", [0, 1])
def test_point_sources_match_oracle(env, problem, precision):
    bem, ctx, _ = env
    p = problem
    ge, gi = bem.bem_grid_create(ctx, p["ve"], p["te"]), bem.bem_grid_create(ctx, p["vi"], p["ti"])
    out, rep = bem.bem_solve_transmission(ctx, ge, gi, p["k_int"], p["k_ext"], p["rho"], sources=SOURCES, amps=AMPS,
                                          opts={"gmres_tol": 1e-12, "precision": precision})
    tol = TOL if precision == 0 else TOL_MIXED
    for r in range(len(SOURCES)):
        ref = _oracle(p, r)
        for key in ("v_ext", "w_ext", "v_int", "w_int"):
            assert rel(out[key][r], ref[key]) < tol, (precision, r, key, rel(out[key][r], ref[key]))
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)


def test_point_source_iteration_count_matches_oracle(env, problem):
    from oracle.mtf import solve_transmission
    bem, ctx, _ = env
    p = problem
    ge, gi = bem.bem_grid_create(ctx, p["ve"], p["te"]), bem.bem_grid_create(ctx, p["vi"], p["ti"])
    _, rep = bem.bem_solve_transmission(ctx, ge, gi, p["k_int"], p["k_ext"], p["rho"], sources=SOURCES[:1],
                                        opts={"gmres_tol": 1e-8})
    ref = solve_transmission(p["ve"], p["te"], p["vi"], p["ti"], p["k_ext"], p["k_int"], p["rho"], None, tol=1e-8,
                             blocks=p["B"], data=tuple(x / AMPS[0] for x in p["data"][0]))
    assert abs(rep["iterations"] - ref["iters"]) <= 1
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)


@pytest.mark.parametrize("on_device", [False, True])
def test_user_traces_equal_the_plane_wave_solve(env, on_device):
    """The oracle's plane-wave data passed as BEM_INC_USER_TRACES give the plane-wave
    solution, from host arrays and from device tensors."""
    from oracle.mtf import plane_wave_data
    bem, ctx, torch = env
    ve, te, vi, ti = bi.transmission_pair(2, 1, seed=8)
    dirs = bi.plane_wave_directions(3, seed=9)
    k_ext, k_int, rho = 1.7, 2.6, 0.6
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    opts = {"gmres_tol": 1e-12}
    ref, _ = bem.bem_solve_transmission(ctx, ge, gi, k_int, k_ext, rho, dirs, opts=opts)
    f = np.stack([plane_wave_data(ve, te, k_ext, d)[0] for d in dirs])
    g = np.stack([plane_wave_data(ve, te, k_ext, d)[1] for d in dirs])
    if on_device:
        f, g = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
        out = {k: torch.zeros((3, n), dtype=torch.complex128, device="cuda") for k, n in
               (("v_ext", len(ve)), ("w_ext", len(ve)), ("v_int", len(vi)), ("w_int", len(vi)))}
        bem.bem_solve_transmission(ctx, ge, gi, k_int, k_ext, rho, traces=(f, g), opts=opts, out=out, on_device=True)
        out = {k: v.cpu().numpy() for k, v in out.items()}
    else:
        out, _ = bem.bem_solve_transmission(ctx, ge, gi, k_int, k_ext, rho, traces=(f, g), opts=opts)
    for key in ref:
        assert rel(out[key], ref[key]) < 1e-11, key
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)


@pytest.mark.parametrize("name,form", [("pmchwt_ext", 1), ("pmchwt_int", 3)])
def test_point_source_data_drive_the_single_trace_formulations(env, problem, name, form):
    """Given data drive the other formulations too: the exterior and interior PMCHWT
    (whose data are mapped to the interior grid) with point-source data as
    BEM_INC_USER_TRACES equal the oracle's solves for the same data."""
    from oracle.pmchwt import solve_single_trace
    bem, ctx, _ = env
    p = problem
    assert form == {"pmchwt_ext": bem.BEM_FORM_PMCHWT, "pmchwt_int": bem.BEM_FORM_PMCHWT_INT}[name]
    ge, gi = bem.bem_grid_create(ctx, p["ve"], p["te"]), bem.bem_grid_create(ctx, p["vi"], p["ti"])
    f, g = p["data"][1]
    out, _ = bem.bem_solve_transmission(ctx, ge, gi, p["k_int"], p["k_ext"], p["rho"], traces=(f[None], g[None]),
                                        opts={"gmres_tol": 1e-12, "formulation": form})
    ref = solve_single_trace(p["ve"], p["te"], p["vi"], p["ti"], p["k_ext"], p["k_int"], p["rho"], None, name,
                             tol=1e-12, blocks=p["B"], data=(f, g))
    for key in ("v_ext", "w_ext", "v_int", "w_int"):
        assert rel(out[key][0], ref[key]) < TOL, key
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)


def test_screen_point_source_equals_its_data(env):
    """On an open surface: the screen solve with a point source equals the screen solve
    with the oracle's point-source g given as data."""
    from oracle.mtf import point_source_data
    bem, ctx, _ = env
    v, t = bi.screen_grid(9, 8, jitter=0.2, seed=3)
    src = np.array([[0.2, 0.1, 1.5]])
    k = 4.0
    gs = bem.bem_grid_create(ctx, v, t)
    a, _ = bem.bem_solve_screen(ctx, gs, k, sources=src, opts={"gmres_tol": 1e-12})
    _, g = point_source_data(v, t, k, src[0])
    b, _ = bem.bem_solve_screen(ctx, gs, k, traces=(None, g[None]), opts={"gmres_tol": 1e-12})
    assert rel(a, b) < 1e-9
    bem.bem_grid_destroy(gs)


def test_invalid_incident_fields_are_rejected(env):
    bem, ctx, _ = env
    ve, te, vi, ti = bi.transmission_pair(1, 1, seed=1)
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    with pytest.raises(bem.BemError) as e:
        bem.bem_solve_transmission(ctx, ge, gi, 2.0, 1.0, 1.0, sources=np.array([[np.nan, 0.0, 3.0]]))
    assert e.value.status == bem.BEM_E_INVALID_ARG
    with pytest.raises(ValueError):
        bem.bem_solve_transmission(ctx, ge, gi, 2.0, 1.0, 1.0, traces=(None, None))
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)
