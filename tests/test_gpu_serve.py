"""Serving on the GPU: requests of different sizes, wavenumbers, density ratios,
numbers of plane waves and precisions run concurrently on the server's streams or
together in lockstep groups, and every result equals the same request solved
alone (FP64: relative L2 <= 1e-10; mixed precision: <= 1e-6, the mode's stated
tolerance).  Timeouts and cancellation
of requests on the GPU return their status without disturbing the others."""
import time

import numpy as np
import pytest

import bem_inputs as bi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2206_00708_gb300 as b
    return b


def _requests():
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(10):
        le, li = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        axes = rng.uniform(0.7, 1.3, 3)
        ve, te, vi, ti = bi.transmission_pair(le, li, seed=100 + i, axes=axes)
        k_ext = float(rng.uniform(1.0, 4.0))
        k_int = k_ext * float(rng.uniform(1.2, 2.0))
        rho = float(np.exp(rng.uniform(np.log(0.2), np.log(5.0))))
        dirs = bi.plane_wave_directions(int(rng.integers(1, 4)), seed=200 + i)
        prec = i % 2  # alternate FP64 / mixed
        reqs.append((ve, te, vi, ti, k_ext, k_int, rho, dirs, prec))
    return reqs


def test_results_in_the_mix_equal_solo_results(bem):
    reqs = _requests()
    srv = bem.bem_serve_create(max_inflight=4)
    try:
        tickets = [bem.bem_serve_submit(srv, ve, te, vi, ti, ke, ki, rho, d, precision=p)
                   for (ve, te, vi, ti, ke, ki, rho, d, p) in reqs]
        served = []
        for t, r in zip(tickets, reqs):
            assert bem.bem_serve_wait(srv, t, 120000.0)
            out, info = bem.bem_serve_take(srv, t, len(r[7]), len(r[0]), len(r[2]))
            assert info["status"] == bem.BEM_OK, info
            served.append(out)
        st = bem.bem_serve_get_stats(srv)
        assert st["completed"] == len(reqs) and st["hbm_reserved_bytes"] == 0
    finally:
        bem.bem_serve_destroy(srv)
    ctx = bem.bem_context_create(0)
    try:
        for (ve, te, vi, ti, ke, ki, rho, d, p), out in zip(reqs, served):
            ge = bem.bem_grid_create(ctx, ve, te)
            gi = bem.bem_grid_create(ctx, vi, ti)
            solo, _ = bem.bem_solve_transmission(ctx, ge, gi, ki, ke, rho, d, opts={"precision": p})
            bem.bem_grid_destroy(ge)
            bem.bem_grid_destroy(gi)
            tol = 1e-10 if p == bem.BEM_PREC_FP64 else 1e-6
            for key in ("v_ext", "w_ext", "v_int", "w_int"):
                e = np.linalg.norm(out[key] - solo[key]) / np.linalg.norm(solo[key])
                assert e < tol, (p, key, e)
    finally:
        bem.bem_context_destroy(ctx)


def test_timeout_and_cancel_on_the_gpu(bem):
    ve, te, vi, ti = bi.transmission_pair(4, 4, seed=1)
    d = np.array([[0.0, 0.0, 1.0]])
    srv = bem.bem_serve_create(max_inflight=2)
    try:
        t_timeout = bem.bem_serve_submit(srv, ve, te, vi, ti, 10.0, 15.0, 2.0, d, precision=0, timeout_ms=5.0)
        t_cancel = bem.bem_serve_submit(srv, ve, te, vi, ti, 10.0, 15.0, 2.0, d, precision=0)
        t_ok = bem.bem_serve_submit(srv, *bi.transmission_pair(1, 1, seed=2), 1.0, 2.0, 1.0, d)
        bem.bem_serve_cancel(srv, t_cancel)
        for t in (t_timeout, t_cancel, t_ok):
            assert bem.bem_serve_wait(srv, t, 120000.0)
        assert bem.bem_serve_poll(srv, t_timeout)["status"] == bem.BEM_E_TIMEOUT
        assert bem.bem_serve_poll(srv, t_cancel)["status"] == bem.BEM_E_CANCELLED
        assert bem.bem_serve_poll(srv, t_ok)["status"] == bem.BEM_OK
    finally:
        bem.bem_serve_destroy(srv)


def test_lockstep_groups_equal_solo_results(bem):
    """Small mixed-precision requests queued behind a running FP64 request are taken
    as one lockstep group (different grids, wavenumbers, density ratios and numbers
    of waves); each member's traces equal its solo solve (1e-6), and a member whose
    deadline passed stops alone with BEM_E_TIMEOUT."""
    rng = np.random.default_rng(21)
    reqs = []
    for i in range(5):
        le, li = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        ve, te, vi, ti = bi.transmission_pair(le, li, seed=300 + i, axes=rng.uniform(0.6, 1.4, 3))
        k_ext = float(rng.uniform(1.0, 5.0))
        k_int = k_ext * float(rng.uniform(1.2, 2.0))
        rho = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
        dirs = bi.plane_wave_directions(int(rng.integers(1, 3)), seed=400 + i)
        reqs.append((ve, te, vi, ti, k_ext, k_int, rho, dirs))
    blocker = bi.transmission_pair(4, 4, seed=7)
    srv = bem.bem_serve_create(max_inflight=1)
    try:
        tb = bem.bem_serve_submit(srv, *blocker, 6.0, 9.0, 2.0, np.array([[0.0, 0.0, 1.0]]), precision=0)
        t0 = time.perf_counter()
        while bem.bem_serve_get_stats(srv)["running"] < 1:
            assert time.perf_counter() - t0 < 30.0
            time.sleep(0.001)
        tickets = [bem.bem_serve_submit(srv, ve, te, vi, ti, ke, ki, rho, d, precision=1)
                   for (ve, te, vi, ti, ke, ki, rho, d) in reqs]
        late = bem.bem_serve_submit(srv, *reqs[0][:4], 2.0, 3.0, 1.0, np.array([[1.0, 0.0, 0.0]]), precision=1,
                                    timeout_ms=1.0)
        served = []
        for t, r in zip(tickets, reqs):
            assert bem.bem_serve_wait(srv, t, 300000.0)
            out, info = bem.bem_serve_take(srv, t, len(r[7]), len(r[0]), len(r[2]))
            assert info["status"] == bem.BEM_OK, info
            assert info["group_size"] == len(reqs) + 1, info
            served.append(out)
        assert bem.bem_serve_wait(srv, late, 300000.0)
        info = bem.bem_serve_poll(srv, late)
        assert info["status"] == bem.BEM_E_TIMEOUT and info["group_size"] == len(reqs) + 1
        assert bem.bem_serve_wait(srv, tb, 300000.0)
        assert bem.bem_serve_poll(srv, tb)["status"] == bem.BEM_OK
        st = bem.bem_serve_get_stats(srv)
        assert st["groups"] == 1 and st["grouped"] == len(reqs) + 1 and st["hbm_reserved_bytes"] == 0
    finally:
        bem.bem_serve_destroy(srv)
    ctx = bem.bem_context_create(0)
    try:
        for (ve, te, vi, ti, ke, ki, rho, d), out in zip(reqs, served):
            ge = bem.bem_grid_create(ctx, ve, te)
            gi = bem.bem_grid_create(ctx, vi, ti)
            solo, _ = bem.bem_solve_transmission(ctx, ge, gi, ki, ke, rho, d, opts={"precision": 1})
            bem.bem_grid_destroy(ge)
            bem.bem_grid_destroy(gi)
            for key in ("v_ext", "w_ext", "v_int", "w_int"):
                e = np.linalg.norm(out[key] - solo[key]) / np.linalg.norm(solo[key])
                assert e < 1e-6, (key, e)
    finally:
        bem.bem_context_destroy(ctx)
