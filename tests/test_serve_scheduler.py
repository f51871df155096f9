"""Host-side tests of the request server (bem_serve_*) in dry-run mode: no GPU
work, each request "runs" for a service time proportional to its unknowns.  They
cover admission by memory budget, FIFO order without starvation, latency
accounting, timeouts, cancellation, poll semantics and concurrent submission."""
import threading
import time

import numpy as np
import pytest

import bem_inputs as bi


@pytest.fixture(scope="module")
def bem():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2206_00708_gb300 as b
    return b


def _req(bem, srv, level=1, n_rhs=1, timeout_ms=0.0):
    ve, te, vi, ti = bi.transmission_pair(level, level, seed=3)
    dirs = bi.plane_wave_directions(n_rhs, seed=5)
    return bem.bem_serve_submit(srv, ve, te, vi, ti, 2.0, 3.0, 1.5, dirs, timeout_ms=timeout_ms)


def test_all_requests_complete_in_fifo_order_with_latency_accounting(bem):
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=2, dry_run_us_per_unknown=60.0)
    try:
        tickets = [_req(bem, srv) for _ in range(6)]
        infos = []
        for t in tickets:
            assert bem.bem_serve_wait(srv, t, 10000.0)
            infos.append(bem.bem_serve_poll(srv, t))
        assert all(i["status"] == bem.BEM_OK for i in infos)
        # two slots: the later requests waited in the queue, and finished in order
        assert infos[-1]["queue_ms"] > infos[0]["queue_ms"]
        for i in infos:
            assert i["total_ms"] >= i["run_ms"] >= 168 * 60e-3 * 0.9
            assert abs(i["total_ms"] - i["queue_ms"] - i["run_ms"]) < 1.0
        st = bem.bem_serve_get_stats(srv)
        assert st["submitted"] == 6 and st["completed"] == 6 and st["running"] == 0 and st["queued"] == 0
        assert st["hbm_reserved_bytes"] == 0 and st["hbm_high_water_bytes"] > 0
    finally:
        bem.bem_serve_destroy(srv)


def test_requests_that_never_fit_are_refused(bem):
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 20, max_inflight=1)
    try:
        with pytest.raises(bem.BemError) as e:
            _req(bem, srv)
        assert e.value.status == bem.BEM_E_ADMISSION_REFUSED
        assert bem.bem_serve_get_stats(srv)["refused"] == 1
    finally:
        bem.bem_serve_destroy(srv)


def test_memory_budget_limits_concurrency(bem):
    probe = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=0.0)
    t = _req(bem, probe)
    bem.bem_serve_wait(probe, t, 10000.0)
    need = bem.bem_serve_poll(probe, t)["bytes_reserved"]
    bem.bem_serve_destroy(probe)
    # four slots, but memory for only one request at a time
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=int(1.5 * need), max_inflight=4,
                               dry_run_us_per_unknown=100.0)
    try:
        t0 = time.perf_counter()
        tickets = [_req(bem, srv) for _ in range(4)]
        for t in tickets:
            assert bem.bem_serve_wait(srv, t, 20000.0)
        wall = time.perf_counter() - t0
        infos = [bem.bem_serve_poll(srv, t) for t in tickets]
        st = bem.bem_serve_get_stats(srv)
        assert st["hbm_high_water_bytes"] <= int(1.5 * need)
        assert wall >= 0.9 * sum(i["run_ms"] for i in infos) / 1e3  # serialised by memory
    finally:
        bem.bem_serve_destroy(srv)


def test_timeout_and_cancellation(bem):
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=2000.0)
    try:
        slow = _req(bem, srv)                      # ~0.34 s of service
        queued = _req(bem, srv)
        timed = _req(bem, srv, timeout_ms=50.0)    # expires while queued
        time.sleep(0.05)
        assert bem.bem_serve_poll(srv, slow) is None  # still running: busy
        bem.bem_serve_cancel(srv, queued)
        i = bem.bem_serve_poll(srv, queued)
        assert i["status"] == bem.BEM_E_CANCELLED and i["run_ms"] == 0.0
        bem.bem_serve_cancel(srv, slow)             # running: stops at its next check
        assert bem.bem_serve_wait(srv, slow, 5000.0)
        assert bem.bem_serve_poll(srv, slow)["status"] == bem.BEM_E_CANCELLED
        assert bem.bem_serve_wait(srv, timed, 5000.0)
        assert bem.bem_serve_poll(srv, timed)["status"] == bem.BEM_E_TIMEOUT
        with pytest.raises(bem.BemError) as e:      # released tickets are gone
            bem.bem_serve_poll(srv, timed)
        assert e.value.status == bem.BEM_E_INVALID_ARG
        st = bem.bem_serve_get_stats(srv)
        assert st["cancelled"] == 2 and st["timed_out"] == 1
    finally:
        bem.bem_serve_destroy(srv)


def test_concurrent_submission_from_threads(bem):
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=3, dry_run_us_per_unknown=5.0)
    tickets, lock = [], threading.Lock()

    def client():
        for _ in range(5):
            t = _req(bem, srv)
            with lock:
                tickets.append(t)

    try:
        th = [threading.Thread(target=client) for _ in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        assert len(set(tickets)) == 20
        for t in tickets:
            assert bem.bem_serve_wait(srv, t, 20000.0)
            assert bem.bem_serve_poll(srv, t)["status"] == bem.BEM_OK
    finally:
        bem.bem_serve_destroy(srv)


def test_destroy_with_pending_requests_returns(bem):
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=5000.0)
    for _ in range(3):
        _req(bem, srv)
    t0 = time.perf_counter()
    bem.bem_serve_destroy(srv)
    assert time.perf_counter() - t0 < 5.0


def test_invalid_requests(bem):
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40)
    try:
        ve, te, vi, ti = bi.transmission_pair(1, 1, seed=1)
        with pytest.raises(bem.BemError) as e:
            bem.bem_serve_submit(srv, ve, te, vi, ti, 1.0, 2.0, -1.0, [[0, 0, 1.0]])
        assert e.value.status == bem.BEM_E_INVALID_ARG
        with pytest.raises(bem.BemError):
            bem.bem_serve_poll(srv, 12345)
    finally:
        bem.bem_serve_destroy(srv)
