"""Host-side tests of the request server (bem_serve_*) in dry-run mode: no GPU
work, each request "runs" for a service time proportional to its unknowns and
waves (a lockstep group for its longest member's).  They cover admission by memory
budget, FIFO order without starvation, latency accounting, timeouts, cancellation,
poll semantics, concurrent submission and the forming of lockstep groups."""
import functools
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


@functools.lru_cache(maxsize=None)
def _pair(level):
    return bi.transmission_pair(level, level, seed=3)


def _req(bem, srv, level=1, n_rhs=1, timeout_ms=0.0, precision=-1):
    ve, te, vi, ti = _pair(level)   # cached: submissions follow one another closely
    dirs = bi.plane_wave_directions(n_rhs, seed=5)
    return bem.bem_serve_submit(srv, ve, te, vi, ti, 2.0, 3.0, 1.5, dirs, timeout_ms=timeout_ms,
                                precision=precision)


def _wait_running(bem, srv, n=1, limit_s=5.0):
    t0 = time.perf_counter()
    while bem.bem_serve_get_stats(srv)["running"] < n:
        assert time.perf_counter() - t0 < limit_s
        time.sleep(0.002)


def _finish(bem, srv, tickets):
    out = []
    for t in tickets:
        assert bem.bem_serve_wait(srv, t, 20000.0)
        out.append(bem.bem_serve_poll(srv, t))
    return out


def test_all_requests_complete_in_fifo_order_with_latency_accounting(bem):
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=2, dry_run_us_per_unknown=60.0, group_max=1)
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
                               dry_run_us_per_unknown=100.0, group_max=1)
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
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=2000.0, group_max=1)
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


# ---------------------------------------------------------------- lockstep groups
# A level-1 pair has 2 * (42 + 42) = 168 unknowns; an FP64 request is never grouped,
# so it serves as a blocker behind which the small mixed-precision requests queue.

def test_queued_small_mixed_requests_run_as_one_lockstep_group(bem):
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=300.0)
    try:
        blocker = _req(bem, srv, precision=0)
        _wait_running(bem, srv)
        ts = [_req(bem, srv, n_rhs=1 + i % 2) for i in range(5)]
        infos = _finish(bem, srv, [blocker] + ts)
        assert all(i["status"] == bem.BEM_OK for i in infos)
        assert infos[0]["group_size"] == 1
        members = infos[1:]
        assert all(i["group_size"] == 5 and i["group_waves"] == 1 + 2 + 1 + 2 + 1 for i in members)
        # one group: started together, finished together, for its longest member's time
        runs = [i["run_ms"] for i in members]
        assert max(runs) - min(runs) < 2.0 and min(runs) >= 0.9 * 168 * 2 * 300e-3
        st = bem.bem_serve_get_stats(srv)
        assert st["groups"] == 1 and st["grouped"] == 5 and st["completed"] == 6
        assert st["hbm_reserved_bytes"] == 0
    finally:
        bem.bem_serve_destroy(srv)


def test_groups_pass_over_requests_that_cannot_join_without_starving_them(bem):
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=200.0)
    try:
        blocker = _req(bem, srv, precision=0)
        _wait_running(bem, srv)
        a, b = _req(bem, srv), _req(bem, srv)
        c = _req(bem, srv, precision=0)          # FP64: passed over, next for the slot
        d = _req(bem, srv)
        e = _req(bem, srv, precision=0)
        ia, ib, ic, idd, ie = _finish(bem, srv, [a, b, c, d, e])
        assert ia["group_size"] == ib["group_size"] == idd["group_size"] == 3
        assert ic["group_size"] == 1 and ie["group_size"] == 1
        # c ran right after the group of a, b, d, and e after c
        assert ic["queue_ms"] >= ia["queue_ms"] + 0.8 * ia["run_ms"]
        assert ie["queue_ms"] >= ic["queue_ms"] + 0.8 * ic["run_ms"]
        bem.bem_serve_wait(srv, blocker, 5000.0)
    finally:
        bem.bem_serve_destroy(srv)


def test_passed_over_requests_keep_their_room_in_the_budget(bem):
    probe = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=0.0)
    t = _req(bem, probe, precision=0)
    bem.bem_serve_wait(probe, t, 10000.0)
    need64 = bem.bem_serve_poll(probe, t)["bytes_reserved"]
    t = _req(bem, probe)
    bem.bem_serve_wait(probe, t, 10000.0)
    need = bem.bem_serve_poll(probe, t)["bytes_reserved"]
    bem.bem_serve_destroy(probe)
    # room for the FP64 request plus two mixed ones: the group takes a and b, passes
    # over c (FP64) and keeps its room, so d does not fit in the group
    budget = need64 + 2 * need + need // 2
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=budget, max_inflight=1, dry_run_us_per_unknown=200.0)
    try:
        blocker = _req(bem, srv, precision=0)
        _wait_running(bem, srv)
        a, b = _req(bem, srv), _req(bem, srv)
        c = _req(bem, srv, precision=0)
        d = _req(bem, srv)
        infos = _finish(bem, srv, [a, b, c, d])
        assert [i["group_size"] for i in infos] == [2, 2, 1, 1]
        assert all(i["status"] == bem.BEM_OK for i in infos)
        bem.bem_serve_wait(srv, blocker, 5000.0)
    finally:
        bem.bem_serve_destroy(srv)


def test_group_limits_requests_waves_and_operator_size(bem):
    # group_max = 2: five queued requests run as groups of 2, 2, 1
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=100.0,
                               group_max=2)
    try:
        blocker = _req(bem, srv, precision=0)
        _wait_running(bem, srv)
        infos = _finish(bem, srv, [_req(bem, srv) for _ in range(5)])
        assert [i["group_size"] for i in infos] == [2, 2, 2, 2, 1]
        bem.bem_serve_wait(srv, blocker, 5000.0)
    finally:
        bem.bem_serve_destroy(srv)
    # requests of more than two waves run alone; group_max = 1: every request alone
    for kw, waves, expect in (({}, (3, 3, 1), [1, 1, 1]), ({"group_max": 1}, (1, 1), [1, 1])):
        srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=10.0,
                                   **kw)
        try:
            blocker = _req(bem, srv, precision=0, n_rhs=100)   # ~0.17 s
            _wait_running(bem, srv)
            infos = _finish(bem, srv, [_req(bem, srv, n_rhs=w) for w in waves])
            assert [i["group_size"] for i in infos] == expect
            assert bem.bem_serve_get_stats(srv)["groups"] == 0
            bem.bem_serve_wait(srv, blocker, 5000.0)
        finally:
            bem.bem_serve_destroy(srv)
    # at most 64 waves per group: 40 two-wave requests with group_max 64 make groups of 32
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=2.0,
                               group_max=64)
    try:
        blocker = _req(bem, srv, precision=0, n_rhs=500)   # ~0.17 s
        _wait_running(bem, srv)
        infos = _finish(bem, srv, [_req(bem, srv, n_rhs=2) for _ in range(40)])
        assert [i["group_size"] for i in infos] == [32] * 32 + [8] * 8
        assert all(i["group_waves"] <= 64 for i in infos)
        bem.bem_serve_wait(srv, blocker, 5000.0)
    finally:
        bem.bem_serve_destroy(srv)
    # level-4 grids: 2 x 3403 complex64 tiles = 223 MB of operators, above the group limit
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 42, max_inflight=1, dry_run_us_per_unknown=2.0)
    try:
        blocker = _req(bem, srv, precision=0, n_rhs=500)   # ~0.17 s
        _wait_running(bem, srv)
        infos = _finish(bem, srv, [_req(bem, srv, level=4) for _ in range(2)])
        assert [i["group_size"] for i in infos] == [1, 1]
        bem.bem_serve_wait(srv, blocker, 5000.0)
    finally:
        bem.bem_serve_destroy(srv)


def test_group_respects_the_memory_budget(bem):
    probe = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=0.0)
    t = _req(bem, probe)
    bem.bem_serve_wait(probe, t, 10000.0)
    need = bem.bem_serve_poll(probe, t)["bytes_reserved"]
    bem.bem_serve_destroy(probe)
    # memory for two small requests at a time: groups of two
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=int(2.5 * need), max_inflight=1,
                               dry_run_us_per_unknown=100.0)
    try:
        first = _req(bem, srv)
        _wait_running(bem, srv)
        infos = _finish(bem, srv, [_req(bem, srv) for _ in range(4)])
        assert [i["group_size"] for i in infos] == [2, 2, 2, 2]
        st = bem.bem_serve_get_stats(srv)
        assert st["hbm_high_water_bytes"] <= int(2.5 * need)
        bem.bem_serve_wait(srv, first, 5000.0)
    finally:
        bem.bem_serve_destroy(srv)


def test_cancel_and_timeout_stop_one_member_of_a_group(bem):
    srv = bem.bem_serve_create(dry_run=1, hbm_budget_bytes=1 << 40, max_inflight=1, dry_run_us_per_unknown=4000.0)
    try:
        blocker = _req(bem, srv, precision=0, n_rhs=1)   # cancelled at once; the group then runs ~0.67 s
        _wait_running(bem, srv)
        a = _req(bem, srv)
        b = _req(bem, srv)
        c = _req(bem, srv, timeout_ms=300.0)
        bem.bem_serve_cancel(srv, blocker)
        _wait_running(bem, srv, 3)                 # the group of a, b, c is running
        bem.bem_serve_cancel(srv, b)
        ia, ib, ic = _finish(bem, srv, [a, b, c])
        assert ia["group_size"] == ib["group_size"] == ic["group_size"] == 3
        assert ia["status"] == bem.BEM_OK
        assert ib["status"] == bem.BEM_E_CANCELLED
        assert ic["status"] == bem.BEM_E_TIMEOUT
        st = bem.bem_serve_get_stats(srv)
        assert st["cancelled"] == 2 and st["timed_out"] == 1 and st["completed"] == 1
    finally:
        bem.bem_serve_destroy(srv)
