"""Scheduling of the continuous-batching server in dry-run mode (no GPU).

In dry-run mode a request holds its solve slot for the service time it is given and no
CUDA call is made, so admission by memory budget, the slot limit, FIFO order, the LRU
cache of finished instances and the warm-start bookkeeping can be checked on the CPU.
"""
import time

import pytest

from paper_2312_11801_gb300 import build as B
from paper_2312_11801_gb300 import instances as I


@pytest.fixture(scope="module")
def U():
    B.build()
    from paper_2312_11801_gb300 import usbs
    usbs.load()
    return usbs


@pytest.fixture(scope="module")
def prob():
    return I.maxcut_er(40, 4, seed=3)


def _need(U, p, r=0):
    nnzC = int(p.C_rowptr[-1])
    return U.usbs_instance_bytes(p.n, nnzC, p.m, len(p.A_con), r, U.PRECISION_MIXED)


def _server(U, **kw):
    kw.setdefault("dry_run", 1)
    solver = kw.pop("solver", {})
    solver.setdefault("r", 0)
    return U.usbs_server_create(solver=solver, **kw)


def _drain(U, srv, count, timeout=20.0):
    out, t0 = [], time.time()
    while len(out) < count and time.time() - t0 < timeout:
        out += U.usbs_server_poll(srv, 64, wait_ms=50)
    assert len(out) == count, out
    return out


def test_instance_bytes_grows_with_size(U):
    small = U.usbs_instance_bytes(1000, 6000, 1000, 1000, 0, U.PRECISION_MIXED)
    big = U.usbs_instance_bytes(10000, 60000, 10000, 10000, 0, U.PRECISION_MIXED)
    fp64 = U.usbs_instance_bytes(1000, 6000, 1000, 1000, 0, U.PRECISION_FP64)
    sk = U.usbs_instance_bytes(1000, 6000, 1000, 1000, 16, U.PRECISION_MIXED)
    assert 0 < small < big and small < fp64 and small < sk
    # the Lanczos basis alone (n x 8 x (3 + 2 x 9) FP32 values) is a lower bound
    assert small >= 1000 * 8 * 21 * 4
    assert U.usbs_instance_bytes(0, 0, 1, 1, 0, U.PRECISION_MIXED) == 0


def test_create_rejects_bad_parameters(U):
    for kw in ({"max_slots": 0}, {"max_slots": 1000}, {"cache_entries": -1}):
        with pytest.raises(U.USBSError) as ei:
            _server(U, **kw)
        assert ei.value.code == U.USBS_EINVAL


def test_slot_limit_and_concurrency(U, prob):
    with _server(U, max_slots=3) as srv:
        t0 = time.time()
        for i in range(6):
            U.usbs_server_submit(srv, i, prob, fake_service_s=0.2)
        done = _drain(U, srv, 6)
        wall = time.time() - t0
        st = U.usbs_server_get_stats(srv)
    assert st["peak_running"] == 3 and st["finished"] == 6 and st["rejected"] == 0
    assert all(c["status"] == U.USBS_OK for c in done)
    assert {c["slot"] for c in done} <= {0, 1, 2}
    # two waves of three 0.2 s requests
    assert 0.35 < wall < 2.0


def test_fifo_order_with_one_slot(U, prob):
    with _server(U, max_slots=1) as srv:
        for i in range(5):
            U.usbs_server_submit(srv, 100 + i, prob, fake_service_s=0.02)
        done = _drain(U, srv, 5)
    assert [c["request_id"] for c in done] == [100, 101, 102, 103, 104]
    admits = [c["t_admit"] for c in done]
    assert admits == sorted(admits)
    for c in done:
        assert c["t_arrival"] <= c["t_admit"] <= c["t_finish"]


def test_memory_budget_limits_admission(U, prob):
    need = _need(U, prob)
    with _server(U, max_slots=8, cache_entries=0, hbm_budget_bytes=int(2.5 * need)) as srv:
        for i in range(6):
            U.usbs_server_submit(srv, i, prob, fake_service_s=0.1)
        done = _drain(U, srv, 6)
        st = U.usbs_server_get_stats(srv)
    assert st["peak_running"] == 2
    assert st["peak_bytes"] <= st["budget_bytes"] == int(2.5 * need)
    assert st["used_bytes"] == 0 and st["cached"] == 0
    assert all(c["bytes"] == need and c["status"] == U.USBS_OK for c in done)


def test_oversize_request_is_rejected_and_others_run(U, prob):
    big = I.maxcut_er(20000, 4, seed=4)
    need_small = _need(U, prob)
    assert _need(U, big) > 2 * need_small
    with _server(U, max_slots=4, hbm_budget_bytes=2 * need_small) as srv:
        U.usbs_server_submit(srv, 1, prob, fake_service_s=0.05)
        U.usbs_server_submit(srv, 2, big, fake_service_s=0.05)
        U.usbs_server_submit(srv, 3, prob, fake_service_s=0.05)
        done = {c["request_id"]: c for c in _drain(U, srv, 3)}
        st = U.usbs_server_get_stats(srv)
    assert done[2]["status"] == U.USBS_EBUSY
    assert done[1]["status"] == done[3]["status"] == U.USBS_OK
    assert st["rejected"] == 1 and st["finished"] == 2


def test_warm_start_from_cached_parent(U, prob):
    with _server(U, max_slots=2, cache_entries=4) as srv:
        U.usbs_server_submit(srv, 1, prob, fake_service_s=0.01)
        first = _drain(U, srv, 1)[0]
        U.usbs_server_submit(srv, 2, prob, parent_id=1, fake_service_s=0.01)
        U.usbs_server_submit(srv, 3, prob, parent_id=99, fake_service_s=0.01)
        done = {c["request_id"]: c for c in _drain(U, srv, 2)}
        st = U.usbs_server_get_stats(srv)
    assert first["warm"] == 0
    assert done[2]["warm"] == 1 and done[3]["warm"] == 0
    # 1 (returned after the grow), 2 and 3 are resident
    assert st["cached"] == 3 and st["used_bytes"] == 3 * _need(U, prob)


def test_lru_eviction_by_entry_count(U, prob):
    with _server(U, max_slots=1, cache_entries=2) as srv:
        for i in range(3):
            U.usbs_server_submit(srv, i, prob, fake_service_s=0.01)
        _drain(U, srv, 3)
        # 0 is the least recently finished and was evicted; 2 is resident
        U.usbs_server_submit(srv, 10, prob, parent_id=0, fake_service_s=0.01)
        U.usbs_server_submit(srv, 11, prob, parent_id=2, fake_service_s=0.01)
        done = {c["request_id"]: c for c in _drain(U, srv, 2)}
        st = U.usbs_server_get_stats(srv)
    assert done[10]["warm"] == 0 and done[11]["warm"] == 1
    assert st["cached"] == 2 and st["used_bytes"] == 2 * _need(U, prob)


def test_cache_is_evicted_for_memory(U, prob):
    need = _need(U, prob)
    with _server(U, max_slots=1, cache_entries=8, hbm_budget_bytes=3 * need) as srv:
        for i in range(5):
            U.usbs_server_submit(srv, i, prob, fake_service_s=0.01)
        done = _drain(U, srv, 5)
        st = U.usbs_server_get_stats(srv)
    assert all(c["status"] == U.USBS_OK for c in done)
    assert st["cached"] == 3 and st["peak_bytes"] <= 3 * need


def test_parent_dropped_when_parent_and_child_do_not_fit(U, prob):
    # budget for one instance only: the cached parent cannot stay resident beside the
    # grown child, so the child starts cold instead of waiting for ever
    need = _need(U, prob)
    with _server(U, max_slots=2, cache_entries=4, hbm_budget_bytes=int(1.5 * need)) as srv:
        U.usbs_server_submit(srv, 1, prob, fake_service_s=0.01)
        _drain(U, srv, 1)
        U.usbs_server_submit(srv, 2, prob, parent_id=1, fake_service_s=0.01)
        c = _drain(U, srv, 1)[0]
        st = U.usbs_server_get_stats(srv)
    assert c["request_id"] == 2 and c["status"] == U.USBS_OK and c["warm"] == 0
    assert st["cached"] == 1 and st["used_bytes"] == need


def test_destroy_finishes_queued_work(U, prob):
    srv = _server(U, max_slots=2)
    for i in range(4):
        U.usbs_server_submit(srv, i, prob, fake_service_s=0.05)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 >= 0.08
