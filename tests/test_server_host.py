"""Serving loop: host-side queue logic with a paused server (no GPU used)."""
import time

import numpy as np
import pytest

from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W


def _qaoa(n=8, p=2, seed=0):
    rng = np.random.default_rng(seed)
    edges = W.random_regular3(n, rng)
    return W.qaoa_circuit(n, edges, p), rng.uniform(0, np.pi, 2 * p), W.zz_on_edges(n, edges)


def test_malformed_request_refused_at_submit():
    s = nt.Server(start_paused=True)
    circ, th, ham = _qaoa()
    ops = circ.ops.copy()
    ops[0]["q1"] = 99
    circ.ops = ops
    with pytest.raises(nt.TcError) as e:
        s.submit(circ, th, ham)
    assert e.value.status == nt.TC_E_INVALID
    bad = W.PauliSum(np.full((1, 8), 7, np.uint8), np.ones(1))
    with pytest.raises(nt.TcError):
        s.submit(_qaoa()[0], th, bad)
    s.close()


def test_pending_then_cancel():
    s = nt.Server(start_paused=True)
    circ, th, ham = _qaoa()
    a = s.submit(circ, th, ham)
    b = s.submit(circ, th, ham)
    assert s.poll(a) is None and s.poll(b) is None
    s.cancel(b)
    r = s.poll(b)
    assert r["status"] == nt.TC_E_CANCELLED
    with pytest.raises(nt.TcError):
        s.poll(b)  # id released
    st = s.stats()
    assert st["submitted"] == 2 and st["cancelled"] == 1 and st["pending"] == 1
    s.close()


def test_queue_limit_returns_busy():
    s = nt.Server(start_paused=True, max_queue=2)
    circ, th, ham = _qaoa()
    s.submit(circ, th, ham)
    s.submit(circ, th, ham)
    with pytest.raises(nt.TcError) as e:
        s.submit(circ, th, ham)
    assert e.value.status == nt.TC_E_BUSY
    assert s.stats()["rejected"] == 1
    s.close()


def test_queued_request_times_out():
    s = nt.Server(start_paused=True, timeout_ms=30)
    circ, th, ham = _qaoa()
    a = s.submit(circ, th, ham)
    t0 = time.monotonic()
    r = None
    while r is None and time.monotonic() - t0 < 5:
        time.sleep(0.01)
        r = s.poll(a)
    assert r is not None and r["status"] == nt.TC_E_TIMEOUT
    s.close()


def test_destroy_with_pending_requests_does_not_hang():
    s = nt.Server(start_paused=True)
    circ, th, ham = _qaoa()
    for _ in range(5):
        s.submit(circ, th, ham)
    t0 = time.monotonic()
    s.close()
    assert time.monotonic() - t0 < 5


def test_requests_are_planned_while_paused():
    """Planner threads compile queued plans on the host before admission."""
    s = nt.Server(start_paused=True, planner_threads=3)
    ids = [s.submit(*_qaoa(n=8 + 2 * (i % 4), p=1 + i % 3, seed=i)) for i in range(12)]
    t0 = time.monotonic()
    while s.stats()["planned"] < len(ids) and time.monotonic() - t0 < 10:
        time.sleep(0.01)
    st = s.stats()
    assert st["planned"] == st["pending"] == len(ids)
    assert st["groups"] == 0 and st["inflight"] == 0
    s.cancel(ids[3])
    assert s.stats()["planned"] == len(ids) - 1
    s.close()


def test_bad_pauli_sum_fails_in_planning_not_at_submit():
    """A Pauli sum that passes tc_submit's checks but not the planner's (a
    non-finite weight) completes with TC_E_INVALID once admitted; while the
    server is paused it stays pending, planned as failed."""
    s = nt.Server(start_paused=True)
    circ, th, ham = _qaoa()
    w = ham.weights.copy()
    w[0] = np.nan
    rid = s.submit(circ, th, W.PauliSum(ham.structures, w))
    time.sleep(0.2)
    st = s.stats()
    assert st["pending"] == 1 and st["planned"] == 0
    assert s.poll(rid) is None
    s.close()
