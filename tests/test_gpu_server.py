"""Serving loop on the GPU: results, alone-vs-mix identity, memory admission."""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import assert_energy_close, assert_grad_close

pytestmark = pytest.mark.gpu


def _requests(widths, seed):
    rng = np.random.default_rng(seed)
    out = []
    for n in widths:
        p = int(rng.integers(1, 4))
        edges = W.random_regular3(n, rng)
        out.append((W.qaoa_circuit(n, edges, p), rng.uniform(0, np.pi, 2 * p), W.zz_on_edges(n, edges)))
    return out


def test_results_match_oracle():
    s = nt.Server()
    reqs = _requests([8, 10, 12, 10, 8], seed=5)
    ids = [s.submit(*r) for r in reqs]
    for rid, (circ, th, ham) in zip(ids, reqs):
        r = s.wait(rid)
        assert r["status"] == nt.TC_OK, r["error"]
        e_ref = sv.energy(sv.run_circuit(circ, th), circ.n, ham)[0]
        assert_energy_close([r["energy"]], [e_ref])
        assert_grad_close(r["grad"], G.parameter_shift(circ, th, ham))
    s.close()


def test_each_result_same_alone_and_in_the_mix():
    reqs = _requests([8, 20, 12, 16, 10, 18, 14, 20, 8, 12], seed=6)
    s = nt.Server(max_inflight=8)
    alone = []
    for r in reqs:
        alone.append(s.wait(s.submit(*r)))
    ids = [s.submit(*r) for r in reqs]  # all in flight together
    mixed = [s.wait(i) for i in ids]
    assert s.stats()["peak_inflight"] > 1
    for a, m in zip(alone, mixed):
        assert a["status"] == m["status"] == nt.TC_OK
        assert a["energy"] == m["energy"] and np.array_equal(a["grad"], m["grad"])
    s.close()


def test_admission_respects_memory_budget():
    budget = 80 << 20  # ~4 twenty-qubit requests (two 8 MiB states each + plan)
    s = nt.Server(mem_budget_bytes=budget, max_inflight=16)
    reqs = _requests([20] * 10, seed=7)
    ids = [s.submit(*r) for r in reqs]
    res = [s.wait(i) for i in ids]
    assert all(r["status"] == nt.TC_OK for r in res)
    st = s.stats()
    assert 0 < st["peak_bytes"] <= budget
    assert st["peak_inflight"] <= 4
    s.close()


def test_request_larger_than_budget_fails_with_nomem():
    s = nt.Server(mem_budget_bytes=10 << 20)
    rid = s.submit(*_requests([20], seed=8)[0])
    r = s.wait(rid)
    assert r["status"] == nt.TC_E_NOMEM
    s.close()


def _wait_planned(s, n, limit_s=30.0):
    import time

    t0 = time.monotonic()
    while s.stats()["planned"] < n and time.monotonic() - t0 < limit_s:
        time.sleep(0.01)
    assert s.stats()["planned"] == n


def test_same_shape_requests_run_as_rows_of_one_group():
    """QAOA instances of one width and depth on different graphs share a plan
    shape (their packed column words differ): queued together they run as the
    rows of one launch sequence, bitwise equal to each request run alone, and
    requests of another shape queued in between form their own group."""
    rng = np.random.default_rng(11)
    reqs = []
    for k in range(12):
        n, p = (10, 2) if k % 2 == 0 else (12, 1)
        edges = W.random_regular3(n, rng)
        reqs.append((W.qaoa_circuit(n, edges, p), rng.uniform(0, np.pi, 2 * p), W.zz_on_edges(n, edges)))
    solo = nt.Server(max_group_rows=1)
    alone = [solo.wait(solo.submit(*r)) for r in reqs]
    assert solo.stats()["grouped_requests"] == 0
    solo.close()
    s = nt.Server(start_paused=True)
    ids = [s.submit(*r) for r in reqs]
    _wait_planned(s, len(ids))
    s.resume()
    got = [s.wait(i) for i in ids]
    st = s.stats()
    assert st["groups"] == 2 and st["grouped_requests"] == 12 and st["peak_inflight"] == 12
    for a, g in zip(alone, got):
        assert a["status"] == g["status"] == nt.TC_OK, g["error"]
        assert a["energy"] == g["energy"] and np.array_equal(a["grad"], g["grad"])
    for k in (0, 5, 10):
        circ, th, ham = reqs[k]
        assert_energy_close([got[k]["energy"]], [sv.energy(sv.run_circuit(circ, th), circ.n, ham)[0]])
        assert_grad_close(got[k]["grad"], G.parameter_shift(circ, th, ham))
    s.close()


def test_group_is_cut_to_the_memory_budget():
    rng = np.random.default_rng(12)
    edges = W.random_regular3(18, rng)
    reqs = [(W.qaoa_circuit(18, edges, 1), rng.uniform(0, np.pi, 2), W.zz_on_edges(18, edges)) for _ in range(8)]
    budget = 24 << 20  # room for about four rows of two 2 MiB states
    s = nt.Server(mem_budget_bytes=budget, start_paused=True)
    ids = [s.submit(*r) for r in reqs]
    _wait_planned(s, len(ids))
    s.resume()
    got = [s.wait(i) for i in ids]
    st = s.stats()
    assert all(g["status"] == nt.TC_OK for g in got)
    assert st["peak_bytes"] <= budget and st["groups"] >= 2
    circ, th, ham = reqs[7]
    assert_energy_close([got[7]["energy"]], [sv.energy(sv.run_circuit(circ, th), circ.n, ham)[0]])
    s.close()
