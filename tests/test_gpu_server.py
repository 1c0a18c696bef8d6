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
