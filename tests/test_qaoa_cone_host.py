"""The QAOA edge light cones used by the 26-qubit parity test: on circuits
small enough for the full FP64 state vector, the sum of the edge terms
evaluated on their cones equals the full oracle energy, and the sum of their
parameter-shift gradients equals the full gradient (QAOA MaxCut, Sec. 5)."""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import workloads as W

from qaoa_cone import edge_cone


@pytest.mark.parametrize("n,p,max_cone", [(10, 1, 6), (12, 2, 14)])
def test_edge_cones_sum_to_the_full_oracle(n, p, max_cone):
    rng = np.random.default_rng(5 + n)
    edges = W.random_regular3(n, rng)
    circ = W.qaoa_circuit(n, edges, p)
    ham = W.zz_on_edges(n, edges)
    theta = rng.uniform(0.0, np.pi, size=2 * p)
    cones = [edge_cone(circ, u, v) for (u, v) in edges]
    assert max(cc.n for cc, _ in cones) <= max_cone
    # p = 1: the two endpoints and their neighbours only
    if p == 1:
        for (u, v), (cc, _) in zip(edges, cones):
            nb = {a for e in edges if u in e or v in e for a in e}
            assert cc.n == len(nb)
    e_cones = sum(sv.energy(sv.run_circuit(cc, theta), cc.n, hh)[0] for cc, hh in cones)
    g_cones = sum(G.parameter_shift(cc, theta, hh) for cc, hh in cones)
    assert abs(e_cones - sv.energy(sv.run_circuit(circ, theta), n, ham)[0]) <= 1e-12
    assert np.abs(g_cones - G.parameter_shift(circ, theta, ham)).max() <= 1e-12
