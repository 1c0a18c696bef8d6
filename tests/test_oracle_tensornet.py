"""Pins for the oracle's tensor-network routes (CPU only)."""
import numpy as np
import pytest

from oracle import statevector as sv
from oracle import tensornet as T
from paper_2205_10091_b300 import workloads as W


def _sv_value(n, gates, obs):
    b = W.OpBuilder(n)
    for (q0, q1, u) in gates:
        b.unitary2(q0, q1, u)
    psi = sv.run_circuit(b.build())
    return sv.energy(psi, n, W.pauli_sum(n, [(1.0, {q: 3 for q in obs})]))[0]


@pytest.mark.parametrize("seed", range(3))
def test_network_equals_statevector_two_paths(seed):
    rng = np.random.default_rng(seed)
    n = 6
    gates = W.brickwork_u4(n, 4, rng)
    obs = (2, 3)
    ref = _sv_value(n, gates, obs)
    net = T.network_expectation(n, gates, obs)
    v1 = T.contract(net, T.greedy_path(net))
    v2 = T.contract(list(reversed(net)), T.greedy_path(list(reversed(net))))
    assert abs(v1 - ref) < 1e-12 and abs(v2 - ref) < 1e-12
    assert abs(v1.imag) < 1e-12


def test_cone_equals_window_and_full():
    # exactly unitary (unrounded) gates: out-of-cone gates cancel to rounding
    rng = np.random.default_rng(31)
    n = 14
    gates = W.brickwork_u4(n, 4, rng, round_c64=False)
    obs = (6, 7)
    cone = T.cone_statevector_expectation(gates, obs)
    win = T.window_statevector_expectation(gates, obs, 1, 12)
    full = _sv_value(n, gates, obs)
    assert abs(cone - full) < 1e-12 and abs(win - full) < 1e-12


def test_brickwork_cone_shape_200_depth8():
    n, gates, obs = W.brick200_workload()
    cone = T.light_cone(gates, obs)
    qs = sorted({q for g in cone for q in g[:2]})
    assert len(cone) == 36
    assert qs[0] == 92 and qs[-1] == 107 and len(qs) == 16


@pytest.mark.parametrize("n,d", [(12, 3), (14, 4)])
def test_circuit_window_equals_full_statevector(n, d):
    # the contraction testbed (Section "Custom contraction settings") small
    # enough to simulate whole: the window n//2 -+ (d + 1) gives the exact
    # value; a window narrower than the string's support does not
    circ = W.example_block_circuit(n, d)
    rng = np.random.default_rng(40 + n)
    theta = rng.uniform(-2, 2, circ.n_params)
    c = n // 2
    psi = sv.run_circuit(circ, theta)
    for pauli in ({c: 3}, {c: 1, c + 1: 2}):
        full = complex(*sv.energy(psi, n, W.pauli_sum(n, [(1.0, pauli)])))
        win = T.circuit_window_expectation(circ, theta, pauli, c - d - 1, c + d + 1)
        assert abs(win - full) < 1e-12
        narrow = T.circuit_window_expectation(circ, theta, pauli, c - 1, c + 2)
        assert abs(narrow - full) > 1e-6


def test_circuit_window_of_whole_register_is_the_statevector():
    rng = np.random.default_rng(5)
    b = W.OpBuilder(5, W.INIT_PLUS)
    for q in range(5):
        b.ry(q, q)
    b.cnot(0, 3)
    b.unitary2(1, 4, W.haar_unitary(4, rng))
    b.cz(2, 4)
    circ = b.build()
    theta = rng.uniform(-3, 3, circ.n_params)
    pauli = {0: 2, 3: 1, 4: 3}
    full = complex(*sv.energy(sv.run_circuit(circ, theta), 5, W.pauli_sum(5, [(1.0, pauli)])))
    assert abs(T.circuit_window_expectation(circ, theta, pauli, 0, 4) - full) < 1e-13
