"""Pins for the oracle's gradient routes (CPU only)."""
import os

import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_batched_vqe_toy_gradient_golden():
    g = np.loadtxt(os.path.join(GOLDEN, "batched_vqe_toy.txt"), comments="#")
    b = W.OpBuilder(2)
    b.rx(0, 0)
    b.cnot(0, 1)
    b.rx(1, 1)
    circ = b.build()
    zz = W.pauli_sum(2, [(1.0, {0: 3, 1: 3})])
    for row in g:
        ps = G.parameter_shift(circ, row[:2], zz)
        fd = G.finite_difference(circ, row[:2], zz)
        np.testing.assert_allclose(ps, row[3:5], atol=1e-14)
        np.testing.assert_allclose(fd, row[3:5], atol=1e-9)


@pytest.mark.parametrize("seed", range(4))
def test_shift_equals_finite_difference(seed):
    rng = np.random.default_rng(100 + seed)
    kinds = [W.OP_H, W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_RZZ, W.OP_CNOT, W.OP_CZ, W.OP_U1, W.OP_U2]
    circ = W.random_circuit(5, 30, rng, n_params=6, kinds=kinds)
    th = rng.uniform(-3, 3, circ.n_params)
    ham = W.random_pauli_sum(5, 7, rng)
    ps = G.parameter_shift(circ, th, ham)
    fd = G.finite_difference(circ, th, ham)
    np.testing.assert_allclose(ps, fd, atol=2e-8)


def test_tfim_zero_angles_zero_gradient():
    n = 6
    circ = W.tfim_circuit(n, 3)
    ham = W.tfim_zz_x(n)
    g = G.parameter_shift(circ, np.zeros(6), ham)
    np.testing.assert_allclose(g, 0, atol=1e-13)


def test_tfim_one_layer_dE_dg():
    # E(g, b=0) = -[(n-2) cos^2 g + 2 cos g]  =>  dE/dg = (n-2) sin 2g + 2 sin g
    n = 7
    circ = W.tfim_circuit(n, 1)
    ham = W.tfim_zz_x(n)
    for gval in (0.2, 1.0, -1.9):
        g = G.parameter_shift(circ, [gval, 0.0], ham)
        assert abs(g[0] - ((n - 2) * np.sin(2 * gval) + 2 * np.sin(gval))) < 1e-12


def test_summed_batch_gradient_is_row_sum():
    # vectorized_value_and_grad with argnums != vectorized_argnums sums the
    # per-row gradients (Section "vmap and vectorized_value_and_grad").
    rng = np.random.default_rng(9)
    circ = W.tfim_circuit(4, 2)
    ham = W.tfim_zz_x(4)
    th = rng.normal(0, 0.3, (3, 4))
    rows = np.stack([G.parameter_shift(circ, t, ham) for t in th])
    # the summed gradient of sum_b E_b is the derivative of the summed energy
    h = 1e-6
    tot = lambda d: sum(G.energy_of(circ, t + d, ham) for t in th)
    for k in range(4):
        e = np.zeros(4)
        e[k] = h
        assert abs((tot(e) - tot(-e)) / (2 * h) - rows[:, k].sum()) < 1e-8


def _qgt_circuit(rng, n=4):
    b = W.OpBuilder(n)
    for q in range(n):
        b.ry(q, q)
    for q in range(n - 1):
        b.rzz(q, q + 1, n, scale=-2.0)  # one shared angle over the chain
    b.cnot(0, 2)
    for q in range(n):
        b.rx(q, n + 1 + q % 2, scale=0.5)
    b.rz(1, 0)  # theta_0 also drives a second gate
    return b.build()


def test_state_derivatives_match_finite_differences():
    rng = np.random.default_rng(77)
    circ = _qgt_circuit(rng)
    theta = rng.uniform(-2, 2, circ.n_params)
    d = G.state_derivatives(circ, theta)
    h = 1e-6
    for p in range(circ.n_params):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd = (sv.run_circuit(circ, tp) - sv.run_circuit(circ, tm)) / (2 * h)
        assert np.abs(d[p] - fd).max() < 1e-8


def test_qgt_bloch_sphere_closed_form():
    # RZ(b) RY(a) |0>: the Fubini-Study metric is diag(1/4, sin^2(a) / 4)
    b = W.OpBuilder(1)
    b.ry(0, 0)
    b.rz(0, 1)
    circ = b.build()
    for a, bb in [(0.3, -1.1), (1.9, 0.4), (np.pi / 2, 2.0)]:
        g = G.quantum_geometric_tensor(circ, [a, bb])
        assert np.allclose(g.real, [[0.25, 0.0], [0.0, np.sin(a) ** 2 / 4]], atol=1e-14)
        assert np.allclose(g, g.conj().T, atol=1e-14)


def test_qgt_global_phase_parameter_is_zero():
    # RZ on |0> only multiplies by a phase: <d psi|d psi> = |<psi|d psi>|^2
    b = W.OpBuilder(2)
    b.rz(0, 0)
    b.ry(1, 1)
    g = G.quantum_geometric_tensor(b.build(), [0.7, 0.2])
    assert np.abs(g[0]).max() < 1e-14 and np.abs(g[:, 0]).max() < 1e-14
    assert abs(g[1, 1] - 0.25) < 1e-14


def test_qgt_positive_semidefinite_and_hermitian():
    rng = np.random.default_rng(78)
    circ = _qgt_circuit(rng)
    g = G.quantum_geometric_tensor(circ, rng.uniform(-2, 2, circ.n_params))
    assert np.allclose(g, g.conj().T, atol=1e-13)
    assert np.linalg.eigvalsh(g).min() > -1e-12


def test_natural_gradient_bloch_closed_form():
    # 4 Re G = diag(1, sin^2 a) for RZ(b) RY(a)|0>: x_i = g_i / (qfi_ii + eps)
    b = W.OpBuilder(1)
    b.ry(0, 0)
    b.rz(0, 1)
    circ = b.build()
    a, eps = 0.8, 1e-3
    g = np.array([0.3, -0.7])
    x = G.natural_gradient(G.quantum_geometric_tensor(circ, [a, 0.4]), g, eps)
    assert np.allclose(x, [0.3 / (1 + eps), -0.7 / (np.sin(a) ** 2 + eps)], rtol=1e-12)
