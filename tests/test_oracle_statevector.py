"""Pins for the FP64 oracle's state-vector semantics (CPU only)."""
import itertools
import os

import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def test_bell_state_order():
    # Section "Basic circuits and outputs": h(0), cnot(0,1); state() lists
    # [a00, a01, a10, a11] with qubit 0 leftmost.
    b = W.OpBuilder(2)
    b.h(0)
    b.cnot(0, 1)
    psi = sv.run_circuit(b.build())
    r = 1 / np.sqrt(2)
    np.testing.assert_allclose(psi, [r, 0, 0, r], atol=1e-15)


def test_qubit_zero_is_msb():
    b = W.OpBuilder(3)
    b.x(0)
    psi = sv.run_circuit(b.build())
    assert abs(psi[0b100] - 1) < 1e-15
    b = W.OpBuilder(3)
    b.x(2)
    psi = sv.run_circuit(b.build())
    assert abs(psi[0b001] - 1) < 1e-15


def test_cnot_control_is_first_argument():
    b = W.OpBuilder(2)
    b.x(1)
    b.cnot(0, 1)  # control 0 is |0>: nothing happens
    assert abs(sv.run_circuit(b.build())[0b01] - 1) < 1e-15
    b = W.OpBuilder(2)
    b.x(1)
    b.cnot(1, 0)  # control 1 is |1>: flips qubit 0
    assert abs(sv.run_circuit(b.build())[0b11] - 1) < 1e-15


@pytest.mark.parametrize("n", [3, 5])
def test_ghz(n):
    b = W.OpBuilder(n)
    b.h(0)
    for i in range(n - 1):
        b.cnot(i, i + 1)
    psi = sv.run_circuit(b.build())
    expect = np.zeros(2 ** n)
    expect[0] = expect[-1] = 1 / np.sqrt(2)
    np.testing.assert_allclose(psi, expect, atol=1e-15)


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.7, -2.5, np.pi])
def test_rotation_closed_forms(theta):
    z = W.pauli_sum(1, [(1.0, {0: 3})])
    x = W.pauli_sum(1, [(1.0, {0: 1})])
    y = W.pauli_sum(1, [(1.0, {0: 2})])
    b = W.OpBuilder(1)
    b.rx(0, 0)
    psi = sv.run_circuit(b.build(), [theta])
    assert abs(sv.energy(psi, 1, z)[0] - np.cos(theta)) < 1e-14
    assert abs(sv.energy(psi, 1, y)[0] + np.sin(theta)) < 1e-14
    b = W.OpBuilder(1)
    b.ry(0, 0)
    psi = sv.run_circuit(b.build(), [theta])
    assert abs(sv.energy(psi, 1, x)[0] - np.sin(theta)) < 1e-14
    assert abs(sv.energy(psi, 1, z)[0] - np.cos(theta)) < 1e-14
    b = W.OpBuilder(1, W.INIT_PLUS)
    b.rz(0, 0)
    psi = sv.run_circuit(b.build(), [theta])
    assert abs(sv.energy(psi, 1, x)[0] - np.cos(theta)) < 1e-14
    assert abs(sv.energy(psi, 1, y)[0] - np.sin(theta)) < 1e-14


def test_rzz_exp1_convention():
    # exp1 with unitary Z(x)Z is exp(i t ZZ) (Section "Circuits and gates");
    # RZZ with scale -2 must equal it: cos(t) I + i sin(t) ZZ.
    t = 0.37
    b = W.OpBuilder(2, W.INIT_PLUS)
    b.rzz(0, 1, 0, scale=-2.0)
    psi = sv.run_circuit(b.build(), [t])
    zz = np.array([1, -1, -1, 1])
    np.testing.assert_allclose(psi, 0.5 * np.exp(1j * t * zz), atol=1e-15)


def test_product_state_factorises():
    rng = np.random.default_rng(0)
    b = W.OpBuilder(4)
    for q in range(4):
        b.ry(q, q)
        b.rz(q, 4 + q)
    th = rng.uniform(-3, 3, 8)
    psi = sv.run_circuit(b.build(), th)
    for i, j in itertools.combinations(range(4), 2):
        zi = sv.energy(psi, 4, W.pauli_sum(4, [(1.0, {i: 3})]))[0]
        zj = sv.energy(psi, 4, W.pauli_sum(4, [(1.0, {j: 3})]))[0]
        zz = sv.energy(psi, 4, W.pauli_sum(4, [(1.0, {i: 3, j: 3})]))[0]
        assert abs(zz - zi * zj) < 1e-14


def test_dense_matrix_golden():
    H = sv.dense_pauli_sum(2, W.pauli_sum(2, [(1.0, {0: 1, 1: 1}), (-1.0, {1: 3}), (-1.0, {0: 3})]))
    np.testing.assert_array_equal(H.real, _load("dense_x0x1_z0_z1.txt"))
    assert np.all(H.imag == 0)


def _full_matrix(n, op, theta, pool):
    """Independent 2^n x 2^n matrix of one op by element-wise definition."""
    m = sv.gate_matrix(op, theta, pool)
    d = 2 ** n
    M = np.zeros((d, d), dtype=np.complex128)
    q0 = int(op["q0"])
    q1 = int(op["q1"])
    bit = lambda x, q: (x >> (n - 1 - q)) & 1
    for xo in range(d):
        for xi in range(d):
            if m.shape[0] == 2:
                if (xo ^ xi) & ~(1 << (n - 1 - q0)):
                    continue
                M[xo, xi] = m[bit(xo, q0), bit(xi, q0)]
            else:
                mask = (1 << (n - 1 - q0)) | (1 << (n - 1 - q1))
                if (xo ^ xi) & ~mask:
                    continue
                M[xo, xi] = m[2 * bit(xo, q0) + bit(xo, q1), 2 * bit(xi, q0) + bit(xi, q1)]
    return M


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_unitary(seed):
    rng = np.random.default_rng(seed)
    n = 4
    circ = W.random_circuit(n, 25, rng)
    th = rng.uniform(-3, 3, circ.n_params)
    U = np.eye(2 ** n, dtype=np.complex128)
    for op in circ.ops:
        U = _full_matrix(n, op, th, circ.pool) @ U
    psi = sv.run_circuit(circ, th)
    np.testing.assert_allclose(psi, U[:, 0], atol=1e-13)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13


def test_pauli_strings_all_against_kron():
    # every Pauli string on 3 qubits, including the Y phase convention
    rng = np.random.default_rng(5)
    n = 3
    psi = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    psi /= np.linalg.norm(psi)
    for s in itertools.product(range(4), repeat=n):
        P = np.array([[1.0 + 0j]])
        for c in s:
            P = np.kron(P, sv.PAULI[c])
        ref = np.vdot(psi, P @ psi)
        got = sv.expect_pauli_string(psi, n, s)
        assert abs(ref - got) < 1e-14


def test_y_phase_explicit():
    # Y|0> = i|1>, Y|1> = -i|0>
    np.testing.assert_allclose(sv.apply_pauli_string(np.array([1, 0], complex), 1, [2]), [0, 1j])
    np.testing.assert_allclose(sv.apply_pauli_string(np.array([0, 1], complex), 1, [2]), [-1j, 0])


def _inverse_circuit(circ):
    b = W.OpBuilder(circ.n, W.INIT_ZERO)
    for op in reversed(circ.ops):
        k, q0, q1, p, s = int(op["kind"]), int(op["q0"]), int(op["q1"]), int(op["param"]), float(op["scale"])
        if k == W.OP_H:
            b.h(q0)
        elif k == W.OP_X:
            b.x(q0)
        elif k == W.OP_RX:
            b.rx(q0, p, -s)
        elif k == W.OP_RY:
            b.ry(q0, p, -s)
        elif k == W.OP_RZ:
            b.rz(q0, p, -s)
        elif k == W.OP_RZZ:
            b.rzz(q0, q1, p, -s)
        elif k == W.OP_CNOT:
            b.cnot(q0, q1)
        elif k == W.OP_CZ:
            b.cz(q0, q1)
        elif k == W.OP_U1:
            o = int(op["mat"])
            b.unitary1(q0, circ.pool[o:o + 4].reshape(2, 2).conj().T)
        elif k == W.OP_U2:
            o = int(op["mat"])
            b.unitary2(q0, q1, circ.pool[o:o + 16].reshape(4, 4).conj().T)
    return b.build(circ.n_params)


def test_apply_then_inverse():
    rng = np.random.default_rng(11)
    circ = W.random_circuit(6, 60, rng)
    th = rng.uniform(-3, 3, circ.n_params)
    psi = sv.run_circuit(circ, th)
    back = sv.run_circuit(_inverse_circuit(circ), th, init_state=psi)
    e0 = np.zeros(64)
    e0[0] = 1
    np.testing.assert_allclose(back, e0, atol=1e-13)


def test_batched_vqe_toy_golden():
    g = _load("batched_vqe_toy.txt")
    b = W.OpBuilder(2)
    b.rx(0, 0)
    b.cnot(0, 1)
    b.rx(1, 1)
    circ = b.build()
    zz = W.pauli_sum(2, [(1.0, {0: 3, 1: 3})])
    for row in g:
        e = sv.energy(sv.run_circuit(circ, row[:2]), 2, zz)[0]
        assert abs(e - row[2]) < 1e-15


@pytest.mark.parametrize("n", [4, 6, 9])
def test_tfim_closed_forms(n):
    circ = W.tfim_circuit(n, 3)
    ham = W.tfim_zz_x(n)
    # zero angles: |+>^n is an X eigenstate, <ZZ> = 0 -> E = -n
    assert abs(sv.energy(sv.run_circuit(circ, np.zeros(6)), n, ham)[0] + n) < 1e-12
    # g = 0, any b: RX only adds a phase on |+>^n
    th = np.array([0.0, 0.7, 0.0, -1.1, 0.0, 2.0])
    assert abs(sv.energy(sv.run_circuit(circ, th), n, ham)[0] + n) < 1e-12
    # one layer, b = 0: E = -[(n-2) cos^2 g + 2 cos g]
    one = W.tfim_circuit(n, 1)
    for g in (0.3, 1.2, -2.2):
        e = sv.energy(sv.run_circuit(one, [g, 0.0]), n, ham)[0]
        assert abs(e + (n - 2) * np.cos(g) ** 2 + 2 * np.cos(g)) < 1e-12


def test_qaoa_p1_cube_closed_form():
    # p = 1 QAOA on a triangle-free 3-regular graph (the 3-cube): with
    # RZZ(gamma) = exp(-i gamma ZZ/2), RX(beta) = exp(-i beta X/2),
    # <Z_u Z_v> = sin(2 beta) sin(gamma) cos^2(gamma) per edge (the p = 1
    # formula of Wang, Hadfield, Jiang, Rieffel, PRA 97, 022304, mapped to
    # these conventions).
    edges = [(a, b) for a in range(8) for b in range(a + 1, 8) if bin(a ^ b).count("1") == 1]
    assert len(edges) == 12
    circ = W.qaoa_circuit(8, edges, 1)
    ham = W.zz_on_edges(8, edges)
    for gam, bet in ((0.4, 0.3), (1.1, -0.7), (2.5, 1.3)):
        e = sv.energy(sv.run_circuit(circ, [gam, bet]), 8, ham)[0]
        assert abs(e - 12 * np.sin(2 * bet) * np.sin(gam) * np.cos(gam) ** 2) < 1e-12


def test_norm_preserved_large():
    rng = np.random.default_rng(3)
    circ = W.random_circuit(12, 80, rng)
    psi = sv.run_circuit(circ, rng.uniform(-3, 3, circ.n_params))
    assert abs(np.linalg.norm(psi) - 1) < 1e-13


@pytest.mark.parametrize("n", [3, 6])
def test_ghz_type_state_closed_forms(n):
    """RY(theta) on qubit 0 and a CNOT chain give cos(theta/2)|0..0> +
    sin(theta/2)|1..1>: <X^(x)n> = sin(theta), <Y Y X..X> = -sin(theta),
    <Z_0> = cos(theta), <Z_0 Z_{n-1}> = 1 (the closed forms of the 30-qubit GPU
    test), and their parameter-shift derivatives."""
    b = W.OpBuilder(n, W.INIT_ZERO)
    b.ry(0, 0)
    for q in range(n - 1):
        b.cnot(q, q + 1)
    circ = b.build(1)
    ystr = {0: 2, 1: 2}
    ystr.update({q: 1 for q in range(2, n)})
    terms = [{q: 1 for q in range(n)}, {0: 3}, {0: 3, n - 1: 3}, ystr]
    for theta in (0.37, 2.9, -1.3):
        psi = sv.run_circuit(circ, [theta])
        assert abs(psi[0] - np.cos(theta / 2)) < 1e-14 and abs(psi[-1] - np.sin(theta / 2)) < 1e-14
        vals = [sv.energy(psi, n, W.pauli_sum(n, [(1.0, t)]))[0] for t in terms]
        assert np.allclose(vals, [np.sin(theta), np.cos(theta), 1.0, -np.sin(theta)], atol=1e-14)
        ders = [G.parameter_shift(circ, [theta], W.pauli_sum(n, [(1.0, t)]))[0] for t in terms]
        assert np.allclose(ders, [np.cos(theta), -np.sin(theta), 0.0, -np.cos(theta)], atol=1e-13)
