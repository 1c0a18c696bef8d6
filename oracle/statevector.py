"""Oracle: plain FP64 state-vector semantics (test infrastructure only).

Pinned by tests/test_oracle_statevector.py against closed forms (Bell/GHZ,
<Z> = cos(theta) after RX, product-state factorisation), the dense
X0X1 - Z0 - Z1 matrix printed in Section "Expectations of Hamiltonians via
operator_expectation", the batched-VQE toy of Section "Batched VQE", brute
force against dense Kronecker products, and the norm invariant.

Index convention (Section "Preliminaries"): qubit 0 is the leftmost register,
i.e. the most significant bit of the amplitude index, so the state of two
qubits is [a00, a01, a10, a11] (Section "Basic circuits and outputs").
"""
from __future__ import annotations

import numpy as np

from paper_2205_10091_b300 import workloads as W

I2 = np.eye(2, dtype=np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = [I2, PX, PY, PZ]  # structure codes 0..3 (Section "Pauli structures and weights")
HAD = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)


def rotation(G: np.ndarray, angle: float) -> np.ndarray:
    """exp(-i angle G / 2) for an involutory generator G (G^2 = I), written
    with the identity exp(i t G) = cos(t) I + i sin(t) G that Section
    "Circuits and gates" uses for its exponential gates.  Reading: RX, RY, RZ
    and RZZ are exp(-i theta G / 2)."""
    d = G.shape[0]
    return np.cos(angle / 2.0) * np.eye(d, dtype=np.complex128) - 1j * np.sin(angle / 2.0) * G


def gate_matrix(op, theta_row: np.ndarray, pool: np.ndarray, angle_shift: float = 0.0) -> np.ndarray:
    """Matrix of one op.  2x2 for one-qubit ops, 4x4 (row index 2*b(q0)+b(q1))
    for two-qubit ops.  ``angle_shift`` is added to the effective angle
    scale*theta[param] (used by the parameter-shift oracle)."""
    k = int(op["kind"])
    ang = 0.0
    if int(op["param"]) >= 0:
        ang = float(op["scale"]) * float(theta_row[int(op["param"])]) + angle_shift
    if k == W.OP_H:
        return HAD
    if k == W.OP_X:
        return PX
    if k == W.OP_RX:
        return rotation(PX, ang)
    if k == W.OP_RY:
        return rotation(PY, ang)
    if k == W.OP_RZ:
        return rotation(PZ, ang)
    if k == W.OP_RZZ:
        return rotation(np.kron(PZ, PZ), ang)
    if k == W.OP_CNOT:
        # first argument is the control (Section "Basic circuits and outputs")
        return np.block([[I2, np.zeros((2, 2))], [np.zeros((2, 2)), PX]]).astype(np.complex128)
    if k == W.OP_CZ:
        return np.diag([1, 1, 1, -1]).astype(np.complex128)
    if k == W.OP_U1:
        o = int(op["mat"])
        return pool[o:o + 4].reshape(2, 2).astype(np.complex128)
    if k == W.OP_U2:
        o = int(op["mat"])
        return pool[o:o + 16].reshape(4, 4).astype(np.complex128)
    raise ValueError(f"no matrix for op kind {k}")


def apply_1q(psi: np.ndarray, n: int, q: int, m: np.ndarray) -> np.ndarray:
    """Apply a 2x2 matrix to qubit q: the amplitude pairs that differ only in
    bit q (MSB order) are multiplied by m."""
    t = psi.reshape(2 ** q, 2, 2 ** (n - q - 1))
    out = np.einsum("ab,ibj->iaj", m, t)
    return out.reshape(-1)


def apply_2q(psi: np.ndarray, n: int, q0: int, q1: int, m: np.ndarray) -> np.ndarray:
    """Apply a 4x4 matrix (row index 2*b(q0)+b(q1)) to qubits q0, q1."""
    t = psi.reshape((2,) * n)
    m4 = m.reshape(2, 2, 2, 2)
    out = np.tensordot(m4, t, axes=([2, 3], [q0, q1]))  # new axes 0,1 = q0,q1
    out = np.moveaxis(out, [0, 1], [q0, q1])
    return np.ascontiguousarray(out).reshape(-1)


def initial_state(n: int, init: int) -> np.ndarray:
    """|0...0> (Section "Specifying the input state") or |+>^n = H^n|0...0>."""
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1.0
    if init == W.INIT_PLUS:
        for q in range(n):
            psi = apply_1q(psi, n, q, HAD)
    return psi


def noise_thresholds(px: float, py: float, pz: float):
    """Left ends of the intervals I_X, I_Y, I_Z of [0,1) for the Pauli channel
    with Kraus weights (1-px-py-pz, px, py, pz) in the order [I, X, Y, Z]
    (Section "Externalizing the randomness": contiguous intervals with
    lengths proportional to the outcome probabilities)."""
    t1 = 1.0 - (px + py + pz)
    t2 = t1 + px
    t3 = t2 + py
    return t1, t2, t3


def select_rotation(u: float, px: float, py: float) -> int:
    """Generator (1, 2, 3 = X, Y, Z) of a random-axis rotation: intervals
    [0, px), [px, px + py), [px + py, 1), left-closed as for noise outcomes."""
    if u < px:
        return 1
    if u < px + py:
        return 2
    return 3


def select_pauli(u: float, px: float, py: float, pz: float) -> int:
    """Outcome i (0..3 = I,X,Y,Z) of the interval containing u; intervals are
    left-closed."""
    t1, t2, t3 = noise_thresholds(px, py, pz)
    if u < t1:
        return 0
    if u < t2:
        return 1
    if u < t3:
        return 2
    return 3


def run_circuit(circ: W.Circuit, theta_row=None, status_row=None, init_state=None,
                shift_op: int = -1, shift: float = 0.0) -> np.ndarray:
    """|psi(theta)> = U_G ... U_1 |psi_0>, one gate at a time in list order.

    ``status_row[e]`` is the uniform number of the e-th noise op (Section
    "Externalizing the randomness"); the selected Pauli is applied after the
    preceding gate, in place of the channel.  ``shift_op``/``shift`` add an
    angle shift to one op occurrence (parameter-shift oracle)."""
    n = circ.n
    psi = initial_state(n, circ.init) if init_state is None else np.array(init_state, dtype=np.complex128)
    theta_row = np.zeros(max(circ.n_params, 1)) if theta_row is None else np.asarray(theta_row, np.float64)
    e = 0
    for idx, op in enumerate(circ.ops):
        k = int(op["kind"])
        if k == W.OP_PAULI_NOISE:
            u = float(status_row[e])
            e += 1
            i = select_pauli(u, float(op["px"]), float(op["py"]), float(op["pz"]))
            if i:
                psi = apply_1q(psi, n, int(op["q0"]), PAULI[i])
            continue
        if k == W.OP_RSEL:
            # Section "Demonstration of barren plateaus": unitary_kraus over
            # [RX, RY, RZ] picks the rotation whose interval contains u
            u = float(status_row[e])
            e += 1
            g = select_rotation(u, float(op["px"]), float(op["py"]))
            ang = float(op["scale"]) * float(theta_row[int(op["param"])]) if int(op["param"]) >= 0 else 0.0
            if idx == shift_op:
                ang += shift
            psi = apply_1q(psi, n, int(op["q0"]), rotation(PAULI[g], ang))
            continue
        m = gate_matrix(op, theta_row, circ.pool, shift if idx == shift_op else 0.0)
        if m.shape[0] == 2:
            psi = apply_1q(psi, n, int(op["q0"]), m)
        else:
            psi = apply_2q(psi, n, int(op["q0"]), int(op["q1"]), m)
    return psi


def apply_pauli_string(psi: np.ndarray, n: int, structure) -> np.ndarray:
    """P|psi> with P = sigma^{v_0} (x) ... (x) sigma^{v_{n-1}}, one
    single-qubit Pauli factor at a time."""
    out = psi
    for q in range(n):
        c = int(structure[q])
        if c:
            out = apply_1q(out, n, q, PAULI[c])
    return out


def expect_pauli_string(psi: np.ndarray, n: int, structure) -> complex:
    """<psi|P|psi> (complex; the imaginary part is ~0 for a Hermitian P)."""
    return complex(np.vdot(psi, apply_pauli_string(psi, n, structure)))


def energy(psi: np.ndarray, n: int, ham: W.PauliSum) -> tuple[float, float]:
    """E = sum_j w_j <psi|P_j|psi> by an explicit loop over terms (Section
    "Explicit loop with c.expectation_ps", Eq. H-pauli).  Returns (Re, Im)."""
    tot = 0j
    for j in range(ham.n_terms):
        tot += float(ham.weights[j]) * expect_pauli_string(psi, n, ham.structures[j])
    return tot.real, tot.imag


def apply_hamiltonian(psi: np.ndarray, n: int, ham: W.PauliSum) -> np.ndarray:
    """H|psi> = sum_j w_j P_j |psi>."""
    out = np.zeros_like(psi)
    for j in range(ham.n_terms):
        out += float(ham.weights[j]) * apply_pauli_string(psi, n, ham.structures[j])
    return out


def dense_pauli_sum(n: int, ham: W.PauliSum) -> np.ndarray:
    """Dense 2^n x 2^n matrix of sum_j w_j P_j by Kronecker products (qubit 0
    leftmost), as PauliStringSum2Dense does in Section "Expectations of
    Hamiltonians via operator_expectation"."""
    H = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    for j in range(ham.n_terms):
        m = np.array([[1.0 + 0j]])
        for q in range(n):
            m = np.kron(m, PAULI[int(ham.structures[j][q])])
        H += float(ham.weights[j]) * m
    return H


def energies(circ: W.Circuit, theta: np.ndarray, ham: W.PauliSum) -> np.ndarray:
    """E_b for every row of a parameter batch (vmap semantics, Section
    "vmap and vectorized_value_and_grad")."""
    return np.array([energy(run_circuit(circ, theta[b]), circ.n, ham)[0] for b in range(theta.shape[0])])
