"""Oracle: gradients of E(theta) = <psi(theta)|H|psi(theta)> (test infrastructure only).

The engine computes gradients with an adjoint sweep; the oracle deliberately
uses two other routes so that neither can hide a mistake in the other:

* parameter shift per gate occurrence: for a gate exp(-i a G/2) with G^2 = I
  and a = s*theta_k, dE/da = [E(a + pi/2) - E(a - pi/2)] / 2 exactly, and
  dE/dtheta_k sums s * dE/da over every occurrence of theta_k (shared angles
  such as one g_l over a whole RZZ layer);
* central finite differences with step h in FP64;
* state derivatives by the product rule (generator inserted after each gate
  occurrence) and the quantum geometric tensor built from them.

Pinned by tests/test_oracle_gradients.py: the batched-VQE toy of Section
"Batched VQE" (closed form cos(w1), gradient (0, -sin w1)), the vvag toy of
Section "vmap and vectorized_value_and_grad" (summed-over-batch gradient),
agreement of the two routes, and TFIM closed forms (zero gradient at zero
angles); the state derivatives against central differences of the state,
and the geometric tensor against closed forms (one qubit RY then RZ: the
Bloch-sphere metric diag(1/4, sin^2(a)/4); a global-phase parameter gives a
zero row).  Batch semantics (Section "vmap and vectorized_value_and_grad"):
with argnums == vectorized_argnums each row gets its own gradient; the
summed variant is the sum over rows.
"""
from __future__ import annotations

import numpy as np

from paper_2205_10091_b300 import workloads as W
from . import statevector as sv


def energy_of(circ: W.Circuit, theta_row, ham: W.PauliSum, shift_op: int = -1, shift: float = 0.0,
              status_row=None) -> float:
    psi = sv.run_circuit(circ, theta_row, status_row=status_row, shift_op=shift_op, shift=shift)
    return sv.energy(psi, circ.n, ham)[0]


def parameter_shift(circ: W.Circuit, theta_row, ham: W.PauliSum, status_row=None) -> np.ndarray:
    """dE/dtheta for one parameter row by the two-term shift rule per gate
    occurrence (valid for the RX, RY, RZ, RZZ family and for random-axis
    rotations, whose generators square to the identity).  ``status_row``:
    the row's event numbers (noise outcomes and rotation axes)."""
    g = np.zeros(circ.n_params)
    for idx, op in enumerate(circ.ops):
        p = int(op["param"])
        if p < 0 or int(op["kind"]) == W.OP_PAULI_NOISE:
            continue
        assert int(op["kind"]) in (W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_RZZ, W.OP_RSEL)
        s = float(op["scale"])
        ep = energy_of(circ, theta_row, ham, idx, +np.pi / 2, status_row)
        em = energy_of(circ, theta_row, ham, idx, -np.pi / 2, status_row)
        g[p] += s * (ep - em) / 2.0
    return g


def finite_difference(circ: W.Circuit, theta_row, ham: W.PauliSum, h: float = 1e-5,
                      params=None) -> np.ndarray:
    """Central differences [E(theta + h e_k) - E(theta - h e_k)] / 2h."""
    theta_row = np.asarray(theta_row, dtype=np.float64)
    ks = range(circ.n_params) if params is None else params
    g = np.full(circ.n_params, np.nan)
    for k in ks:
        tp = theta_row.copy()
        tp[k] += h
        tm = theta_row.copy()
        tm[k] -= h
        g[k] = (energy_of(circ, tp, ham) - energy_of(circ, tm, ham)) / (2.0 * h)
    return g


_GENERATOR = {W.OP_RX: 1, W.OP_RY: 2, W.OP_RZ: 3}  # Pauli code of G in exp(-i a G / 2)


def state_derivatives(circ: W.Circuit, theta_row) -> np.ndarray:
    """[n_params][2^n]: d|psi>/d theta_p by the product rule, one gate
    occurrence at a time: for an occurrence exp(-i a G / 2), a = s theta_p,
    the term is U_after (-i s / 2) G U_upto |psi_0>, the generator applied
    right after the gate (the two commute).  RZZ has G = Z (x) Z."""
    n = circ.n
    theta_row = np.asarray(theta_row, np.float64)
    out = np.zeros((circ.n_params, 2 ** n), np.complex128)
    for idx, op in enumerate(circ.ops):
        p = int(op["param"])
        if p < 0:
            continue
        k = int(op["kind"])
        assert k in (W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_RZZ), "state derivatives need RX/RY/RZ/RZZ gates"
        head = W.Circuit(n, circ.ops[:idx + 1], circ.n_params, circ.pool, circ.init)
        psi = sv.run_circuit(head, theta_row)
        if k == W.OP_RZZ:
            psi = sv.apply_1q(psi, n, int(op["q0"]), sv.PZ)
            psi = sv.apply_1q(psi, n, int(op["q1"]), sv.PZ)
        else:
            psi = sv.apply_1q(psi, n, int(op["q0"]), sv.PAULI[_GENERATOR[k]])
        psi = psi * (-0.5j * float(op["scale"]))
        tail = W.Circuit(n, circ.ops[idx + 1:], circ.n_params, circ.pool, circ.init)
        out[p] += sv.run_circuit(tail, theta_row, init_state=psi)
    return out


def quantum_geometric_tensor(circ: W.Circuit, theta_row) -> np.ndarray:
    """G_ij = <d_i psi|d_j psi> - <d_i psi|psi><psi|d_j psi> (Section
    "Quantum Fisher Information"); the QFI is 4 Re G."""
    psi = sv.run_circuit(circ, theta_row)
    d = state_derivatives(circ, theta_row)
    ov = d.conj() @ psi  # <d_i psi|psi>
    return d.conj() @ d.T - np.outer(ov, ov.conj())


def natural_gradient(qgt, grad, eps: float) -> np.ndarray:
    """x solving (4 Re G + eps I) x = grad (Section "Quantum Fisher
    Information": the natural gradient solves the QFI system; eps > 0 is a
    Tikhonov shift that makes the positive semidefinite QFI invertible)."""
    qfi = 4.0 * np.asarray(qgt).real
    return np.linalg.solve(qfi + eps * np.eye(qfi.shape[0]), np.asarray(grad, np.float64))
