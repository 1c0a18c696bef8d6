"""Oracle: gradients of E(theta) = <psi(theta)|H|psi(theta)> (test infrastructure only).

The engine computes gradients with an adjoint sweep; the oracle deliberately
uses two other routes so that neither can hide a mistake in the other:

* parameter shift per gate occurrence: for a gate exp(-i a G/2) with G^2 = I
  and a = s*theta_k, dE/da = [E(a + pi/2) - E(a - pi/2)] / 2 exactly, and
  dE/dtheta_k sums s * dE/da over every occurrence of theta_k (shared angles
  such as one g_l over a whole RZZ layer);
* central finite differences with step h in FP64.

Pinned by tests/test_oracle_gradients.py: the batched-VQE toy of Section
"Batched VQE" (closed form cos(w1), gradient (0, -sin w1)), the vvag toy of
Section "vmap and vectorized_value_and_grad" (summed-over-batch gradient),
agreement of the two routes, and TFIM closed forms (zero gradient at zero
angles).  Batch semantics (Section "vmap and vectorized_value_and_grad"):
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
