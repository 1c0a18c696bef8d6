"""Oracle: Monte Carlo Pauli-channel trajectories (test infrastructure only).

* ``philox4x32_10``: the counter-based generator of Salmon, Moraes, Dror and
  Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC'11), written from
  its published definition; pinned by the algorithm's published
  known-answer vectors (tests/golden/philox4x32_10_kat.txt), by
  uniformity/independence statistics, and by bit-equality with the engine's
  own independent implementation.
* Trajectory selection follows Section "Externalizing the randomness": the
  uniform number u picks the outcome whose interval contains it; intervals
  are contiguous with lengths proportional to the probabilities, in the
  order [I, X, Y, Z] (Section "Monte Carlo simulation with tc.Circuit").
* ``density_matrix``: exact evolution rho -> sum_i K_i rho K_i^dagger
  (Section "Density matrix simulation with tc.DMCircuit"), used to pin the
  trajectory estimator statistically for small n.

Status stream layout shared with the engine (a definition of this library,
not the paper's): noise event e of trajectory b uses Philox with counter
(e // 4, b, 0, 0) and key (seed & 0xffffffff, seed >> 32), output word
e % 4, and u = (word >> 8) * 2^-24.
"""
from __future__ import annotations

import numpy as np

from paper_2205_10091_b300 import workloads as W
from . import statevector as sv

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.  ``ctr``: 4 arrays of uint32 values,
    ``key``: 2 arrays/ints; returns 4 uint64 arrays holding 32-bit words.

    One round maps (x0, x1, x2, x3) with key (k0, k1) to
      (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)),
    and the key is bumped by the Weyl constants between rounds."""
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in ctr)
    k0 = np.asarray(key[0], dtype=np.uint64) & _MASK
    k1 = np.asarray(key[1], dtype=np.uint64) & _MASK
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * x0  # < 2^64, exact in uint64
        p1 = _M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return x0, x1, x2, x3


def status_from_seed(seed: int, n_traj: int, n_events: int, traj_offset: int = 0) -> np.ndarray:
    """u[b][e] in [0,1) for trajectories traj_offset..traj_offset+n_traj-1."""
    b = np.arange(traj_offset, traj_offset + n_traj, dtype=np.uint64)[:, None]
    e = np.arange(n_events, dtype=np.uint64)[None, :]
    shape = (n_traj, n_events)
    ctr = (np.broadcast_to(e >> np.uint64(2), shape), np.broadcast_to(b, shape),
           np.zeros(shape, np.uint64), np.zeros(shape, np.uint64))
    key = (np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    words = philox4x32_10(ctr, key)
    sel = np.broadcast_to(e & np.uint64(3), shape)
    w = np.choose(sel.astype(np.int64), words)
    return (w >> np.uint64(8)).astype(np.float64) * 2.0 ** -24


def trajectory_expectations(circ: W.Circuit, status: np.ndarray, observables) -> np.ndarray:
    """Exact per-trajectory <O> for each observable (a PauliSum):
    out[b][o]."""
    out = np.zeros((status.shape[0], len(observables)))
    for b in range(status.shape[0]):
        psi = sv.run_circuit(circ, None, status_row=status[b])
        for o, obs in enumerate(observables):
            out[b, o] = sv.energy(psi, circ.n, obs)[0]
    return out


def estimate(values: np.ndarray):
    """Mean over trajectories and its standard error (sample std, ddof=1,
    over sqrt(N))."""
    n = values.shape[0]
    mean = values.mean(axis=0)
    se = values.std(axis=0, ddof=1) / np.sqrt(n) if n > 1 else np.zeros_like(mean)
    return mean, se


def density_matrix(circ: W.Circuit, theta=None) -> np.ndarray:
    """rho after the circuit, channels applied as sum_i K_i rho K_i^dagger
    with K = sqrt(1-px-py-pz) I, sqrt(px) X, sqrt(py) Y, sqrt(pz) Z; gates
    with a parameter take theta[param] * scale as in run_circuit (theta =
    None: all parameters 0)."""
    n = circ.n
    psi0 = sv.initial_state(n, circ.init)
    rho = np.outer(psi0, psi0.conj())
    theta = np.zeros(max(circ.n_params, 1)) if theta is None else np.asarray(theta, dtype=np.float64)

    def conj_apply(rho, q, m, q1=None):
        # rho -> M rho M^dagger: apply M to the column index of rho (rows are
        # the ket side) and conj(M) to the row index, each with the 1q/2q
        # state-vector routines over a doubled register.
        d = 2 ** n
        cols = rho.T.reshape(d, d)  # each row of cols is a column of rho
        cols = np.stack([sv.apply_1q(c, n, q, m) if q1 is None else sv.apply_2q(c, n, q, q1, m) for c in cols])
        rho = cols.T
        rows = np.stack([sv.apply_1q(r, n, q, m.conj()) if q1 is None else sv.apply_2q(r, n, q, q1, m.conj())
                         for r in rho])
        return rows

    for op in circ.ops:
        k = int(op["kind"])
        q = int(op["q0"])
        if k == W.OP_PAULI_NOISE:
            px, py, pz = float(op["px"]), float(op["py"]), float(op["pz"])
            acc = (1.0 - px - py - pz) * rho
            for p, P in ((px, sv.PX), (py, sv.PY), (pz, sv.PZ)):
                if p:
                    acc = acc + p * conj_apply(rho, q, P)
            rho = acc
            continue
        m = sv.gate_matrix(op, theta, circ.pool)
        rho = conj_apply(rho, q, m) if m.shape[0] == 2 else conj_apply(rho, q, m, int(op["q1"]))
    return rho


def dm_expectation(rho: np.ndarray, n: int, obs: W.PauliSum) -> float:
    """tr(rho O) with O = sum_j w_j P_j."""
    return float(np.real(np.trace(rho @ sv.dense_pauli_sum(n, obs))))
