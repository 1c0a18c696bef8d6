"""Oracle: tensor-network expectation values (test infrastructure only).

Section "Tensor network engine" / "Custom contraction settings": a circuit
expectation <0|U^dagger O U|0> is a tensor network (ket gates, the observable,
conjugated bra gates) whose value does not depend on the contraction path.

* ``light_cone``: the gates that can influence <O>; every other gate meets
  its own inverse in the doubled network and cancels (U^dagger U = I).
* ``cone_statevector_expectation``: the oracle's own route for large circuits:
  a dense FP64 state vector over the cone's qubits, the cone gates applied one
  at a time, then <O>.
* ``window_statevector_expectation``: every gate inside a qubit window wider
  than the cone (pins the cone: must give the same scalar).
* ``circuit_window_expectation``: <P> of a parameterised op-list circuit
  over a qubit window: every op inside the window applied to a dense FP64
  window state, ops touching the outside dropped.  Exact whenever every
  dropped op commutes with the Heisenberg-evolved string at its position
  (outside its support, or diagonal against diagonal support), which holds
  for the contraction testbed with the window n//2 - d - 1 .. n//2 + d + 1.
* ``network_expectation`` + ``contract``: the doubled network contracted
  pairwise with np.einsum along any given path (pins path independence and
  agreement with the state vector on tiny circuits).

Pinned by tests/test_oracle_tensornet.py (state vector == network on tiny
brickworks along two different paths; cone == window; cone of a brickwork
has the expected gate count; the circuit window equals the full state
vector on circuits small enough to simulate whole, and a window narrower
than the string's support does not).
"""
from __future__ import annotations

import numpy as np

from paper_2205_10091_b300 import workloads as W
from . import statevector as sv

PZ = sv.PZ


def light_cone(gates, obs_qubits):
    """Gates (in forward order) in the backward causal cone of obs_qubits."""
    active = set(obs_qubits)
    keep = []
    for g in reversed(gates):
        q0, q1 = g[0], g[1]
        if q0 in active or q1 in active:
            keep.append(g)
            active.add(q0)
            active.add(q1)
    keep.reverse()
    return keep


def _local_statevector_expectation(gates, obs_qubits, qubits):
    qubits = sorted(qubits)
    loc = {q: i for i, q in enumerate(qubits)}
    m = len(qubits)
    psi = np.zeros(2 ** m, dtype=np.complex128)
    psi[0] = 1.0
    for (q0, q1, u) in gates:
        psi = sv.apply_2q(psi, m, loc[q0], loc[q1], np.asarray(u, np.complex128))
    phi = psi
    for q in obs_qubits:
        phi = sv.apply_1q(phi, m, loc[q], PZ)
    return complex(np.vdot(psi, phi))


def cone_statevector_expectation(gates, obs_qubits):
    """<Z..Z> over the light cone only, as a dense state vector."""
    cone = light_cone(gates, obs_qubits)
    qubits = set(obs_qubits)
    for (q0, q1, _) in cone:
        qubits.update((q0, q1))
    return _local_statevector_expectation(cone, obs_qubits, qubits)


def window_statevector_expectation(gates, obs_qubits, lo, hi):
    """<Z..Z> with every gate whose qubits lie in [lo, hi] applied."""
    inside = [g for g in gates if lo <= g[0] <= hi and lo <= g[1] <= hi]
    return _local_statevector_expectation(inside, obs_qubits, range(lo, hi + 1))


def circuit_window_expectation(circ: W.Circuit, theta_row, pauli: dict, lo: int, hi: int) -> complex:
    """<P> for the Pauli string ``pauli`` ({qubit: 1..3 = X, Y, Z}) with
    the ops of ``circ`` that lie inside [lo, hi] applied to the window."""
    ops = circ.ops
    q1 = ops["q1"]
    inside = (ops["q0"] >= lo) & (ops["q0"] <= hi) & ((q1 < 0) | ((q1 >= lo) & (q1 <= hi)))
    sub = ops[inside].copy()
    sub["q0"] -= lo
    sub["q1"] = np.where(sub["q1"] >= 0, sub["q1"] - lo, -1)
    m = hi - lo + 1
    psi = sv.run_circuit(W.Circuit(m, sub, circ.n_params, circ.pool, circ.init), theta_row)
    phi = psi
    for q, c in pauli.items():
        assert lo <= q <= hi
        phi = sv.apply_1q(phi, m, q - lo, sv.PAULI[c])
    return complex(np.vdot(psi, phi))


def network_expectation(n, gates, obs_qubits):
    """Doubled network for <0|U^dagger Z..Z U|0> on n qubits as a list of
    (tensor, labels).  Gate tensors are U[o0,o1,i0,i1]."""
    nxt = [0]

    def new():
        nxt[0] += 1
        return nxt[0] - 1

    tensors = []
    ket = [new() for _ in range(n)]
    for q in range(n):
        tensors.append((np.array([1.0, 0.0], np.complex128), [ket[q]]))
    # bra side starts from the same |0> vectors, conjugated, with fresh labels
    bra = [new() for _ in range(n)]
    for q in range(n):
        tensors.append((np.array([1.0, 0.0], np.complex128), [bra[q]]))
    for (q0, q1, u) in gates:
        t = np.asarray(u, np.complex128).reshape(2, 2, 2, 2)
        a, b = new(), new()
        tensors.append((t, [a, b, ket[q0], ket[q1]]))
        ket[q0], ket[q1] = a, b
        c, d = new(), new()
        tensors.append((t.conj(), [c, d, bra[q0], bra[q1]]))
        bra[q0], bra[q1] = c, d
    for q in range(n):
        if q in obs_qubits:
            tensors.append((PZ.copy(), [bra[q], ket[q]]))
        else:
            tensors.append((np.eye(2, dtype=np.complex128), [bra[q], ket[q]]))
    return tensors


def contract_pair(ta, la, tb, lb, keep_labels):
    """Contract two tensors over their shared labels (np.einsum), keeping
    labels that still appear elsewhere."""
    out = [l for l in la if l in keep_labels] + [l for l in lb if l in keep_labels and l not in la]
    sym = {}
    for l in la + lb + out:
        if l not in sym:
            sym[l] = chr(ord("a") + len(sym)) if len(sym) < 26 else chr(ord("A") + len(sym) - 26)
    expr = "".join(sym[l] for l in la) + "," + "".join(sym[l] for l in lb) + "->" + "".join(sym[l] for l in out)
    return np.einsum(expr, ta, tb), out


def contract(tensors, path):
    """Contract along an opt_einsum-style path of position pairs (the two
    operands are removed and the result appended)."""
    ts = list(tensors)
    for (i, j) in path:
        i, j = sorted((i, j))
        (tb, lb) = ts.pop(j)
        (ta, la) = ts.pop(i)
        rest = set()
        for (_, l) in ts:
            rest.update(l)
        t, l = contract_pair(ta, la, tb, lb, rest)
        ts.append((t, l))
    while len(ts) > 1:
        (tb, lb) = ts.pop()
        (ta, la) = ts.pop()
        rest = set()
        for (_, l) in ts:
            rest.update(l)
        t, l = contract_pair(ta, la, tb, lb, rest)
        ts.append((t, l))
    return complex(ts[0][0])


def sequential_path(n_tensors):
    """Path that folds tensors in list order: (0,1), then (0, last), ..."""
    path = []
    cnt = n_tensors
    while cnt > 1:
        path.append((0, cnt - 1) if path else (0, 1))
        cnt -= 1
    return path


def greedy_path(tensors):
    """A simple path: repeatedly contract the connected pair with the
    smallest result (ties: first pair found); unconnected pairs last."""
    sizes = [(list(l), t.shape) for (t, l) in tensors]
    items = [(l, dict(zip(l, s))) for (l, s) in sizes]
    path = []
    while len(items) > 1:
        best = None
        for i in range(len(items)):
            for j in range(i + 1, len(items)):
                la, da = items[i]
                lb, db = items[j]
                if not set(la) & set(lb):
                    continue
                rest = set()
                for k, (lk, _) in enumerate(items):
                    if k != i and k != j:
                        rest.update(lk)
                out = [l for l in la if l in rest] + [l for l in lb if l in rest and l not in la]
                size = 1
                for l in out:
                    size *= (da.get(l) or db.get(l))
                if best is None or size < best[0]:
                    best = (size, i, j, out, {**da, **db})
        if best is None:
            best = (0, 0, 1, items[0][0] + items[1][0], {**items[0][1], **items[1][1]})
        _, i, j, out, dims = best
        path.append((i, j))
        items.pop(j)
        items.pop(i)
        items.append((out, {l: dims[l] for l in out}))
    return path
