"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module only *describes* work: circuits as op lists, parameter batches,
Pauli-sum Hamiltonians as (structure, weight) pairs, random graphs and Haar
matrices.  It holds none of the method's arithmetic (no gate application, no
expectation values, no gradients), so both the CUDA engine and the FP64
oracle may import it without sharing code.

Conventions (readings of the paper, each stated where it is used):

* Qubit 0 is the most significant bit of the amplitude index (Section
  "Preliminaries": qubit 0 is the leftmost register).
* A Pauli structure is a length-n vector over {0,1,2,3} = {I,X,Y,Z}
  (Section "Pauli structures and weights"); weights are real (Eq. H-pauli).
* A parameterised gate uses the angle ``scale * theta[param]``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---------------------------------------------------------------------------
# Op list encoding (mirrors ``tc_op`` in include/tc.h; tests check the layout)
# ---------------------------------------------------------------------------
OP_H, OP_X, OP_RX, OP_RY, OP_RZ, OP_RZZ, OP_CNOT, OP_CZ, OP_U1, OP_U2, OP_PAULI_NOISE, OP_RSEL = range(12)
OP_NAMES = ["H", "X", "RX", "RY", "RZ", "RZZ", "CNOT", "CZ", "U1", "U2", "PAULI_NOISE", "RSEL"]

INIT_ZERO, INIT_PLUS = 0, 1

OP_DTYPE = np.dtype(
    [
        ("kind", np.int32),
        ("q0", np.int32),
        ("q1", np.int32),
        ("param", np.int32),
        ("scale", np.float64),
        ("mat", np.int32),
        ("pad", np.int32),
        ("px", np.float64),
        ("py", np.float64),
        ("pz", np.float64),
    ],
    align=True,
)
assert OP_DTYPE.itemsize == 56


@dataclasses.dataclass
class Circuit:
    """A parameterised circuit: the op list plus what it refers to.

    ``pool`` is a flat complex128 array; a U1 op reads 4 entries (row-major
    2x2) and a U2 op reads 16 entries (row-major 4x4, row index
    2*b(q0)+b(q1)) starting at ``op["mat"]``.
    """

    n: int
    ops: np.ndarray
    n_params: int
    pool: np.ndarray
    init: int = INIT_ZERO

    @property
    def n_noise(self) -> int:
        return int(np.count_nonzero(self.ops["kind"] == OP_PAULI_NOISE))


class OpBuilder:
    """Append-only op list builder (the paper's ``tc.Circuit`` method calls)."""

    def __init__(self, n: int, init: int = INIT_ZERO):
        self.n = n
        self.init = init
        self.rows: list[tuple] = []
        self.pool: list[complex] = []
        self.n_params = 0

    def _add(self, kind, q0, q1=-1, param=-1, scale=1.0, mat=-1, px=0.0, py=0.0, pz=0.0):
        assert 0 <= q0 < self.n and -1 <= q1 < self.n
        self.rows.append((kind, q0, q1, param, float(scale), mat, 0, float(px), float(py), float(pz)))
        if param >= 0:
            self.n_params = max(self.n_params, param + 1)

    def h(self, q):
        self._add(OP_H, q)

    def x(self, q):
        self._add(OP_X, q)

    def rx(self, q, param, scale=1.0):
        self._add(OP_RX, q, param=param, scale=scale)

    def ry(self, q, param, scale=1.0):
        self._add(OP_RY, q, param=param, scale=scale)

    def rz(self, q, param, scale=1.0):
        self._add(OP_RZ, q, param=param, scale=scale)

    def rzz(self, q0, q1, param, scale=1.0):
        self._add(OP_RZZ, q0, q1, param=param, scale=scale)

    def cnot(self, c, t):
        self._add(OP_CNOT, c, t)

    def cz(self, q0, q1):
        self._add(OP_CZ, q0, q1)

    def unitary1(self, q, m):
        m = np.asarray(m, dtype=np.complex128).reshape(2, 2)
        off = len(self.pool)
        self.pool.extend(m.ravel().tolist())
        self._add(OP_U1, q, mat=off)

    def unitary2(self, q0, q1, m):
        m = np.asarray(m, dtype=np.complex128).reshape(4, 4)
        off = len(self.pool)
        self.pool.extend(m.ravel().tolist())
        self._add(OP_U2, q0, q1, mat=off)

    def depolarizing(self, q, px, py, pz):
        self._add(OP_PAULI_NOISE, q, px=px, py=py, pz=pz)

    def rsel(self, q, param, scale=1.0, px=1.0 / 3, py=1.0 / 3, pz=1.0 / 3):
        """RX, RY or RZ(scale * theta[param]), chosen per row with
        probabilities (px, py, pz) by the row's uniform number for this event."""
        self._add(OP_RSEL, q, param=param, scale=scale, px=px, py=py, pz=pz)

    def build(self, n_params: int | None = None) -> Circuit:
        ops = np.array(self.rows, dtype=OP_DTYPE) if self.rows else np.zeros(0, OP_DTYPE)
        return Circuit(
            n=self.n,
            ops=ops,
            n_params=self.n_params if n_params is None else n_params,
            pool=np.array(self.pool, dtype=np.complex128),
            init=self.init,
        )


# ---------------------------------------------------------------------------
# Hamiltonians as Pauli structures + real weights (Eq. H-pauli)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class PauliSum:
    structures: np.ndarray  # uint8 [T][n], 0..3 = I,X,Y,Z
    weights: np.ndarray  # float64 [T]

    @property
    def n_terms(self) -> int:
        return int(self.weights.shape[0])


def pauli_sum(n: int, terms: list[tuple[float, dict[int, int]]]) -> PauliSum:
    """Build a PauliSum from [(weight, {qubit: code})]."""
    s = np.zeros((len(terms), n), dtype=np.uint8)
    w = np.zeros(len(terms), dtype=np.float64)
    for j, (wt, d) in enumerate(terms):
        w[j] = wt
        for q, c in d.items():
            s[j, q] = c
    return PauliSum(s, w)


def tfim_zz_x(n: int, J: float = 1.0, h: float = 1.0) -> PauliSum:
    """H = -J sum_i Z_i Z_{i+1} (open chain) - h sum_i X_i."""
    terms = [(-J, {i: 3, i + 1: 3}) for i in range(n - 1)]
    terms += [(-h, {i: 1}) for i in range(n)]
    return pauli_sum(n, terms)


def zz_on_edges(n: int, edges, weight: float = 1.0) -> PauliSum:
    return pauli_sum(n, [(weight, {u: 3, v: 3}) for (u, v) in edges])


# ---------------------------------------------------------------------------
# Random objects
# ---------------------------------------------------------------------------
def haar_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random U(d): QR of a complex Ginibre matrix with the phases of
    R's diagonal moved into Q (Mezzadri, Notices AMS 54, 2007)."""
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diagonal(r) / np.abs(np.diagonal(r))
    return q * ph[None, :]


def haar_su2(rng: np.random.Generator) -> np.ndarray:
    u = haar_unitary(2, rng)
    return u / np.sqrt(np.linalg.det(u))


def random_regular3(n: int, rng: np.random.Generator, max_tries: int = 10000) -> list[tuple[int, int]]:
    """Random simple 3-regular graph by configuration-model pairing with
    rejection of self-loops and multi-edges."""
    assert n % 2 == 0 and n >= 4
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        ok = True
        seen = set()
        for u, v in pairs:
            u, v = int(u), int(v)
            if u == v:
                ok = False
                break
            e = (min(u, v), max(u, v))
            if e in seen:
                ok = False
                break
            seen.add(e)
        if ok:
            return sorted(seen)
    raise RuntimeError("no simple 3-regular graph found")


# ---------------------------------------------------------------------------
# The workloads (named by what they are)
# ---------------------------------------------------------------------------
def hea_circuit(n: int, layers: int) -> Circuit:
    """Hardware-efficient ansatz: per layer RX(a_i), RZ(b_i) on every qubit
    (RX then RZ per qubit), then a CNOT ladder 0->1, ..., n-2->n-1.
    theta[2n*l + i] = a_i, theta[2n*l + n + i] = b_i."""
    b = OpBuilder(n, INIT_ZERO)
    for l in range(layers):
        for i in range(n):
            b.rx(i, 2 * n * l + i)
            b.rz(i, 2 * n * l + n + i)
        for i in range(n - 1):
            b.cnot(i, i + 1)
    return b.build(2 * n * layers)


def tfim_circuit(n: int, layers: int) -> Circuit:
    """TFIM VQE ansatz from |+>^n: per layer RZZ(g_l) on all nearest-neighbour
    bonds, then RX(b_l) on all qubits; theta[2l] = g_l, theta[2l+1] = b_l."""
    b = OpBuilder(n, INIT_PLUS)
    for l in range(layers):
        for i in range(n - 1):
            b.rzz(i, i + 1, 2 * l)
        for i in range(n):
            b.rx(i, 2 * l + 1)
    return b.build(2 * layers)


def qaoa_circuit(n: int, edges, p: int) -> Circuit:
    """QAOA MaxCut from |+>^n: per layer RZZ(gamma_l) on every edge, then
    RX(beta_l) mixer; theta[2l] = gamma_l, theta[2l+1] = beta_l."""
    b = OpBuilder(n, INIT_PLUS)
    for l in range(p):
        for (u, v) in edges:
            b.rzz(u, v, 2 * l)
        for i in range(n):
            b.rx(i, 2 * l + 1)
    return b.build(2 * p)


def noisy_su2_cz_circuit(n: int, layers: int, p: float, rng: np.random.Generator) -> Circuit:
    """Per layer a Haar SU(2) on every qubit, then CZ on pairs (2i,2i+1) in
    even layers and (2i+1,2i+2) in odd layers.  Single-qubit depolarising
    noise with px=py=pz=p/3 follows every gate: one event on the SU(2)'s
    qubit, one on each qubit of a CZ."""
    b = OpBuilder(n, INIT_ZERO)
    q3 = p / 3.0
    for l in range(layers):
        for i in range(n):
            b.unitary1(i, haar_su2(rng))
            b.depolarizing(i, q3, q3, q3)
        start = 0 if l % 2 == 0 else 1
        for i in range(start, n - 1, 2):
            b.cz(i, i + 1)
            b.depolarizing(i, q3, q3, q3)
            b.depolarizing(i + 1, q3, q3, q3)
    return b.build(0)


def random_circuit(n: int, n_gates: int, rng: np.random.Generator, n_params: int = 8,
                   kinds=None) -> Circuit:
    """Random mix of every gate kind on random qubits (parity coverage)."""
    if kinds is None:
        kinds = [OP_H, OP_X, OP_RX, OP_RY, OP_RZ, OP_RZZ, OP_CNOT, OP_CZ, OP_U1, OP_U2]
    b = OpBuilder(n, INIT_ZERO)
    for _ in range(n_gates):
        k = kinds[int(rng.integers(len(kinds)))]
        q0 = int(rng.integers(n))
        q1 = int(rng.integers(n - 1))
        if q1 >= q0:
            q1 += 1
        prm = int(rng.integers(n_params))
        sc = float(rng.choice([1.0, -2.0, 0.5]))
        if k == OP_H:
            b.h(q0)
        elif k == OP_X:
            b.x(q0)
        elif k == OP_RX:
            b.rx(q0, prm, sc)
        elif k == OP_RY:
            b.ry(q0, prm, sc)
        elif k == OP_RZ:
            b.rz(q0, prm, sc)
        elif k == OP_RZZ:
            b.rzz(q0, q1, prm, sc)
        elif k == OP_CNOT:
            b.cnot(q0, q1)
        elif k == OP_CZ:
            b.cz(q0, q1)
        elif k == OP_U1:
            b.unitary1(q0, haar_unitary(2, rng))
        elif k == OP_U2:
            b.unitary2(q0, q1, haar_unitary(4, rng))
        elif k == OP_PAULI_NOISE:
            px, py, pz = rng.uniform(0, 0.2, 3)
            b.depolarizing(q0, px, py, pz)
    return b.build(n_params)


def random_pauli_sum(n: int, n_terms: int, rng: np.random.Generator) -> PauliSum:
    s = rng.integers(0, 4, size=(n_terms, n)).astype(np.uint8)
    w = rng.standard_normal(n_terms)
    return PauliSum(s, w)


def chem_pauli_sum(n: int = 12, n_terms: int = 1390, seed: int = 1006) -> PauliSum:
    """A chemistry-shaped Pauli sum with the structure of a Jordan-Wigner
    molecular Hamiltonian (the paper's H2O example has 12 qubits and 1390
    terms; its data is not used here): Z_p and Z_p Z_q terms, hopping terms
    X_p Z..Z X_q and Y_p Z..Z Y_q, and four-body terms O_p Z..Z O_q O_r Z..Z O_s
    with O in {X, Y} and an even number of Y (a real Hamiltonian).  Weights are
    N(0, 1) with a decaying envelope, largest for the one-body terms."""
    rng = np.random.default_rng(seed)
    terms = []

    def zs(a, b):
        return {k: 3 for k in range(a + 1, b)}

    for p_ in range(n):
        terms.append({p_: 3})
    for p_ in range(n):
        for q in range(p_ + 1, n):
            terms.append({p_: 3, q: 3})
    for p_ in range(n):
        for q in range(p_ + 1, n):
            for o in (1, 2):
                d = zs(p_, q)
                d[p_] = o
                d[q] = o
                terms.append(d)
    quads = [(a, b, c, d) for a in range(n) for b in range(a + 1, n) for c in range(b + 1, n) for d in range(c + 1, n)]
    pats = [(1, 1, 1, 1), (2, 2, 2, 2), (1, 1, 2, 2), (2, 2, 1, 1), (1, 2, 1, 2), (2, 1, 2, 1), (1, 2, 2, 1), (2, 1, 1, 2)]
    cand = [(qd, pt) for qd in quads for pt in pats]
    pick = rng.choice(len(cand), size=max(0, n_terms - len(terms)), replace=False)
    for i in sorted(pick):
        (a, b, c, d), (oa, ob, oc, od) = cand[i]
        t = zs(a, b)
        t.update(zs(c, d))
        t.update({a: oa, b: ob, c: oc, d: od})
        terms.append(t)
    w = rng.standard_normal(len(terms)) * np.exp(-np.arange(len(terms)) / 400.0)
    return pauli_sum(n, [(float(wi), t) for wi, t in zip(w, terms[:n_terms])])


def brickwork_u4(n: int, depth: int, rng: np.random.Generator, round_c64: bool = True
                 ) -> list[tuple[int, int, np.ndarray]]:
    """1D brickwork of Haar U(4): layer 0 acts on pairs (2i, 2i+1), layer 1 on
    (2i+1, 2i+2), alternating.  Matrices are drawn in complex128 and, by
    default, rounded to complex64 (returned upcast, so both sides see the same
    numbers; the rounded gates are unitary only to ~1e-8)."""
    gates = []
    for l in range(depth):
        start = 0 if l % 2 == 0 else 1
        for i in range(start, n - 1, 2):
            u = haar_unitary(4, rng)
            if round_c64:
                u = u.astype(np.complex64).astype(np.complex128)
            gates.append((i, i + 1, u))
    return gates


# ---------------------------------------------------------------------------
# Named configurations (sizes of the paper-shaped workloads)
# ---------------------------------------------------------------------------
SEED_HEA10, SEED_TFIM20, SEED_BRICK200, SEED_QAOA_STREAM, SEED_NOISY16 = 1001, 1002, 1003, 1004, 1005


def hea10_workload():
    """10-qubit HEA, 4 layers, 80 angles U[0, 2pi), complex128, |0...0>;
    observables <Z0 Z1> and <X5>."""
    rng = np.random.default_rng(SEED_HEA10)
    circ = hea_circuit(10, 4)
    theta = rng.uniform(0.0, 2.0 * np.pi, size=(1, circ.n_params))
    obs = [pauli_sum(10, [(1.0, {0: 3, 1: 3})]), pauli_sum(10, [(1.0, {5: 1})])]
    return circ, theta, obs


def tfim_workload(n: int = 20, layers: int = 10, batch: int = 1024, seed: int = SEED_TFIM20):
    """TFIM VQE: n qubits, `layers` layers, batch of parameter sets with
    angles ~ N(0, 0.3^2); H = -sum Z_i Z_{i+1} - sum X_i."""
    rng = np.random.default_rng(seed)
    circ = tfim_circuit(n, layers)
    theta = rng.normal(0.0, 0.3, size=(batch, circ.n_params))
    return circ, theta, tfim_zz_x(n)


def noisy16_workload(n: int = 16, layers: int = 12, p: float = 0.01, trajectories: int = 8192,
                     seed: int = SEED_NOISY16):
    rng = np.random.default_rng(seed)
    circ = noisy_su2_cz_circuit(n, layers, p, rng)
    obs = [pauli_sum(n, [(1.0, {0: 3})]), pauli_sum(n, [(1.0, {i: 3, i + 1: 3}) for i in range(n - 1)])]
    return circ, trajectories, seed, obs


def bp_workload(n: int = 10, layers: int = 10, structures: int = 100, seed: int = 1008):
    """The gradient-variance workload of Section "Demonstration of barren
    plateaus": per layer a random choice of RX/RY/RZ (probability 1/3 each,
    one weight per gate, theta[i * layers + l]) on every qubit, then CZ on
    (i, i+1); one batch row per random structure (the structure comes from
    the row's event stream) with weights ~ U[0, 2 pi); cost <Z0 Z1>."""
    b = OpBuilder(n, INIT_ZERO)
    for l in range(layers):
        for i in range(n):
            b.rsel(i, i * layers + l)
        for i in range(n - 1):
            b.cz(i, i + 1)
    circ = b.build(n * layers)
    theta = np.random.default_rng(seed).uniform(0, 2 * np.pi, size=(structures, n * layers))
    return circ, theta, seed, pauli_sum(n, [(1.0, {0: 3, 1: 3})])


def example_block_circuit(n: int = 40, d: int = 6) -> Circuit:
    """The contraction testbed of Section "Custom contraction settings": d
    layers, each exp(i t Z_i Z_{i+1}) along the chain i = 0..n-2 followed by
    RX on every qubit, on |0...0>.  Weights: theta[2 j n + i] for the ZZ gate
    (i, i+1) of layer j, theta[(2 j + 1) n + i] for RX on qubit i; the paper
    sets all 2 d n of them to one.  exp(i t ZZ) = RZZ(-2 t), hence scale -2.
    The observable is Z on qubit n // 2."""
    b = OpBuilder(n, INIT_ZERO)
    for j in range(d):
        for i in range(n - 1):
            b.rzz(i, i + 1, 2 * j * n + i, scale=-2.0)
        for i in range(n):
            b.rx(i, (2 * j + 1) * n + i)
    return b.build(2 * d * n)


def brick200_workload(n: int = 200, depth: int = 8, seed: int = SEED_BRICK200):
    rng = np.random.default_rng(seed)
    gates = brickwork_u4(n, depth, rng)
    return n, gates, (99, 100)


@dataclasses.dataclass
class QaoaRequest:
    rid: int
    t_arrive: float
    n: int
    p: int
    edges: list
    theta: np.ndarray  # [2p]


def qaoa_stream(rate_hz: float = 2000.0, duration_s: float = 10.0, seed: int = SEED_QAOA_STREAM,
                widths=tuple(range(8, 27, 2)), max_p: int = 6) -> list[QaoaRequest]:
    """Poisson arrivals; n uniform over `widths`, p uniform in 1..max_p,
    random 3-regular graph, angles uniform in [0, pi)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    rid = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        n = int(rng.choice(widths))
        p = int(rng.integers(1, max_p + 1))
        edges = random_regular3(n, rng)
        theta = rng.uniform(0.0, np.pi, size=2 * p)
        out.append(QaoaRequest(rid, t, n, p, edges, theta))
        rid += 1
    return out
