"""GPU parity: small circuits in one launch (tc_apply_expect).

States and Pauli-sum expectations of circuits of 5..10 qubits, computed in
one cluster launch per row (the "Plain method" of Section "Basic circuits and
outputs": the state, then one expectation per observable), against the FP64
oracle and against the tile-pass path (tc_apply_layers + tc_expect_pauli_sum).
Gates land on lane, warp and cluster-rank bits of the index; wider or noisy
circuits take the general path through the same call.
"""
import numpy as np
import pytest

from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64, TOL_AMP_C128, cuda_params

pytestmark = pytest.mark.gpu

KINDS = [W.OP_H, W.OP_X, W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_RZZ, W.OP_CNOT, W.OP_CZ, W.OP_U1, W.OP_U2]


def _check(circ, theta, sums, dtype, B):
    import torch

    c = nt.Circuit(circ, dtype=dtype)
    obs = nt.Observables(sums)
    st, val = c.apply_expect(cuda_params(theta), obs, B)
    _, val2 = c.apply_expect(cuda_params(theta), obs, B, store_state=False)
    torch.cuda.synchronize()
    st, val, val2 = st.cpu().numpy(), val.cpu().numpy(), val2.cpu().numpy()
    tol = TOL_AMP_C128 if dtype == nt.TC_C128 else TOL_AMP_C64
    etol = 1e-11 if dtype == nt.TC_C128 else 1e-5
    assert np.array_equal(val, val2)
    for b in range(B):
        ref = sv.run_circuit(circ, theta[b] if theta is not None else None)
        assert np.abs(st[b] - ref).max() <= tol
        for k, s in enumerate(sums):
            e_ref = sv.energy(ref, circ.n, s)[0]
            assert abs(val[b, k] - e_ref) <= etol * max(1.0, np.abs(s.weights).sum())
    # the tile-pass path on the same rows
    st2 = c.apply(cuda_params(theta), B).cpu().numpy()
    assert np.abs(st - st2).max() <= 2 * tol
    return st, val


def test_hea10_complex128_state_and_observables():
    circ, theta, obs = W.hea10_workload()
    st, val = _check(circ, theta, obs, nt.TC_C128, 1)
    ref = sv.run_circuit(circ, theta[0])
    assert abs(val[0, 0] - sv.energy(ref, 10, obs[0])[0]) <= 1e-12
    assert abs(val[0, 1] - sv.energy(ref, 10, obs[1])[0]) <= 1e-12


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n", [5, 6, 7, 8, 10])
def test_random_circuits_every_kind(n, dtype):
    rng = np.random.default_rng(900 + n)
    circ = W.random_circuit(n, 6 * n, rng, n_params=5, kinds=KINDS)
    theta = rng.uniform(-3, 3, size=(3, 5))
    sums = [W.random_pauli_sum(n, 5, rng), W.random_pauli_sum(n, 1, rng), W.pauli_sum(n, [(0.7, {0: 1, n - 1: 2})])]
    _check(circ, theta, sums, dtype, 3)


def test_gates_across_the_cluster_rank_bits():
    """10 qubits: qubits 0..2 are the rank bits. One-qubit matrices, CNOTs
    and 4x4 matrices on every kind of pair (rank-rank, rank-warp, rank-lane,
    warp-lane), with X/Y strings that flip rank bits."""
    rng = np.random.default_rng(5)
    n = 10
    b = W.OpBuilder(n)
    for q in range(n):
        b.unitary1(q, W.haar_unitary(2, rng))
    for (q0, q1) in [(0, 1), (2, 0), (1, 5), (6, 2), (0, 9), (9, 1), (3, 8), (7, 4), (2, 9)]:
        b.cnot(q0, q1)
        b.unitary2(q0, q1, W.haar_unitary(4, rng))
        b.cz(q1, q0)
        b.rzz(q0, q1, 0)
        b.ry(q0, 1)
    circ = b.build(2)
    theta = rng.uniform(-3, 3, size=(2, 2))
    sums = [W.pauli_sum(n, [(1.0, {0: 1}), (0.5, {1: 2, 2: 1}), (-0.3, {0: 3, 9: 1})]),
            W.pauli_sum(n, [(1.0, {q: 1 for q in range(n)})])]
    for dtype in (nt.TC_C64, nt.TC_C128):
        _check(circ, theta, sums, dtype, 2)


def test_wide_and_noisy_circuits_take_the_general_path():
    rng = np.random.default_rng(8)
    circ = W.random_circuit(12, 40, rng, n_params=4, kinds=KINDS)
    theta = rng.uniform(-3, 3, size=(2, 4))
    _check(circ, theta, [W.random_pauli_sum(12, 4, rng)], nt.TC_C128, 2)
    noisy = W.noisy_su2_cz_circuit(8, 2, 0.2, rng)
    c = nt.Circuit(noisy, dtype=nt.TC_C128)
    _, val = c.apply_expect(None, nt.Observables([W.pauli_sum(8, [(1.0, {0: 3})])]), 3)
    st = c.apply(None, 3)
    ref = c.expect(st, nt.Hamiltonian(W.pauli_sum(8, [(1.0, {0: 3})])))
    assert np.abs(val.cpu().numpy()[:, 0] - ref.cpu().numpy()).max() <= 1e-12


def test_empty_observable_and_no_observables():
    import torch

    circ, theta, _ = W.hea10_workload()
    c = nt.Circuit(circ, dtype=nt.TC_C128)
    empty = W.PauliSum(np.zeros((0, 10), np.uint8), np.zeros(0))
    _, val = c.apply_expect(cuda_params(theta), nt.Observables([empty, W.pauli_sum(10, [(2.0, {})])]), 1)
    assert val.cpu().numpy()[0, 0] == 0.0 and abs(val.cpu().numpy()[0, 1] - 2.0) <= 1e-12
    st, _ = c.apply_expect(cuda_params(theta), nt.Observables([]), 1)
    torch.cuda.synchronize()
    assert np.abs(st.cpu().numpy()[0] - sv.run_circuit(circ, theta[0])).max() <= TOL_AMP_C128
