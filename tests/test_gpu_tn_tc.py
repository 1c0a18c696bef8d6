"""GPU parity: tensor-core contraction steps (TC_TN_TF32X3, TC_TN_BF16X6).

Section "Tensor network engine": every pairwise contraction is a matrix
product.  In the split-precision modes the steps above a threshold run on
the tensor cores (tcgen05) with split operands; each mode is checked against
the FP64 oracle on the 200-qubit light cone, on small brickwork networks with
every step on the tensor cores (steps of all shapes: M, N below the tile,
K below one stage, either side on the MMA rows), and on the 40-qubit
contraction testbed of Table "contractor" whose largest steps are the dense
intermediate-by-intermediate products.

Tolerance (complex64 inputs, FP32 sums): both split modes keep the products
to ~2^-22 relative and round the sums to nearest every 16 complex terms, so
each step adds at most ~(K/16 + 4) 2^-24 relative error to entries of
magnitude <= 1 (the networks are unitary contractions of unit-norm
factors); over the ~100 (light cone) to ~1500 (whole 40-qubit network) steps
this stays far below the 1e-5 absolute bound on <Z Z> used throughout.
"""
import numpy as np
import pytest

from oracle import tensornet as T
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5
PRECS = [nt.TC_TN_TF32X3, nt.TC_TN_BF16X6]


def _gates_tensor(gate_lists):
    import torch

    arr = np.stack([np.stack([u for (_, _, u) in g]) for g in gate_lists]).astype(np.complex64)
    return torch.as_tensor(arr, device="cuda")


def _params(theta):
    import torch

    return torch.as_tensor(np.asarray(theta, np.float32), device="cuda")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("all_steps", [True, False])
def test_brick200_lightcone_tensor_cores(prec, all_steps):
    n, gates, obs = W.brick200_workload()
    lc = nt.LightCone(n, [(a, b) for a, b, _ in gates], obs)
    if all_steps:
        lc.set_tc_threshold(0)
        assert lc.info()["tc_steps"] >= 90
    g = _gates_tensor([gates])
    out = lc.contract(g, precision=prec).cpu().numpy()
    ref = T.cone_statevector_expectation(gates, obs)
    assert abs(out[0, 0] - ref.real) <= TOL and abs(out[0, 1]) <= TOL
    f32 = lc.contract(g).cpu().numpy()
    assert abs(out[0, 0] - f32[0, 0]) <= TOL


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", range(3))
def test_small_networks_every_step_on_tensor_cores(prec, seed):
    rng = np.random.default_rng(seed)
    for n, depth in ((6, 4), (8, 5), (10, 6)):
        gates = W.brickwork_u4(n, depth, rng)
        for obs in ((n // 2 - 1, n // 2), (0,), (1, n - 2)):
            lc = nt.LightCone(n, [(a, b) for a, b, _ in gates], obs)
            lc.set_tc_threshold(0)
            out = lc.contract(_gates_tensor([gates]), precision=prec).cpu().numpy()
            net = T.network_expectation(n, gates, obs)
            ref = T.contract(net, T.greedy_path(net))
            assert abs(out[0, 0] - ref.real) <= TOL and abs(out[0, 1] - ref.imag) <= TOL, (n, obs)


@pytest.mark.parametrize("prec", PRECS)
def test_whole_network_40_qubits(prec):
    """The whole 40-qubit testbed network (474 ops, no pruning), the plan the
    benchmark times: its dense steps on the tensor cores."""
    n, d, c = 40, 6, 20
    circ = W.example_block_circuit(n, d)
    rng = np.random.default_rng(41)
    theta = rng.uniform(-1.5, 1.5, size=(3, circ.n_params))
    theta[0] = 1.0
    theta = theta.astype(np.float32).astype(np.float64)
    net = nt.CircuitNetwork(circ, {c: 3}, prune=0, split=True, rank_cap=26, greedy_trials=16)
    info = net.info()
    assert info["tc_steps"] >= 10 and info["tc_cmacs"] >= 0.5 * info["cmacs"]
    out = net.expect(_params(theta), precision=prec).cpu().numpy()
    f32 = net.expect(_params(theta)).cpu().numpy()
    for b in range(3):
        ref = T.circuit_window_expectation(circ, theta[b], {c: 3}, c - d - 1, c + d + 1)
        assert abs(out[b, 0] - ref.real) <= TOL and abs(out[b, 1]) <= TOL, (b, out[b], ref)
        assert abs(out[b, 0] - f32[b, 0]) <= TOL


@pytest.mark.parametrize("prec", PRECS)
def test_batched_instances_and_repeat(prec):
    """A batch of weight rows in one graph: each row equals its own oracle
    value; repeated calls replay the graph bit for bit; switching precision
    re-captures."""
    n, d, c = 40, 6, 20
    circ = W.example_block_circuit(n, d)
    theta = np.random.default_rng(7).uniform(-1.5, 1.5, size=(16, circ.n_params)).astype(np.float32)
    net = nt.CircuitNetwork(circ, {c: 3}, prune=0, split=True, rank_cap=26, greedy_trials=16)
    p = _params(theta)
    a = net.expect(p, precision=prec).cpu().numpy()
    b = net.expect(p, precision=prec).cpu().numpy()
    assert np.array_equal(a, b)
    f32 = net.expect(p).cpu().numpy()
    assert np.abs(a[:, 0] - f32[:, 0]).max() <= TOL
    for r in (0, 9, 15):
        ref = T.circuit_window_expectation(circ, theta[r].astype(np.float64), {c: 3}, c - d - 1, c + d + 1)
        assert abs(a[r, 0] - ref.real) <= TOL
