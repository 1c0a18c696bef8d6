"""GPU parity: checkpointed gradients (TC_GRAD_CHECKPOINT).

The op list is cut into segments, each planned as a circuit of its own; the
forward sweep stores the state after every segment and the adjoint sweep of
each segment starts from its stored state (the adjoint method of Section
"Gradients, optimization and variational algorithms" with checkpoints).
Energies and gradients are checked against the FP64 oracle (parameter shift,
central differences on a deep circuit) and against the uncompute mode, for
segment lengths from one op (every gate its own segment) to the default.
"""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import assert_energy_close, assert_grad_close, cuda_params

pytestmark = pytest.mark.gpu

KINDS = [W.OP_H, W.OP_X, W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_RZZ, W.OP_CNOT, W.OP_CZ, W.OP_U1, W.OP_U2]


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("seg_ops", [1, 7, 0])
def test_random_circuit_checkpointed_gradients(dtype, seg_ops):
    n = 11
    rng = np.random.default_rng(300 + seg_ops)
    circ = W.random_circuit(n, 40, rng, n_params=6, kinds=KINDS)
    ham = W.random_pauli_sum(n, 6, rng)
    theta = rng.uniform(-3, 3, size=(3, 6))
    c = nt.Circuit(circ, dtype=dtype)
    H = nt.Hamiltonian(ham)
    e, g = c.expect_grad(cuda_params(theta), H, checkpoint_ops=seg_ops)
    eu, gu = c.expect_grad(cuda_params(theta), H)
    e, g, eu, gu = (x.cpu().numpy() for x in (e, g, eu, gu))
    for b in range(3):
        e_ref = sv.energy(sv.run_circuit(circ, theta[b]), n, ham)[0]
        g_ref = G.parameter_shift(circ, theta[b], ham)
        if dtype == nt.TC_C128:
            assert abs(e[b] - e_ref) <= 1e-11 * max(1, abs(e_ref))
            assert np.abs(g[b] - g_ref).max() <= 1e-10 * max(1, np.abs(g_ref).max())
        else:
            assert_energy_close(e[b:b + 1], [e_ref])
            assert_grad_close(g[b], g_ref)
    tol = 1e-12 if dtype == nt.TC_C128 else 1e-5
    assert np.abs(e - eu).max() <= tol * max(1, np.abs(eu).max())
    assert np.abs(g - gu).max() <= 10 * tol * max(1, np.abs(gu).max())


def test_deep_tfim_checkpointed_gradients():
    """16 qubits, 48 layers, complex64, a segment every four layers."""
    n, layers = 16, 48
    circ, theta, ham = W.tfim_workload(n=n, layers=layers, batch=2, seed=48)
    c = nt.Circuit(circ)
    layer_ops = (n - 1) + n
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham), checkpoint_ops=4 * layer_ops)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    b = 1
    assert_energy_close(e[b:b + 1], [sv.energy(sv.run_circuit(circ, theta[b]), n, ham)[0]])
    ks = [0, 1, 2, 3, layers - 1, layers, 2 * layers - 2, 2 * layers - 1]
    fd = G.finite_difference(circ, theta[b], ham, h=1e-5, params=ks)
    assert_grad_close(g[b, ks], fd[ks])


def test_checkpoint_rows_in_chunks_match_one_chunk():
    circ, theta, ham = W.tfim_workload(n=12, layers=6, batch=9, seed=5)
    c = nt.Circuit(circ)
    H = nt.Hamiltonian(ham)
    e1, g1 = c.expect_grad(cuda_params(theta), H, checkpoint_ops=23)
    e2, g2 = c.expect_grad(cuda_params(theta), H, checkpoint_ops=23, max_rows=4)
    assert np.array_equal(e1.cpu().numpy(), e2.cpu().numpy())
    assert np.array_equal(g1.cpu().numpy(), g2.cpu().numpy())


def test_checkpoint_refuses_noise_events():
    rng = np.random.default_rng(3)
    circ = W.noisy_su2_cz_circuit(10, 2, 0.1, rng)
    c = nt.Circuit(circ)
    ham = W.pauli_sum(10, [(1.0, {0: 3})])
    with pytest.raises(nt.TcError) as err:
        c.expect_grad(cuda_params(np.zeros((1, 0))), nt.Hamiltonian(ham), checkpoint_ops=5)
    assert err.value.status == nt.TC_E_UNSUPPORTED
