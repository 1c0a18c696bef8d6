"""GPU parity: pass kernels specialised per circuit at plan time (tc_options.specialize).

The specialised kernels run the same gate-pass code as the plan-interpreting
kernels with the plan compiled in; their states, energies and gradients are
checked against the FP64 oracle (states of random circuits with every gate
kind and noise outcomes, adjoint gradients against parameter shift) and
against the interpreting kernels on the same inputs.
"""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import noise as N
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64, TOL_AMP_C128, assert_energy_close, assert_grad_close, cuda_params

pytestmark = pytest.mark.gpu

KINDS = [W.OP_H, W.OP_X, W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_RZZ, W.OP_CNOT, W.OP_CZ, W.OP_U1, W.OP_U2]


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n", [10, 14])
def test_random_circuit_states_and_gradients(n, dtype):
    import torch

    rng = np.random.default_rng(4000 + n)
    circ = W.random_circuit(n, 4 * n, rng, n_params=6, kinds=KINDS)
    ham = W.random_pauli_sum(n, 6, rng)
    theta = rng.uniform(-3, 3, size=(2, 6))
    cs = nt.Circuit(circ, dtype=dtype, specialize=True)
    ci = nt.Circuit(circ, dtype=dtype)
    st_s = cs.apply(cuda_params(theta), 2)
    st_i = ci.apply(cuda_params(theta), 2)
    torch.cuda.synchronize()
    tol = TOL_AMP_C128 if dtype == nt.TC_C128 else TOL_AMP_C64
    got = st_s.cpu().numpy()
    for b in range(2):
        assert np.abs(got[b] - sv.run_circuit(circ, theta[b])).max() <= tol
    assert np.abs(got - st_i.cpu().numpy()).max() <= tol
    e, g = cs.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    for b in range(2):
        e_ref = sv.energy(sv.run_circuit(circ, theta[b]), n, ham)[0]
        g_ref = G.parameter_shift(circ, theta[b], ham)
        if dtype == nt.TC_C128:
            assert abs(e[b] - e_ref) <= 1e-11 * max(1, abs(e_ref))
            assert np.abs(g[b] - g_ref).max() <= 1e-10 * max(1, np.abs(g_ref).max())
        else:
            assert_energy_close(e[b:b + 1], [e_ref])
            assert_grad_close(g[b], g_ref)


def test_tfim20_batch_matches_interpreter_and_oracle():
    """The benchmark's circuit (20 qubits, 10 layers) on 64 rows."""
    circ, theta, ham = W.tfim_workload(n=20, layers=10, batch=64, seed=77)
    H = nt.Hamiltonian(ham)
    e_s, g_s = nt.Circuit(circ, specialize=True).expect_grad(cuda_params(theta), H)
    e_i, g_i = nt.Circuit(circ).expect_grad(cuda_params(theta), H)
    e_s, g_s, e_i, g_i = (x.cpu().numpy() for x in (e_s, g_s, e_i, g_i))
    assert np.abs(e_s - e_i).max() <= 1e-5 * max(1.0, np.abs(e_i).max())
    assert np.abs(g_s - g_i).max() <= 1e-5 * max(1.0, np.abs(g_i).max())
    b = 17
    assert_energy_close(e_s[b:b + 1], [sv.energy(sv.run_circuit(circ, theta[b]), 20, ham)[0]])


def test_noise_outcomes_match_oracle_stream():
    rng = np.random.default_rng(31)
    circ = W.noisy_su2_cz_circuit(11, 5, 0.3, rng)
    c = nt.Circuit(circ, specialize=True)
    out = c.apply(None, 12, seed=987654321, row_offset=5).cpu().numpy()
    st = N.status_from_seed(987654321, 12, circ.n_noise, traj_offset=5)
    for b in range(12):
        assert np.abs(out[b] - sv.run_circuit(circ, None, status_row=st[b])).max() <= TOL_AMP_C64
