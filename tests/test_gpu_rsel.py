"""GPU parity for random-axis rotations (unitary_kraus over RX, RY, RZ with a
status number per gate, Section "Demonstration of barren plateaus"): one
batch row per random circuit structure; states, energies and adjoint
gradients against the oracle on each row's structure."""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import noise as N
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64, TOL_AMP_C128, assert_energy_close, assert_grad_close, cuda_params

pytestmark = pytest.mark.gpu


def _rsel_circuit(n, layers, rng):
    b = W.OpBuilder(n)
    p = 0
    for l in range(layers):
        for q in range(n):
            b.rsel(q, p % 7, scale=float(rng.choice([1.0, 0.5, -2.0])))
            p += 1
        for q in range(l % 2, n - 1, 2):
            b.cz(q, q + 1)
        b.rzz(0, n - 1, 7)
        b.rx(n // 2, 8)
    return b.build(9)


def _n_events(circ):
    return int(np.sum((circ.ops["kind"] == W.OP_RSEL) | (circ.ops["kind"] == W.OP_PAULI_NOISE)))


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n", [4, 11, 14])
def test_rsel_states_with_status(n, dtype):
    import torch

    rng = np.random.default_rng(700 + n)
    circ = _rsel_circuit(n, 3, rng)
    B = 3
    theta = rng.uniform(-3, 3, size=(B, circ.n_params))
    status = rng.uniform(0, 1, size=(B, _n_events(circ))).astype(np.float32)
    c = nt.Circuit(circ, dtype=dtype)
    st = c.apply(cuda_params(theta), B, status=torch.as_tensor(status, device="cuda")).cpu().numpy()
    tol = TOL_AMP_C128 if dtype == nt.TC_C128 else TOL_AMP_C64
    for b in range(B):
        ref = sv.run_circuit(circ, theta[b], status_row=status[b].astype(np.float64))
        assert np.abs(st[b] - ref).max() <= tol


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n", [4, 11])
def test_rsel_energy_and_gradient_per_structure(n, dtype):
    rng = np.random.default_rng(710 + n)
    circ = _rsel_circuit(n, 3, rng)
    ham = W.random_pauli_sum(n, 6, rng)
    B, seed = 4, 711
    theta = rng.uniform(-3, 3, size=(B, circ.n_params))
    c = nt.Circuit(circ, dtype=dtype)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham), seed=seed)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    status = N.status_from_seed(seed, B, _n_events(circ))
    for b in range(B):
        e_ref = sv.energy(sv.run_circuit(circ, theta[b], status_row=status[b]), n, ham)[0]
        g_ref = G.parameter_shift(circ, theta[b], ham, status_row=status[b])
        if dtype == nt.TC_C128:
            assert abs(e[b] - e_ref) <= 1e-11 * max(1, abs(e_ref))
            assert np.abs(g[b] - g_ref).max() <= 1e-10 * max(1, np.abs(g_ref).max())
        else:
            assert_energy_close(e[b:b + 1], [e_ref])
            assert_grad_close(g[b], g_ref)


def test_bp_workload_rows_match_oracle():
    circ, theta, seed, ham = W.bp_workload(n=6, layers=4, structures=6)
    c = nt.Circuit(circ)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham), seed=seed)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    status = N.status_from_seed(seed, theta.shape[0], _n_events(circ))
    for b in range(theta.shape[0]):
        assert_energy_close(e[b:b + 1], [sv.energy(sv.run_circuit(circ, theta[b], status_row=status[b]), 6, ham)[0]])
        assert_grad_close(g[b], G.parameter_shift(circ, theta[b], ham, status_row=status[b]))


def test_bp_workload_full_size_sampled_rows():
    # the bench launch: 10 qubits x 10 layers, 100 structures in one call
    circ, theta, seed, ham = W.bp_workload()
    c = nt.Circuit(circ)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham), seed=seed)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    status = N.status_from_seed(seed, theta.shape[0], _n_events(circ))
    for b in (0, 57, 99):
        e_ref = sv.energy(sv.run_circuit(circ, theta[b], status_row=status[b]), circ.n, ham)[0]
        assert_energy_close(e[b:b + 1], [e_ref])
        assert_grad_close(g[b], G.parameter_shift(circ, theta[b], ham, status_row=status[b]))
