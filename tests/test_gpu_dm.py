"""GPU parity for density-matrix circuits (Section "Density matrix simulator"):
rho under gates and exact Pauli channels, held as a vectorised 2n-qubit state,
against the oracle's density matrix; expectations tr(rho H); and the
trajectory estimate of Section "Batched Monte Carlo trajectory noise
simulation" against the exact value."""
import numpy as np
import pytest

from oracle import noise as N
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64, TOL_AMP_C128, assert_energy_close, cuda_params

pytestmark = pytest.mark.gpu

KINDS = [W.OP_H, W.OP_X, W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_RZZ, W.OP_CNOT, W.OP_CZ, W.OP_U1, W.OP_U2,
         W.OP_PAULI_NOISE, W.OP_PAULI_NOISE]


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n", [2, 3, 5, 7])
def test_dm_matches_oracle(n, dtype):
    import torch

    rng = np.random.default_rng(600 + n)
    circ = W.random_circuit(n, 6 * n + 6, rng, n_params=4, kinds=KINDS)
    theta = rng.uniform(-3, 3, size=(2, 4))
    c = nt.DensityMatrixCircuit(circ, dtype=dtype)
    rho = c.apply(cuda_params(theta), 2)
    torch.cuda.synchronize()
    got = rho.cpu().numpy()
    ham = W.random_pauli_sum(n, 6, rng)
    e = c.expect(rho, nt.Hamiltonian(ham)).cpu().numpy()
    tol = TOL_AMP_C128 if dtype == nt.TC_C128 else TOL_AMP_C64
    d = 1 << n
    for b in range(2):
        ref = N.density_matrix(circ, theta[b])
        err = np.abs(got[b].reshape(d, d) - ref).max()
        assert err <= tol, f"row {b}: max |d rho| {err:.3e}"
        e_ref = N.dm_expectation(ref, n, ham)
        if dtype == nt.TC_C128:
            assert abs(e[b] - e_ref) <= 1e-11 * max(1.0, abs(e_ref))
        else:
            assert_energy_close(e[b:b + 1], [e_ref])


def test_dm_trace_hermitian_and_pure_limit():
    import torch

    n = 6
    rng = np.random.default_rng(610)
    circ = W.random_circuit(n, 40, rng, n_params=3, kinds=KINDS[:10])  # no channels: rho stays pure
    theta = rng.uniform(-3, 3, size=(1, 3))
    c = nt.DensityMatrixCircuit(circ, dtype=nt.TC_C128)
    rho = c.apply(cuda_params(theta), 1)
    torch.cuda.synchronize()
    r = rho.cpu().numpy()[0].reshape(1 << n, 1 << n)
    psi = sv.run_circuit(circ, theta[0])
    assert np.abs(r - np.outer(psi, psi.conj())).max() <= 1e-12
    assert np.abs(r - r.conj().T).max() <= 1e-13
    ident = W.pauli_sum(n, [(1.0, {})])
    assert abs(c.expect(rho, nt.Hamiltonian(ident)).item() - 1.0) <= 1e-12


def test_dm_exact_vs_trajectories():
    n, layers, p = 8, 6, 0.03
    circ = W.noisy_su2_cz_circuit(n, layers, p, np.random.default_rng(620))
    obs = [W.pauli_sum(n, [(1.0, {0: 3})]), W.pauli_sum(n, [(1.0, {i: 3, i + 1: 3}) for i in range(n - 1)])]
    dm = nt.DensityMatrixCircuit(circ)
    rho = dm.apply(None, 1)
    exact = [dm.expect(rho, nt.Hamiltonian(o)).item() for o in obs]
    ref = N.density_matrix(circ)
    for o, x in zip(obs, exact):
        assert abs(x - N.dm_expectation(ref, n, o)) <= 1e-5
    c = nt.Circuit(circ)
    n_traj = 8192
    st = c.apply(None, n_traj, seed=621)
    for o, x in zip(obs, exact):
        v = c.expect(st, nt.Hamiltonian(o))
        ms = nt.mean_stderr(v).cpu().numpy()
        assert abs(ms[0] - x) <= 5 * ms[1] + 1e-6, (ms, x)
