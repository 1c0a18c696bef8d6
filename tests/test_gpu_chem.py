"""GPU parity for a many-term, chemistry-shaped Pauli sum (12 qubits, 1390
terms in 531 flip groups: the shape of the paper's H2O example in Section
"Expectations of Hamiltonians"), energies and gradients against the oracle."""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import assert_energy_close, assert_grad_close, cuda_params

pytestmark = pytest.mark.gpu


def _states(n, B, dtype, seed):
    rng = np.random.default_rng(seed)
    circ = W.random_circuit(n, 8 * n, rng)
    theta = rng.uniform(-3, 3, size=(B, circ.n_params))
    import torch

    c = nt.Circuit(circ, dtype=dtype)
    st = c.apply(cuda_params(theta), B)
    torch.cuda.synchronize()
    return c, st, [sv.run_circuit(circ, theta[b]) for b in range(B)]


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_chem12_energy(dtype):
    n = 12
    ham = W.chem_pauli_sum(n)
    c, st, refs = _states(n, 3, dtype, 91)
    e = c.expect(st, nt.Hamiltonian(ham)).cpu().numpy()
    ref = np.array([sv.energy(r, n, ham)[0] for r in refs])
    if dtype == nt.TC_C128:
        np.testing.assert_allclose(e, ref, rtol=0, atol=1e-11 * max(1.0, np.abs(ref).max()))
    else:
        assert_energy_close(e, ref)


def test_chem12_gradient():
    n = 12
    ham = W.chem_pauli_sum(n)
    b = W.OpBuilder(n)
    for layer in range(2):
        for q in range(n):
            b.ry(q, 2 * layer)
        for q in range(n - 1):
            b.rzz(q, q + 1, 2 * layer + 1)
        for q in range(n):
            b.rx(q, 4 + layer, scale=0.5 + 0.1 * q)
    circ = b.build(n_params=6)
    theta = np.random.default_rng(92).uniform(-2, 2, size=(2, 6))
    c = nt.Circuit(circ)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    for r in range(2):
        assert_energy_close(e[r:r + 1], [sv.energy(sv.run_circuit(circ, theta[r]), n, ham)[0]])
        assert_grad_close(g[r], G.finite_difference(circ, theta[r], ham))
