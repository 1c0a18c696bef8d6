"""GPU edge cases through the bindings: zero rows on every batched call
(empty tensors, whose device pointers are NULL), an empty Pauli sum, and a
circuit without gates, against what the definitions give (Eq. H-pauli: an
empty sum is 0; no gates leave the initial state)."""
import numpy as np
import pytest

from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64, assert_energy_close, cuda_params

pytestmark = pytest.mark.gpu


def _circuit(n):
    b = W.OpBuilder(n, W.INIT_PLUS)
    for q in range(n):
        b.rx(q, 0)
    for q in range(n - 1):
        b.rzz(q, q + 1, 1)
    return b.build(2)


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_zero_rows_everywhere(dtype):
    import torch

    n = 12
    c = nt.Circuit(_circuit(n), dtype=dtype)
    H = nt.Hamiltonian(W.tfim_zz_x(n))
    p0 = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    st = c.apply(p0, 0)
    assert st.shape == (0, 1 << n)
    assert c.expect(st, H).shape == (0,)
    e, g = c.expect_grad(p0, H)
    assert e.shape == (0,) and g.shape == (0, 2)
    assert c.norms(st).shape == (0,)
    assert c.qgt(p0).shape == (0, 2, 2)
    states, vals = c.apply_expect(p0, nt.Observables([W.tfim_zz_x(n)]), 0)
    assert vals.shape == (0, 1)
    n_lc, gates, zq = W.brick200_workload()
    lc = nt.LightCone(n_lc, [(a, q) for a, q, _ in gates], zq, greedy_trials=64)
    assert lc.contract(torch.empty((0, len(gates), 4, 4), dtype=torch.complex64, device="cuda")).shape == (0, 2)
    net = nt.CircuitNetwork(W.example_block_circuit(40, 6), {20: 3}, prune=2)
    assert net.expect(torch.empty((0, net.n_params), dtype=torch.float32, device="cuda")).shape == (0, 2)
    torch.cuda.synchronize()


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_empty_pauli_sum_gives_zero_energy_and_gradient(dtype):
    n = 14
    c = nt.Circuit(_circuit(n), dtype=dtype)
    empty = nt.Hamiltonian(W.PauliSum(np.zeros((0, n), np.uint8), np.zeros(0)))
    theta = np.random.default_rng(3).uniform(-1, 1, size=(3, 2))
    e, g = c.expect_grad(cuda_params(theta), empty)
    assert np.all(e.cpu().numpy() == 0.0) and np.all(g.cpu().numpy() == 0.0)
    st = c.apply(cuda_params(theta), 3)
    assert np.all(c.expect(st, empty).cpu().numpy() == 0.0)


@pytest.mark.parametrize("init", [W.INIT_ZERO, W.INIT_PLUS])
def test_circuit_without_gates(init):
    n = 16
    circ = W.OpBuilder(n, init).build()
    c = nt.Circuit(circ)
    st = c.apply(None, 2).cpu().numpy()
    ref = sv.run_circuit(circ)
    assert np.abs(st - ref[None]).max() <= TOL_AMP_C64
    ham = W.pauli_sum(n, [(0.5, {0: 3}), (-1.25, {3: 1, 9: 1}), (2.0, {15: 2})])
    e, _ = c.expect_grad(cuda_params(np.zeros((2, 0))), nt.Hamiltonian(ham))
    # |0..0>: <Z_0> = 1, X X and Y give 0; |+>^n: <X_3 X_9> = 1, Z and Y give 0
    want = 0.5 if init == W.INIT_ZERO else -1.25
    assert_energy_close(e.cpu().numpy(), [want, want])
    assert_energy_close(e.cpu().numpy(), [sv.energy(ref, n, ham)[0]] * 2)
