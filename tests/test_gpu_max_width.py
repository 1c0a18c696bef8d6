"""GPU parity at the engine's widest register, 30 qubits (8 GiB per complex64
state), against closed forms.

RY(theta) on qubit 0, then CNOT(q, q + 1) for q = 0..28, from |0...0> gives
cos(theta/2)|0...0> + sin(theta/2)|1...1> (Section "Circuits and gates"; RY =
exp(-i theta Y / 2), qubit 0 the most significant bit).  Its expectations:
  <Z_0> = cos(theta),  <Z_0 Z_29> = 1,  <X^(x)30> = sin(theta),
  <Y_0 Y_1 X_2 ... X_29> = -sin(theta)
(both strings flip every qubit, so only the cross terms of the two basis states
contribute; Y|0> = i|1>, Y|1> = -i|0> gives the factor -1 for two Y), and
dE/dtheta follows term by term.  The full-width strings run as paired
Pauli-sum passes, the CNOT chain crosses every tile boundary."""
import numpy as np
import pytest

from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64, assert_energy_close, assert_grad_close, cuda_params

pytestmark = pytest.mark.gpu

N = 30
WEIGHTS = (0.7, -0.4, 0.3, 0.9)  # X^30, Z_0, Z_0 Z_29, Y_0 Y_1 X_2..X_29


def _circuit():
    b = W.OpBuilder(N, W.INIT_ZERO)
    b.ry(0, 0)
    for q in range(N - 1):
        b.cnot(q, q + 1)
    return b.build(1)


def _hamiltonian():
    ystr = {0: 2, 1: 2}
    ystr.update({q: 1 for q in range(2, N)})
    return W.pauli_sum(N, [(WEIGHTS[0], {q: 1 for q in range(N)}), (WEIGHTS[1], {0: 3}),
                           (WEIGHTS[2], {0: 3, N - 1: 3}), (WEIGHTS[3], ystr)])


def _closed_form(theta):
    wx, wz, wzz, wy = WEIGHTS
    e = (wx - wy) * np.sin(theta) + wz * np.cos(theta) + wzz
    g = (wx - wy) * np.cos(theta) - wz * np.sin(theta)
    return e, g


def test_state_at_30_qubits():
    import torch

    theta = np.array([[0.37], [2.9]])
    c = nt.Circuit(_circuit())
    st = c.apply(cuda_params(theta), 2)
    norms = c.norms(st).cpu().numpy()
    rng = np.random.default_rng(30)
    others = torch.as_tensor(rng.integers(1, (1 << N) - 1, size=64), device="cuda")
    for b in range(2):
        a0 = complex(st[b, 0].item())
        a1 = complex(st[b, (1 << N) - 1].item())
        assert abs(a0 - np.cos(theta[b, 0] / 2)) <= TOL_AMP_C64
        assert abs(a1 - np.sin(theta[b, 0] / 2)) <= TOL_AMP_C64
        assert float(st[b, others].abs().max().item()) == 0.0
        assert abs(norms[b] - 1.0) <= 1e-5
    del st
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_energy_gradient_at_30_qubits(dtype):
    import torch

    theta = np.array([[0.37], [2.9]]) if dtype == nt.TC_C64 else np.array([[1.1]])
    c = nt.Circuit(_circuit(), dtype=dtype)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(_hamiltonian()))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    for b in range(theta.shape[0]):
        e_ref, g_ref = _closed_form(theta[b, 0])
        if dtype == nt.TC_C128:
            assert abs(e[b] - e_ref) <= 1e-11 * max(1.0, abs(e_ref))
            assert abs(g[b, 0] - g_ref) <= 1e-10 * max(1.0, abs(g_ref))
        else:
            assert_energy_close(e[b:b + 1], [e_ref])
            assert_grad_close(g[b], [g_ref])
    torch.cuda.empty_cache()
