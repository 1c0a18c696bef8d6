"""GPU parity: the torch.autograd.Function over the adjoint sweep.

Section "Gradients, optimization and variational algorithms" (value_and_grad)
and Section "vmap and vectorized_value_and_grad" (per-row and summed forms):
gradients taken through torch.autograd.grad must equal the oracle's
parameter-shift gradients, weighted by the incoming gradient of each energy.
"""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import assert_energy_close, assert_grad_close

pytestmark = pytest.mark.gpu


def test_autograd_per_row_weighted_gradients():
    import torch

    circ, theta, ham = W.tfim_workload(n=12, layers=4, batch=5, seed=12)
    c = nt.Circuit(circ)
    H = nt.Hamiltonian(ham)
    th = torch.as_tensor(theta, device="cuda").requires_grad_(True)
    e = nt.expectation(c, th, H)
    w = torch.as_tensor(np.linspace(-1.0, 2.0, theta.shape[0]), device="cuda")
    (g,) = torch.autograd.grad((w * e).sum(), th)
    e, g, w = e.detach().cpu().numpy(), g.cpu().numpy(), w.cpu().numpy()
    for b in range(theta.shape[0]):
        e_ref = sv.energy(sv.run_circuit(circ, theta[b]), circ.n, ham)[0]
        assert_energy_close(e[b:b + 1], [e_ref])
        assert_grad_close(g[b], w[b] * G.parameter_shift(circ, theta[b], ham))


def test_autograd_summed_over_rows():
    """One parameter vector shared by every row (expanded to [B][P]): its
    gradient is the sum of the rows' gradients."""
    import torch

    circ, theta, ham = W.tfim_workload(n=10, layers=3, batch=1, seed=3)
    c = nt.Circuit(circ, dtype=nt.TC_C128)
    H = nt.Hamiltonian(ham)
    base = torch.as_tensor(theta[0], device="cuda").requires_grad_(True)
    B = 4
    e = nt.expectation(c, base.expand(B, -1), H)
    (g,) = torch.autograd.grad(e.sum(), base)
    ref = B * G.parameter_shift(circ, theta[0], ham)
    assert np.abs(g.cpu().numpy() - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


def test_autograd_optimiser_step_lowers_energy():
    """A few Adam steps through the Function lower the TFIM energy (a use of
    the Function, as the paper's VQE loops use value_and_grad)."""
    import torch

    circ, theta, ham = W.tfim_workload(n=10, layers=3, batch=2, seed=8)
    c = nt.Circuit(circ)
    H = nt.Hamiltonian(ham)
    th = torch.nn.Parameter(torch.as_tensor(theta, device="cuda"))
    opt = torch.optim.Adam([th], lr=0.05)
    e0 = nt.expectation(c, th, H).detach().clone()
    for _ in range(20):
        opt.zero_grad()
        nt.expectation(c, th, H).sum().backward()
        opt.step()
    e1 = nt.expectation(c, th, H).detach()
    assert torch.all(e1 < e0)
