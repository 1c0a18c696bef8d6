"""GPU parity: Pauli strings whose X/Y support is wider than one tile.

Section "Pauli structures and weights" (Eq. H-pauli) allows any structure
per term.  A term whose flip mask does not fit one shared-memory tile runs in
a paired Pauli-sum pass (each CTA holds a tile and its partner tile).  These
tests use full-width strings (X^n, Y^n, random X/Y/Z strings, several terms
sharing the bits outside the tile) at 14-20 qubits in both dtypes, energies
and adjoint gradients, against the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import assert_energy_close, assert_grad_close, cuda_params

pytestmark = pytest.mark.gpu


def _wide_sum(n, rng, n_random=6):
    """X^n, Y^n, an alternating X/Y string with a Z, strings that share their
    high flip bits, random X/Y-heavy strings and a few narrow terms."""
    terms = [
        (0.7, {q: 1 for q in range(n)}),
        (-0.4, {q: 2 for q in range(n)}),
        (0.3, {**{q: 1 + (q % 2) for q in range(n - 1)}, n - 1: 3}),
        # X on qubits 0..11 plus different low qubits: the same flip bits
        # outside the tile, so both share one paired pass
        (0.25, {**{q: 1 for q in range(12)}, n - 1: 2}),
        (-0.15, {**{q: 1 for q in range(12)}, n - 2: 1}),
        (0.5, {0: 3, 1: 3}),
        (-0.6, {n // 2: 1}),
    ]
    out = W.pauli_sum(n, terms)
    codes = rng.choice([0, 1, 2, 3], p=[0.1, 0.35, 0.35, 0.2], size=(n_random, n)).astype(np.uint8)
    w = rng.standard_normal(n_random)
    return W.PauliSum(np.concatenate([out.structures, codes]), np.concatenate([out.weights, w]))


def _random_states(rng, B, n):
    psi = rng.standard_normal((B, 2 ** n)) + 1j * rng.standard_normal((B, 2 ** n))
    return psi / np.linalg.norm(psi, axis=1, keepdims=True)


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n", [14, 16, 20])
def test_wide_strings_energy(n, dtype):
    import torch

    rng = np.random.default_rng(900 + n)
    psi = _random_states(rng, 2, n)
    ham = _wide_sum(n, rng)
    if dtype == nt.TC_C64:
        psi = psi.astype(np.complex64).astype(np.complex128)  # the oracle sees the stored values
    c = nt.Circuit(W.OpBuilder(n).build(), dtype=dtype)
    st = torch.as_tensor(psi.astype(np.complex64 if dtype == nt.TC_C64 else np.complex128), device="cuda")
    got = c.expect(st, nt.Hamiltonian(ham)).cpu().numpy()
    for b in range(2):
        ref = sv.energy(psi[b], n, ham)[0]
        if dtype == nt.TC_C128:
            assert abs(got[b] - ref) <= 1e-11 * max(1.0, abs(ref)), (b, got[b], ref)
        else:
            assert_energy_close(got[b:b + 1], [ref])


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_single_wide_terms_each(dtype):
    """One term at a time (X^n, Y^n and a Y-heavy string) on a 16-qubit GHZ-like
    state with phases, where <X^n> and <Y^n> are known in closed form too."""
    import torch

    n = 16
    # (|0..0> + e^{i phi}|1..1>)/sqrt(2): Y^n|0..0> = i^n |1..1>, so
    # <X^n> = cos(phi) and <Y^n> = Re(i^n e^{-i phi})
    phi = 0.37
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1 / np.sqrt(2)
    psi[-1] = np.exp(1j * phi) / np.sqrt(2)
    c = nt.Circuit(W.OpBuilder(n).build(), dtype=dtype)
    st = torch.as_tensor(psi[None].astype(np.complex64 if dtype == nt.TC_C64 else np.complex128), device="cuda")
    closed = {1: np.cos(phi), 2: np.real((1j) ** n * np.exp(-1j * phi))}
    tol = 1e-12 if dtype == nt.TC_C128 else 1e-6
    for code in (1, 2):
        ham = W.pauli_sum(n, [(1.0, {q: code for q in range(n)})])
        got = c.expect(st, nt.Hamiltonian(ham)).cpu().numpy()[0]
        assert abs(got - closed[code]) <= tol, (code, got, closed[code])
        assert abs(got - sv.energy(psi, n, ham)[0]) <= tol
    mixed = W.pauli_sum(n, [(1.0, {q: (2 if q % 3 else 1) for q in range(n)})])
    got = c.expect(st, nt.Hamiltonian(mixed)).cpu().numpy()[0]
    assert abs(got - sv.energy(psi, n, mixed)[0]) <= tol


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n", [14, 16])
def test_wide_strings_adjoint_gradient(n, dtype):
    rng = np.random.default_rng(950 + n)
    kinds = [W.OP_H, W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_RZZ, W.OP_CNOT, W.OP_CZ, W.OP_U1]
    circ = W.random_circuit(n, 2 * n + 6, rng, n_params=5, kinds=kinds)
    ham = _wide_sum(n, rng, n_random=4)
    theta = rng.uniform(-3, 3, size=(2, 5))
    c = nt.Circuit(circ, dtype=dtype)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
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


def test_wide_strings_gradient_20_qubits():
    """20 qubits, complex64, the TFIM ansatz with X^n, Y^n and random wide
    strings added to H; all 4 gradients of one row by central differences."""
    circ, theta, _ = W.tfim_workload(n=20, layers=2, batch=2, seed=31)
    rng = np.random.default_rng(31)
    ham = _wide_sum(20, rng, n_random=3)
    c = nt.Circuit(circ)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    e_ref = sv.energy(sv.run_circuit(circ, theta[1]), 20, ham)[0]
    assert_energy_close(e[1:2], [e_ref])
    fd = G.finite_difference(circ, theta[1], ham, h=1e-5)
    assert_grad_close(g[1], fd)


def test_wide_groups_share_a_pass_and_chunked_rows_agree():
    """Terms with the same bits outside the tile, and energy-only calls whose
    flip groups are split over several blocks, give the same energies as the
    gradient path's single-block passes."""
    import torch

    n = 18
    rng = np.random.default_rng(77)
    circ, theta, _ = W.tfim_workload(n=n, layers=2, batch=3, seed=77)
    ham = _wide_sum(n, rng, n_random=10)
    c = nt.Circuit(circ)
    H = nt.Hamiltonian(ham)
    e_grad, _ = c.expect_grad(cuda_params(theta), H)
    states = c.apply(cuda_params(theta), 3)
    e_only = c.expect(states, H)
    torch.cuda.synchronize()
    ref = [sv.energy(sv.run_circuit(circ, theta[b]), n, ham)[0] for b in range(3)]
    assert_energy_close(e_grad.cpu().numpy(), ref)
    assert_energy_close(e_only.cpu().numpy(), ref)
