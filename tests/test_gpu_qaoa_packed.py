"""GPU parity: QAOA cost layers evaluated as packed diagonal groups.

A cost layer on a random 3-regular graph has ZZ pairs at many index
distances; the planner turns it into one 64-bit column word per qubit
position and the kernels count the cut edges of an amplitude index with an
XOR walk and a popcount.  States, energies and adjoint gradients are checked
against the FP64 oracle (Sec. 5: the QAOA MaxCut example; gradients by the
parameter-shift rule), through the plan-interpreting and the specialised
kernels, at widths that put graph edges inside and outside a tile.
"""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64, TOL_AMP_C128, assert_energy_close, assert_grad_close, cuda_params
from qaoa_cone import edge_cone

pytestmark = pytest.mark.gpu


def _maxcut(n, edges):
    return W.pauli_sum(n, [(0.5, {u: 3, v: 3}) for (u, v) in edges])


@pytest.mark.parametrize("specialize", [False, True])
@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n", [12, 18])
def test_qaoa_states_energies_gradients(n, dtype, specialize):
    import torch

    rng = np.random.default_rng(600 + n)
    edges = W.random_regular3(n, rng)
    # the shift rule runs the circuit twice per gate occurrence: one layer at 18 qubits
    p = 3 if n <= 12 else 1
    circ = W.qaoa_circuit(n, edges, p)
    ham = _maxcut(n, edges)
    theta = rng.uniform(0.0, np.pi, size=(3, 2 * p))
    c = nt.Circuit(circ, dtype=dtype, specialize=specialize)
    assert c.info()["packed_diag_groups"] >= p
    st = c.apply(cuda_params(theta), 3)
    torch.cuda.synchronize()
    got = st.cpu().numpy()
    tol = TOL_AMP_C128 if dtype == nt.TC_C128 else TOL_AMP_C64
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    for b in range(3):
        ref = sv.run_circuit(circ, theta[b])
        assert np.abs(got[b] - ref).max() <= tol
        e_ref = sv.energy(ref, n, ham)[0]
        if n > 12 and b > 0:
            assert_energy_close(e[b:b + 1], [e_ref])
            continue
        g_ref = G.parameter_shift(circ, theta[b], ham)
        if dtype == nt.TC_C128:
            assert abs(e[b] - e_ref) <= 1e-11 * max(1, abs(e_ref))
            assert np.abs(g[b] - g_ref).max() <= 1e-10 * max(1, np.abs(g_ref).max())
        else:
            assert_energy_close(e[b:b + 1], [e_ref])
            assert_grad_close(g[b], g_ref)


def test_qaoa_64_edge_layer_at_the_word_limit():
    """A layer of exactly 64 terms fills the column word."""
    rng = np.random.default_rng(77)
    n = 16
    pairs = [(u, v) for u in range(n) for v in range(u + 1, n)]
    idx = rng.choice(len(pairs), size=64, replace=False)
    edges = [pairs[i] for i in sorted(idx)]
    circ = W.qaoa_circuit(n, edges, 1)
    ham = _maxcut(n, edges)
    theta = rng.uniform(0.0, np.pi, size=(2, 2))
    c = nt.Circuit(circ)
    assert c.info()["packed_diag_groups"] >= 1
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    for b in range(2):
        assert_energy_close(e[b:b + 1], [sv.energy(sv.run_circuit(circ, theta[b]), n, ham)[0]])
        assert_grad_close(g[b], G.finite_difference(circ, theta[b], ham))


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_packed_pauli_sum_terms_next_to_other_terms(dtype):
    """Pauli sum with a packed group (ZZ of one weight on a 3-regular graph)
    followed by single Z, a ZZ bond of another weight, a ZZZ parity term and
    X / Y strings: energies and gradients against the oracle."""
    rng = np.random.default_rng(91)
    n = 14
    edges = W.random_regular3(n, rng)
    terms = [(0.75, {u: 3, v: 3}) for (u, v) in edges]
    terms += [(0.3, {q: 3}) for q in range(0, n, 3)]
    terms += [(-1.1, {2: 3, 3: 3}), (0.4, {1: 3, 6: 3, 11: 3}), (0.6, {5: 1}), (-0.2, {0: 2, 9: 1})]
    ham = W.pauli_sum(n, terms)
    circ = W.random_circuit(n, 3 * n, rng, n_params=5, kinds=[W.OP_RX, W.OP_RY, W.OP_RZZ, W.OP_CNOT, W.OP_H])
    theta = rng.uniform(-3, 3, size=(2, 5))
    c = nt.Circuit(circ, dtype=dtype)
    H = nt.Hamiltonian(ham)
    assert c.pauli_sum_info(H)["packed_diag_groups"] == 1
    e, g = c.expect_grad(cuda_params(theta), H)
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


@pytest.mark.parametrize("p,dtype,specialize", [(1, nt.TC_C64, False), (1, nt.TC_C64, True), (1, nt.TC_C128, False),
                                                (2, nt.TC_C64, False)])
def test_qaoa26_full_width_against_edge_light_cones(p, dtype, specialize):
    """The serving stream's widest request: MaxCut QAOA on a random 3-regular
    graph of 26 qubits (H = sum over edges of Z_u Z_v).  The oracle evaluates
    each edge's term and its parameter-shift gradient on that edge's light cone
    (at most 6 qubits for p = 1, 14 for p = 2) in FP64; the sums are the exact
    26-qubit energy and gradient."""
    n = 26
    rng = np.random.default_rng(2600 + p)
    edges = W.random_regular3(n, rng)
    circ = W.qaoa_circuit(n, edges, p)
    ham = W.zz_on_edges(n, edges)
    theta = rng.uniform(0.0, np.pi, size=(2, 2 * p))
    c = nt.Circuit(circ, dtype=dtype, specialize=specialize)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    cones = [edge_cone(circ, u, v) for (u, v) in edges]
    assert max(cc.n for cc, _ in cones) <= (6 if p == 1 else 14)
    for b in range(2):
        e_ref = sum(sv.energy(sv.run_circuit(cc, theta[b]), cc.n, hh)[0] for cc, hh in cones)
        g_ref = sum(G.parameter_shift(cc, theta[b], hh) for cc, hh in cones)
        if dtype == nt.TC_C128:
            assert abs(e[b] - e_ref) <= 1e-10 * max(1, abs(e_ref))
            assert np.abs(g[b] - g_ref).max() <= 1e-9 * max(1, np.abs(g_ref).max())
        else:
            assert_energy_close(e[b:b + 1], [e_ref])
            assert_grad_close(g[b], g_ref)
