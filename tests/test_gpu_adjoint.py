"""GPU parity: adjoint energy + gradient against oracle parameter shift / finite differences."""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import assert_energy_close, assert_grad_close, cuda_params

pytestmark = pytest.mark.gpu


def _run(circ, theta, ham, dtype=nt.TC_C64, **kw):
    c = nt.Circuit(circ, dtype=dtype, **{k: v for k, v in kw.items() if k.startswith("tile")})
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham), max_rows=kw.get("max_rows", 0))
    return e.cpu().numpy(), g.cpu().numpy()


def test_batched_vqe_toy():
    b = W.OpBuilder(2)
    b.rx(0, 0)
    b.cnot(0, 1)
    b.rx(1, 1)
    circ = b.build()
    W_ = np.array([[0.1, 0.2], [0.3, 0.4]])
    zz = W.pauli_sum(2, [(1.0, {0: 3, 1: 3})])
    e, g = _run(circ, W_, zz, dtype=nt.TC_C128)
    np.testing.assert_allclose(e, np.cos(W_[:, 1]), atol=1e-13)
    np.testing.assert_allclose(g[:, 0], 0, atol=1e-13)
    np.testing.assert_allclose(g[:, 1], -np.sin(W_[:, 1]), atol=1e-13)


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n,tiles", [(4, (0, 0)), (10, (0, 0)), (12, (0, 0)), (14, (9, 9)), (15, (10, 9))])
def test_random_circuit_gradients(n, tiles, dtype):
    rng = np.random.default_rng(500 + n)
    kinds = [W.OP_H, W.OP_X, W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_RZZ, W.OP_CNOT, W.OP_CZ, W.OP_U1, W.OP_U2]
    circ = W.random_circuit(n, 3 * n + 8, rng, n_params=6, kinds=kinds)
    ham = W.random_pauli_sum(n, 8, rng)  # any structure, including flips wider than a tile
    theta = rng.uniform(-3, 3, size=(2, 6))
    e, g = _run(circ, theta, ham, dtype=dtype, tile_fwd=tiles[0], tile_bwd=tiles[1])
    for b in range(2):
        e_ref = sv.energy(sv.run_circuit(circ, theta[b]), n, ham)[0]
        g_ref = G.parameter_shift(circ, theta[b], ham)
        if dtype == nt.TC_C128:
            assert abs(e[b] - e_ref) <= 1e-11 * max(1, abs(e_ref))
            assert np.abs(g[b] - g_ref).max() <= 1e-10 * max(1, np.abs(g_ref).max())
        else:
            assert_energy_close(e[b:b + 1], [e_ref])
            assert_grad_close(g[b], g_ref)


@pytest.mark.parametrize("n,layers", [(8, 3), (12, 5), (16, 4)])
def test_tfim_gradients_vs_parameter_shift(n, layers):
    circ, theta, ham = W.tfim_workload(n=n, layers=layers, batch=3, seed=40 + n)
    e, g = _run(circ, theta, ham)
    for b in range(3):
        e_ref = sv.energy(sv.run_circuit(circ, theta[b]), n, ham)[0]
        assert_energy_close(e[b:b + 1], [e_ref])
        if n <= 12:
            assert_grad_close(g[b], G.parameter_shift(circ, theta[b], ham))
        else:
            assert_grad_close(g[b], G.finite_difference(circ, theta[b], ham, h=1e-5))


def test_tfim_zero_angles():
    circ, theta, ham = W.tfim_workload(n=20, layers=10, batch=2, seed=1)
    theta[:] = 0
    e, g = _run(circ, theta, ham)
    assert np.abs(e + 20).max() <= 1e-5 * 20
    assert np.abs(g).max() <= 1e-4


def test_chunked_rows_equal_unchunked():
    circ, theta, ham = W.tfim_workload(n=14, layers=3, batch=7, seed=3)
    e1, g1 = _run(circ, theta, ham)
    e2, g2 = _run(circ, theta, ham, max_rows=3)
    assert np.array_equal(e1, e2) and np.array_equal(g1, g2)


def test_tfim20_full_size_sampled_rows():
    """Full-size TFIM workload (20 qubits, 10 layers, batch 1024) in the launch
    configuration the benchmark times; rows sampled for the oracle."""
    circ, theta, ham = W.tfim_workload()
    e, g = _run(circ, theta, ham)
    assert e.shape == (1024,) and g.shape == (1024, 20)
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(g))
    rows = [0, 517, 1023]
    e_ref = [sv.energy(sv.run_circuit(circ, theta[b]), 20, ham)[0] for b in rows]
    assert_energy_close(e[rows], e_ref)
    # gradient: two (row, parameter) samples by central differences
    for b, k in ((517, 3), (1023, 18)):
        fd = G.finite_difference(circ, theta[b], ham, h=1e-4, params=[k])[k]
        assert abs(g[b, k] - fd) <= 1e-4 * max(1.0, np.abs(g[b]).max())
