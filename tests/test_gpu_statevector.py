"""GPU parity: state vectors and Pauli sums against the FP64 oracle."""
import numpy as np
import pytest

from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64, TOL_AMP_C128, assert_energy_close, cuda_params

pytestmark = pytest.mark.gpu


def _gpu_states(circ, theta, dtype, **kw):
    import torch

    c = nt.Circuit(circ, dtype=dtype, **kw)
    out = c.apply(cuda_params(theta), theta.shape[0])
    torch.cuda.synchronize()
    return out.cpu().numpy(), c


def test_hea10_complex128_state_and_observables():
    circ, theta, obs = W.hea10_workload()
    got, c = _gpu_states(circ, theta, nt.TC_C128)
    ref = sv.run_circuit(circ, theta[0])
    assert np.abs(got[0] - ref).max() <= TOL_AMP_C128
    import torch

    st = torch.as_tensor(got, device="cuda")
    for o in obs:
        e = c.expect(st, nt.Hamiltonian(o)).cpu().numpy()
        assert abs(e[0] - sv.energy(ref, 10, o)[0]) <= 1e-12


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n,tile", [(2, 0), (5, 0), (9, 0), (11, 0), (13, 0), (14, 0), (15, 9), (16, 10)])
def test_random_circuits(n, tile, dtype):
    rng = np.random.default_rng(1000 + n + 17 * tile)
    circ = W.random_circuit(n, 6 * n + 10, rng)
    theta = rng.uniform(-3, 3, size=(3, circ.n_params))
    got, _ = _gpu_states(circ, theta, dtype, tile_fwd=tile)
    tol = TOL_AMP_C128 if dtype == nt.TC_C128 else TOL_AMP_C64
    for b in range(3):
        ref = sv.run_circuit(circ, theta[b])
        assert np.abs(got[b] - ref).max() <= tol, f"row {b}: {np.abs(got[b] - ref).max():.3e}"


@pytest.mark.parametrize("kind", [W.OP_H, W.OP_X, W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_U1])
def test_every_qubit_position_1q(kind):
    n = 14
    rng = np.random.default_rng(kind)
    for q in range(n):
        b = W.OpBuilder(n)
        for p in range(n):
            b.ry(p, p)  # generic product state
        if kind == W.OP_U1:
            b.unitary1(q, W.haar_unitary(2, rng))
        else:
            b._add(kind, q, param=n if kind in (W.OP_RX, W.OP_RY, W.OP_RZ) else -1)
        circ = b.build(n + 1)
        theta = rng.uniform(-3, 3, size=(1, n + 1))
        got, _ = _gpu_states(circ, theta, nt.TC_C128, tile_fwd=9)
        ref = sv.run_circuit(circ, theta[0])
        assert np.abs(got[0] - ref).max() <= 1e-12, f"qubit {q}"


@pytest.mark.parametrize("kind", [W.OP_CNOT, W.OP_CZ, W.OP_RZZ, W.OP_U2])
def test_every_qubit_pair_2q(kind):
    n = 11
    rng = np.random.default_rng(50 + kind)
    pairs = [(a, c) for a in range(n) for c in range(n) if a != c]
    rng.shuffle(pairs)
    for (q0, q1) in pairs[:40]:
        b = W.OpBuilder(n)
        for p in range(n):
            b.ry(p, p)
            b.rz(p, n + p)
        if kind == W.OP_U2:
            b.unitary2(q0, q1, W.haar_unitary(4, rng))
        else:
            b._add(kind, q0, q1, param=2 * n if kind == W.OP_RZZ else -1)
        circ = b.build(2 * n + 1)
        theta = rng.uniform(-3, 3, size=(1, 2 * n + 1))
        got, _ = _gpu_states(circ, theta, nt.TC_C128, tile_fwd=9)
        ref = sv.run_circuit(circ, theta[0])
        assert np.abs(got[0] - ref).max() <= 1e-12, f"pair {(q0, q1)}"


def test_init_states_and_batch_input():
    import torch

    rng = np.random.default_rng(3)
    for n in (4, 12):
        circ = W.random_circuit(n, 20, rng)
        theta = rng.uniform(-3, 3, size=(2, circ.n_params))
        psi0 = rng.standard_normal((2, 2 ** n)) + 1j * rng.standard_normal((2, 2 ** n))
        psi0 /= np.linalg.norm(psi0, axis=1, keepdims=True)
        c = nt.Circuit(circ, dtype=nt.TC_C128)
        out = c.apply(cuda_params(theta), 2, init=torch.as_tensor(psi0, device="cuda"))
        got = out.cpu().numpy()
        for b in range(2):
            ref = sv.run_circuit(circ, theta[b], init_state=psi0[b])
            assert np.abs(got[b] - ref).max() <= 1e-12


@pytest.mark.parametrize("n,tile", [(3, 0), (9, 0), (12, 0), (14, 9), (16, 11)])
def test_pauli_sum_random_terms(n, tile):
    import torch

    rng = np.random.default_rng(77 + n)
    psi = rng.standard_normal((3, 2 ** n)) + 1j * rng.standard_normal((3, 2 ** n))
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    ham = W.random_pauli_sum(n, 25, rng)  # any structure, including flips wider than a tile
    c = nt.Circuit(W.OpBuilder(n).build(), dtype=nt.TC_C128, tile_fwd=tile)
    got = c.expect(torch.as_tensor(psi, device="cuda"), nt.Hamiltonian(ham)).cpu().numpy()
    for b in range(3):
        ref = sv.energy(psi[b], n, ham)[0]
        assert abs(got[b] - ref) <= 1e-12 * max(1, abs(ref)) * 10


def test_pauli_sum_complex64_tfim():
    import torch

    n = 16
    rng = np.random.default_rng(8)
    psi = (rng.standard_normal((2, 2 ** n)) + 1j * rng.standard_normal((2, 2 ** n)))
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    ham = W.tfim_zz_x(n)
    c = nt.Circuit(W.OpBuilder(n).build(), dtype=nt.TC_C64)
    got = c.expect(torch.as_tensor(psi.astype(np.complex64), device="cuda"), nt.Hamiltonian(ham)).cpu().numpy()
    ref = [sv.energy(psi[b].astype(np.complex64).astype(np.complex128), n, ham)[0] for b in range(2)]
    assert_energy_close(got, ref)


def test_batch_row_alone_equals_in_batch():
    import torch

    circ, theta, ham = W.tfim_workload(n=14, layers=4, batch=8, seed=5)
    c = nt.Circuit(circ)
    allb = c.apply(cuda_params(theta), 8)
    one = c.apply(cuda_params(theta[5:6]), 1)
    torch.cuda.synchronize()
    assert torch.equal(allb[5:6], one)
    H = nt.Hamiltonian(ham)
    e_all = c.expect(allb, H)
    e_one = c.expect(one, H)
    assert torch.equal(e_all[5:6], e_one)


def test_plain_path_matches_fused():
    import torch

    circ, theta, ham = W.tfim_workload(n=12, layers=3, batch=2, seed=9)
    c = nt.Circuit(circ)
    H = nt.Hamiltonian(ham)
    work = torch.empty((2, 1 << 12), dtype=torch.complex64, device="cuda")
    e_plain = c.expect_plain(cuda_params(theta), H, work).cpu().numpy()
    ref = [sv.energy(sv.run_circuit(circ, theta[b]), 12, ham)[0] for b in range(2)]
    assert_energy_close(e_plain, ref)
