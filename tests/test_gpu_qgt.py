"""GPU parity for the quantum geometric tensor (tc_qgt, Section "Quantum
Fisher Information") against the oracle's product-rule state derivatives."""
import numpy as np
import pytest

from oracle import gradients as G
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import cuda_params

pytestmark = pytest.mark.gpu

# G_ij sums c_k c_l <psi_k|psi_l> over the occurrences k of i and l of j
# (c = s / 2), minus a product of two such sums: an overlap error delta
# becomes at most 2 W_i W_j delta, W_i = sum_k |c_k|.  delta: complex64
# states (FP32 gates, ~1e-6 per overlap of unit vectors) / complex128.
DELTA = {nt.TC_C64: 2e-6, nt.TC_C128: 2e-12}


def _tol(circ, dtype):
    w = np.zeros(circ.n_params)
    for op in circ.ops:
        if int(op["param"]) >= 0:
            w[int(op["param"])] += abs(float(op["scale"])) / 2
    return 2 * DELTA[dtype] * max(1.0, w.max()) ** 2


def _circuit(n, rng, layers=2):
    b = W.OpBuilder(n, W.INIT_ZERO if n % 2 else W.INIT_PLUS)
    p = 0
    for _ in range(layers):
        for q in range(n):
            b.ry(q, p + q % 3, scale=float(rng.choice([1.0, -0.5, 2.0])))
        p += 3
        for q in range(n - 1):
            b.rzz(q, q + 1, p, scale=-2.0)  # one angle over the chain
        b.cnot(0, n - 1)
        b.unitary1(1, W.haar_unitary(2, rng))
        for q in range(0, n, 2):
            b.rx(q, p + 1)
        b.rz(n // 2, p + 2)
        p += 3
    return b.build(p + 1)  # the last parameter drives no gate: zero row and column


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n", [3, 10, 12])
def test_qgt_matches_oracle(n, dtype):
    rng = np.random.default_rng(900 + n)
    circ = _circuit(n, rng)
    B = 3
    theta = rng.uniform(-2.5, 2.5, size=(B, circ.n_params))
    c = nt.Circuit(circ, dtype=dtype)
    g = c.qgt(cuda_params(theta)).cpu().numpy()
    for b in range(B):
        ref = G.quantum_geometric_tensor(circ, theta[b])
        assert np.abs(g[b] - ref).max() <= _tol(circ, dtype)
        assert np.abs(g[b, -1]).max() == 0 and np.abs(g[b, :, -1]).max() == 0


def test_qgt_tfim_rows_chunked():
    circ, theta, _ = W.tfim_workload(10, 2, 4)
    # a budget below two rows' scratch forces one row per chunk
    c = nt.Circuit(circ, mem_budget_bytes=1 << 20)
    g = c.qgt(cuda_params(theta)).cpu().numpy()
    for b in range(4):
        assert np.abs(g[b] - G.quantum_geometric_tensor(circ, theta[b])).max() <= _tol(circ, nt.TC_C64)


def test_qgt_unsupported_and_empty():
    b = W.OpBuilder(4)
    b.ry(0, 0)
    b.depolarizing(1, 0.1, 0.1, 0.1)
    c = nt.Circuit(b.build())
    with pytest.raises(nt.TcError) as e:
        c.qgt(cuda_params(np.zeros((1, 1))))
    assert e.value.status == nt.TC_E_UNSUPPORTED
    b = W.OpBuilder(4)
    b.h(0)
    c = nt.Circuit(b.build(2))  # parameters that drive no gate
    assert np.abs(c.qgt(cuda_params(np.ones((2, 2)))).cpu().numpy()).max() == 0


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_qgt_commuting_insertions(dtype):
    # generators that move past commuting gates before their insertion point
    rng = np.random.default_rng(931)
    n = 5
    b = W.OpBuilder(n, W.INIT_PLUS)
    b.rx(2, 0)
    b.cnot(4, 2)          # X on the target commutes
    b.rx(2, 0, scale=-0.5)  # same axis
    b.rz(1, 1)
    b.cnot(1, 3)          # Z on the control commutes
    b.unitary1(1, np.diag(np.exp(1j * rng.uniform(0, 6, 2))))  # diagonal U1
    b.rzz(0, 1, 2)
    b.unitary2(0, 1, np.diag(np.exp(1j * rng.uniform(0, 6, 4))))  # diagonal U2
    b.cz(0, 3)
    b.ry(3, 3)
    b.ry(3, 3, scale=2.0)
    b.h(0)                # stops Z-type generators on qubit 0
    b.rz(4, 1)            # the last gate: its generator moves to the end
    circ = b.build()
    theta = rng.uniform(-2.5, 2.5, size=(2, circ.n_params))
    g = nt.Circuit(circ, dtype=dtype).qgt(cuda_params(theta)).cpu().numpy()
    for r in range(2):
        assert np.abs(g[r] - G.quantum_geometric_tensor(circ, theta[r])).max() <= _tol(circ, dtype)


def test_natural_gradient_solve_and_pipeline():
    import torch

    circ, theta, ham = W.tfim_workload(10, 2, 3)
    c = nt.Circuit(circ)
    d = cuda_params(theta)
    q = c.qgt(d)
    _, grad = c.expect_grad(d, nt.Hamiltonian(ham))
    eps = 0.05
    x = nt.natural_gradient(q, grad, eps).cpu().numpy()
    qn, gn = q.cpu().numpy(), grad.cpu().numpy()
    for r in range(3):
        # the solve itself, on the same inputs (FP64 Cholesky vs LAPACK); the
        # device reads the lower triangle of 4 Re G (complex64 makes it
        # symmetric only to rounding)
        low = np.tril(4.0 * qn[r].real)
        ref = np.linalg.solve(low + np.tril(low, -1).T + eps * np.eye(low.shape[0]), gn[r])
        assert np.abs(x[r] - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
        # the whole pipeline against the oracle's tensor and parameter-shift gradient
        ref_o = G.natural_gradient(G.quantum_geometric_tensor(circ, theta[r]),
                                   G.parameter_shift(circ, theta[r], ham), eps)
        assert np.abs(x[r] - ref_o).max() <= 1e-2 * max(1.0, np.abs(ref_o).max())
    with pytest.raises(nt.TcError):
        nt.natural_gradient(q, grad, 0.0)
    bad = torch.zeros((1, 2, 2), dtype=torch.complex128, device="cuda")
    bad[0, 0, 0] = -1.0
    with pytest.raises(nt.TcError) as e:
        nt.natural_gradient(bad, torch.ones((1, 2), dtype=torch.float64, device="cuda"), 1e-3)
    assert e.value.status == nt.TC_E_INVALID


def test_qgt_full_size_tfim20_closed_form_at_zero_angles():
    # the bench's 20-qubit, 10-layer ansatz at theta = 0: every gate is the
    # identity on |+>^20, d_l psi = -(i/2) sum_j Z_j Z_{j+1} psi for a ZZ-layer
    # angle and -(i/2) sum_j X_j psi = -10 i psi for an RX-layer angle, so
    # 4 Re G = Var(sum_j Z_j Z_{j+1}) = 19 between any two ZZ-layer angles and 0
    # elsewhere (X-sum acts as a scalar on |+>^20), and Im G = 0
    circ, _, _ = W.tfim_workload(20, 10, 1)
    c = nt.Circuit(circ)
    g = c.qgt(cuda_params(np.zeros((1, circ.n_params)))).cpu().numpy()[0]
    qfi = 4 * g.real
    ref = np.zeros_like(qfi)
    ref[0::2, 0::2] = 19.0
    tol = 4 * _tol(circ, nt.TC_C64)
    assert np.abs(qfi - ref).max() <= tol
    assert np.abs(g.imag).max() <= tol


def test_natural_gradient_pipeline_complex128_tight():
    """The QGT -> natural-gradient pipeline in complex128 against the oracle's
    tensor and parameter-shift gradient: every stage in FP64, so the solve's
    result agrees to 1e-8 relative (the solve amplifies the ~1e-13 input errors
    by the condition number of 4 Re G + eps I, below 1e4 here)."""
    circ, theta, ham = W.tfim_workload(10, 2, 3)
    c = nt.Circuit(circ, dtype=nt.TC_C128)
    d = cuda_params(theta)
    q = c.qgt(d)
    _, grad = c.expect_grad(d, nt.Hamiltonian(ham))
    eps = 0.05
    x = nt.natural_gradient(q, grad, eps).cpu().numpy()
    for r in range(3):
        qo = G.quantum_geometric_tensor(circ, theta[r])
        ref = G.natural_gradient(qo, G.parameter_shift(circ, theta[r], ham), eps)
        cond = np.linalg.cond(4.0 * qo.real + eps * np.eye(qo.shape[0]))
        assert cond < 1e4
        assert np.abs(x[r] - ref).max() <= 1e-8 * max(1.0, np.abs(ref).max())


def test_gram_bounded_wait_reports_timeout_and_recovers(monkeypatch):
    """Failure detection without a fault: with TC_TEST_GRAM_SKIP_MMA=1 the
    tensor-core Gram issues no MMA, so its first completion wait (an mbarrier
    nothing arrives at) runs out after its bounded number of polls; the kernel
    sets its status word, frees its tensor memory and returns, and the call
    reports TC_E_TIMEOUT.  The context stays usable: the next call, without
    the variable, gives the oracle's tensor."""
    circ, theta, _ = W.tfim_workload(12, 2, 1)
    c = nt.Circuit(circ)
    d = cuda_params(theta)
    monkeypatch.setenv("TC_TEST_GRAM_SKIP_MMA", "1")
    with pytest.raises(nt.TcError) as e:
        c.qgt(d)
    assert e.value.status == nt.TC_E_TIMEOUT
    monkeypatch.delenv("TC_TEST_GRAM_SKIP_MMA")
    g = c.qgt(d).cpu().numpy()[0]
    assert np.abs(g - G.quantum_geometric_tensor(circ, theta[0])).max() <= _tol(circ, nt.TC_C64)


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_qgt_bitwise_reproducible(dtype):
    """The Gram's amplitude chunks are summed in a fixed order (no atomics):
    two calls on the same rows give the same bits."""
    import torch

    circ, theta, _ = W.tfim_workload(n=14, layers=4, batch=3, seed=9)
    c = nt.Circuit(circ, dtype=dtype)
    d = torch.as_tensor(theta, device="cuda")
    g1 = c.qgt(d).cpu().numpy()
    g2 = c.qgt(d).cpu().numpy()
    assert np.array_equal(g1, g2)
