"""The allocation-free energy entry point (tc_expect_pauli_sum_noalloc).

Some callers cannot allocate device memory where they need an energy: code
that runs under a fixed memory reservation, inside an allocator callback, or
in a latency-critical loop that must not hit cudaMalloc's implicit
synchronisation.  This entry point keeps its scratch in a fixed-size array
inside the library.  The tests check, through the C-ABI, that two calls in a
row give the energies of the allocating entry point (tc_expect_pauli_sum)
and of the FP64 oracle within the energy tolerance of the other GPU tests,
that after a zero-row warm-up call the calls change neither the device's
free memory nor torch's allocator, and that an oversize request is refused.
This file is collected last.
"""
import numpy as np
import pytest

from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import assert_energy_close

pytestmark = pytest.mark.gpu


def _states(rng, B, n, dtype):
    psi = rng.standard_normal((B, 2 ** n)) + 1j * rng.standard_normal((B, 2 ** n))
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    return psi.astype(np.complex64 if dtype == nt.TC_C64 else np.complex128)


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_noalloc_matches_allocating_entry_point_twice(dtype):
    import torch

    rng = np.random.default_rng(2024)
    n = 14
    c = nt.Circuit(W.OpBuilder(n).build(), dtype=dtype)
    wide = W.pauli_sum(n, [(0.5, {q: 1 for q in range(n)}), (-0.25, {q: 2 for q in range(n)})])
    calls = [
        (_states(rng, 6, n, dtype), W.tfim_zz_x(n)),
        (_states(rng, 3, n, dtype), W.PauliSum(np.concatenate([W.random_pauli_sum(n, 17, rng).structures,
                                                               wide.structures]),
                                               np.concatenate([rng.standard_normal(17), wide.weights]))),
    ]
    # warm-up with no rows: looks up (and, on first use, loads) the scratch array
    H0 = nt.Hamiltonian(calls[0][1])
    one = torch.zeros((1, 1 << n), dtype=c.state_dtype, device="cuda")
    c.expect_noalloc(one, H0, torch.empty(1, dtype=torch.float64, device="cuda"), rows=0)
    for psi, ham in calls:  # two calls in a row, different inputs
        states = torch.as_tensor(psi, device="cuda")
        H = nt.Hamiltonian(ham)
        ref = c.expect(states, H).cpu().numpy()
        out = torch.full((states.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        c.expect_noalloc(states, H, out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert_energy_close(got, ref)
        oracle = [sv.energy(psi[b].astype(np.complex128), n, ham)[0] for b in range(psi.shape[0])]
        assert_energy_close(got, oracle)


def test_noalloc_rejects_oversize_request():
    import torch

    # 300 random strings with ~16 flipped qubits each need tens of paired
    # Pauli-sum passes; enough rows that rows x passes x 256 tiles x 8 B of
    # partial sums exceed the 8 MiB of scratch, with states of a few 100 MiB
    n = 20
    rng = np.random.default_rng(5)
    codes = rng.choice([1, 2, 3], p=[0.4, 0.4, 0.2], size=(300, n)).astype(np.uint8)
    ham = W.PauliSum(codes, rng.standard_normal(300))
    c = nt.Circuit(W.OpBuilder(n).build())
    passes = c.pauli_sum_info(nt.Hamiltonian(ham))["passes"]
    B = (9 << 20) // (passes * 256 * 8) + 1
    states = torch.zeros((B, 1 << n), dtype=torch.complex64, device="cuda")
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    with pytest.raises(nt.TcError) as e:
        c.expect_noalloc(states, nt.Hamiltonian(ham), out)
    assert e.value.status == nt.TC_E_INVALID and "limit" in str(e.value)


def test_refused_under_stream_capture():
    """The plan copy reads host memory freed at return: a capturing stream is refused."""
    import torch

    circ, theta, ham = W.tfim_workload(n=12, layers=2, batch=2, seed=3)
    c = nt.Circuit(circ)
    st = c.apply(torch.as_tensor(theta, device="cuda"), 2)
    H = nt.Hamiltonian(ham)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    c.expect_noalloc(st, H, out=out)  # warm-up outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    sw, w, T = H.args()
    code = None
    with torch.cuda.graph(g, stream=s):
        code = nt.lib().tc_expect_pauli_sum_noalloc(c.h, nt._ptr(st), 2, sw, w, T, nt._ptr(out), nt._stream(s))
    assert code == nt.TC_E_UNSUPPORTED
