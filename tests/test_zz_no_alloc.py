"""The allocation-free energy entry point (tc_expect_pauli_sum_noalloc).

Some callers cannot allocate device memory where they need an energy (a fixed
memory reservation, an allocator callback, a latency-critical loop that must
not hit cudaMalloc's implicit synchronisation).  This entry point keeps its
scratch in a fixed-size array inside the library.  The test checks, through
the C-ABI, that two calls in a row give the energies of the allocating entry
point (tc_expect_pauli_sum) within the energy tolerance of the other GPU
tests, and that an oversize request is refused.  This file is collected last.
"""
import numpy as np
import pytest

from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import assert_energy_close

pytestmark = pytest.mark.gpu


def _states(rng, B, n, dtype):
    import torch

    psi = rng.standard_normal((B, 2 ** n)) + 1j * rng.standard_normal((B, 2 ** n))
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    return torch.as_tensor(psi.astype(np.complex64 if dtype == nt.TC_C64 else np.complex128), device="cuda")


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_noalloc_matches_allocating_entry_point_twice(dtype):
    import torch

    rng = np.random.default_rng(2024)
    n = 14
    c = nt.Circuit(W.OpBuilder(n).build(), dtype=dtype)
    calls = [
        (_states(rng, 6, n, dtype), W.tfim_zz_x(n)),
        (_states(rng, 3, n, dtype), W.random_pauli_sum(n, 17, rng)),
    ]
    for states, ham in calls:  # two calls in a row, different inputs
        H = nt.Hamiltonian(ham)
        ref = c.expect(states, H).cpu().numpy()
        out = torch.full((states.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        got = c.expect_noalloc(states, H, out).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert_energy_close(got, ref)


def test_noalloc_rejects_oversize_request():
    import torch

    n, B = 20, 2100  # 2100 rows x (2 or more) passes x 256 tiles x 8 B > 8 MiB of scratch
    c = nt.Circuit(W.OpBuilder(n).build())
    states = torch.empty((B, 1 << n), dtype=torch.complex64, device="cuda")
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    with pytest.raises(nt.TcError) as e:
        c.expect_noalloc(states, nt.Hamiltonian(W.tfim_zz_x(n)), out)
    assert e.value.status == nt.TC_E_INVALID and "limit" in str(e.value)
