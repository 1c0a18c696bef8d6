"""GPU parity: the FP64 per-row norm check (tc_state_norms).

Unitary gates preserve ||psi|| (Section "Circuits and gates": every gate is a
unitary matrix), so ||psi||^2 = 1 after any noiseless or trajectory circuit
from a normalised input; for arbitrary inputs the result is the plain sum of
squares, checked against numpy's FP64 sum of the stored values.
"""
import numpy as np
import pytest

from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import cuda_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
@pytest.mark.parametrize("n", [1, 3, 10, 17, 20])
def test_norms_of_arbitrary_states(n, dtype):
    import torch

    rng = np.random.default_rng(300 + n)
    B = 5
    x = (rng.standard_normal((B, 2 ** n)) + 1j * rng.standard_normal((B, 2 ** n))) * rng.uniform(0.1, 3, (B, 1))
    x = x.astype(np.complex64 if dtype == nt.TC_C64 else np.complex128)
    c = nt.Circuit(W.OpBuilder(n).build(), dtype=dtype)
    got = c.norms(torch.as_tensor(x, device="cuda")).cpu().numpy()
    xd = x.astype(np.complex128)
    ref = np.sum(xd.real ** 2 + xd.imag ** 2, axis=1)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_norm_preserved_by_circuits(dtype):
    import torch

    circ, theta, _ = W.tfim_workload(n=16, layers=6, batch=4, seed=61)
    c = nt.Circuit(circ, dtype=dtype)
    st = c.apply(cuda_params(theta), 4)
    dev = np.abs(c.norms(st).cpu().numpy() - 1.0).max()
    assert dev <= (1e-6 if dtype == nt.TC_C64 else 1e-13), dev
    circ_n, n_traj, seed, _ = W.noisy16_workload(trajectories=64)
    cn = nt.Circuit(circ_n)
    sn = cn.apply(None, n_traj, seed=seed)
    assert np.abs(cn.norms(sn).cpu().numpy() - 1.0).max() <= 1e-5
    torch.cuda.synchronize()


def test_norm_row_alone_equals_in_batch():
    import torch

    rng = np.random.default_rng(9)
    x = torch.as_tensor((rng.standard_normal((7, 2 ** 18)) + 1j * rng.standard_normal((7, 2 ** 18))).astype(np.complex64),
                        device="cuda")
    c = nt.Circuit(W.OpBuilder(18).build())
    allb = c.norms(x)
    one = c.norms(x[3:4].contiguous())
    assert torch.equal(allb[3:4], one)
