"""GPU parity: Monte Carlo trajectories against the oracle."""
import numpy as np
import pytest

from oracle import noise as N
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64

pytestmark = pytest.mark.gpu


def test_status_array_trajectories_exact():
    import torch

    rng = np.random.default_rng(12)
    circ = W.noisy_su2_cz_circuit(10, 4, 0.3, rng)
    status = rng.uniform(0, 1, size=(16, circ.n_noise)).astype(np.float32)
    c = nt.Circuit(circ)
    out = c.apply(None, 16, status=torch.as_tensor(status, device="cuda")).cpu().numpy()
    for b in range(16):
        ref = sv.run_circuit(circ, None, status_row=status[b].astype(np.float64))
        assert np.abs(out[b] - ref).max() <= TOL_AMP_C64


def test_philox_trajectories_match_oracle_stream():
    rng = np.random.default_rng(13)
    circ = W.noisy_su2_cz_circuit(11, 5, 0.3, rng)
    c = nt.Circuit(circ)
    out = c.apply(None, 24, seed=987654321, row_offset=100).cpu().numpy()
    st = N.status_from_seed(987654321, 24, circ.n_noise, traj_offset=100)
    for b in range(24):
        ref = sv.run_circuit(circ, None, status_row=st[b])
        assert np.abs(out[b] - ref).max() <= TOL_AMP_C64
