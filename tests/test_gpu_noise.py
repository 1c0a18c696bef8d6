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


def test_mean_stderr_kernel_matches_numpy():
    import torch

    x = np.random.default_rng(3).standard_normal(10007) * 2.5 + 0.7
    out = nt.mean_stderr(torch.as_tensor(x, device="cuda")).cpu().numpy()
    assert abs(out[0] - x.mean()) < 1e-12
    assert abs(out[1] - x.std(ddof=1) / np.sqrt(x.size)) < 1e-12


def test_trajectory_mean_within_4_sigma_of_density_matrix():
    import torch

    rng = np.random.default_rng(61)
    n = 6
    circ = W.noisy_su2_cz_circuit(n, 5, 0.3, rng)
    obs = [W.pauli_sum(n, [(1.0, {0: 3})]), W.pauli_sum(n, [(1.0, {i: 3, i + 1: 3}) for i in range(n - 1)])]
    c = nt.Circuit(circ)
    B = 20000
    states = c.apply(None, B, seed=77)
    rho = N.density_matrix(circ)
    for o in obs:
        vals = c.expect(states, nt.Hamiltonian(o))
        mean, se = nt.mean_stderr(vals).cpu().numpy()
        exact = N.dm_expectation(rho, n, o)
        assert abs(mean - exact) <= 4 * se + 1e-9, (mean, se, exact)


def test_noisy16_full_size_sampled_trajectories():
    """The 16-qubit, 12-layer noisy workload at full size (8192 trajectories,
    Philox seed 1005) in one call; sampled trajectories are recomputed by the
    oracle from the same Philox stream."""
    import torch

    circ, n_traj, seed, obs = W.noisy16_workload()
    c = nt.Circuit(circ)
    states = c.apply(None, n_traj, seed=seed)
    vals = [c.expect(states, nt.Hamiltonian(o)).cpu().numpy() for o in obs]
    for v in vals:
        assert v.shape == (n_traj,) and np.all(np.isfinite(v))
    for b in (0, 1, 4095, 8191):
        st = N.status_from_seed(seed, 1, circ.n_noise, traj_offset=b)
        ref = N.trajectory_expectations(circ, st, obs)[0]
        for o in range(2):
            assert abs(vals[o][b] - ref[o]) <= 1e-5 * max(1.0, abs(ref[o])), (b, o, vals[o][b], ref[o])
    est = [nt.mean_stderr(torch.as_tensor(v, device="cuda")).cpu().numpy() for v in vals]
    assert 0 < est[0][1] < 0.05 and 0 < est[1][1] < 0.2
