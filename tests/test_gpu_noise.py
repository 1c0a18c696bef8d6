"""GPU parity: Monte Carlo trajectories against the oracle."""
import numpy as np
import pytest

from oracle import noise as N
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64, assert_energy_close, assert_grad_close, cuda_params

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


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_folded_noise_gradients_per_trajectory(dtype):
    # noise events next to a U1 on their qubit are folded into its per-row
    # matrix (after it, or before the next one); the rest stay instructions
    from oracle import gradients as G
    from oracle import noise as N

    rng = np.random.default_rng(4242)
    n = 5
    b = W.OpBuilder(n)
    for q in range(n):
        b.unitary1(q, W.haar_unitary(2, rng))
        b.depolarizing(q, 0.2, 0.15, 0.25)          # after the U1: folded after it
    for q in range(n - 1):
        b.cz(q, q + 1)
        b.depolarizing(q, 0.1, 0.3, 0.2)            # before the next U1 on q: folded before it
    for q in range(n):
        b.unitary1(q, W.haar_unitary(2, rng))
        b.ry(q, q % 3)
    b.depolarizing(2, 0.3, 0.3, 0.3)                # next to RY only: stays an instruction
    circ = b.build(3)
    ham = W.random_pauli_sum(n, 5, rng)
    B, seed = 6, 77
    theta = rng.uniform(-2, 2, size=(B, circ.n_params))
    c = nt.Circuit(circ, dtype=dtype)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham), seed=seed)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    status = N.status_from_seed(seed, B, circ.n_noise)
    for r in range(B):
        e_ref = sv.energy(sv.run_circuit(circ, theta[r], status_row=status[r]), n, ham)[0]
        g_ref = G.parameter_shift(circ, theta[r], ham, status_row=status[r])
        if dtype == nt.TC_C128:
            assert abs(e[r] - e_ref) <= 1e-11 and np.abs(g[r] - g_ref).max() <= 1e-10
        else:
            assert_energy_close(e[r:r + 1], [e_ref])
            assert_grad_close(g[r], g_ref)


def test_shard_moments_merge_to_mean_stderr():
    """Trajectory values split in three shards: each shard's (count, mean, M2)
    from tc_shard_moments, merged on the host, equals tc_mean_stderr of the
    whole set and numpy's estimate."""
    import torch

    rng = np.random.default_rng(12)
    x = rng.normal(0.3, 1.0, size=10_000)
    xd = torch.as_tensor(x, device="cuda")
    parts = [nt.shard_moments(xd[a:b]).cpu().numpy() for a, b in [(0, 3000), (3000, 3001), (3001, 10_000)]]
    for (a, b), p in zip([(0, 3000), (3000, 3001), (3001, 10_000)], parts):
        s = x[a:b]
        assert p[0] == len(s) and abs(p[1] - s.mean()) <= 1e-14 and abs(p[2] - ((s - s.mean()) ** 2).sum()) <= 1e-9
    m, se = nt.merge_moments(parts)
    whole = nt.mean_stderr(xd).cpu().numpy()
    assert abs(m - whole[0]) <= 1e-14 and abs(se - whole[1]) <= 1e-15
    assert abs(m - x.mean()) <= 1e-14 and abs(se - x.std(ddof=1) / np.sqrt(len(x))) <= 1e-15
