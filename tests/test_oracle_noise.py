"""Pins for the oracle's trajectory machinery (CPU only)."""
import os
import numpy as np
import pytest

from oracle import noise as N
from oracle import statevector as sv
from paper_2205_10091_b300 import workloads as W


def test_philox_uniformity_chi2():
    u = N.status_from_seed(1234, 1000, 1000).ravel()
    assert u.min() >= 0 and u.max() < 1
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    exp = u.size / 64
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 120  # 63 dof: p ~ 1e-5 threshold


def test_philox_streams_differ_and_are_deterministic():
    a = N.status_from_seed(7, 4, 64)
    b = N.status_from_seed(7, 4, 64)
    c = N.status_from_seed(8, 4, 64)
    np.testing.assert_array_equal(a, b)
    assert np.mean(a == c) < 0.01
    # trajectory offset gives the same rows as a larger draw
    d = N.status_from_seed(7, 2, 64, traj_offset=2)
    np.testing.assert_array_equal(d, a[2:])
    # adjacent-event serial correlation ~ 0
    u = N.status_from_seed(99, 200, 512)
    r = np.corrcoef(u[:, :-1].ravel(), u[:, 1:].ravel())[0, 1]
    assert abs(r) < 0.01


def test_philox_avalanche():
    x = N.philox4x32_10((np.uint64(5), 0, 0, 0), (1, 2))
    y = N.philox4x32_10((np.uint64(4), 0, 0, 0), (1, 2))
    flips = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(x, y))
    assert 40 < flips < 88


def test_selection_intervals_left_closed():
    px, py, pz = 0.1, 0.2, 0.3
    t1, t2, t3 = sv.noise_thresholds(px, py, pz)
    assert sv.select_pauli(0.0, px, py, pz) == 0
    assert sv.select_pauli(np.nextafter(t1, 0), px, py, pz) == 0
    assert sv.select_pauli(t1, px, py, pz) == 1
    assert sv.select_pauli(t2, px, py, pz) == 2
    assert sv.select_pauli(t3, px, py, pz) == 3
    assert sv.select_pauli(np.nextafter(1.0, 0), px, py, pz) == 3


def test_zero_noise_equals_noiseless():
    rng = np.random.default_rng(2)
    circ = W.noisy_su2_cz_circuit(6, 4, 0.0, rng)
    st = N.status_from_seed(5, 3, circ.n_noise)
    obs = [W.pauli_sum(6, [(1.0, {0: 3})])]
    vals = N.trajectory_expectations(circ, st, obs)
    assert np.ptp(vals) < 1e-14
    mean, se = N.estimate(vals)
    assert se[0] < 1e-14


def test_depolarizing_closed_form():
    # |0> through a depolarising channel with px=py=pz=p/3: <Z> = 1 - 4p/3
    for p in (0.01, 0.3, 0.75):
        b = W.OpBuilder(1)
        b.depolarizing(0, p / 3, p / 3, p / 3)
        rho = N.density_matrix(b.build())
        assert abs(N.dm_expectation(rho, 1, W.pauli_sum(1, [(1.0, {0: 3})])) - (1 - 4 * p / 3)) < 1e-14
        assert abs(np.trace(rho) - 1) < 1e-14


def test_density_matrix_noiseless_is_pure_state():
    rng = np.random.default_rng(4)
    circ = W.noisy_su2_cz_circuit(4, 3, 0.0, rng)
    rho = N.density_matrix(circ)
    psi = sv.run_circuit(circ, None, status_row=np.zeros(circ.n_noise))
    np.testing.assert_allclose(rho, np.outer(psi, psi.conj()), atol=1e-13)


def test_trajectory_mean_matches_density_matrix():
    rng = np.random.default_rng(6)
    n = 4
    circ = W.noisy_su2_cz_circuit(n, 4, 0.3, rng)
    obs = [W.pauli_sum(n, [(1.0, {0: 3})]), W.pauli_sum(n, [(1.0, {i: 3, i + 1: 3}) for i in range(n - 1)])]
    st = N.status_from_seed(21, 3000, circ.n_noise)
    mean, se = N.estimate(N.trajectory_expectations(circ, st, obs))
    rho = N.density_matrix(circ)
    for o in range(2):
        exact = N.dm_expectation(rho, n, obs[o])
        assert abs(mean[o] - exact) < 4 * se[o] + 1e-12


def test_random_axis_rotation_selects_by_interval():
    """unitary_kraus over [RX, RY, RZ] (Section "Demonstration of barren
    plateaus"): u in [0, 1/3) gives RX, [1/3, 2/3) RY, [2/3, 1) RZ; each
    case equals the fixed rotation, and the shift rule holds for it."""
    import numpy as np

    from oracle import gradients as G
    from oracle import statevector as sv
    from paper_2205_10091_b300 import workloads as W

    rng = np.random.default_rng(5)
    theta = rng.uniform(-3, 3, size=2)
    for u, fixed in ((0.0, "rx"), (0.2, "rx"), (1.0 / 3, "ry"), (0.5, "ry"), (2.0 / 3, "rz"), (0.99, "rz")):
        b = W.OpBuilder(3)
        b.h(0)
        b.h(1)
        b.rsel(1, 0, scale=0.7)
        b.cz(0, 1)
        b.rsel(2, 1)
        got = sv.run_circuit(b.build(2), theta, status_row=[u, 0.1])
        f = W.OpBuilder(3)
        f.h(0)
        f.h(1)
        getattr(f, fixed)(1, 0, 0.7)
        f.cz(0, 1)
        f.rx(2, 1)
        np.testing.assert_allclose(got, sv.run_circuit(f.build(2), theta), atol=1e-14)
        ham = W.pauli_sum(3, [(1.0, {1: 1}), (0.5, {1: 2, 2: 3})])
        gs = G.parameter_shift(b.build(2), theta, ham, status_row=[u, 0.1])
        gf = G.parameter_shift(f.build(2), theta, ham)
        np.testing.assert_allclose(gs, gf, atol=1e-12)


def test_philox_known_answer_vectors():
    # published known-answer vectors of Philox4x32-10 (tests/golden/philox4x32_10_kat.txt)
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        got = N.philox4x32_10(tuple(v[0:4]), tuple(v[4:6]))
        assert [int(x) for x in got] == v[6:10]
