"""GPU parity: light-cone contraction against the FP64 oracle."""
import numpy as np
import pytest

from oracle import tensornet as T
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_ZZ = 1e-5  # absolute: |<Z Z>| <= 1


def _gates_tensor(gate_lists):
    import torch

    arr = np.stack([np.stack([u for (_, _, u) in g]) for g in gate_lists]).astype(np.complex64)
    return torch.as_tensor(arr, device="cuda")


@pytest.mark.parametrize("trials", [1, 64])  # per-step graph / fused executor
def test_brick200_depth8_zz_vs_oracle(trials):
    n, gates, obs = W.brick200_workload()
    lc = nt.LightCone(n, [(a, b) for a, b, _ in gates], obs, greedy_trials=trials)
    assert lc.info()["fused"] == (1 if trials > 1 else 0)
    out = lc.contract(_gates_tensor([gates])).cpu().numpy()
    ref = T.cone_statevector_expectation(gates, obs)
    assert abs(out[0, 0] - ref.real) <= TOL_ZZ and abs(out[0, 1]) <= TOL_ZZ


def test_brick200_seed_batch_fused_sampled():
    # the bench launch: 1024 seeds of the 200-qubit brickwork in one fused launch
    n, gates0, obs = W.brick200_workload()
    lc = nt.LightCone(n, [(a, b) for a, b, _ in gates0], obs, greedy_trials=64)
    gl = [W.brickwork_u4(n, 8, np.random.default_rng(s)) for s in range(1024)]
    out = lc.contract(_gates_tensor(gl)).cpu().numpy()
    for b in (0, 1, 511, 1023):
        ref = T.cone_statevector_expectation(gl[b], obs)
        assert abs(out[b, 0] - ref.real) <= TOL_ZZ


def test_batch_of_seeds_each_matches():
    n, depth, obs = 60, 8, (29, 30)
    gl = [W.brickwork_u4(n, depth, np.random.default_rng(s)) for s in range(6)]
    lc = nt.LightCone(n, [(a, b) for a, b, _ in gl[0]], obs)
    out = lc.contract(_gates_tensor(gl)).cpu().numpy()
    for b in range(6):
        ref = T.cone_statevector_expectation(gl[b], obs).real
        assert abs(out[b, 0] - ref) <= TOL_ZZ
    # batch row alone equals in batch
    one = lc.contract(_gates_tensor(gl[3:4])).cpu().numpy()
    assert np.array_equal(one[0], out[3])


@pytest.mark.parametrize("seed", range(3))
def test_small_brickwork_vs_full_network(seed):
    n = 6
    gates = W.brickwork_u4(n, 4, np.random.default_rng(seed))
    for obs in ((2, 3), (0,), (1, 4)):
        lc = nt.LightCone(n, [(a, b) for a, b, _ in gates], obs)
        out = lc.contract(_gates_tensor([gates])).cpu().numpy()
        net = T.network_expectation(n, gates, obs)
        ref = T.contract(net, T.greedy_path(net)).real
        assert abs(out[0, 0] - ref) <= TOL_ZZ


def test_repeated_calls_reuse_graph_and_agree():
    n, gates, obs = W.brick200_workload()
    lc = nt.LightCone(n, [(a, b) for a, b, _ in gates], obs)
    g = _gates_tensor([gates])
    a = lc.contract(g).cpu().numpy()
    b = lc.contract(g).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("cluster,split_min", [(8, 2048), (8, 1), (2, 1), (4, 64)])
def test_cluster_fused_bitwise_equals_one_cta(cluster, split_min):
    # few instances run on a thread-block cluster (large groups split over its
    # CTAs, outputs written through distributed shared memory); every output is
    # computed by the same code as in the one-CTA launch, so the results agree
    # bit for bit, and with the oracle to the FP32 bound.  split_min = 1 splits
    # every group, the smallest ones included.
    n, gates0, obs = W.brick200_workload()
    lc = nt.LightCone(n, [(a, b) for a, b, _ in gates0], obs, greedy_trials=64)
    assert lc.info()["fused"] == 1 and lc.info()["max_cluster"] == 8
    assert 0 < lc.info()["blob_ints"] <= 6144  # group blocks staged once, whole
    gl = [gates0] + [W.brickwork_u4(n, 8, np.random.default_rng(s)) for s in (7, 8, 9)]
    g = _gates_tensor(gl)
    lc.set_cluster(cluster, split_min)
    info = lc.info()
    assert info["max_cluster"] == cluster and info["split_min_items"] == split_min
    assert 1 <= info["split_groups"] <= info["fused_groups"]
    if split_min == 1:
        assert info["split_groups"] == info["fused_groups"]
    c1 = lc.contract(g[:1]).cpu().numpy()
    c4 = lc.contract(g).cpu().numpy()
    c1b = lc.contract(g[:1]).cpu().numpy()
    lc.set_cluster(1)
    o1 = lc.contract(g[:1]).cpu().numpy()
    o4 = lc.contract(g).cpu().numpy()
    assert np.array_equal(c1, o1) and np.array_equal(c4, o4) and np.array_equal(c1, c1b)
    assert np.array_equal(c1[0], c4[0])
    for b in (0, 3):
        ref = T.cone_statevector_expectation(gl[b], obs)
        assert abs(c4[b, 0] - ref.real) <= TOL_ZZ and abs(c4[b, 1]) <= TOL_ZZ


def test_cluster_fused_one_instance_equals_batch_row():
    # B = 1 (cluster launch) against the same gates as row 5 of a 1024-row
    # batch (one CTA per instance): bitwise equal
    n, gates0, obs = W.brick200_workload()
    lc = nt.LightCone(n, [(a, b) for a, b, _ in gates0], obs, greedy_trials=64)
    gl = [W.brickwork_u4(n, 8, np.random.default_rng(s)) for s in range(1024)]
    g = _gates_tensor(gl)
    full = lc.contract(g).cpu().numpy()
    one = lc.contract(g[5:6].contiguous()).cpu().numpy()
    assert np.array_equal(one[0], full[5])
