"""Light-cone planner host checks (CPU only: plans are built on the host)."""
import math

import numpy as np
import pytest

from oracle import tensornet as T
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W


def _plan(n, depth, obs, seed=0, cap=18, path=None):
    gates = W.brickwork_u4(n, depth, np.random.default_rng(seed))
    return nt.LightCone(n, [(a, b) for a, b, _ in gates], obs, rank_cap=cap, path=path), gates


def test_brick200_cone_matches_oracle_cone():
    n, gates, obs = W.brick200_workload()
    lc = nt.LightCone(n, [(a, b) for a, b, _ in gates], obs)
    info = lc.info()
    cone = T.light_cone(gates, obs)
    assert info["n_cone_gates"] == len(cone) == 36
    assert (info["cone_lo"], info["cone_hi"]) == (92, 107)
    # 16 qubits x (|0> ket + |0> bra) + 36 x (gate + conjugate) + 2 Z
    assert info["n_inputs"] == 32 + 72 + 2
    assert info["n_steps"] == info["n_inputs"] - 1
    assert info["max_rank"] <= 18
    assert info["flops"] == 8 * info["cmacs"]
    assert info["size"] <= info["write"]


@pytest.mark.parametrize("cap", [6, 8, 12])
def test_rank_cap_respected_or_refused(cap):
    try:
        lc, _ = _plan(40, 6, (19, 20), cap=cap)
    except nt.TcError as e:
        assert e.status == nt.TC_E_INVALID and "rank cap" in str(e)
        return
    assert lc.info()["max_rank"] <= cap


def test_user_path_accepted_and_checked():
    lc, gates = _plan(6, 2, (2, 3))
    n_in = lc.info()["n_inputs"]
    seq = [(0, 1)] + [(0, k) for k in range(n_in - 2, 0, -1)]
    try:
        p = nt.LightCone(6, [(a, b) for a, b, _ in gates], (2, 3), rank_cap=26, path=seq)
        assert p.info()["n_steps"] == n_in - 1
    except nt.TcError as e:  # a sequential fold may create outer products; must be a clean refusal
        assert e.status == nt.TC_E_INVALID
    with pytest.raises(nt.TcError):
        nt.LightCone(6, [(a, b) for a, b, _ in gates], (2, 3), path=[(0, 0)])


def test_bad_inputs_rejected():
    with pytest.raises(nt.TcError):
        nt.LightCone(4, [(0, 4)], (0,))
    with pytest.raises(nt.TcError):
        nt.LightCone(4, [(1, 1)], (0,))
    with pytest.raises(nt.TcError):
        nt.LightCone(4, [(0, 1)], (7,))


def test_example_block_shaped_metrics_reported():
    # the contractor-table testbed shape (n=40, d=6, <Z_20>), with brickwork
    # gates: the greedy path and its log10 FLOPs / log2 SIZE / log2 WRITE
    n = 40
    gates = W.brickwork_u4(n, 6, np.random.default_rng(1))
    info = nt.LightCone(n, [(a, b) for a, b, _ in gates], (20,)).info()
    assert 0 < math.log10(info["flops"]) < 10
    assert math.log2(info["size"]) <= 18


def test_example_block_commuting_cone_shape():
    # Section "Custom contraction settings" testbed, n = 40, d = 6, <Z_20>.
    # Walking back from Z_20, layer j (0-based) keeps RX on 2 (5 - j) + 1
    # qubits and the 2 (5 - j) + 2 ZZ gates touching them; the first layer's
    # ZZ gates leave qubits 14 and 26 with diagonal support only.
    c = W.example_block_circuit(40, 6)
    net = nt.CircuitNetwork(c, {20: 3}, prune=2, split=True)
    info = net.info()
    assert info["n_cone_gates"] == 36 + 42
    assert (info["cone_lo"], info["cone_hi"], info["n_active"]) == (14, 26, 13)
    # 13 x (|0> ket + bra) + 2 x (36 RX + 42 x 2 halves) + Z
    assert info["n_inputs"] == 26 + 2 * (36 + 84) + 1
    assert info["n_steps"] == info["n_inputs"] - 1
    unsplit = nt.CircuitNetwork(c, {20: 3}, prune=2, split=False).info()
    assert unsplit["n_inputs"] == 26 + 2 * (36 + 42) + 1


def test_example_block_whole_network_and_causal_cone():
    c = W.example_block_circuit(40, 6)
    whole = nt.CircuitNetwork(c, {20: 3}, prune=0, split=True, rank_cap=26).info()
    assert whole["n_cone_gates"] == len(c.ops) and whole["n_active"] == 40
    cone = nt.CircuitNetwork(c, {20: 3}, prune=1, split=True, rank_cap=26).info()
    # in circuit order the chain ZZ(i, i+1), i = 0..38, drags every qubit left of 20 into the cone
    assert (cone["cone_lo"], cone["cone_hi"]) == (0, 26)
    comm = nt.CircuitNetwork(c, {20: 3}, prune=2).info()
    assert comm["cmacs"] < cone["cmacs"] < whole["cmacs"]


def test_circuit_network_rejects_bad_input():
    b = W.OpBuilder(4)
    b.rx(0, 0)
    b.depolarizing(1, 0.1, 0.1, 0.1)
    with pytest.raises(nt.TcError) as e:
        nt.CircuitNetwork(b.build(), {0: 3})
    assert e.value.status == nt.TC_E_UNSUPPORTED
    b = W.OpBuilder(4)
    b.rx(0, 0)
    with pytest.raises(nt.TcError):
        nt.CircuitNetwork(b.build(), {})
    with pytest.raises(nt.TcError):
        nt.CircuitNetwork(b.build(), {0: 3}, prune=3)


def test_greedy_trials_deterministic_and_no_worse():
    c = W.example_block_circuit(40, 6)
    one = nt.CircuitNetwork(c, {20: 3}, prune=2, greedy_trials=1).info()
    a = nt.CircuitNetwork(c, {20: 3}, prune=2, greedy_trials=16).info()
    b = nt.CircuitNetwork(c, {20: 3}, prune=2, greedy_trials=16).info()
    assert a == b
    assert a["cmacs"] <= one["cmacs"]
    with pytest.raises(nt.TcError):
        nt.CircuitNetwork(c, {20: 3}, greedy_trials=-1)


def test_executor_choice():
    # small live sets run as one fused launch; the whole 40-qubit network and
    # the 200-qubit light cone (live tensors above 200 KiB) as per-step GEMMs
    c = W.example_block_circuit(40, 6)
    fused = nt.CircuitNetwork(c, {20: 3}, prune=2).info()
    assert fused["fused"] == 1 and 0 < fused["smem_bytes"] <= 200 * 1024
    assert 0 < fused["fused_groups"] < fused["n_steps"]
    whole = nt.CircuitNetwork(c, {20: 3}, prune=0, rank_cap=26).info()
    assert whole["fused"] == 0 and whole["smem_bytes"] > 200 * 1024
    n, gates, obs = W.brick200_workload()
    assert nt.LightCone(n, [(a, b) for a, b, _ in gates], obs).info()["fused"] == 0


def test_cluster_setting_validated_and_reported():
    n, gates, obs = W.brick200_workload()
    lc = nt.LightCone(n, [(a, b) for a, b, _ in gates], obs, greedy_trials=64)
    info = lc.info()
    assert info["max_cluster"] == 8 and info["split_min_items"] == 2048
    assert 1 <= info["split_groups"] < info["fused_groups"]
    assert 0 < info["blob_ints"] <= 6144
    for bad in ((0, 2048), (3, 2048), (16, 2048), (8, 0)):
        with pytest.raises(RuntimeError):
            lc.set_cluster(*bad)
    lc.set_cluster(4, 1)
    assert lc.info()["split_groups"] == lc.info()["fused_groups"]
    lc.set_cluster(1, 4096)
    assert lc.info()["max_cluster"] == 1
