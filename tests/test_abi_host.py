"""C-ABI host-side checks (CPU only: no compute calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tc.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"TC_API\s+[\w\s\*]+?\b(tc_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 9
    L = nt.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(nt.SIGNATURES), set(names) - set(nt.SIGNATURES)


def test_enum_values_match_generator():
    src = open(HEADER).read()
    for i, name in enumerate(W.OP_NAMES):
        m = re.search(r"TC_OP_%s\s*=\s*(\d+)" % name, src)
        assert m and int(m.group(1)) == i, name
    assert re.search(r"TC_INIT_ZERO\s*=\s*0", src) and re.search(r"TC_INIT_PLUS\s*=\s*1", src)


def test_op_struct_layout():
    assert C.sizeof(nt.tc_op) == 56 == W.OP_DTYPE.itemsize
    for f, _ in nt.tc_op._fields_:
        assert getattr(nt.tc_op, f).offset == W.OP_DTYPE.fields[f][1], f


def test_plan_tfim20_fuses_layers():
    info = nt.Circuit(W.tfim_circuit(20, 10)).info()
    assert info["n_ops"] == 390 and info["n_params"] == 20
    # fewer HBM sweeps than layers: commuting gates of consecutive layers share passes
    assert 1 <= info["fwd_passes"] <= 10
    assert info["tile_qubits_fwd"] == 13


def test_plan_narrow_circuit_is_padded():
    info = nt.Circuit(W.tfim_circuit(3, 2)).info()
    assert info["n_qubits"] == 3 and info["n_qubits_internal"] == 10


def test_noise_events_counted():
    circ, _, _, _ = W.noisy16_workload()
    assert nt.Circuit(circ).info()["n_noise"] == circ.n_noise == 372


@pytest.mark.parametrize("bad", ["q0", "q1", "param", "mat", "noise"])
def test_invalid_ops_rejected(bad):
    b = W.OpBuilder(4)
    b.rx(0, 0)
    b.cnot(1, 2)
    b.unitary1(3, np.eye(2))
    b.depolarizing(2, 0.1, 0.1, 0.1)
    circ = b.build()
    ops = circ.ops.copy()
    if bad == "q0":
        ops[0]["q0"] = 4
    elif bad == "q1":
        ops[1]["q1"] = 1
    elif bad == "param":
        ops[0]["param"] = 5
    elif bad == "mat":
        ops[2]["mat"] = 1
    else:
        ops[3]["px"] = 0.9
    circ.ops = ops
    with pytest.raises(nt.TcError) as e:
        nt.Circuit(circ)
    assert e.value.status == nt.TC_E_INVALID
    assert "op " in str(e.value)


def test_bad_sizes_rejected():
    h = C.c_void_p()
    assert nt.lib().tc_circuit_create(0, 0, 0, None, 0, 0, None, 0, None, C.byref(h)) == nt.TC_E_INVALID
    assert nt.lib().tc_circuit_create(31, 0, 0, None, 0, 0, None, 0, None, C.byref(h)) == nt.TC_E_INVALID
    assert nt.lib().tc_circuit_create(4, 7, 0, None, 0, 0, None, 0, None, C.byref(h)) == nt.TC_E_INVALID


def test_noise_events_next_to_u1_fold_into_its_matrix():
    # an event right after a U1 on its qubit (or right before the next one)
    # costs no instruction; one next to an RY stays an instruction
    rng = np.random.default_rng(3)
    b = W.OpBuilder(12)
    b.unitary1(0, W.haar_unitary(2, rng))
    b.depolarizing(0, 0.1, 0.1, 0.1)   # after U1 on 0: folded
    b.depolarizing(1, 0.1, 0.1, 0.1)   # before U1 on 1: folded
    b.unitary1(1, W.haar_unitary(2, rng))
    b.ry(2, 0)
    b.depolarizing(2, 0.1, 0.1, 0.1)   # next to RY: stays
    noisy = nt.Circuit(b.build(1)).info()
    b = W.OpBuilder(12)
    b.unitary1(0, W.haar_unitary(2, rng))
    b.unitary1(1, W.haar_unitary(2, rng))
    b.ry(2, 0)
    plain = nt.Circuit(b.build(1)).info()
    assert noisy["n_noise"] == 3
    assert noisy["fwd_instrs"] == plain["fwd_instrs"] + 1
    assert noisy["bwd_instrs"] == plain["bwd_instrs"] + 1


def test_pauli_sum_plan_pairs_wide_flip_masks():
    """Flip masks wider than a tile go to paired passes; masks with the same
    bits outside the tile share one; tile-sized masks stay in ordinary passes."""
    n = 20
    c = nt.Circuit(W.OpBuilder(n).build())
    tfim = c.pauli_sum_info(nt.Hamiltonian(W.tfim_zz_x(n)))
    assert tfim["paired_passes"] == 0 and tfim["passes"] == 2 and tfim["flip_groups"] == 20
    xn = W.pauli_sum(n, [(1.0, {q: 1 for q in range(n)}), (0.5, {q: 2 for q in range(n)})])
    i = c.pauli_sum_info(nt.Hamiltonian(xn))
    # X^n and Y^n share one flip mask: one group, one paired pass (plus the first pass)
    assert i["flip_groups"] == 1 and i["paired_passes"] == 1 and i["passes"] == 2
    shared = W.pauli_sum(n, [(1.0, {**{q: 1 for q in range(12)}, n - 1: 2}),
                             (1.0, {**{q: 1 for q in range(12)}, n - 2: 1}),
                             (1.0, {**{q: 1 for q in range(12)}, n - 3: 1, n - 4: 2})])
    i = c.pauli_sum_info(nt.Hamiltonian(shared))
    assert i["flip_groups"] == 3 and i["paired_passes"] == 1
    rng = np.random.default_rng(1)
    codes = rng.choice([1, 2, 3], p=[0.4, 0.4, 0.2], size=(40, n)).astype(np.uint8)
    i = c.pauli_sum_info(nt.Hamiltonian(W.PauliSum(codes, np.ones(40))))
    # strings whose masks differ only in bits that fit the tile share a pass
    assert 1 <= i["paired_passes"] <= 40 and i["passes"] == 1 + i["paired_passes"] and i["flip_groups"] == 40
    # two wide masks (10 flipped qubits each, none among the 3 lowest index
    # bits) that differ in 14 qubits: more than the 9 free tile bits
    far = np.zeros((2, n), dtype=np.uint8)
    far[0, 7:17] = 1
    far[1, 0:10] = 1
    i = c.pauli_sum_info(nt.Hamiltonian(W.PauliSum(far, np.ones(2))))
    assert i["paired_passes"] == 2
    # a whole-state tile never pairs
    c12 = nt.Circuit(W.OpBuilder(12).build())
    i = c12.pauli_sum_info(nt.Hamiltonian(W.pauli_sum(12, [(1.0, {q: 1 for q in range(12)})])))
    assert i["paired_passes"] == 0


@pytest.mark.parametrize("dtype", [nt.TC_C64, nt.TC_C128])
def test_specialised_passes_compile_for_every_instruction_kind(dtype):
    """Plan-time specialisation (NVRTC, host only) compiles the forward and
    adjoint passes of circuits with every gate kind: rotations, H, X, CNOT,
    CZ, RZZ at several distances, 2x2 and 4x4 matrices, a channel-shaped 4x4,
    noise events and random-axis rotations."""
    rng = np.random.default_rng(12)
    b = W.OpBuilder(12)
    for q in range(12):
        b.ry(q, q % 5)
    for q in range(11):
        b.rzz(q, (q + 3) % 12, 5)
        b.cnot(q, q + 1)
    b.cz(0, 7)
    b.rx(3, 6)
    b.rz(4, 7)
    b.h(5)
    b.x(6)
    b.unitary1(2, W.haar_unitary(2, rng))
    b.unitary2(8, 9, W.haar_unitary(4, rng))
    chan = np.diag([0.9, 0.8, 0.8, 0.9]).astype(np.complex128)
    chan[0, 3] = chan[3, 0] = 0.1
    chan[1, 2] = chan[2, 1] = 0.05
    b.unitary2(10, 11, chan)
    b.depolarizing(1, 0.1, 0.05, 0.02)
    b.rsel(2, 8)
    circ = b.build(9)
    c = nt.Circuit(circ, dtype=dtype, specialize=True)
    info = c.info()
    assert info["specialized_passes"] == info["fwd_passes"] + info["bwd_passes"] > 0
    assert nt.Circuit(circ, dtype=dtype).info()["specialized_passes"] == 0


def test_qaoa_layers_use_packed_diag_groups():
    """A QAOA cost layer on a 3-regular graph has ZZ pairs at many distances;
    the planner evaluates such a group as one linear map per amplitude.  A
    nearest-neighbour layer (one distance) keeps the entry form."""
    rng = np.random.default_rng(5)
    edges = W.random_regular3(16, rng)
    info = nt.Circuit(W.qaoa_circuit(16, edges, 3)).info()
    assert info["packed_diag_groups"] >= 3
    assert nt.Circuit(W.tfim_circuit(16, 3)).info()["packed_diag_groups"] == 0


def test_specialised_passes_compile_with_packed_groups():
    rng = np.random.default_rng(6)
    c = nt.Circuit(W.qaoa_circuit(14, W.random_regular3(14, rng), 2), specialize=True)
    info = c.info()
    assert info["packed_diag_groups"] >= 2
    assert info["specialized_passes"] == info["fwd_passes"] + info["bwd_passes"]


def test_pauli_sum_packs_zz_terms_of_one_weight():
    rng = np.random.default_rng(8)
    n = 16
    edges = W.random_regular3(n, rng)
    c = nt.Circuit(W.OpBuilder(n).build())
    i = c.pauli_sum_info(nt.Hamiltonian(W.zz_on_edges(n, edges)))
    assert i["packed_diag_groups"] == 1 and i["diag_entries"] == 1 + n
    # nearest-neighbour bonds (one distance) keep the entry form
    nn = W.pauli_sum(n, [(1.0, {q: 3, q + 1: 3}) for q in range(n - 1)])
    assert c.pauli_sum_info(nt.Hamiltonian(nn))["packed_diag_groups"] == 0


def test_grad_options_validated_before_any_device_work():
    """Bad gradient options fail on the host (no GPU needed): an unknown
    mode, a negative segment length, checkpoints of a noisy circuit."""
    import ctypes as C

    L = nt.lib()
    c = nt.Circuit(W.OpBuilder(10).build())
    s, w, T = nt.Hamiltonian(W.pauli_sum(10, [(1.0, {0: 3})])).args()
    fake = C.c_void_p(16)  # never dereferenced: validation fails first
    for mode, ops, want in [(7, 0, nt.TC_E_UNSUPPORTED), (nt.TC_GRAD_CHECKPOINT, -1, nt.TC_E_INVALID)]:
        go = nt.tc_grad_options(mode, 0, ops)
        assert L.tc_expect_grad(c.h, None, 1, s, w, T, C.c_uint64(0), fake, None, C.byref(go), None) == want
    circ = W.noisy_su2_cz_circuit(10, 1, 0.1, np.random.default_rng(1))
    cn = nt.Circuit(circ)
    go = nt.tc_grad_options(nt.TC_GRAD_CHECKPOINT, 0, 3)
    assert L.tc_expect_grad(cn.h, None, 1, s, w, T, C.c_uint64(0), fake, None, C.byref(go), None) == \
        nt.TC_E_UNSUPPORTED


def test_apply_expect_validates_on_the_host():
    import ctypes as C

    L = nt.lib()
    c = nt.Circuit(W.hea10_workload()[0], dtype=nt.TC_C128)
    fake = C.c_void_p(16)  # never dereferenced: validation fails first
    T = (C.c_int * 1)(-1)
    assert L.tc_apply_expect(c.h, fake, 1, 1, None, None, None, None, fake, None) == nt.TC_E_INVALID
    assert L.tc_apply_expect(c.h, fake, 1, 1, C.cast(T, C.c_void_p), None, None, None, fake, None) == nt.TC_E_INVALID
    assert L.tc_apply_expect(c.h, fake, -1, 0, None, None, None, None, None, None) == nt.TC_E_INVALID
    assert L.tc_apply_expect(c.h, fake, 0, 0, None, None, None, None, None, None) == nt.TC_OK


def test_zero_rows_accept_null_buffers_and_one_row_refuses_them():
    """B = 0 is a valid call on every batched entry point: it returns TC_OK
    after the argument checks, before any launch, with NULL device buffers.
    The same NULL buffers with B = 1 are refused (TC_E_INVALID).  No GPU is
    touched either way."""
    import ctypes as C

    n = 12
    b = W.OpBuilder(n, W.INIT_PLUS)
    for q in range(n):
        b.rx(q, 0)
    b.rzz(0, 1, 1)
    c = nt.Circuit(b.build(2))
    L = nt.lib()
    s = np.zeros((1, n), np.uint8)
    s[0, 0] = 3
    w = np.ones(1)
    sp, wp = s.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p)
    T = (C.c_int * 1)(1)
    calls = {
        "apply_layers": lambda B: L.tc_apply_layers(c.h, None, B, None, 0, None, 0, None, None),
        "expect_pauli_sum": lambda B: L.tc_expect_pauli_sum(c.h, None, B, sp, wp, 1, None, None),
        "expect_grad": lambda B: L.tc_expect_grad(c.h, None, B, sp, wp, 1, 0, None, None, None, None),
        "expect_plain": lambda B: L.tc_expect_plain(c.h, None, B, sp, wp, 1, None, None, None),
        "state_norms": lambda B: L.tc_state_norms(c.h, None, B, None, None),
        "qgt": lambda B: L.tc_qgt(c.h, None, B, None, None),
        "natural_gradient": lambda B: L.tc_natural_gradient(None, None, B, 2, C.c_double(1e-3), None, None),
        "apply_expect": lambda B: L.tc_apply_expect(c.h, None, B, 1, T, sp, wp, None, None, None),
    }
    n_lc, gates, zq = W.brick200_workload()
    lc = nt.LightCone(n_lc, [(a, q) for a, q, _ in gates], zq)
    net = nt.CircuitNetwork(W.example_block_circuit(40, 6), {20: 3}, prune=2)
    calls["contract_path"] = lambda B: L.tc_contract_path(lc.h, B, None, nt.TC_TN_FP32, None, None)
    calls["tn_circuit_expect"] = lambda B: L.tc_tn_circuit_expect(net.h, B, None, nt.TC_TN_FP32, None, None)
    for name, call in calls.items():
        assert call(0) == nt.TC_OK, name
        assert call(1) == nt.TC_E_INVALID, name
    # the other arguments are still checked with no rows
    assert L.tc_contract_path(lc.h, 0, None, 7, None, None) == nt.TC_E_INVALID
    assert L.tc_tn_circuit_expect(net.h, 0, None, 7, None, None) == nt.TC_E_INVALID
    assert L.tc_natural_gradient(None, None, 0, 2, C.c_double(-1.0), None, None) == nt.TC_E_INVALID
    assert L.tc_expect_grad(c.h, None, -1, sp, wp, 1, 0, None, None, None, None) == nt.TC_E_INVALID
