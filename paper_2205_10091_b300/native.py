"""ctypes binding for libtc_b300.so (argument marshalling only).

Every computation runs in the CUDA library; this module converts Python/
torch objects to the pointers and sizes that include/tc.h declares.  Device
buffers are torch CUDA tensors (torch is used for device memory and streams
only).  There is no fallback: if the library is missing, loading fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc_b300.so")

TC_OK, TC_E_INVALID, TC_E_NOMEM, TC_E_CUDA, TC_E_TIMEOUT, TC_E_UNSUPPORTED, TC_E_BUSY, TC_E_CANCELLED = range(8)
TC_C64, TC_C128 = 0, 1
TC_TN_FP32, TC_TN_TF32X3, TC_TN_BF16X6 = 0, 1, 2  # tc_tn_precision
TC_GRAD_UNCOMPUTE, TC_GRAD_CHECKPOINT = 0, 1  # tc_grad_mode


class TcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tc status {status}: {msg}")
        self.status = status


class tc_op(C.Structure):
    _fields_ = [
        ("kind", C.c_int32),
        ("q0", C.c_int32),
        ("q1", C.c_int32),
        ("param", C.c_int32),
        ("scale", C.c_double),
        ("mat", C.c_int32),
        ("pad", C.c_int32),
        ("px", C.c_double),
        ("py", C.c_double),
        ("pz", C.c_double),
    ]


class tc_options(C.Structure):
    _fields_ = [
        ("tile_qubits_fwd", C.c_int32),
        ("tile_qubits_bwd", C.c_int32),
        ("mem_budget_bytes", C.c_int64),
        ("max_gates_per_pass", C.c_int32),
        ("specialize", C.c_int32),
        ("reserved", C.c_int32 * 6),
    ]


class tc_plan_info(C.Structure):
    _fields_ = [
        ("n_qubits", C.c_int32),
        ("n_qubits_internal", C.c_int32),
        ("n_ops", C.c_int32),
        ("n_params", C.c_int32),
        ("n_noise", C.c_int32),
        ("fwd_passes", C.c_int32),
        ("bwd_passes", C.c_int32),
        ("fwd_stages", C.c_int32),
        ("bwd_stages", C.c_int32),
        ("tile_qubits_fwd", C.c_int32),
        ("tile_qubits_bwd", C.c_int32),
        ("fwd_instrs", C.c_int32),
        ("bwd_instrs", C.c_int32),
        ("specialized_passes", C.c_int32),
        ("packed_diag_groups", C.c_int32),
        ("reserved", C.c_int32 * 1),
    ]


class tc_pauli_sum_plan_info(C.Structure):
    _fields_ = [("passes", C.c_int32), ("paired_passes", C.c_int32), ("flip_groups", C.c_int32),
                ("diag_entries", C.c_int32), ("tile_qubits", C.c_int32), ("packed_diag_groups", C.c_int32),
                ("reserved", C.c_int32 * 2)]


class tc_grad_options(C.Structure):
    _fields_ = [("mode", C.c_int32), ("max_rows", C.c_int32), ("checkpoint_ops", C.c_int32),
                ("reserved", C.c_int32 * 5)]


class tc_path_info(C.Structure):
    _fields_ = [("flops", C.c_double), ("cmacs", C.c_double), ("write", C.c_double), ("size", C.c_double),
                ("n_steps", C.c_int32), ("max_rank", C.c_int32), ("n_cone_gates", C.c_int32), ("cone_lo", C.c_int32),
                ("cone_hi", C.c_int32), ("n_inputs", C.c_int32), ("n_active", C.c_int32), ("fused", C.c_int32),
                ("smem_bytes", C.c_int32), ("fused_groups", C.c_int32), ("tc_steps", C.c_int32),
                ("tc_cmacs", C.c_double), ("max_cluster", C.c_int32), ("split_min_items", C.c_int32),
                ("split_groups", C.c_int32), ("blob_ints", C.c_int32)]


class tc_server_options(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_int64), ("max_inflight", C.c_int32), ("max_queue", C.c_int32),
                ("timeout_ms", C.c_int32), ("start_paused", C.c_int32), ("max_group_rows", C.c_int32),
                ("planner_threads", C.c_int32), ("reserved", C.c_int32 * 4)]


class tc_request(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("init", C.c_int32), ("n_ops", C.c_int32), ("n_params", C.c_int32),
                ("n_pool", C.c_int32), ("T", C.c_int32), ("ops", C.c_void_p), ("pool", C.c_void_p),
                ("theta", C.c_void_p), ("structures", C.c_void_p), ("weights", C.c_void_p)]


class tc_result(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int32), ("n_params", C.c_int32), ("energy", C.c_double),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double)]


class tc_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("cancelled", C.c_int64),
                ("timed_out", C.c_int64), ("failed", C.c_int64), ("rejected", C.c_int64), ("pending", C.c_int32),
                ("inflight", C.c_int32), ("peak_inflight", C.c_int32), ("planned", C.c_int32),
                ("bytes_in_use", C.c_int64), ("peak_bytes", C.c_int64), ("groups", C.c_int64),
                ("grouped_requests", C.c_int64)]


class tc_kernel_stat(C.Structure):
    _fields_ = [("kind", C.c_int32), ("launches", C.c_int32), ("total_ms", C.c_double), ("algo_bytes", C.c_double)]


KERNEL_KINDS = ["tile_pass_forward", "tile_pass_adjoint", "pauli_sum_pass", "finalize", "pad", "plain_term",
                "gate_tables", "one_launch_small"]

assert C.sizeof(tc_op) == W.OP_DTYPE.itemsize == 56

_lib = None

# name -> (restype, argtypes); every symbol include/tc.h declares
SIGNATURES = {
    "tc_circuit_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                    C.c_void_p, C.POINTER(C.c_void_p)]),
    "tc_circuit_destroy": (None, [C.c_void_p]),
    "tc_dm_circuit_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                       C.c_void_p, C.POINTER(C.c_void_p)]),
    "tc_dm_expect_pauli_sum": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                         C.c_void_p]),
    "tc_circuit_info": (C.c_int, [C.c_void_p, C.POINTER(tc_plan_info)]),
    "tc_pauli_sum_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                    C.POINTER(tc_pauli_sum_plan_info)]),
    "tc_apply_layers": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_uint64, C.c_void_p, C.c_int64,
                                  C.c_void_p, C.c_void_p]),
    "tc_expect_pauli_sum": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                      C.c_void_p]),
    "tc_apply_expect": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    "tc_expect_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_uint64,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tc_expect_plain": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "tc_expect_pauli_sum_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                              C.c_void_p, C.c_void_p]),
    "tc_tn_lightcone_create": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                         C.c_int, C.POINTER(C.c_void_p)]),
    "tc_tn_info": (C.c_int, [C.c_void_p, C.POINTER(tc_path_info)]),
    "tc_contract_path": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "tc_tn_set_tc_threshold": (C.c_int, [C.c_void_p, C.c_double]),
    "tc_tn_set_cluster": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "tc_tn_destroy": (None, [C.c_void_p]),
    "tc_qgt": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "tc_natural_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p,
                                      C.c_void_p]),
    "tc_tn_circuit_create": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                       C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                       C.POINTER(C.c_void_p)]),
    "tc_tn_circuit_expect": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "tc_mean_stderr": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "tc_shard_moments": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "tc_merge_moments": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "tc_state_norms": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "tc_server_create": (C.c_int, [C.POINTER(tc_server_options), C.POINTER(C.c_void_p)]),
    "tc_submit": (C.c_int, [C.c_void_p, C.POINTER(tc_request), C.POINTER(C.c_uint64)]),
    "tc_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(tc_result), C.c_void_p, C.c_int]),
    "tc_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "tc_server_resume": (C.c_int, [C.c_void_p]),
    "tc_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(tc_server_stats)]),
    "tc_server_destroy": (C.c_int, [C.c_void_p]),
    "tc_profile_begin": (C.c_int, []),
    "tc_profile_end": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "tc_last_error": (C.c_char_p, []),
    "tc_version": (C.c_char_p, []),
}


def lib():
    """Load libtc_b300.so (raises if it is missing: no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2205_10091_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int):
    if st != TC_OK:
        raise TcError(st, lib().tc_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch

        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream.cuda_stream)


def profile_begin():
    _check(lib().tc_profile_begin())


def profile_end() -> dict:
    """Per kernel kind: launches, device ms (CUDA events) and algorithmic bytes."""
    arr = (tc_kernel_stat * 16)()
    n = C.c_int()
    _check(lib().tc_profile_end(arr, 16, C.byref(n)))
    return {KERNEL_KINDS[arr[i].kind]: {"launches": arr[i].launches, "ms": arr[i].total_ms,
                                        "algo_bytes": arr[i].algo_bytes} for i in range(min(n.value, 16))}


def natural_gradient(qgt, grad, eps: float, out=None, stream=None):
    """x = (4 Re G + eps I)^-1 grad per row on the device: qgt CUDA complex128
    [B][P][P] (Circuit.qgt), grad CUDA float64 [B][P]; returns CUDA float64 [B][P]."""
    import torch

    B, P = grad.shape
    if out is None:
        out = torch.empty((B, P), dtype=torch.float64, device="cuda")
    _check(lib().tc_natural_gradient(_ptr(qgt), _ptr(grad), B, P, C.c_double(eps), _ptr(out), _stream(stream)))
    return out


def mean_stderr(x, out=None, stream=None):
    """(mean, standard error) of a CUDA float64 vector, computed on the device."""
    import torch

    if out is None:
        out = torch.empty(2, dtype=torch.float64, device="cuda")
    _check(lib().tc_mean_stderr(_ptr(x), x.numel(), _ptr(out), _stream(stream)))
    return out


def shard_moments(x, out=None, stream=None):
    """(count, mean, M2) of this rank's CUDA float64 values (tc_shard_moments)."""
    import torch

    if out is None:
        out = torch.empty(3, dtype=torch.float64, device="cuda")
    _check(lib().tc_shard_moments(_ptr(x), x.numel(), _ptr(out), _stream(stream)))
    return out


def merge_moments(parts) -> tuple:
    """(mean, standard error) from the ranks' (count, mean, M2) triples, in
    rank order (tc_merge_moments, host)."""
    p = np.ascontiguousarray(np.asarray(parts, dtype=np.float64).reshape(-1, 3))
    out = np.zeros(2)
    _check(lib().tc_merge_moments(p.ctypes.data_as(C.c_void_p), p.shape[0], out.ctypes.data_as(C.c_void_p)))
    return float(out[0]), float(out[1])


def mean_stderr_across_ranks(x, group=None):
    """Monte Carlo estimate over trajectories split across torch.distributed
    ranks: each rank's triple on its GPU, an all-gather of the triples, the
    same rank-ordered merge on every rank."""
    import torch
    import torch.distributed as dist

    m = shard_moments(x)
    if dist.get_backend(group) != "nccl":
        m = m.cpu()
    parts = [torch.empty_like(m) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, m, group=group)
    return merge_moments(torch.stack(parts).cpu().numpy())


class Hamiltonian:
    """Host copy of a Pauli sum in the ABI's layout (structures [T][n] u8, weights [T] f64)."""

    def __init__(self, ps: W.PauliSum):
        self.structures = np.ascontiguousarray(ps.structures, dtype=np.uint8)
        self.weights = np.ascontiguousarray(ps.weights, dtype=np.float64)
        self.T = int(self.weights.shape[0])

    def args(self):
        return (self.structures.ctypes.data_as(C.c_void_p), self.weights.ctypes.data_as(C.c_void_p), self.T)


class Observables:
    """K Pauli sums in tc_apply_expect's layout (term counts, concatenated
    structures and weights), marshalled once."""

    def __init__(self, sums):
        hs = [s if isinstance(s, Hamiltonian) else Hamiltonian(s) for s in sums]
        self.K = len(hs)
        self.T = (C.c_int * max(self.K, 1))(*[h.T for h in hs])
        n = hs[0].structures.shape[1] if hs else 0
        self.structures = np.ascontiguousarray(
            np.concatenate([h.structures.reshape(-1, n) for h in hs]) if hs else np.zeros((0, 0)), dtype=np.uint8)
        self.weights = np.ascontiguousarray(np.concatenate([h.weights for h in hs]) if hs else np.zeros(0),
                                            dtype=np.float64)
        self._args = (C.cast(self.T, C.c_void_p), self.structures.ctypes.data_as(C.c_void_p),
                      self.weights.ctypes.data_as(C.c_void_p))


class Circuit:
    """Owns a tc_circuit handle compiled from a workloads.Circuit."""

    def __init__(self, circ: W.Circuit, dtype: int = TC_C64, tile_fwd: int = 0, tile_bwd: int = 0,
                 mem_budget_bytes: int = 0, max_gates_per_pass: int = 0, specialize: bool = False):
        self.circ = circ
        self.n = circ.n
        self.dtype = dtype
        self.n_params = circ.n_params
        ops = np.ascontiguousarray(circ.ops, dtype=W.OP_DTYPE)
        pool = np.ascontiguousarray(np.stack([circ.pool.real, circ.pool.imag], -1).ravel(), dtype=np.float64)
        opt = tc_options(tile_fwd, tile_bwd, mem_budget_bytes, max_gates_per_pass, int(specialize))
        h = C.c_void_p()
        _check(lib().tc_circuit_create(circ.n, dtype, circ.init, ops.ctypes.data_as(C.c_void_p), len(ops),
                                       circ.n_params, pool.ctypes.data_as(C.c_void_p) if len(circ.pool) else None,
                                       len(circ.pool), C.byref(opt), C.byref(h)))
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and _lib is not None:
            _lib.tc_circuit_destroy(h)
            self.h = None

    def info(self) -> dict:
        o = tc_plan_info()
        _check(lib().tc_circuit_info(self.h, C.byref(o)))
        return {f: getattr(o, f) for f, _ in tc_plan_info._fields_ if f != "reserved"}

    def pauli_sum_info(self, ham: Hamiltonian) -> dict:
        """Host-only plan of a Pauli sum: passes, paired passes, flip groups."""
        o = tc_pauli_sum_plan_info()
        s, w, T = ham.args()
        _check(lib().tc_pauli_sum_info(self.h, s, w, T, C.byref(o)))
        return {f: getattr(o, f) for f, _ in tc_pauli_sum_plan_info._fields_ if f != "reserved"}

    @property
    def state_dtype(self):
        import torch

        return torch.complex128 if self.dtype == TC_C128 else torch.complex64

    def apply(self, params, B: int, init=None, seed: int = 0, status=None, row_offset: int = 0, out=None,
              stream=None):
        import torch

        if out is None:
            out = torch.empty((B, 1 << self.n), dtype=self.state_dtype, device="cuda")
        _check(lib().tc_apply_layers(self.h, _ptr(params), B, _ptr(init), C.c_uint64(seed), _ptr(status),
                                     C.c_int64(row_offset), _ptr(out), _stream(stream)))
        return out

    def apply_expect(self, params, obs: Observables, B: int, states=None, values=None, store_state: bool = True,
                     stream=None):
        """States and K expectations in one call (tc_apply_expect): (states or
        None, values [B][K] float64)."""
        import torch

        if states is None and store_state:
            states = torch.empty((B, 1 << self.n), dtype=self.state_dtype, device="cuda")
        if values is None:
            values = torch.empty((B, obs.K), dtype=torch.float64, device="cuda")
        t, s, w = obs._args
        _check(lib().tc_apply_expect(self.h, _ptr(params), B, obs.K, t, s, w, _ptr(states), _ptr(values),
                                     _stream(stream)))
        return states, values

    def expect(self, states, ham: Hamiltonian, out=None, stream=None):
        import torch

        B = states.shape[0]
        if out is None:
            out = torch.empty(B, dtype=torch.float64, device="cuda")
        s, w, T = ham.args()
        _check(lib().tc_expect_pauli_sum(self.h, _ptr(states), B, s, w, T, _ptr(out), _stream(stream)))
        return out

    def norms(self, states, out=None, stream=None):
        """||psi_b||^2 of each row (FP64 sums on the device): CUDA float64 [B]."""
        import torch

        B = states.shape[0]
        if out is None:
            out = torch.empty(B, dtype=torch.float64, device="cuda")
        _check(lib().tc_state_norms(self.h, _ptr(states), B, _ptr(out), _stream(stream)))
        return out

    def expect_noalloc(self, states, ham: Hamiltonian, out, stream=None, rows=None):
        """Energies through the allocation-free entry point (`out` is caller-owned;
        ``rows`` defaults to states.shape[0], 0 makes the per-device warm-up call)."""
        B = states.shape[0] if rows is None else rows
        s, w, T = ham.args()
        _check(lib().tc_expect_pauli_sum_noalloc(self.h, _ptr(states), B, s, w, T, _ptr(out), _stream(stream)))
        return out

    def qgt(self, params, out=None, stream=None):
        """Quantum geometric tensor G_ij = <d_i psi|d_j psi> - <d_i psi|psi><psi|d_j psi>
        per row: CUDA complex128 [B][P][P] (the QFI is 4 G.real)."""
        import torch

        B = params.shape[0]
        if out is None:
            out = torch.empty((B, self.n_params, self.n_params), dtype=torch.complex128, device="cuda")
        _check(lib().tc_qgt(self.h, _ptr(params), B, _ptr(out), _stream(stream)))
        return out

    def expect_grad(self, params, ham: Hamiltonian, seed: int = 0, energy=None, grad=None, max_rows: int = 0,
                    stream=None, checkpoint_ops=None):
        """Energies and gradients of every row (tc_expect_grad).  checkpoint_ops:
        None = uncompute mode; an int = TC_GRAD_CHECKPOINT with that many ops
        per segment (0 = four segments)."""
        import torch

        B = params.shape[0]
        if energy is None:
            energy = torch.empty(B, dtype=torch.float64, device="cuda")
        if grad is None:
            grad = torch.empty((B, self.n_params), dtype=torch.float64, device="cuda")
        s, w, T = ham.args()
        go = tc_grad_options(TC_GRAD_UNCOMPUTE if checkpoint_ops is None else TC_GRAD_CHECKPOINT, max_rows,
                             0 if checkpoint_ops is None else int(checkpoint_ops))
        _check(lib().tc_expect_grad(self.h, _ptr(params), B, s, w, T, C.c_uint64(seed), _ptr(energy), _ptr(grad),
                                    C.byref(go), _stream(stream)))
        return energy, grad

    def expect_plain(self, params, ham: Hamiltonian, work, energy=None, stream=None):
        import torch

        B = params.shape[0]
        if energy is None:
            energy = torch.empty(B, dtype=torch.float64, device="cuda")
        s, w, T = ham.args()
        _check(lib().tc_expect_plain(self.h, _ptr(params), B, s, w, T, _ptr(work), _ptr(energy), _stream(stream)))
        return energy


_EXPECT_FN = None


def _expect_fn():
    """torch.autograd.Function over tc_expect_grad (built on first use, so
    that importing this module does not import torch)."""
    global _EXPECT_FN
    if _EXPECT_FN is None:
        import torch

        class ExpectGrad(torch.autograd.Function):
            # forward: one tc_expect_grad call (energies and per-row
            # gradients from the adjoint sweep); backward: the cached gradient
            # rows scaled by the incoming gradient of each energy
            @staticmethod
            def forward(ctx, params, circuit, ham, seed):
                e, g = circuit.expect_grad(params.detach().to(torch.float64).contiguous(), ham, seed=seed)
                ctx.save_for_backward(g)
                return e

            @staticmethod
            def backward(ctx, grad_e):
                (g,) = ctx.saved_tensors
                return grad_e[:, None] * g, None, None, None

        _EXPECT_FN = ExpectGrad
    return _EXPECT_FN


def expectation(circuit: "Circuit", params, ham: Hamiltonian, seed: int = 0):
    """E_b = <psi(theta_b)|H|psi(theta_b)> for every row of ``params`` (CUDA
    float64 [B][P]) as a differentiable torch function: the paper's
    value_and_grad (Section "Gradients, optimization and variational
    algorithms") with the gradient from the library's adjoint sweep.  Rows
    are independent (vectorized_value_and_grad with argnums equal to
    vectorized_argnums); a parameter vector shared by all rows, expanded to
    [B][P], gets the row sum (the summed form)."""
    return _expect_fn().apply(params, circuit, ham, seed)


class DensityMatrixCircuit(Circuit):
    """A tc_dm_circuit_create handle: rho under the circuit's gates and exact
    Pauli channels, held as [B][4^n] vectorised density matrices."""

    def __init__(self, circ: W.Circuit, dtype: int = TC_C64):
        self.circ = circ
        self.n = 2 * circ.n  # qubits of the vectorised state (apply() returns [B][4^n])
        self.n_rho = circ.n
        self.dtype = dtype
        self.n_params = circ.n_params
        ops = np.ascontiguousarray(circ.ops, dtype=W.OP_DTYPE)
        pool = np.ascontiguousarray(np.stack([circ.pool.real, circ.pool.imag], -1).ravel(), dtype=np.float64)
        h = C.c_void_p()
        _check(lib().tc_dm_circuit_create(circ.n, dtype, circ.init, ops.ctypes.data_as(C.c_void_p), len(ops),
                                          circ.n_params, pool.ctypes.data_as(C.c_void_p) if len(circ.pool) else None,
                                          len(circ.pool), None, C.byref(h)))
        self.h = h

    def expect(self, rho, ham: Hamiltonian, out=None, stream=None):
        """tr(rho_b H) for every row of rho ([B][4^n])."""
        import torch

        B = rho.shape[0]
        if out is None:
            out = torch.empty(B, dtype=torch.float64, device="cuda")
        s, w, T = ham.args()
        _check(lib().tc_dm_expect_pauli_sum(self.h, _ptr(rho), B, s, w, T, _ptr(out), _stream(stream)))
        return out


class LightCone:
    """Light-cone tensor-network plan for <Z..Z> of a two-qubit-gate circuit."""

    def __init__(self, n_qubits: int, gate_qubits, z_qubits, rank_cap: int = 18, path=None, greedy_trials: int = 1):
        gq = np.ascontiguousarray(np.asarray(gate_qubits, dtype=np.int32).reshape(-1, 2))
        zq = np.ascontiguousarray(np.asarray(z_qubits, dtype=np.int32))
        pth = None if path is None else np.ascontiguousarray(np.asarray(path, dtype=np.int32).reshape(-1, 2))
        h = C.c_void_p()
        _check(lib().tc_tn_lightcone_create(n_qubits, gq.ctypes.data_as(C.c_void_p), len(gq),
                                            zq.ctypes.data_as(C.c_void_p), len(zq), rank_cap, greedy_trials,
                                            None if pth is None else pth.ctypes.data_as(C.c_void_p),
                                            0 if pth is None else len(pth), C.byref(h)))
        self.h = h
        self.n_gates = len(gq)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and _lib is not None:
            _lib.tc_tn_destroy(h)
            self.h = None

    def info(self) -> dict:
        o = tc_path_info()
        _check(lib().tc_tn_info(self.h, C.byref(o)))
        return {f: getattr(o, f) for f, _ in tc_path_info._fields_ if f != "reserved"}

    def set_tc_threshold(self, min_cmacs: float):
        """Steps of at least min_cmacs complex multiply-adds run on tensor cores
        in the split-precision modes."""
        _check(lib().tc_tn_set_tc_threshold(self.h, C.c_double(min_cmacs)))

    def set_cluster(self, max_cluster: int = 8, split_min_items: int = 2048):
        """Fused launch with few instances: CTAs per instance (1 = off) and the
        group size from which a group is split over them."""
        _check(lib().tc_tn_set_cluster(self.h, int(max_cluster), int(split_min_items)))

    def contract(self, d_gates, out=None, stream=None, precision: int = TC_TN_FP32):
        """d_gates: CUDA complex64 tensor [B][n_gates][4][4]; returns CUDA float64 [B][2]."""
        import torch

        B = d_gates.shape[0]
        if out is None:
            out = torch.empty((B, 2), dtype=torch.float64, device="cuda")
        _check(lib().tc_contract_path(self.h, B, _ptr(d_gates), precision, _ptr(out), _stream(stream)))
        return out


class CircuitNetwork:
    """<P> of a parameterised circuit contracted as one tensor network
    (tc_tn_circuit_create / tc_tn_circuit_expect).  ``pauli``: {qubit: code}
    with codes 1..3 = X, Y, Z; ``prune``: 0 whole network, 1 causal cone,
    2 cone without commuting diagonal gates; ``split``: rank-2 gates (RZZ, CZ,
    CNOT) as two tensors; ``greedy_trials``: > 1 keeps the cheapest of that
    many greedy paths (the first deterministic, the rest randomised)."""

    def __init__(self, circ: W.Circuit, pauli: dict, prune: int = 2, split: bool = True, rank_cap: int = 18,
                 greedy_trials: int = 1, path=None):
        ops = np.ascontiguousarray(circ.ops, dtype=W.OP_DTYPE)
        pool = np.ascontiguousarray(np.stack([circ.pool.real, circ.pool.imag], -1).ravel(), dtype=np.float64)
        codes = np.zeros(circ.n, dtype=np.uint8)
        for q, c in pauli.items():
            codes[q] = c
        pth = None if path is None else np.ascontiguousarray(np.asarray(path, dtype=np.int32).reshape(-1, 2))
        h = C.c_void_p()
        _check(lib().tc_tn_circuit_create(circ.n, circ.init, ops.ctypes.data_as(C.c_void_p), len(ops), circ.n_params,
                                          pool.ctypes.data_as(C.c_void_p) if len(circ.pool) else None,
                                          len(circ.pool), codes.ctypes.data_as(C.c_void_p), prune, int(split),
                                          rank_cap, greedy_trials,
                                          None if pth is None else pth.ctypes.data_as(C.c_void_p),
                                          0 if pth is None else len(pth), C.byref(h)))
        self.h = h
        self.n_params = circ.n_params

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and _lib is not None:
            _lib.tc_tn_destroy(h)
            self.h = None

    def info(self) -> dict:
        o = tc_path_info()
        _check(lib().tc_tn_info(self.h, C.byref(o)))
        return {f: getattr(o, f) for f, _ in tc_path_info._fields_ if f != "reserved"}

    def set_tc_threshold(self, min_cmacs: float):
        """Steps of at least min_cmacs complex multiply-adds run on tensor cores
        in the split-precision modes."""
        _check(lib().tc_tn_set_tc_threshold(self.h, C.c_double(min_cmacs)))

    def set_cluster(self, max_cluster: int = 8, split_min_items: int = 2048):
        """Fused launch with few instances: CTAs per instance (1 = off) and the
        group size from which a group is split over them."""
        _check(lib().tc_tn_set_cluster(self.h, int(max_cluster), int(split_min_items)))

    def expect(self, d_params, B: int | None = None, out=None, stream=None, precision: int = TC_TN_FP32):
        """d_params: CUDA float32 [B][n_params]; returns CUDA float64 [B][2] (Re, Im)."""
        import torch

        if B is None:
            B = d_params.shape[0]
        if out is None:
            out = torch.empty((B, 2), dtype=torch.float64, device="cuda")
        _check(lib().tc_tn_circuit_expect(self.h, B, _ptr(d_params), precision, _ptr(out), _stream(stream)))
        return out


class Server:
    """Continuous-batching request server (tc_server_*)."""

    def __init__(self, mem_budget_bytes: int = 0, max_inflight: int = 0, max_queue: int = 0, timeout_ms: int = 0,
                 start_paused: bool = False, max_group_rows: int = 0, planner_threads: int = 0):
        o = tc_server_options(mem_budget_bytes, max_inflight, max_queue, timeout_ms, int(start_paused),
                              max_group_rows, planner_threads)
        h = C.c_void_p()
        _check(lib().tc_server_create(C.byref(o), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().tc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        if _lib is not None:
            self.close()

    def submit(self, circ: W.Circuit, theta, ham: W.PauliSum) -> int:
        ops = np.ascontiguousarray(circ.ops, dtype=W.OP_DTYPE)
        pool = np.ascontiguousarray(np.stack([circ.pool.real, circ.pool.imag], -1).ravel(), dtype=np.float64)
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).ravel())
        st = np.ascontiguousarray(ham.structures, dtype=np.uint8)
        w = np.ascontiguousarray(ham.weights, dtype=np.float64)
        req = tc_request(circ.n, circ.init, len(ops), circ.n_params, len(circ.pool), len(w),
                         ops.ctypes.data, pool.ctypes.data if len(circ.pool) else None, th.ctypes.data,
                         st.ctypes.data, w.ctypes.data)
        rid = C.c_uint64()
        _check(lib().tc_submit(self.h, C.byref(req), C.byref(rid)))
        return rid.value

    def poll(self, rid: int, max_params: int = 256):
        """None while pending/running, else a dict (the id is then released)."""
        r = tc_result()
        g = np.zeros(max_params)
        st = lib().tc_poll(self.h, C.c_uint64(rid), C.byref(r), g.ctypes.data_as(C.c_void_p), max_params)
        if st == TC_E_BUSY:
            return None
        _check(st)
        return {"id": r.id, "status": r.status, "energy": r.energy, "grad": g[:r.n_params].copy(),
                "t_submit": r.t_submit, "t_start": r.t_start, "t_done": r.t_done,
                "error": None if r.status == TC_OK else lib().tc_last_error().decode()}

    def cancel(self, rid: int):
        _check(lib().tc_cancel(self.h, C.c_uint64(rid)))

    def resume(self):
        _check(lib().tc_server_resume(self.h))

    def stats(self) -> dict:
        o = tc_server_stats()
        _check(lib().tc_server_get_stats(self.h, C.byref(o)))
        return {f: getattr(o, f) for f, _ in tc_server_stats._fields_}

    def wait(self, rid: int, timeout_s: float = 60.0, sleep_s: float = 0.0002):
        import time

        t0 = time.monotonic()
        while True:
            r = self.poll(rid)
            if r is not None:
                return r
            if time.monotonic() - t0 > timeout_s:
                raise TimeoutError(f"request {rid} not done after {timeout_s} s")
            time.sleep(sleep_s)
