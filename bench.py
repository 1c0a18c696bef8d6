"""Benchmark: batched energy + gradient evaluations per second.

Workload: 20-qubit 1D TFIM VQE, H = -sum Z_i Z_{i+1} - sum X_i, 10 layers of
[RZZ(g_l) on all 19 bonds, RX(b_l) on all qubits] from |+>^20, a batch of 1024
parameter sets per GPU with angles ~ N(0, 0.3^2), complex64 states (8 MiB
each).  One step = energy and full gradient for every row of the batch
(tc_expect_grad: forward sweep, Pauli-sum pass, adjoint sweep, reduction).

Timed region: W untimed warm-up steps, then K steps bracketed by a barrier and
torch.cuda.synchronize(), timed with CUDA events on the launch stream; the
states (2 x 8 GiB) are larger than L2, so no flush is needed.  `value` is the
whole-job rate: rows of all ranks / max-over-ranks time.  `e2e` repeats the
measurement with the parameters in pinned host memory, copied in each step,
and energies + gradients copied back each step.

--impl reference times the FP64 oracle on the host cores (the reference arm of
this benchmark; a deliberately slow restatement, not a target).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2205_10091_b300 import workloads as W  # noqa: E402

METRIC = "batched energy+grad evals/s"
UNIT = "evals/s"
N_QUBITS, LAYERS, BATCH = 20, 10, 1024
WORKLOAD = "tfim20_l10_b1024_c64_energy_grad"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------
# oracle (CPU) legs: the FP64 numpy oracle in worker processes (spawn start
# method, one BLAS thread each), never inside a timed GPU region
# ---------------------------------------------------------------------------
# the oracle is memory-bound (numpy einsum over 16 MiB complex128 states), so
# more processes than this add little on the host; the reference arm's
# steps use fewer still, so that K + W steps end within a few minutes
MAX_ORACLE_WORKERS = 8
REFERENCE_STEP_ROWS = 2


def host_info() -> dict:
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or None}


def _worker_init():
    global _WORKER_LIMIT
    try:
        from threadpoolctl import threadpool_limits

        _WORKER_LIMIT = threadpool_limits(1)
    except Exception:  # pragma: no cover
        _WORKER_LIMIT = None


def oracle_pool(workers: int):
    import multiprocessing as mp

    return mp.get_context("spawn").Pool(workers, initializer=_worker_init)


def tfim_energy_task(args):
    """Oracle energy of one TFIM row, optionally with theta[k] shifted by h:
    returns (energy, seconds)."""
    from oracle import statevector as sv

    n, layers, batch, seed, row, k, h = args
    circ, theta, ham = W.tfim_workload(n, layers, batch, seed)
    th = theta[row].copy()
    if k >= 0:
        th[k] += h
    t0 = time.perf_counter()
    e = sv.energy(sv.run_circuit(circ, th), n, ham)[0]
    return e, time.perf_counter() - t0


def oracle_rows_wall(pool, workers: int, seed: int, first_row: int = 0):
    """Forward + energy of `workers` rows, one per worker, in parallel: wall seconds."""
    tasks = [(N_QUBITS, LAYERS, BATCH, seed, (first_row + i) % BATCH, -1, 0.0) for i in range(workers)]
    t0 = time.perf_counter()
    pool.map(tfim_energy_task, tasks, chunksize=1)
    return time.perf_counter() - t0


def _evals_per_grad() -> int:
    # central differences: the energy plus two shifted energies per parameter
    return 2 * 2 * LAYERS + 1


def cpu_baseline(pool, workers: int) -> dict:
    wall = oracle_rows_wall(pool, workers, W.SEED_TFIM20)
    value = workers / (wall * _evals_per_grad())
    hi = host_info()
    return {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", **hi,
            "sample": (f"{workers} rows of the workload, FP64 numpy forward+energy, one row per process "
                       f"({workers} spawn processes x 1 thread on {hi['nproc']} host cores): {wall:.2f} s wall; "
                       f"energy+gradient by central differences costs {_evals_per_grad()} such evaluations "
                       f"per row, so value = rows / (wall x {_evals_per_grad()}) (extrapolated)")}


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    workers = min(os.cpu_count() or 1, REFERENCE_STEP_ROWS)
    with oracle_pool(workers) as pool:
        for w in range(args.warmup):
            oracle_rows_wall(pool, workers, W.SEED_TFIM20, first_row=w * workers)
        walls = [oracle_rows_wall(pool, workers, W.SEED_TFIM20, first_row=(args.warmup + k) * workers)
                 for k in range(args.steps)]
    wall = float(np.mean(walls))
    value = workers / (wall * _evals_per_grad())
    hi = host_info()
    sample = (f"each step: FP64 numpy forward+energy of {workers} rows of the workload, one per process "
              f"({workers} spawn processes x 1 thread on {hi['nproc']} host cores); ms_per_step is that "
              f"measured wall time.  value extrapolates: energy+gradient by central differences costs "
              f"{_evals_per_grad()} forward+energy evaluations per row")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_qubits": N_QUBITS, "layers": LAYERS, "batch_per_gpu": BATCH},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample, **hi},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def headline_errors(pool, energy, grad, seed: int, rows=(0, 517, 1023), grad_samples=((517, 3), (1023, 18)),
                    h: float = 1e-4) -> dict:
    """Sampled rows of the timed batch against the FP64 oracle: energies, and
    gradient entries by central differences (run in the oracle pool)."""
    tasks = [(N_QUBITS, LAYERS, BATCH, seed, r, -1, 0.0) for r in rows]
    for r, k in grad_samples:
        tasks += [(N_QUBITS, LAYERS, BATCH, seed, r, k, h), (N_QUBITS, LAYERS, BATCH, seed, r, k, -h)]
    res = [e for e, _ in pool.map(tfim_energy_task, tasks, chunksize=1)]
    e_ref = res[:len(rows)]
    fd = [(res[len(rows) + 2 * i] - res[len(rows) + 2 * i + 1]) / (2 * h) for i in range(len(grad_samples))]
    de = [abs(float(energy[r]) - e_ref[i]) for i, r in enumerate(rows)]
    dg = [abs(float(grad[r, k]) - fd[i]) for i, (r, k) in enumerate(grad_samples)]
    return {"energy_max_abs": max(de), "energy_rows": list(rows), "energy_tol": "1e-5 max(|E|, 1)",
            "grad_max_abs": max(dg), "grad_samples": [list(x) for x in grad_samples],
            "grad_ref": f"central differences, h = {h:g}", "grad_tol": "1e-4 max(|g|_inf, 1)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def rank_workload(rank: int):
    """Each rank's own batch of parameter rows (weak scaling: rows are
    independent problems, no data-path collective)."""
    return W.tfim_workload(N_QUBITS, LAYERS, BATCH, seed=W.SEED_TFIM20 + rank)


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's time (the job's time), identical on every rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(rows_per_rank: int, world: int, ms: float) -> float:
    """Whole-job rows per second: every rank's rows over the slowest rank's time."""
    return world * rows_per_rank / (ms / 1e3)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2205_10091_b300 import native as nt

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    # the oracle's worker processes (rank 0 at N=1 only): spawned, outside
    # every timed region
    pool, workers = None, 0
    if world == 1 and not args.no_oracle:
        workers = min(os.cpu_count() or 1, MAX_ORACLE_WORKERS)
        pool = oracle_pool(workers)

    # each rank owns an independent batch of parameter sets (weak scaling)
    circ, theta, ham = rank_workload(rank)
    # the forward and adjoint passes compiled for this circuit at plan time
    # (before any timing; the default plan-interpreting kernels with --no-specialize)
    t_plan = time.perf_counter()
    c = nt.Circuit(circ, specialize=not args.no_specialize)
    t_plan = time.perf_counter() - t_plan
    H = nt.Hamiltonian(ham)
    B, P = theta.shape
    stream = torch.cuda.current_stream()
    d_theta = torch.as_tensor(theta, device="cuda")
    energy = torch.empty(B, dtype=torch.float64, device="cuda")
    grad = torch.empty((B, P), dtype=torch.float64, device="cuda")

    for _ in range(args.warmup):
        c.expect_grad(d_theta, H, energy=energy, grad=grad)
    torch.cuda.synchronize()

    # ---- device-resident timed region --------------------------------------
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    nt.profile_begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        c.expect_grad(d_theta, H, energy=energy, grad=grad)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = nt.profile_end()
    clk = clocks.stop()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    value = job_rate(B, world, ms)

    # ---- end to end through host buffers -------------------------------------
    h_theta = torch.as_tensor(theta).pin_memory()
    h_e = torch.empty(B, dtype=torch.float64).pin_memory()
    h_g = torch.empty((B, P), dtype=torch.float64).pin_memory()
    for _ in range(2):
        d_theta.copy_(h_theta, non_blocking=True)
        c.expect_grad(d_theta, H, energy=energy, grad=grad)
        h_e.copy_(energy, non_blocking=True)
        h_g.copy_(grad, non_blocking=True)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        d_theta.copy_(h_theta, non_blocking=True)
        c.expect_grad(d_theta, H, energy=energy, grad=grad)
        h_e.copy_(energy, non_blocking=True)
        h_g.copy_(grad, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    e2e = {"value": job_rate(B, world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": int(h_theta.numel() * 8),
           "d2h_bytes_per_step": int((h_e.numel() + h_g.numel()) * 8)}

    # ---- plain per-circuit path: one row, unfused sweeps, forward + energy ----
    work = torch.empty((1, 1 << N_QUBITS), dtype=torch.complex64, device="cuda")
    e_plain = torch.empty(1, dtype=torch.float64, device="cuda")
    one = d_theta[:1].contiguous()
    for _ in range(2):
        c.expect_plain(one, H, work, energy=e_plain)
    torch.cuda.synchronize()
    n_plain = 20
    e0.record(stream)
    for _ in range(n_plain):
        c.expect_plain(one, H, work, energy=e_plain)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / n_plain

    # ---- FP64 norm check of every row's final state (after the timed region) --
    st_all = c.apply(d_theta, B)
    norm_dev = float((c.norms(st_all) - 1.0).abs().max().item())
    del st_all
    torch.cuda.synchronize()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel --------------------------------------
    peaks, peak_src = _peaks()
    top = max(prof.items(), key=lambda kv: kv[1]["ms"])
    kname, kst = top
    achieved = kst["algo_bytes"] / (kst["ms"] / 1e3) / 1e9
    hbm = float(peaks["hbm_gbs"])
    traffic = _traffic(kname)
    launches = sum(v["launches"] for v in prof.values())
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_qubits": N_QUBITS, "layers": LAYERS, "batch_per_gpu": B,
                   "params_per_row": P, "hamiltonian_terms": int(H.T), "parallelism": f"dp{world}",
                   "pass_kernels": "specialised at plan time" if not args.no_specialize else "plan-interpreting",
                   "plan_seconds": t_plan,
                   "l2": "inputs larger than L2 (psi and lambda: 2 x 8 GiB per 1024 rows)"},
        "e2e": e2e,
        "gpu_launches": launches,
        "kernels": {k: {"launches": v["launches"], "ms_per_launch": v["ms"] / max(v["launches"], 1),
                        "share": v["ms"] / max(sum(x["ms"] for x in prof.values()), 1e-9),
                        "algo_gb_per_launch": v["algo_bytes"] / max(v["launches"], 1) / 1e9}
                    for k, v in prof.items()},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": f"{peak_src} hbm_gbs",
                     "traffic": traffic, "binding": _binding(kname)},
        "plain_path": {"value": 1e3 / plain_ms, "unit": "forward+energy evals/s", "rows": 1,
                       "ms_per_eval": plain_ms, "what": "unfused: one HBM sweep per gate, one per Pauli term"},
        "clocks": clk,
    }
    err = {"norm_max_dev": norm_dev, "norm_rows": B, "norm_tol": 1e-5}
    if pool is not None:
        err.update(headline_errors(pool, energy.cpu().numpy(), grad.cpu().numpy(), W.SEED_TFIM20 + rank))
    out["err_vs_oracle"] = err
    if world == 1 and not args.no_extra:
        out["workloads"] = extra_workloads(check=not args.no_oracle)
    if pool is not None and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(pool, workers)
    if pool is not None:
        pool.close()
        pool.join()
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# the other hot-path workloads (bounded, rank 0 at N=1)
# ---------------------------------------------------------------------------
# FP32 FMA rate of this B300 measured by a CUDA-core FMA probe (34 T lane-FMA/s)
FP32_TFLOPS_PROBE = 68.0


def _time_cuda(fn, reps: int, warm: int = 3) -> float:
    """Mean ms per call of fn() on the current stream (CUDA events)."""
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extra_workloads(serve_rates=(250.0, 500.0, 1000.0, 2000.0), serve_seconds: float = 2.0,
                    check: bool = True) -> dict:
    """Each block times one workload of the hot path and, with check=True,
    states the error of sampled results against the FP64 oracle
    (`err_vs_oracle`, computed after the timing)."""
    import time

    import torch

    from paper_2205_10091_b300 import native as nt

    if check:
        from oracle import gradients as G
        from oracle import noise as NZ
        from oracle import statevector as sv
        from oracle import tensornet as T
    out = {}
    # ---- HEA-10, complex128: one circuit, state + two observables ----------
    circ, theta, obs = W.hea10_workload()
    c = nt.Circuit(circ, dtype=nt.TC_C128)
    d_th = torch.as_tensor(theta, device="cuda")
    st = torch.empty((1, 1 << 10), dtype=torch.complex128, device="cuda")
    Hs = [nt.Hamiltonian(o) for o in obs]
    O2 = nt.Observables(obs)
    vals = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    e_out = [torch.empty(1, dtype=torch.float64, device="cuda") for _ in Hs]

    def one():  # the state and both observables in one call (one launch)
        c.apply_expect(d_th, O2, 1, states=st, values=vals)

    def one_tile():  # the same through the tile passes: state, then one Pauli-sum call per observable
        c.apply(d_th, 1, out=st)
        for H, e in zip(Hs, e_out):
            c.expect(st, H, out=e)

    def median_us(fn, n=1000):
        # per-call latency: CUDA events around each call, median
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for e0, e1 in ev:
            e0.record()
            fn()
            e1.record()
        torch.cuda.synchronize()
        return float(np.median([e0.elapsed_time(e1) for e0, e1 in ev])) * 1e3

    one_tile()
    med_tile = median_us(one_tile)
    zz_tile, x5_tile = float(e_out[0].item()), float(e_out[1].item())
    ms1 = _time_cuda(one, 200)
    med1 = median_us(one)
    Bb = 65536
    d_thb = torch.as_tensor(np.tile(theta, (Bb, 1)), device="cuda")
    stb = torch.empty((Bb, 1 << 10), dtype=torch.complex128, device="cuda")
    valb = torch.empty((Bb, 2), dtype=torch.float64, device="cuda")
    msb = _time_cuda(lambda: c.apply(d_thb, Bb, out=stb), 5, warm=2)
    msb1 = _time_cuda(lambda: c.apply_expect(d_thb, O2, Bb, states=stb, values=valb), 5, warm=2)
    v = vals.cpu().numpy()[0]
    out["hea10_c128"] = {"us_per_circuit_state_and_2_observables": ms1 * 1e3,
                         "us_median_of_1000": med1, "path": "tc_apply_expect, one cluster launch",
                         "us_median_of_1000_tile_passes": med_tile,
                         "batched_states_per_s": Bb / (msb / 1e3),
                         "batched_states_and_2_observables_per_s": Bb / (msb1 / 1e3), "batch": Bb,
                         "zz01": float(v[0]), "x5": float(v[1])}
    if check:
        ref = sv.run_circuit(circ, theta[0])
        got = st[0].cpu().numpy()
        out["hea10_c128"]["err_vs_oracle"] = {
            "amp_max_abs": float(np.abs(got - ref).max()), "amp_tol": 1e-12,
            "obs_max_abs": max(abs(float(v[i]) - sv.energy(ref, 10, o)[0]) for i, o in enumerate(obs)),
            "obs_tile_path_max_abs": max(abs(x - sv.energy(ref, 10, o)[0]) for x, o in zip((zz_tile, x5_tile), obs)),
            "batched_amp_max_abs": float(np.abs(stb[Bb - 1].cpu().numpy() - ref).max())}
    del stb, d_thb
    # ---- light-cone TN, 200-qubit brickwork depth 8, <Z99 Z100> -----------
    n, gates, zq = W.brick200_workload()
    lc = nt.LightCone(n, [(a, b) for a, b, _ in gates], zq, greedy_trials=64)
    g1 = torch.as_tensor(np.stack([u for (_, _, u) in gates])[None].astype(np.complex64), device="cuda")
    o1 = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    ms_tn = _time_cuda(lambda: lc.contract(g1, out=o1), 200)
    Bt = 1024
    gb = torch.as_tensor(np.stack([np.stack([u for (_, _, u) in W.brickwork_u4(n, 8, np.random.default_rng(s))])
                                   for s in range(Bt)]).astype(np.complex64), device="cuda")
    ob = torch.empty((Bt, 2), dtype=torch.float64, device="cuda")
    ms_tnb = _time_cuda(lambda: lc.contract(gb, out=ob), 20)
    info = lc.info()
    tn_err = None
    if check:
        seeds = (0, 511, 1023)
        d_b = [abs(float(ob[sd, 0].item()) - T.cone_statevector_expectation(
            W.brickwork_u4(n, 8, np.random.default_rng(sd)), zq).real) for sd in seeds]
        tn_err = {"zz_abs": abs(float(o1[0, 0].item()) - T.cone_statevector_expectation(gates, zq).real),
                  "batched_zz_max_abs": max(d_b), "batched_seeds": list(seeds), "tol": 1e-5,
                  "oracle": "FP64 state vector of the 16-qubit light cone"}
    modes = {}
    for mname, prec in (("tf32x3", nt.TC_TN_TF32X3), ("bf16x6", nt.TC_TN_BF16X6)):
        om = torch.empty((1, 2), dtype=torch.float64, device="cuda")
        ms_m = _time_cuda(lambda: lc.contract(g1, out=om, precision=prec), 50)
        modes[mname] = {"us_per_contraction": ms_m * 1e3, "tc_steps": lc.info()["tc_steps"],
                        "zz_abs_err_vs_oracle": (abs(float(om[0, 0].item()) -
                                                     T.cone_statevector_expectation(gates, zq).real)
                                                 if check else None)}
    out["brick200_lightcone_tn"] = {
        "err_vs_oracle": tn_err,
        "precision_modes": modes,
        "zz": float(o1[0, 0].item()), "us_per_contraction": ms_tn * 1e3,
        "batched_contractions_per_s": Bt / (ms_tnb / 1e3), "batch_seeds": Bt,
        "log10_flops": float(np.log10(info["flops"])), "log2_size": float(np.log2(info["size"])),
        "log2_write": float(np.log2(info["write"])), "steps": info["n_steps"], "cone_gates": info["n_cone_gates"],
        "executor": {"fused": info["fused"], "level_groups": info["fused_groups"],
                     "live_kib": info["smem_bytes"] / 1024, "b1": f"{info['max_cluster']}-CTA cluster",
                     "split_groups_b1": info["split_groups"], "batched": "one CTA per seed"},
        "timing": "CUDA events around back-to-back calls (B = 1: 200 calls; batched: 20)"}
    del gb, ob
    # ---- contraction testbed: 40 qubits, 6 layers of ZZ + RX, <Z_20> -------
    cb40 = W.example_block_circuit(40, 6)
    paths = {}
    for name, kw in (("whole_network_greedy", dict(prune=0, rank_cap=26)),
                     ("whole_network_best_of_16", dict(prune=0, rank_cap=26, greedy_trials=16)),
                     ("causal_cone_greedy", dict(prune=1, rank_cap=26)),
                     ("commuting_cone_greedy", dict(prune=2)),
                     ("commuting_cone_best_of_64", dict(prune=2, greedy_trials=64))):
        pi = nt.CircuitNetwork(cb40, {20: 3}, split=True, **kw).info()
        paths[name] = {"log10_flops_2_per_cmac": float(np.log10(2 * pi["cmacs"])),
                       "log2_size": float(np.log2(pi["size"])), "log2_write": float(np.log2(pi["write"])),
                       "steps": pi["n_steps"], "kept_ops": pi["n_cone_gates"], "qubits": pi["n_active"]}
    net40 = nt.CircuitNetwork(cb40, {20: 3}, split=True, prune=2, greedy_trials=64)
    th1 = torch.ones((1, cb40.n_params), dtype=torch.float32, device="cuda")
    o40 = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    ms40 = _time_cuda(lambda: net40.expect(th1, out=o40), 200)
    B40 = 1024
    th40 = torch.as_tensor(np.random.default_rng(1009).uniform(-1.5, 1.5, (B40, cb40.n_params)).astype(np.float32),
                           device="cuda")
    o40b = torch.empty((B40, 2), dtype=torch.float64, device="cuda")
    ms40b = _time_cuda(lambda: net40.expect(th40, out=o40b), 20)
    whole = nt.CircuitNetwork(cb40, {20: 3}, split=True, prune=0, rank_cap=26, greedy_trials=16)
    o40w = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    ms40w = _time_cuda(lambda: whole.expect(th1, out=o40w), 20)
    # the whole network per precision mode: one instance, and 1024 weight rows per launch
    Bw = 1024
    thw = th40[:Bw].contiguous()
    ref_w = (T.circuit_window_expectation(cb40, np.ones(cb40.n_params), {20: 3}, 13, 27).real if check else None)
    wmodes = {}
    for mname, prec in (("fp32", nt.TC_TN_FP32), ("tf32x3", nt.TC_TN_TF32X3), ("bf16x6", nt.TC_TN_BF16X6)):
        o1m = torch.empty((1, 2), dtype=torch.float64, device="cuda")
        obm = torch.empty((Bw, 2), dtype=torch.float64, device="cuda")
        ms1m = _time_cuda(lambda: whole.expect(th1, out=o1m, precision=prec), 20)
        msbm = _time_cuda(lambda: whole.expect(thw, out=obm, precision=prec), 5, warm=2)
        wi = whole.info()
        wmodes[mname] = {"us_per_contraction": ms1m * 1e3, "batched_contractions_per_s": Bw / (msbm / 1e3),
                         "batch": Bw, "tc_steps": wi["tc_steps"] if prec else 0,
                         "tflops_batched": 8 * wi["cmacs"] * Bw / (msbm / 1e3) / 1e12,
                         "z20_abs_err_vs_oracle": abs(float(o1m[0, 0].item()) - ref_w) if check else None}
    eb_err = None
    if check:
        win = lambda th: T.circuit_window_expectation(cb40, th, {20: 3}, 13, 27).real  # noqa: E731
        ref1 = win(np.ones(cb40.n_params))
        th40h = th40.cpu().numpy().astype(np.float64)
        eb_err = {"z20_abs": abs(float(o40[0, 0].item()) - ref1),
                  "z20_whole_network_abs": abs(float(o40w[0, 0].item()) - ref1),
                  "batched_max_abs": max(abs(float(o40b[b, 0].item()) - win(th40h[b])) for b in (0, 1023)),
                  "oracle": "FP64 state vector of qubits 13..27 (exact: the gates outside commute with the "
                            "evolved Z_20)"}
    out["example_block40_tn"] = {
        "err_vs_oracle": eb_err,
        "z20_all_ones": float(o40[0, 0].item()), "z20_whole_network": float(o40w[0, 0].item()),
        "us_per_contraction": ms40 * 1e3, "batched_contractions_per_s": B40 / (ms40b / 1e3), "batch": B40,
        "us_per_whole_network_contraction": ms40w * 1e3,
        "whole_network_precision_modes": wmodes,
        "paper_default_row": {"log10_flops": 7.373, "log2_size": 12, "log2_write": 20.171},
        "paths": paths}
    del net40, whole
    # ---- noisy 16-qubit trajectories ---------------------------------------
    circ, n_traj, seed, obs = W.noisy16_workload()
    t_nz = time.monotonic()
    c = nt.Circuit(circ, specialize=True)  # pass kernels compiled for the circuit (outside the timed region)
    t_nz = time.monotonic() - t_nz
    sts = torch.empty((n_traj, 1 << 16), dtype=torch.complex64, device="cuda")
    Hs = [nt.Hamiltonian(o) for o in obs]
    vals = [torch.empty(n_traj, dtype=torch.float64, device="cuda") for _ in Hs]
    ests = [torch.empty(2, dtype=torch.float64, device="cuda") for _ in Hs]

    def traj():
        c.apply(None, n_traj, seed=seed, out=sts)
        for H, v, e in zip(Hs, vals, ests):
            c.expect(sts, H, out=v)
            nt.mean_stderr(v, out=e)

    ms_tr = _time_cuda(traj, 5, warm=2)
    ms_ap = _time_cuda(lambda: c.apply(None, n_traj, seed=seed, out=sts), 5, warm=2)
    # algorithmic arithmetic: a generic 2x2 complex gate is 14 real FLOP per amplitude
    flop = int(np.count_nonzero(circ.ops["kind"] == W.OP_U1)) * 14 * (1 << circ.n) * n_traj
    nz_err = None
    if check:
        kk = 4
        ex = NZ.trajectory_expectations(circ, NZ.status_from_seed(seed, kk, circ.n_noise), obs)
        nz_err = {"per_trajectory_max_abs": max(abs(float(vals[o][b].item()) - ex[b][o])
                                                for b in range(kk) for o in range(len(obs))),
                  "trajectories": kk, "tol": 1e-5,
                  "oracle": "exact FP64 state of each trajectory under the same Philox outcomes",
                  "norm_max_dev": float((c.norms(sts[:256]) - 1.0).abs().max().item())}
    out["noisy16_trajectories"] = {
        "err_vs_oracle": nz_err,
        "trajectories_per_s": n_traj / (ms_tr / 1e3), "ms_per_run": ms_tr, "trajectories": n_traj,
        "ms_forward": ms_ap, "forward_tflops": flop / (ms_ap / 1e3) / 1e12,
        "fp32_frac": flop / (ms_ap / 1e3) / 1e12 / FP32_TFLOPS_PROBE,
        "pass_kernels": "compiled for the circuit at plan time", "plan_seconds": t_nz,
        "z0": [float(x) for x in ests[0].tolist()], "sum_zz": [float(x) for x in ests[1].tolist()]}
    del sts
    torch.cuda.synchronize()
    # ---- exact density matrix of a 12-qubit noisy circuit --------------------
    ndm, ldm = 12, 12
    cdm = W.noisy_su2_cz_circuit(ndm, ldm, 0.01, np.random.default_rng(1007))
    dmc = nt.DensityMatrixCircuit(cdm)
    rho = torch.empty((1, 1 << (2 * ndm)), dtype=torch.complex64, device="cuda")
    obs_dm = [nt.Hamiltonian(W.pauli_sum(ndm, [(1.0, {0: 3})])),
              nt.Hamiltonian(W.pauli_sum(ndm, [(1.0, {i: 3, i + 1: 3}) for i in range(ndm - 1)]))]
    vals_dm = [torch.empty(1, dtype=torch.float64, device="cuda") for _ in obs_dm]

    def dm_run():
        dmc.apply(None, 1, out=rho)
        for H, v in zip(obs_dm, vals_dm):
            dmc.expect(rho, H, out=v)

    ms_dm = _time_cuda(dm_run, 20)
    out["dm12_noisy_exact"] = {"err_vs_oracle": None if not check else
                               "not checked here: the oracle's dense density matrix is run at 2..7 qubits in "
                               "the parity tests",
                               "ms_per_run": ms_dm, "qubits": ndm, "layers": ldm, "p": 0.01,
                               "z0": float(vals_dm[0].item()), "sum_zz": float(vals_dm[1].item()),
                               "plan": {k: v for k, v in dmc.info().items() if k in ("fwd_passes", "fwd_stages")}}
    del rho
    # ---- gradient variance over random structures: 10 qubits x 10 layers ----
    cbp, thbp, seedbp, hbp = W.bp_workload()
    cb = nt.Circuit(cbp)
    Hbp = nt.Hamiltonian(hbp)
    d_bp = torch.as_tensor(thbp, device="cuda")
    e_bp = torch.empty(thbp.shape[0], dtype=torch.float64, device="cuda")
    g_bp = torch.empty(thbp.shape, dtype=torch.float64, device="cuda")
    ms_bp = _time_cuda(lambda: cb.expect_grad(d_bp, Hbp, seed=seedbp, energy=e_bp, grad=g_bp), 50)
    bp_err = None
    if check:
        n_ev = int(np.count_nonzero((cbp.ops["kind"] == W.OP_PAULI_NOISE) | (cbp.ops["kind"] == W.OP_RSEL)))
        stat = NZ.status_from_seed(seedbp, thbp.shape[0], n_ev)
        de, dg = [], []
        for b in (0, 57):
            de.append(abs(float(e_bp[b].item()) - sv.energy(sv.run_circuit(cbp, thbp[b], status_row=stat[b]),
                                                               cbp.n, hbp)[0]))
            dg.append(float(np.abs(g_bp[b].cpu().numpy()
                                   - G.parameter_shift(cbp, thbp[b], hbp, status_row=stat[b])).max()))
        bp_err = {"energy_max_abs": max(de), "grad_max_abs": max(dg), "rows": [0, 57],
                  "grad_ref": "parameter shift per gate occurrence"}
    out["bp10_gradient_variance"] = {
        "err_vs_oracle": bp_err,
        "ms_per_run": ms_bp, "qubits": cbp.n, "layers": 10, "structures": int(thbp.shape[0]),
        "var_dtheta0": float(g_bp[:, 0].var(unbiased=False).item()),
        "mean_var_over_params": float(g_bp.var(dim=0, unbiased=False).mean().item())}
    # ---- quantum geometric tensor (QFI = 4 Re G) of the TFIM ansatz -------
    qgt = {}
    for nq, Bq in ((20, 2), (12, 64)):
        cq_circ, thq, _ = W.tfim_workload(nq, 10, Bq)
        cq = nt.Circuit(cq_circ)
        d_thq = torch.as_tensor(thq, device="cuda")
        gq = torch.empty((Bq, cq_circ.n_params, cq_circ.n_params), dtype=torch.complex128, device="cuda")
        msq = _time_cuda(lambda: cq.qgt(d_thq, out=gq), 3 if nq == 20 else 10, warm=1)
        occ = int(np.count_nonzero(cq_circ.ops["param"] >= 0))
        qgt[f"tfim{nq}_l10"] = {"rows": Bq, "ms_per_row": msq / Bq, "params": cq_circ.n_params,
                                "gate_occurrences": occ, "states_per_row": occ + 1,
                                "qfi00_row0": float(4 * gq[0, 0, 0].real.item())}
        if check and nq == 12:
            ref = G.quantum_geometric_tensor(cq_circ, thq[0])
            qgt[f"tfim{nq}_l10"]["err_vs_oracle"] = {
                "G_max_abs": float(np.abs(gq[0].cpu().numpy() - ref).max()), "G_max_abs_ref": float(np.abs(ref).max()),
                "row": 0, "oracle": "product-rule state derivatives, FP64"}
        del cq, gq
    out["qgt_tfim"] = qgt
    # ---- many-term Pauli sum: 12-qubit, 1390-term chemistry-shaped H ------
    hc = W.chem_pauli_sum(12)
    Hc = nt.Hamiltonian(hc)
    cc = nt.Circuit(W.OpBuilder(12).build())
    rngc = np.random.default_rng(1006)
    chem = {"terms": int(hc.n_terms), "qubits": 12}
    for Bc in (1, 1024):
        xs = rngc.standard_normal((Bc, 1 << 12)) + 1j * rngc.standard_normal((Bc, 1 << 12))
        xs /= np.linalg.norm(xs, axis=1, keepdims=True)
        stc = torch.as_tensor(xs.astype(np.complex64), device="cuda")
        ec = torch.empty(Bc, dtype=torch.float64, device="cuda")
        msc = _time_cuda(lambda: cc.expect(stc, Hc, out=ec), 50 if Bc == 1 else 10)
        chem[f"b{Bc}"] = {"us_per_call": msc * 1e3, "states_per_s": Bc / (msc / 1e3)}
        if check:
            x0 = xs[0].astype(np.complex64).astype(np.complex128)
            chem[f"b{Bc}"]["err_vs_oracle"] = {"energy_abs_row0": abs(float(ec[0].item()) - sv.energy(x0, 12, hc)[0])}
    out["chem12_pauli_sum"] = chem
    # ---- QAOA serving: Poisson arrivals, continuous admission ---------------
    serv = {}
    sampled = []
    for rate in serve_rates:
        reqs = W.qaoa_stream(rate_hz=rate, duration_s=serve_seconds)
        prep = [(W.qaoa_circuit(r.n, r.edges, r.p), r.theta, W.zz_on_edges(r.n, r.edges), r.t_arrive)
                for r in reqs]
        srv = nt.Server(mem_budget_bytes=48 << 30, max_inflight=32)
        for w in range(8, 27, 2):  # warm one request per width
            for cc, th, hh, _ in [p for p in prep if p[0].n == w][:1]:
                srv.wait(srv.submit(cc, th, hh), timeout_s=300)
        t0 = time.monotonic()
        ids = []
        for cc, th, hh, ta in prep:
            while time.monotonic() - t0 < ta:
                pass
            ids.append((srv.submit(cc, th, hh), ta))
        lat, svc, last = [], [], 0.0
        for i, (rid, ta) in enumerate(ids):
            r = srv.wait(rid, timeout_s=600)
            lat.append(r["t_done"] - (t0 + ta))
            svc.append(r["t_done"] - r["t_start"])
            last = max(last, r["t_done"] - t0)
            if check and len(sampled) < 3 and prep[i][0].n <= 14:
                sampled.append((prep[i], r))
        stt = srv.stats()
        srv.close()
        lat = np.asarray(lat)
        serv[f"{rate:g}_per_s"] = {"requests": len(lat), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                                  "p99_ms": float(np.percentile(lat, 99) * 1e3),
                                  "completed_per_s": len(lat) / last, "peak_inflight": stt["peak_inflight"],
                                  "mean_admitted_to_done_ms": float(np.mean(svc) * 1e3)}
    # offered load against the saturated throughput (the highest completion rate seen)
    cap = max(v["completed_per_s"] for v in serv.values())
    for k, v in serv.items():
        v["rho_offered_over_capacity"] = float(k.split("_")[0]) / cap
    out["qaoa_serving"] = {"n_qubits": "8..26 (even)", "layers": "1..6", "arrivals": "Poisson",
                           "seconds_per_rate": serve_seconds, "capacity_per_s": cap, "by_offered_rate": serv}
    if check and sampled:
        de, dg = [], []
        for (cc, th, hh, _), r in sampled:
            thr = np.asarray(th, dtype=np.float64).ravel()
            de.append(abs(r["energy"] - sv.energy(sv.run_circuit(cc, thr), cc.n, hh)[0]))
            dg.append(float(np.abs(r["grad"] - G.finite_difference(cc, thr, hh, h=1e-5)).max()))
        out["qaoa_serving"]["err_vs_oracle"] = {"energy_max_abs": max(de), "grad_max_abs": max(dg),
                                                "requests": len(sampled), "qubits": [p[0][0].n for p in sampled],
                                                "grad_ref": "central differences, h = 1e-5"}
    return out


def _profile_kv(kernel: str):
    """'key: value' lines of the committed ncu summary of `kernel`
    (profiles/traffic_<kernel>.txt), or None when the file is absent or the
    tile-pass sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    return kv if kv.get("source_hash") == _source_hash() else None


def _binding(kernel: str):
    """The roof that binds `kernel`, from the same ncu capture as its traffic."""
    kv = _profile_kv(kernel)
    if not kv or "binding" not in kv:
        return None
    out = {"roof": kv["binding"], "source": f"profiles/traffic_{kernel}.txt (ncu, same source hash)"}
    for k in ("issue_active", "fp32_tflops", "fp32_peak_tflops"):
        if k in kv:
            out[k] = float(kv[k])
    if "fp32_tflops" in out and "fp32_peak_tflops" in out:
        out["fp32_frac"] = out["fp32_tflops"] / out["fp32_peak_tflops"]
    return out


def _traffic(kernel: str):
    """DRAM bytes per full-size launch of `kernel` from the committed ncu
    summary (profiles/traffic_<kernel>.txt, 'key: value' lines), or None when
    the tile-pass sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("source_hash") != _source_hash():
        return None
    try:
        return float(kv["bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


# the sources that define the tile-pass kernels and the plans they run
TILE_PASS_SOURCES = ("plan.h", "planner.cpp", "planner.h", "sv_args.h", "sv_core.cuh", "sv_kernels.cu",
                     "sv_kernels.cuh", "jit.cpp")


def _source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2205_10091_b300", "csrc")
    for f in TILE_PASS_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other hot-path workloads")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle checks and the CPU baseline")
    ap.add_argument("--no-specialize", action="store_true",
                    help="run the headline circuit on the plan-interpreting pass kernels")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
