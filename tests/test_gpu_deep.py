"""GPU parity: long circuits and whole rows at the benchmark's size.

- Uncompute drift: the adjoint sweep recovers each layer's state by applying
  the inverse gates to the final state (psi <- U^dagger psi, Section
  "Gradients, optimization and variational algorithms" restated as an adjoint
  method) instead of storing it, so rounding accumulates over the whole
  depth, most in the earliest layers.  A 16-qubit, 48-layer complex64 TFIM
  circuit checks the first layers' gradients (reached last by the sweep),
  middle and last ones against oracle central differences at the usual
  gradient tolerance.
- One full row of the 20-qubit, 10-layer, 1024-row TFIM batch: all 20
  gradients against oracle central differences (the oracle's energies run in
  worker processes).
"""
import multiprocessing as mp

import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import assert_energy_close, assert_grad_close, cuda_params

pytestmark = pytest.mark.gpu


def test_deep_circuit_uncompute_gradients():
    n, layers = 16, 48
    circ, theta, ham = W.tfim_workload(n=n, layers=layers, batch=2, seed=48)
    c = nt.Circuit(circ)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    b = 1
    assert_energy_close(e[b:b + 1], [sv.energy(sv.run_circuit(circ, theta[b]), n, ham)[0]])
    ks = [0, 1, 2, 3, layers - 1, layers, 2 * layers - 2, 2 * layers - 1]
    fd = G.finite_difference(circ, theta[b], ham, h=1e-5, params=ks)
    assert_grad_close(g[b, ks], fd[ks])
    # the same row in complex128 (the uncompute's own rounding is ~1e-16 there)
    c2 = nt.Circuit(circ, dtype=nt.TC_C128)
    _, g2 = c2.expect_grad(cuda_params(theta[b:b + 1]), nt.Hamiltonian(ham))
    assert np.abs(g2.cpu().numpy()[0, ks] - fd[ks]).max() <= 1e-6 * max(1.0, np.abs(fd[ks]).max())


def _tfim20_energy(args):
    row, k, h = args
    circ, theta, ham = W.tfim_workload()
    th = theta[row].copy()
    if k >= 0:
        th[k] += h
    return sv.energy(sv.run_circuit(circ, th), circ.n, ham)[0]


def test_tfim20_full_row_all_gradients(monkeypatch):
    import os

    # the spawned workers import this module: give them the repository and tests/
    here = os.path.dirname(os.path.abspath(__file__))
    monkeypatch.setenv("PYTHONPATH", os.pathsep.join([os.path.dirname(here), here, os.environ.get("PYTHONPATH", "")]))
    monkeypatch.setenv("OMP_NUM_THREADS", "1")  # one BLAS thread per worker
    monkeypatch.setenv("OPENBLAS_NUM_THREADS", "1")
    circ, theta, ham = W.tfim_workload()
    c = nt.Circuit(circ)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    row, h = 700, 1e-4
    tasks = [(row, -1, 0.0)] + [(row, k, s * h) for k in range(circ.n_params) for s in (1, -1)]
    with mp.get_context("spawn").Pool(min(mp.cpu_count(), 16)) as pool:
        res = pool.map(_tfim20_energy, tasks, chunksize=1)
    assert_energy_close(e[row:row + 1], [res[0]])
    fd = np.array([(res[1 + 2 * k] - res[2 + 2 * k]) / (2 * h) for k in range(circ.n_params)])
    assert_grad_close(g[row], fd)
