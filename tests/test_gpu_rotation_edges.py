"""GPU parity at the numerical edges of the complex64 rotation kernels.

Complex64 RY runs in tangent form c [[1, -t], [t, 1]] (t = tan(a/2)) with the
factor c kept in a running scale; RX runs as a framed RY.  These cases pin
the angles where c vanishes (a = pi, 3 pi), angles a hair away from them,
and chains of rotations whose scale product underflows FP32 unless it is
folded back into the registers.  References are the FP64 oracle's states,
energies and central-difference gradients.
"""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import statevector as sv
from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W

from gpu_util import TOL_AMP_C64, assert_energy_close, assert_grad_close, cuda_params

pytestmark = pytest.mark.gpu

EDGE_ANGLES = np.array([np.pi, -np.pi, 3 * np.pi, np.pi + 1e-7, np.pi - 1e-6, 2 * np.pi, 0.0, 1e-30,
                        np.pi / 2, -3 * np.pi / 2])


def _layered(n, layers, kinds):
    """Layers of rotations on every qubit (one shared angle per layer and kind)
    and a ZZ chain, so rotations on a qubit alternate with phase groups."""
    b = W.OpBuilder(n)
    p = 0
    for _ in range(layers):
        for kind in kinds:
            for q in range(n):
                (b.ry if kind == "ry" else b.rx)(q, p)
            p += 1
        for q in range(n - 1):
            b.rzz(q, q + 1, p)
        p += 1
    return b.build(n_params=p)


def _states(circ, theta):
    import torch

    c = nt.Circuit(circ, dtype=nt.TC_C64)
    out = c.apply(cuda_params(theta), theta.shape[0])
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("kinds", [("ry",), ("rx",), ("ry", "rx")])
def test_edge_angles_states(kinds):
    n, layers = 12, 3
    circ = _layered(n, layers, kinds)
    rng = np.random.default_rng(71)
    rows = []
    for a in EDGE_ANGLES:
        th = rng.uniform(-3, 3, size=circ.n_params)
        th[:: len(kinds) + 1] = a  # every first rotation layer of a block takes the edge angle
        rows.append(th)
    theta = np.array(rows)
    got = _states(circ, theta)
    for b in range(theta.shape[0]):
        ref = sv.run_circuit(circ, theta[b])
        err = np.abs(got[b] - ref).max()
        assert err <= TOL_AMP_C64, f"angle {EDGE_ANGLES[b]!r}: max amplitude error {err:.3e}"


def test_edge_angles_energy_and_gradient():
    n, layers = 10, 2
    circ = _layered(n, layers, ("rx",))
    ham = W.tfim_zz_x(n)
    rng = np.random.default_rng(72)
    theta = rng.uniform(-3, 3, size=(len(EDGE_ANGLES), circ.n_params))
    theta[:, 0] = EDGE_ANGLES
    theta[:, 2] = EDGE_ANGLES[::-1]
    c = nt.Circuit(circ, dtype=nt.TC_C64)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    for b in range(theta.shape[0]):
        e_ref = sv.energy(sv.run_circuit(circ, theta[b]), n, ham)[0]
        assert_energy_close(e[b:b + 1], [e_ref])
        assert_grad_close(g[b], G.finite_difference(circ, theta[b], ham))


@pytest.mark.parametrize("distinct", [False, True])
def test_scale_renormalisation_long_chain(distinct):
    # 48 RY layers at |cos(a/2)| ~ 0.02..0.25: the running scale passes 2^-20
    # every few gates and would underflow FP32 long before the end without
    # folding.  distinct=False reuses four angles (rounding that repeats over
    # 120 gates is the harshest case for norm drift); distinct=True gives every
    # layer its own angle near pi, a fifth of them exactly pi.
    n, layers = 10, 48
    n_rot = layers if distinct else 4
    b = W.OpBuilder(n)
    for layer in range(layers):
        for q in range(n):
            b.ry(q, layer % n_rot)
        if layer % 8 == 7:
            for q in range(n - 1):
                b.rzz(q, q + 1, n_rot)
    circ = b.build(n_params=n_rot + 1)
    if distinct:
        rng = np.random.default_rng(73)
        theta = np.pi + rng.uniform(-0.25, 0.25, (3, n_rot + 1)) * rng.choice([-1, 1], (3, n_rot + 1))
        theta[:, ::5] = np.pi
        theta[:, -1] = [0.3, -0.7, 0.1]
    else:
        theta = np.array([[2.94, -2.94, 3.04, 2.9, 0.3], [3.1, 3.1, -3.1, 3.1, -0.7],
                          [np.pi, 2.94, np.pi, -np.pi, 0.1]])
    got = _states(circ, theta)
    ham = W.tfim_zz_x(n)
    c = nt.Circuit(circ, dtype=nt.TC_C64)
    e, g = c.expect_grad(cuda_params(theta), nt.Hamiltonian(ham))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    for r in range(theta.shape[0]):
        ref = sv.run_circuit(circ, theta[r])
        err = np.abs(got[r] - ref).max()
        assert err <= TOL_AMP_C64, f"row {r}: max amplitude error {err:.3e}"
        assert_energy_close(e[r:r + 1], [sv.energy(ref, n, ham)[0]])
        assert_grad_close(g[r], G.finite_difference(circ, theta[r], ham))
