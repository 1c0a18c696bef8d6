"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

from paper_2205_10091_b300 import native as nt

# tolerances: c128 amplitudes, c64 amplitudes, energies |dE| <= 1e-5 max(|E|, 1),
# gradients max |dg| <= 1e-4 max(max |g|, 1)
TOL_AMP_C128 = 1e-12
TOL_AMP_C64 = 2e-6
TOL_E_REL = 1e-5
TOL_G_REL = 1e-4


def cuda_params(theta):
    import torch

    return torch.as_tensor(np.asarray(theta, dtype=np.float64), device="cuda").contiguous()


def assert_energy_close(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(got - ref)
    bound = TOL_E_REL * np.maximum(np.abs(ref), 1.0)
    assert np.all(err <= bound), f"max |dE| {err.max():.3e} vs bound {bound.min():.3e}"


def assert_grad_close(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(np.abs(ref).max() if ref.size else 0.0, 1.0)
    err = np.abs(got - ref).max() if ref.size else 0.0
    assert err <= TOL_G_REL * scale, f"max |dg| {err:.3e} vs {TOL_G_REL * scale:.3e}"
