"""The device-side input generator (make_waters_device, torch float64) gives
the orbitals of the host generator (make_waters) from the same seeded
parameters; run here on the CPU device."""
import numpy as np
import pytest

from paper_2208_06097_gb300 import synth

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("args", [(3, 6.0, (20, 18, 22), 5), (2, 5.0, 16, 41)])
def test_device_generator_matches_host(args):
    n_mol, L, grid, seed = args
    s = synth.make_waters(n_mol, L, grid, seed)
    phi, cell, g = synth.make_waters_device(n_mol, L, grid, seed, "cpu")
    assert cell == s.cell and g == s.grid
    assert np.abs(phi.numpy() - s.phi).max() <= 1e-12 * np.abs(s.phi).max()
    # orthonormal on the grid
    F = phi.numpy().reshape(phi.shape[0], -1)
    assert np.abs(F @ F.T * s.dV - np.eye(F.shape[0])).max() <= 1e-12
