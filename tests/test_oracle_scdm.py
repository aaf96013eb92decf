"""Pins of the oracle's SCDM: U is orthogonal, the localized orbitals are
orthonormal and span the input space, and a rotated set of well-separated
localized orbitals is recovered (up to order and sign) -- the case where a
localized basis exists and SCDM must find it."""
import numpy as np

from oracle import scdm as S
from paper_2208_06097_gb300.synth import separated_gaussians


def test_scdm_invariants(rng):
    phi, dV = separated_gaussians(8, 24, 12.0)
    R, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    can = (R.T @ phi.reshape(8, -1)).reshape(phi.shape)
    C, U, pt = S.scdm(can)
    assert np.abs(U.T @ U - np.eye(8)).max() <= 1e-12
    G = pt.reshape(8, -1) @ pt.reshape(8, -1).T * dV
    assert np.abs(G - np.eye(8)).max() <= 1e-10
    # same space: each input orbital is its own projection on the output span
    a, b = can.reshape(8, -1), pt.reshape(8, -1)
    proj = (a @ b.T * dV) @ b
    assert np.abs(proj - a).max() <= 1e-10 * np.abs(a).max()
    assert len(set(C.tolist())) == 8


def test_scdm_recovers_separated_orbitals(rng):
    phi, dV = separated_gaussians(8, 24, 12.0)
    R, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    can = (R.T @ phi.reshape(8, -1)).reshape(phi.shape)
    _, _, pt = S.scdm(can)
    O = np.abs(pt.reshape(8, -1) @ phi.reshape(8, -1).T * dV)
    # each localized orbital matches exactly one original one
    assert np.all(np.abs(O.max(axis=1) - 1.0) <= 1e-6)
    assert sorted(O.argmax(axis=1).tolist()) == list(range(8))
