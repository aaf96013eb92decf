"""Pins of the whole oracle application (Eqs. tDxx, DxxVxx, exxGen_mlwf).

* Brute force: an isolated water (wide Gaussians, fine grid) whose exact
  free-space D^i = sum_j v_ij phi_j over the whole cell is computed by FFT;
  as eps -> 0 (delta = 0) the truncated result must converge to it
  monotonically until the finite-difference floor (Sec. II B: the error due
  to domain truncation vanishes as eps -> 0).
* Invariants on the (H2O)8-like case: E_xx < 0, sum_i <phi_i|V_xx phi_i>
  ~ E_xx, and <phi_i|V_xx phi_j> ~ <phi_j|V_xx phi_i>.
"""
import numpy as np
import pytest

from oracle import freespace
from oracle import oracle as O
from paper_2208_06097_gb300 import synth


@pytest.fixture(scope="module")
def isolated():
    s = synth.make_waters(1, 12.0 * 0.529177210903, 48, seed=7, alpha_range=(0.6, 0.9),
                          centre_first=True)
    h = tuple(c / g for c, g in zip(s.cell, s.grid))
    D = np.zeros_like(s.phi)
    E = 0.0
    n = s.n_orb
    for i in range(n):
        for j in range(i, n):
            rho = s.phi[i] * s.phi[j]
            v = freespace.freespace_potential(rho, h)
            w = 1.0 if i == j else 2.0
            E -= w * (rho * v).sum() * s.dV
            D[i] += v * s.phi[j]
            if j != i:
                D[j] += v * s.phi[i]
    return s, -D, E


def test_converges_to_free_space_brute_force(isolated):
    s, V_bf, E_bf = isolated
    ev, ee = [], []
    for eps in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        r = O.apply_vxx(s.phi, s.cell, O.Params(eps=eps, delta=0.0, cg_tol=1e-12))
        assert r["rc"] == 0 and len(r["pair"]) == 10
        ev.append(np.abs(r["vxx"] - V_bf).max())
        ee.append(abs(r["exx"] - E_bf))
    assert all(b < a for a, b in zip(ev, ev[1:])), ev
    assert all(b < a for a, b in zip(ee, ee[1:])), ee
    assert ee[-1] < 5e-6 * abs(E_bf) and ev[-1] < 2e-5


def test_energy_negative_and_consistent(h2o8, h2o8_oracle):
    r = h2o8_oracle
    assert r["rc"] == 0
    assert r["exx"] < 0
    F = h2o8.phi.reshape(h2o8.n_orb, -1)
    V = r["vxx"].reshape(h2o8.n_orb, -1)
    M = F @ V.T * h2o8.dV
    # truncation-level agreement (eps = 10^-3.5)
    assert abs(np.trace(M) - r["exx"]) < 1e-3 * abs(r["exx"])
    assert np.abs(M - M.T).max() < 1e-2 * np.abs(M).max()


def test_pair_energies_positive(h2o8_oracle):
    # self pairs: (rho|rho) > 0 for a positive-definite Coulomb kernel
    r = h2o8_oracle
    self_ = r["pair"][:, 0] == r["pair"][:, 1]
    assert np.all(r["epair"][self_] > 0)
    assert np.all(r["iters"] > 0)


def test_deterministic(h2o8, h2o8_oracle):
    r2 = O.apply_vxx(h2o8.phi, h2o8.cell, O.Params())
    assert np.array_equal(r2["vxx"], h2o8_oracle["vxx"]) and r2["exx"] == h2o8_oracle["exx"]
