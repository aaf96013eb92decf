"""Pins of the oracle's ACE steps (Eq. Vace, Eq. exx_ace, App. A)."""
import numpy as np
import pytest

from oracle import ace


@pytest.fixture(scope="module")
def ace_c1(h2o8, h2o8_oracle):
    F = h2o8.phi.reshape(h2o8.n_orb, -1)
    W = h2o8_oracle["vxx"].reshape(h2o8.n_orb, -1)
    return F, W, ace.build_ace(F, W, h2o8.dV)


def test_cholesky_matches_lapack(ace_c1):
    F, W, a = ace_c1
    np.testing.assert_allclose(a["L"], np.linalg.cholesky(-a["Mbar"]), rtol=1e-12, atol=1e-13)


def test_cholesky_rejects_indefinite():
    with pytest.raises(ace.NotPositiveDefinite):
        ace.cholesky_lower(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_xi_solves_triangular_system(ace_c1):
    F, W, a = ace_c1
    np.testing.assert_allclose(a["L"] @ a["Xi"], W, rtol=0, atol=1e-11 * np.abs(W).max())


def test_reproduces_vxx_on_occupied_when_M_symmetric(h2o8, rng):
    # W = -Phi G with G SPD gives a symmetric M = -G: then V^ACE Phi = W exactly.
    F = h2o8.phi.reshape(h2o8.n_orb, -1)
    B = rng.normal(size=(h2o8.n_orb, h2o8.n_orb))
    G = B @ B.T + h2o8.n_orb * np.eye(h2o8.n_orb)
    W = -(G @ F)  # rows: W_j = -sum_i G_ji phi_i
    a = ace.build_ace(F, W, h2o8.dV)
    Y = ace.apply_ace(a["Xi"], F, h2o8.dV)
    np.testing.assert_allclose(Y, W, rtol=0, atol=1e-10 * np.abs(W).max())
    assert ace.exx_ace(F, a["Xi"], h2o8.dV) == pytest.approx(np.trace(a["Mbar"]), rel=1e-12)


def test_occupied_action_error_is_the_skew_part(ace_c1, h2o8):
    # rows: V^ACE Phi = M Mbar^-1 W (= W when M is symmetric); the gap is the skew part of M
    F, W, a = ace_c1
    Y = ace.apply_ace(a["Xi"], F, h2o8.dV)
    pred = a["M"] @ np.linalg.solve(a["Mbar"], W)
    np.testing.assert_allclose(Y, pred, rtol=0, atol=1e-9 * np.abs(W).max())
    E = ace.exx_ace(F, a["Xi"], h2o8.dV)
    M, Mb = a["M"], a["Mbar"]
    assert E == pytest.approx(np.trace(M @ np.linalg.solve(Mb, M.T)), rel=1e-10)
    assert E < 0


def test_operator_is_symmetric_negative_semidefinite(ace_c1, h2o8, rng):
    F, W, a = ace_c1
    psi = rng.normal(size=(3, F.shape[1]))
    Y = ace.apply_ace(a["Xi"], psi, h2o8.dV)
    G = psi @ Y.T * h2o8.dV
    np.testing.assert_allclose(G, G.T, rtol=1e-12, atol=1e-12 * np.abs(G).max())
    assert np.all(np.linalg.eigvalsh(0.5 * (G + G.T)) <= 1e-12 * np.abs(G).max())
    # rank <= n: vectors orthogonal to every xi_k are annihilated
    Q, _ = np.linalg.qr(a["Xi"].T)
    z = psi[0] - Q @ (Q.T @ psi[0])
    assert np.abs(ace.apply_ace(a["Xi"], z[None], h2o8.dV)).max() < 1e-10 * np.abs(Y).max()


def test_eigen_form_equals_cholesky_form_when_pd(ace_c1, h2o8, rng):
    F, W, a = ace_c1
    e = ace.build_ace_eigen(F, W, h2o8.dV)
    assert np.all(e["lam"] > 0) and e["zeta"].shape[0] == F.shape[0]
    psi = rng.normal(size=(3, F.shape[1]))
    np.testing.assert_allclose(ace.apply_ace_eigen(e["zeta"], psi, h2o8.dV),
                               ace.apply_ace(a["Xi"], psi, h2o8.dV), rtol=0,
                               atol=1e-9 * np.abs(ace.apply_ace(a["Xi"], psi, h2o8.dV)).max())


def test_eigen_form_indefinite(h2o8, rng):
    # W = -Phi G with G symmetric indefinite: -Mbar = G.  The Cholesky form
    # fails; the eigen form gives a negative semidefinite operator whose action
    # on the occupied orbitals is W Q sign(Lambda) Q^T.
    F = h2o8.phi.reshape(h2o8.n_orb, -1)
    n = F.shape[0]
    B = rng.normal(size=(n, n))
    G = 0.5 * (B + B.T)
    W = -(G @ F)
    with pytest.raises(ace.NotPositiveDefinite):
        ace.build_ace(F, W, h2o8.dV)
    e = ace.build_ace_eigen(F, W, h2o8.dV)
    assert np.any(e["lam"] < 0)
    np.testing.assert_allclose(np.sort(e["lam"]), np.sort(np.linalg.eigvalsh(G)), atol=1e-10)
    Y = ace.apply_ace_eigen(e["zeta"], F, h2o8.dV)
    Q, lam = e["Q"], e["lam"]
    pred = (Q @ np.diag(np.sign(lam)) @ Q.T).T @ W  # rows: sum_i (Q sign Q^T)_{ij} W_i
    np.testing.assert_allclose(Y, pred, rtol=0, atol=1e-9 * np.abs(W).max())
    psi = rng.normal(size=(4, F.shape[1]))
    Yp = ace.apply_ace_eigen(e["zeta"], psi, h2o8.dV)
    Gm = psi @ Yp.T * h2o8.dV
    assert np.all(np.linalg.eigvalsh(0.5 * (Gm + Gm.T)) <= 1e-10 * np.abs(Gm).max())
