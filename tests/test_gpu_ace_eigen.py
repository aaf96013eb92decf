"""The eigen-decomposition form of the ACE build (App. A) on the GPU
(cyclic Jacobi on -Mbar) against the oracle's eigen form (library
eigensolver, complex zeta, Hermitian products)."""
import numpy as np
import pytest

from oracle import ace as OA
from paper_2208_06097_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ctx(s, **kw):
    from paper_2208_06097_gb300 import sea
    c = sea.Context(s.cell, s.grid, **kw)
    c.set_orbitals(np.ascontiguousarray(s.phi))
    return c


@pytest.mark.parametrize("precision", [0, 1])
def test_indefinite_w_uses_eigen_form(h2o8, precision):
    rng = np.random.default_rng(5)
    F = h2o8.phi.reshape(h2o8.n_orb, -1)
    n = F.shape[0]
    B = rng.normal(size=(n, n))
    G = 0.5 * (B + B.T)
    W = np.ascontiguousarray(-(G @ F)).reshape(h2o8.phi.shape)
    e = OA.build_ace_eigen(F, W.reshape(n, -1), h2o8.dV)
    psi = synth.random_trial_vectors(3, h2o8.grid, 21)
    yr = OA.apply_ace_eigen(e["zeta"], psi.reshape(3, -1), h2o8.dV)
    with _ctx(h2o8, precision=precision) as ctx:
        ctx.build_ace_from(W)
        st = ctx.stats()
        assert st["ace_eigen"] == 1
        assert st["ace_negative_eigenvalues"] == int(np.sum(e["lam"] < 0))
        M, L = ctx.ace_matrices()
        assert np.abs(M - e["M"]).max() <= 1e-10 * np.abs(e["M"]).max()
        lam = np.sort(np.diag(L))
        np.testing.assert_allclose(lam, np.sort(e["lam"]), atol=1e-9 * np.abs(e["lam"]).max())
        y = np.empty_like(psi)
        ctx.apply_ace(psi, y)
        assert np.abs(y.reshape(3, -1) - yr).max() <= 1e-9 * np.abs(yr).max()
        # Eq. exx_ace, first form: sum_i <phi_i|V^ACE|phi_i> with the oracle's operator
        yF = OA.apply_ace_eigen(e["zeta"], F, h2o8.dV)
        e_ref = float(np.sum(F * yF) * h2o8.dV)
        assert abs(st["exx_ace"] - e_ref) <= 1e-10 * abs(e_ref)


def test_forced_eigen_form_equals_cholesky_form(h2o8):
    from oracle import oracle as O
    ref = O.apply_vxx(h2o8.phi, h2o8.cell, O.Params(cg_tol=1e-12))
    F = h2o8.phi.reshape(h2o8.n_orb, -1)
    a = OA.build_ace(F, ref["vxx"].reshape(h2o8.n_orb, -1), h2o8.dV)
    psi = synth.random_trial_vectors(3, h2o8.grid, 22)
    yr = OA.apply_ace(a["Xi"], psi.reshape(3, -1), h2o8.dV)
    with _ctx(h2o8, ace_decomp=2, cg_tol=1e-12) as ctx:
        out = np.empty_like(h2o8.phi)
        ctx.apply_vxx(out)
        ctx.build_ace()
        assert ctx.stats()["ace_eigen"] == 1
        y = np.empty_like(psi)
        ctx.apply_ace(psi, y)
        e_ace = ctx.stats()["exx_ace"]
    assert np.abs(y.reshape(3, -1) - yr).max() <= 1e-9 * np.abs(yr).max()
    # the eigen form's E_xx^ACE equals the Cholesky form's (Eq. exx_ace)
    e_ref = OA.exx_ace(F, a["Xi"], h2o8.dV)
    assert abs(e_ace - e_ref) <= 1e-10 * abs(e_ref)


def test_singular_mbar_drops_the_zero_mode(h2o8):
    s = synth.make_waters(2, 6.21, 32, seed=77)
    phi = np.ascontiguousarray(s.phi.copy())
    phi[0] = 0.0
    s.phi = phi
    from paper_2208_06097_gb300 import sea
    with _ctx(s, orth_tol=0.0) as ctx:  # a zero orbital has norm 0
        out = np.empty_like(phi)
        ctx.apply_vxx(out)
        ctx.build_ace()
        st = ctx.stats()
        assert st["ace_eigen"] == 1 and st["ace_dropped_eigenvalues"] == 1
        F = phi.reshape(phi.shape[0], -1)
        e = OA.build_ace_eigen(F, out.reshape(phi.shape[0], -1), s.dV)
        psi = synth.random_trial_vectors(2, s.grid, 23)
        y = np.empty_like(psi)
        ctx.apply_ace(psi, y)
        yr = OA.apply_ace_eigen(e["zeta"], psi.reshape(2, -1), s.dV)
        assert np.abs(y.reshape(2, -1) - yr).max() <= 1e-9 * np.abs(yr).max()
        with pytest.raises(sea.SeaError) as err:
            ctx.ace_vectors(np.empty_like(phi))
        assert err.value.code == 2
