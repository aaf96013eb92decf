"""Pins for the oracle's CG (Eq. pe): it must return the unique solution of
the SPD system, which a dense library solve of the same operator gives."""
import numpy as np

from oracle import oracle as O


def _dense(ex, ey, ez, h):
    n = ex * ey * ez
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = O.neg_laplacian(e.reshape(ez, ey, ex), h).ravel()
    return A


def test_cg_matches_dense_solve(rng):
    ex, ey, ez = 6, 5, 7
    h = (0.25, 0.2, 0.3)
    A = _dense(ex, ey, ez, h)
    b = rng.normal(size=(ez, ey, ex))
    x, it, res = O.cg(b, h, tol=1e-14)
    assert it > 0 and res <= 1e-14
    xs = np.linalg.solve(A, b.ravel())
    assert np.abs(x.ravel() - xs).max() < 1e-11 * np.abs(xs).max()


def test_cg_residual_definition(rng):
    b = rng.normal(size=(8, 8, 8))
    h = (0.25, 0.25, 0.25)
    x, it, res = O.cg(b, h, tol=1e-6)
    r = b - O.neg_laplacian(x, h)
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(b) * 1.0001
    # one iteration fewer must not meet the tolerance (stops at the first hit)
    x2, it2, res2 = O.cg(b, h, tol=1e-6, max_iter=it - 1)
    assert it2 == -(it - 1) and res2 > 1e-6


def test_cg_zero_rhs():
    x, it, res = O.cg(np.zeros((4, 4, 4)), (0.3, 0.3, 0.3), tol=1e-8)
    assert it == 0 and np.all(x == 0)


def test_cg_absolute_mode(rng):
    b = rng.normal(size=(6, 6, 6))
    h = (0.25, 0.25, 0.25)
    x, it, _ = O.cg(b, h, tol=1e-5, tol_mode=1)
    r = b - O.neg_laplacian(x, h)
    assert np.sqrt(np.mean(r * r)) / (4 * np.pi) <= 1e-5 * 1.0001
