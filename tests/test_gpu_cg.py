"""GPU parity of the per-pair Poisson solver (Eq. pe, App. C stencil)
through sea_poisson_batch, against the oracle's CG and a dense solve."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EXTS = [(1, 1, 1), (3, 5, 7), (13, 12, 11), (20, 9, 14), (6, 6, 6), (2, 17, 4), (16, 16, 16)]


def _batch(h, exts, seed, tol, max_iter=5000):
    from paper_2208_06097_gb300 import sea
    rng = np.random.default_rng(seed)
    bs = [rng.normal(size=(e[2], e[1], e[0])) for e in exts]
    flat = np.concatenate([b.ravel() for b in bs])
    rhs = torch.from_numpy(flat).cuda()
    x = torch.empty_like(rhs)
    it, rc = sea.poisson_batch(h, exts, rhs, x, tol=tol, max_iter=max_iter)
    xs, off = [], 0
    xh = x.cpu().numpy()
    for e in exts:
        n = e[0] * e[1] * e[2]
        xs.append(xh[off:off + n].reshape(e[2], e[1], e[0]))
        off += n
    return bs, xs, it, rc


def test_matches_oracle_cg_tight():
    h = (0.25, 0.23, 0.27)
    bs, xs, it, rc = _batch(h, EXTS, 1, 1e-13)
    assert rc == 0
    for b, x, k in zip(bs, xs, it):
        xr, kr, _ = O.cg(b, h, tol=1e-13)
        assert np.abs(x - xr).max() <= 1e-11 * max(1.0, np.abs(xr).max())
        assert abs(int(k) - kr) <= 2


def test_dense_solve_small_box():
    h = (0.3, 0.3, 0.3)
    e = (5, 4, 6)
    bs, xs, it, rc = _batch(h, [e], 3, 1e-14)
    n = e[0] * e[1] * e[2]
    A = np.zeros((n, n))
    for k in range(n):
        u = np.zeros(n)
        u[k] = 1
        A[:, k] = O.neg_laplacian(u.reshape(e[2], e[1], e[0]), h).ravel()
    xs_ref = np.linalg.solve(A, bs[0].ravel())
    assert np.abs(xs[0].ravel() - xs_ref).max() <= 1e-11 * np.abs(xs_ref).max()


def test_iteration_cap_reports_status():
    h = (0.25, 0.25, 0.25)
    bs, xs, it, rc = _batch(h, [(12, 12, 12)], 5, 1e-14, max_iter=3)
    assert rc == 5 and it[0] == -3
    xr, kr, _ = O.cg(bs[0], h, tol=1e-14, max_iter=3)
    assert np.abs(xs[0] - xr).max() <= 1e-12 * np.abs(xr).max()


def test_empty_batch():
    from paper_2208_06097_gb300 import sea
    it, rc = sea.poisson_batch((0.3, 0.3, 0.3), np.zeros((0, 3), np.int32),
                               torch.zeros(1, dtype=torch.float64, device="cuda"),
                               torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert rc == 0 and len(it) == 0
