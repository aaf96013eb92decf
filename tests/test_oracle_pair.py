"""End-to-end pins of one pair problem (Eqs. pe, me, mepole) against closed
forms: a product of two Gaussians is a Gaussian charge whose potential is
q erf(sqrt(p) r)/r and whose self-interaction is q^2 sqrt(2p/pi)."""
import numpy as np
import pytest
from scipy.special import erf

from oracle import oracle as O


def _grid_gauss(n, hh, a, A):
    z, y, x = np.meshgrid(*(np.arange(n) * hh for _ in range(3)), indexing="ij")
    d2 = (x - A[0]) ** 2 + (y - A[1]) ** 2 + (z - A[2]) ** 2
    return (2 * a / np.pi) ** 0.75 * np.exp(-a * d2)


def _case(n, hh, a=1.1, b=1.6):
    L = n * hh
    A = np.array([0.52, 0.47, 0.5]) * L
    B = A + np.array([0.35, -0.2, 0.25])
    fi, fj = _grid_gauss(n, hh, a, A), _grid_gauss(n, hh, b, B)
    p = a + b
    P = (a * A + b * B) / p
    q = (2 * a / np.pi) ** 0.75 * (2 * b / np.pi) ** 0.75 * np.exp(-a * b / p * np.sum((A - B) ** 2)) * (np.pi / p) ** 1.5
    return fi, fj, P, p, q, (L, L, L)


def _solve(n, hh, **kw):
    fi, fj, P, p, q, cell = _case(n, hh, **kw)
    m = int(round(2.2 * 2 * np.sqrt(3.0) / hh))  # box of about +-4.4 sigma around P
    lo = [int(np.floor(P[a] / hh)) - m // 2 for a in range(3)]
    ext = [m, m, m]
    v, Q, e, it = O.pair_solve(fi, fj, cell, lo, ext, O.Params(cg_tol=1e-13))
    z, y, x = np.meshgrid(*(np.arange(m) for _ in range(3)), indexing="ij")
    X = (x + lo[0]) * hh - P[0]
    Y = (y + lo[1]) * hh - P[1]
    Z = (z + lo[2]) * hh - P[2]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    vex = q * erf(np.sqrt(p) * r) / r
    return v, vex, e, q * q * np.sqrt(2 * p / np.pi), it


def test_gaussian_product_potential_and_energy_converge():
    errs, eerrs = [], []
    for n, hh in ((40, 0.3), (60, 0.2)):
        v, vex, e, eex, it = _solve(n, hh)
        assert it > 0
        errs.append(np.abs(v - vex).max())
        eerrs.append(abs(e - eex))
    assert errs[1] < errs[0] / 20 and errs[1] < 2e-5
    assert eerrs[1] < eerrs[0] / 20 and eerrs[1] < 1e-6


def test_pair_is_symmetric_in_i_j():
    fi, fj, P, p, q, cell = _case(32, 0.3)
    lo, ext = (10, 9, 11), (13, 12, 14)
    v1, Q1, e1, _ = O.pair_solve(fi, fj, cell, lo, ext)
    v2, Q2, e2, _ = O.pair_solve(fj, fi, cell, lo, ext)
    assert np.array_equal(v1, v2) and np.array_equal(Q1, Q2) and e1 == e2


def test_pair_monopole_is_box_charge():
    fi, fj, P, p, q, cell = _case(32, 0.3)
    lo, ext = (8, 8, 8), (16, 16, 16)
    v, Q, e, _ = O.pair_solve(fi, fj, cell, lo, ext)
    hh = cell[0] / 32
    idx = np.arange(8, 24)
    charge = (fi[np.ix_(idx, idx, idx)] * fj[np.ix_(idx, idx, idx)]).sum() * hh ** 3
    assert Q[0] * np.sqrt(4 * np.pi) == pytest.approx(charge, rel=1e-12)
