"""Pins for the real solid harmonics used by Eqs. me and mepole."""
import numpy as np
import pytest
from numpy.polynomial import legendre

from oracle import oracle as O

LMAX = 6


def _leg(l, x):
    c = np.zeros(l + 1)
    c[l] = 1.0
    return legendre.legval(x, c)


def test_addition_theorem(rng):
    # sum_m S_lm(a) S_lm(b) = (2l+1)/(4 pi) |a|^l |b|^l P_l(cos gamma)
    for _ in range(20):
        a = rng.normal(size=3)
        b = rng.normal(size=3)
        Sa = O.solid_harmonics_all(LMAX, a)[0]
        Sb = O.solid_harmonics_all(LMAX, b)[0]
        ra, rb = np.linalg.norm(a), np.linalg.norm(b)
        cg = a @ b / (ra * rb)
        for l in range(LMAX + 1):
            sl = slice(l * l, (l + 1) * (l + 1))
            lhs = np.dot(Sa[sl], Sb[sl])
            rhs = (2 * l + 1) / (4 * np.pi) * ra ** l * rb ** l * _leg(l, cg)
            assert abs(lhs - rhs) < 1e-12 * max(1.0, (2 * l + 1) * ra ** l * rb ** l)


def test_orthonormal_on_sphere():
    nt, nphi = 24, 48
    x, w = legendre.leggauss(nt)
    ph = 2 * np.pi * np.arange(nphi) / nphi
    pts, wts = [], []
    for ct, wt in zip(x, w):
        st = np.sqrt(1 - ct * ct)
        for p in ph:
            pts.append((st * np.cos(p), st * np.sin(p), ct))
            wts.append(wt * 2 * np.pi / nphi)
    S = O.solid_harmonics_all(LMAX, np.array(pts))
    G = S.T @ (S * np.array(wts)[:, None])
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-12


def test_single_and_all_agree(rng):
    p = rng.normal(size=3)
    S = O.solid_harmonics_all(LMAX, p)[0]
    for l in range(LMAX + 1):
        for m in range(-l, l + 1):
            assert O.solid_harmonic(l, m, *p) == pytest.approx(S[l * l + l + m], rel=1e-14, abs=1e-15)


def test_homogeneous_degree_l(rng):
    p = rng.normal(size=3)
    S1 = O.solid_harmonics_all(LMAX, p)[0]
    S2 = O.solid_harmonics_all(LMAX, 1.7 * p)[0]
    for l in range(LMAX + 1):
        sl = slice(l * l, (l + 1) * (l + 1))
        np.testing.assert_allclose(S2[sl], 1.7 ** l * S1[sl], rtol=1e-12, atol=1e-14)


def test_origin():
    S = O.solid_harmonics_all(LMAX, np.zeros(3))[0]
    assert S[0] == pytest.approx(1 / np.sqrt(4 * np.pi))
    assert np.all(S[1:] == 0)
