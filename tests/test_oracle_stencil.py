"""Pins for the O(h^12) discrete Laplacian of the oracle (App. C).

The 2p-order central second difference is the unique symmetric stencil of
half width p that is exact on polynomials of degree <= 2p+1; degree 2p+2 is
the first it gets wrong, and on smooth functions the error falls as h^2p.
"""
import numpy as np
import pytest

from oracle import oracle as O


def _box_poly(ex, ey, ez, h, a, b, c, off):
    z, y, x = np.meshgrid(np.arange(ez), np.arange(ey), np.arange(ex), indexing="ij")
    X = (x - off[0]) * h[0]
    Y = (y - off[1]) * h[1]
    Z = (z - off[2]) * h[2]
    f = X ** a * Y ** b * Z ** c
    lap = np.zeros_like(f)
    if a >= 2:
        lap += a * (a - 1) * X ** (a - 2) * Y ** b * Z ** c
    if b >= 2:
        lap += b * (b - 1) * X ** a * Y ** (b - 2) * Z ** c
    if c >= 2:
        lap += c * (c - 1) * X ** a * Y ** b * Z ** (c - 2)
    return f, lap


@pytest.mark.parametrize("abc", [(0, 0, 0), (2, 0, 0), (0, 3, 1), (5, 4, 2), (13, 0, 0),
                                 (0, 13, 0), (0, 0, 13), (7, 6, 5), (13, 13, 13)])
def test_exact_on_polynomials_up_to_degree_13(abc):
    h = (0.31, 0.27, 0.23)  # anisotropic: each axis must use its own h^2
    ex, ey, ez = 15, 14, 13
    off = (7.2, 6.4, 5.9)
    f, lap = _box_poly(ex, ey, ez, h, *abc, off)
    out = -O.neg_laplacian(f, h)
    sl = (slice(6, ez - 6), slice(6, ey - 6), slice(6, ex - 6))  # stencil fully inside
    scale = max(1.0, np.abs(lap[sl]).max(), np.abs(f).max() / min(h) ** 2)
    assert np.abs(out[sl] - lap[sl]).max() <= 1e-9 * scale


def test_degree_14_is_not_exact():
    h = (0.3, 0.3, 0.3)
    f, lap = _box_poly(13, 13, 13, h, 14, 0, 0, (6.0, 6.0, 6.0))
    out = -O.neg_laplacian(f, h)
    # at the centre the truncation term (p!)^2 2/(2p+2)! h^12 f^(14) is non-zero
    assert abs(out[6, 6, 6] - lap[6, 6, 6]) > 1e-3


def test_order_twelve_on_trig():
    errs = []
    for n in (8, 12):  # coarse enough to stay above the rounding floor
        hh = 2 * np.pi / n
        x = np.arange(n + 12) * hh
        f = np.sin(0.9 * x)[None, None, :] * np.ones((13, 13, 1))
        out = -O.neg_laplacian(f, (hh, 1.0, 1.0))
        i = (n + 12) // 2
        errs.append(abs(out[6, 6, i] - (-0.81 * np.sin(0.9 * x[i]))))
    rate = np.log(errs[0] / errs[1]) / np.log(12 / 8)
    assert 11.0 < rate < 13.5


def test_zero_dirichlet_outside_box():
    # A delta in a corner: neighbours beyond the box are treated as zero, so
    # the operator is a finite Toeplitz section: symmetric and positive.
    h = (0.25, 0.25, 0.25)
    n = 5
    A = np.zeros((n ** 3, n ** 3))
    for k in range(n ** 3):
        e = np.zeros(n ** 3)
        e[k] = 1.0
        A[:, k] = O.neg_laplacian(e.reshape(n, n, n), h).ravel()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
