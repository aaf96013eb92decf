"""Pins for the multipole moments (Eq. mepole) and expansion (Eq. me).

Closed forms: for a spherical Gaussian charge q centred at d, r^l Y_lm is a
harmonic polynomial, so by the mean-value property its moments about the
origin are exactly q S_lm(d).  Outside the charge the potential is q/|r-d|,
which the l <= 6 expansion reproduces up to O((|d|/r)^7).
"""
import numpy as np

from oracle import oracle as O


def _gauss_box(n, hh, p, d, q=1.0):
    c = (n - 1) / 2
    z, y, x = np.meshgrid(*(np.arange(n) - c for _ in range(3)), indexing="ij")
    X, Y, Z = x * hh - d[0], y * hh - d[1], z * hh - d[2]
    return q * (p / np.pi) ** 1.5 * np.exp(-p * (X * X + Y * Y + Z * Z))


def test_moments_of_displaced_gaussian():
    n, hh, p = 56, 0.15, 3.0  # box half width 4.2 bohr: r^6 tails negligible
    d = np.array([0.31, -0.22, 0.17])
    rho = _gauss_box(n, hh, p, d, q=0.8)
    Q = O.moments(rho, (hh, hh, hh), hh ** 3, 6)
    S = O.solid_harmonics_all(6, d)[0]
    np.testing.assert_allclose(Q, 0.8 * S, rtol=0, atol=1e-9)


def test_moments_center_is_box_centre_anisotropic():
    # an off-centre point charge: Q_1m picks up the offset from the box centre
    ex, ey, ez = 9, 7, 5
    h = (0.2, 0.3, 0.4)
    rho = np.zeros((ez, ey, ex))
    rho[1, 5, 2] = 1.0 / np.prod(h)
    Q = O.moments(rho, h, np.prod(h), 1)
    off = np.array([(2 - 4) * 0.2, (5 - 3) * 0.3, (1 - 2) * 0.4])
    S = O.solid_harmonics_all(1, off)[0]
    np.testing.assert_allclose(Q, S, atol=1e-14)


def test_me_far_field_of_displaced_charge(rng):
    d = np.array([0.2, -0.1, 0.15])
    q = 1.3
    Q = q * O.solid_harmonics_all(6, d)[0]
    pts = rng.normal(size=(50, 3))
    pts = 6.0 * pts / np.linalg.norm(pts, axis=1)[:, None]
    v = O.me_eval(Q, 6, pts)
    exact = q / np.linalg.norm(pts - d, axis=1)
    ratio = np.linalg.norm(d) / 6.0
    assert np.abs(v - exact).max() < 5 * q / 6.0 * ratio ** 7


def test_me_monopole_is_coulomb():
    Q = np.zeros(49)
    Q[0] = 2.0 * np.sqrt(1 / (4 * np.pi))  # charge 2 at the centre
    pts = np.array([[1.0, 0, 0], [0, 2.0, 0], [0.3, 0.4, 1.2]])
    np.testing.assert_allclose(O.me_eval(Q, 6, pts), 2.0 / np.linalg.norm(pts, axis=1), rtol=1e-14)
