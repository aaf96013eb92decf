"""Fixtures under tests/golden/ against the oracle and the library's defaults.

`fd12_second_difference.txt` holds the exact weights of the order-12 centred
second difference, the per-axis operator of the paper's O(h^12) Laplacian.
They are fixed by its moment conditions, which are checked here in rational
arithmetic; the oracle derives its weights from a closed form, so the two are
independent.  `paper_settings.txt` holds the settings the paper states for its
calculations (l_max, stencil order, CG residual, the epsilon range).
"""
import math
import pathlib
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = pathlib.Path(__file__).parent / "golden"


def _rows(name):
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if line and not line.startswith("#"):
            yield line.split()


def _fd12():
    return {int(k): Fraction(int(n), int(d)) for k, n, d in _rows("fd12_second_difference.txt")}


def _settings():
    return {k: v for k, v in _rows("paper_settings.txt")}


def test_fd12_fixture_is_consistent():
    w = _fd12()
    assert sorted(w) == list(range(7))
    # exact on 1 and x^2 (f'' = 0 and 2), exact zero on x^4..x^12 moments
    assert w[0] + 2 * sum(w[k] for k in range(1, 7)) == 0
    assert 2 * sum(w[k] * k * k for k in range(1, 7)) == 2
    for m in range(4, 13, 2):
        assert sum(w[k] * k ** m for k in range(1, 7)) == 0


def test_oracle_weights_match_exact_weights():
    w = _fd12()
    c = O.fd_coeffs(6)
    for k in range(7):
        assert c[k] == pytest.approx(float(w[k]), rel=4e-16, abs=0.0)


def test_oracle_laplacian_uses_the_published_weights():
    # -Lap_h of a unit spike at the box centre returns -c_|k|/h^2 along each axis
    h = (0.4, 0.5, 0.6)
    v = np.zeros((13, 13, 13))
    v[6, 6, 6] = 1.0
    out = O.neg_laplacian(v, h)
    w = _fd12()
    for k in range(1, 7):
        assert out[6, 6, 6 + k] == pytest.approx(-float(w[k]) / h[0] ** 2, rel=1e-14)
        assert out[6, 6 - k, 6] == pytest.approx(-float(w[k]) / h[1] ** 2, rel=1e-14)
        assert out[6 + k, 6, 6] == pytest.approx(-float(w[k]) / h[2] ** 2, rel=1e-14)
    centre = -float(w[0]) * sum(1 / x ** 2 for x in h)
    assert out[6, 6, 6] == pytest.approx(centre, rel=1e-14)


def test_defaults_follow_the_paper_settings():
    s = _settings()
    p = O.Params()
    assert 2 * p.fd_half == int(s["laplacian_order"])
    assert p.lmax == int(s["lmax"])
    assert float(s["eps_log10_min"]) <= math.log10(p.eps) <= float(s["eps_log10_max"])


def test_library_defaults_follow_the_paper_settings():
    from paper_2208_06097_gb300 import build, sea
    build.build()
    s = _settings()
    p = sea.default_params()
    assert p.fd_order == int(s["laplacian_order"]) and p.lmax == int(s["lmax"])
    assert float(s["eps_log10_min"]) <= math.log10(p.eps) <= float(s["eps_log10_max"])
