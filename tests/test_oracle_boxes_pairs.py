"""Pins for domain truncation (Eq. oii) and pair selection (Eq. sij)."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O


def _brute_interval(m, tail):
    n = len(m)
    for L in range(1, n + 1):
        for s in range(n):
            out = [x for x in range(n) if (x - s) % n >= L]
            if sum(m[x] for x in out) <= tail:
                return s, L
    return 0, n


@pytest.mark.parametrize("seed", range(12))
def test_fit_interval_is_shortest_then_leftmost(seed):
    r = np.random.default_rng(seed)
    n = int(r.integers(3, 13))
    m = r.exponential(size=n) ** 3
    m /= m.sum()
    tail = float(r.choice([0.0, 0.01, 0.05, 0.2]))
    assert O.fit_interval(m, tail) == _brute_interval(m, tail)


def test_fit_interval_wraps():
    m = np.zeros(10)
    m[[9, 0, 1]] = [0.3, 0.4, 0.3]
    assert O.fit_interval(m, 1e-12) == (9, 3)


def test_marginals_sum_to_total(h2o8):
    f = h2o8.phi[3]
    mx, my, mz = O.marginals(f, h2o8.dV)
    tot = (f * f).sum() * h2o8.dV
    for m, ax in ((mx, (0, 1)), (my, (0, 2)), (mz, (1, 2))):
        # squares below the 2^-64 grid count as zero: at most one grid unit
        # per point of the plane
        plane = f.size // m.size
        np.testing.assert_allclose(m, (f * f).sum(axis=ax) * h2o8.dV, rtol=1e-12,
                                   atol=plane * 2.0 ** -64 * h2o8.dV)
        assert m.sum() == pytest.approx(tot, rel=1e-13)


def _exact_marginals(f, dV):
    """Eq. oii marginals under the exact reading, with Python integers: each
    square on the grid 2^-64 (floor, saturated at 2^96), exact sums, one
    rounding to nearest of the sum (fractions.Fraction -> float) and one of
    the product with dV."""
    from fractions import Fraction
    def F(v):
        p, q = float(v).as_integer_ratio()  # |v| = p/q, q a power of two
        val = (p * p << 64) // (q * q)
        return min(val, 1 << 96)
    nz, ny, nx = f.shape
    Fs = [[[F(f[z, y, x]) for x in range(nx)] for y in range(ny)] for z in range(nz)]
    mx = [sum(Fs[z][y][x] for z in range(nz) for y in range(ny)) for x in range(nx)]
    my = [sum(Fs[z][y][x] for z in range(nz) for x in range(nx)) for y in range(ny)]
    mz = [sum(Fs[z][y][x] for y in range(ny) for x in range(nx)) for z in range(nz)]
    conv = lambda S: float(Fraction(S, 1 << 64)) * dV
    return [np.array([conv(S) for S in m]) for m in (mx, my, mz)]


@pytest.mark.parametrize("seed", range(4))
def test_marginals_are_exact_fixed_point_sums(seed):
    r = np.random.default_rng(seed)
    shape = (3, 4, 5)
    # magnitudes from far below the 2^-64 grid of the squares up to the
    # saturation point, both signs, a few exact zeros
    f = r.standard_normal(shape) * 10.0 ** r.uniform(-14, 5, size=shape)
    f[0, 0, 0] = 0.0
    f[1, 2, 3] = 2.0 ** 16  # square exactly 2^32: saturates to 2^96
    f[2, 3, 4] = -(2.0 ** 16) * (1 - 2.0 ** -52)  # just below saturation
    f[0, 1, 2] = 2.0 ** -32  # square exactly one grid unit
    f[0, 1, 3] = 2.0 ** -32 * (1 - 2.0 ** -53)  # square just below one unit
    dV = 0.0146
    got = O.marginals(f, dV)
    for g, e in zip(got, _exact_marginals(f, dV)):
        np.testing.assert_array_equal(g, e)


def test_boxes_cover_mass_and_are_tight(h2o8):
    eps = 10 ** -3.5
    box = O.boxes(h2o8.phi, h2o8.dV, eps)
    N = h2o8.grid
    for i, b in enumerate(box):
        f = h2o8.phi[i]
        idx = [(b[a] + np.arange(b[3 + a])) % N[a] for a in range(3)]
        inside = (f[np.ix_(idx[2], idx[1], idx[0])] ** 2).sum() * h2o8.dV
        assert inside >= 1 - eps  # Eq. oii (orbitals are normalized)
        mx, my, mz = O.marginals(f, h2o8.dV)
        for a, m in enumerate((mx, my, mz)):
            s, L = b[a], b[3 + a]
            assert m.sum() - m[(s + np.arange(L)) % N[a]].sum() <= eps / 3 + 1e-15
            # one point shorter (either end) breaks the per-axis tail
            for s2 in (s, s + 1):
                assert m.sum() - m[(s2 + np.arange(L - 1)) % N[a]].sum() > eps / 3


@pytest.mark.parametrize("seed", range(200))
def test_intersect_matches_ring_sets(seed):
    r = np.random.default_rng(seed)
    n = int(r.integers(5, 30))
    L1 = int(r.integers(1, n))
    L2 = int(r.integers(1, n - L1 + 1))  # single-piece intersections
    s1, s2 = int(r.integers(0, n)), int(r.integers(0, n))
    A = {(s1 + t) % n for t in range(L1)}
    B = {(s2 + t) % n for t in range(L2)}
    res = O.intersect(s1, L1, s2, L2, n)
    if not (A & B):
        assert res is None
        return
    lo, ext, k = res
    assert {(lo + t) % n for t in range(ext)} == A & B
    assert s1 <= lo and lo + ext <= s1 + L1          # inside i's frame
    assert s2 + k * n <= lo and lo + ext <= s2 + k * n + L2


def test_intersect_full_axis():
    assert O.intersect(3, 10, 7, 4, 10) == (7, 4, 0)
    assert O.intersect(7, 4, 3, 10, 10) == (7, 4, 0)


def test_overlap_abs_matches_numpy(h2o8):
    fi, fj = h2o8.phi[0], h2o8.phi[1]
    lo, ext = (40, -3, 5), (12, 10, 9)
    N = h2o8.grid
    idx = [(lo[a] + np.arange(ext[a])) % N[a] for a in range(3)]
    ref = np.abs(fi[np.ix_(idx[2], idx[1], idx[0])] * fj[np.ix_(idx[2], idx[1], idx[0])]).sum() * h2o8.dV
    assert O.overlap_abs(fi, fj, lo, ext, h2o8.dV) == pytest.approx(ref, rel=1e-13)


def test_pairs_match_brute_force(h2o8):
    eps, delta = 10 ** -3.5, 1e-3
    box = O.boxes(h2o8.phi, h2o8.dV, eps)
    P = O.pairs(h2o8.phi, h2o8.dV, box, delta)
    N = h2o8.grid
    want = []
    for i, j in itertools.combinations_with_replacement(range(h2o8.n_orb), 2):
        sets = []
        for a in range(3):
            A = {(box[i][a] + t) % N[a] for t in range(box[i][3 + a])}
            B = {(box[j][a] + t) % N[a] for t in range(box[j][3 + a])}
            sets.append(sorted(A & B))
        if not all(sets):
            continue
        f = h2o8.phi
        S = np.abs(f[i][np.ix_(sets[2], sets[1], sets[0])] * f[j][np.ix_(sets[2], sets[1], sets[0])]).sum() * h2o8.dV
        if i == j or S >= delta:
            want.append((i, j, S))
    got = [(int(a), int(b)) for a, b in P["pair"]]
    assert got == [(i, j) for i, j, _ in want]
    np.testing.assert_allclose(P["S"], [s for _, _, s in want], rtol=1e-12)
    assert all(i == j for i, j in got[:1])


def test_scale2x():
    assert O.scale2x(10, 4, 96) == (8, 8)      # even: [s - L/2, s + 3L/2)
    assert O.scale2x(10, 5, 96) == (7, 11)     # odd: [c - L, c + L], c = 12
    assert O.scale2x(0, 40, 48) == (-4, 48)    # capped at N, centred on 19.5
