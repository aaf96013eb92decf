"""Seeded synthetic water-like localized orbitals (input generator only).

This module builds the inputs that both the CPU oracle and the CUDA path
consume.  It holds none of the exchange method's arithmetic: it only draws
molecules, places Gaussian-type orbitals on a periodic real-space grid and
orthonormalizes them (Loewdin) so that the orbitals are the kind of localized,
orthonormal occupied set the method starts from (Sec. II B: localized orbitals
on the real-space mesh of a periodic cell, Gamma point, real valued).

Recipe (stands in for the paper's (H2O)64 configurations, which are not
available):

* ``n_mol`` rigid waters, O-H = 0.96 A, H-O-H = 104.5 deg; O positions
  uniform in the cell with minimum-image O-O >= 2.5 A (random sequential
  addition, 10^4 tries per molecule, then a seeded soft-sphere relaxation
  when the density is above the random-addition jamming limit); orientations
  from uniform random unit quaternions.
* Four orbitals per molecule: two bond Gaussians 0.45 A from O along each
  O-H, two lone-pair Gaussians 0.35 A from O along
  -b cos(54.75 deg) +/- n sin(54.75 deg) (b = H-O-H bisector, n = plane
  normal).
* Each orbital is exp(-alpha |d|^2) (1 + 0.1 d^T A d), d in bohr,
  alpha ~ U[1.5, 3.0] bohr^-2, A symmetric with entries ~ U[-1, 1]; periodic
  images with |n_a| <= 1 are summed.
* Loewdin orthonormalization on the grid: Phi <- Phi S^{-1/2},
  S = Phi^T Phi dV.

Layout: ``phi[n_orb][nz][ny][nx]`` float64, x fastest.  Units: bohr.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ANGSTROM = 1.0 / 0.529177210903  # bohr per angstrom

R_OH = 0.96  # A
THETA_HOH = 104.5  # deg
D_BOND = 0.45  # A, bond-orbital centre from O along O-H
D_LONE = 0.35  # A, lone-pair centre from O
LONE_ANGLE = 54.75  # deg, half angle between the two lone pairs
MIN_OO = 2.5  # A


@dataclasses.dataclass
class System:
    """One synthetic configuration."""

    phi: np.ndarray  # [n_orb, nz, ny, nx] float64, orthonormal on the grid
    cell: tuple  # (Lx, Ly, Lz) bohr, orthorhombic
    grid: tuple  # (nx, ny, nz)
    centers: np.ndarray  # [n_orb, 3] bohr, Gaussian centres before Loewdin
    alphas: np.ndarray  # [n_orb]
    oxygens: np.ndarray  # [n_mol, 3] bohr

    @property
    def n_orb(self) -> int:
        return self.phi.shape[0]

    @property
    def dV(self) -> float:
        return (self.cell[0] * self.cell[1] * self.cell[2]) / (
            self.grid[0] * self.grid[1] * self.grid[2])


def _min_image(d, L):
    return d - L * np.round(d / L)


def _place_oxygens(rng, n_mol, L, dmin, tries=10_000):
    pos = np.zeros((0, 3))
    for _ in range(n_mol):
        ok = False
        for _t in range(tries):
            p = rng.uniform(0.0, L, size=3)
            if pos.shape[0] == 0:
                ok = True
            else:
                d = _min_image(pos - p, L)
                ok = bool(np.all(np.einsum("ij,ij->i", d, d) >= dmin * dmin))
            if ok:
                pos = np.vstack([pos, p])
                break
        if not ok:
            return _relax(rng, n_mol, L, dmin)
    return pos


def _relax(rng, n_mol, L, dmin, max_sweeps=200_000):
    """Seeded soft-sphere relaxation: push overlapping pairs apart."""
    pos = rng.uniform(0.0, L, size=(n_mol, 3))
    target = dmin * 1.0005
    for _ in range(max_sweeps):
        d = pos[:, None, :] - pos[None, :, :]
        d = _min_image(d, L)
        r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
        np.fill_diagonal(r, np.inf)
        if r.min() >= dmin:
            return np.mod(pos, L)
        over = np.clip(target - r, 0.0, None)
        with np.errstate(invalid="ignore", divide="ignore"):
            push = np.where(r[..., None] > 0, d / r[..., None], 0.0)
        pos = pos + 0.5 * np.einsum("ij,ijk->ik", over, push)
        pos = np.mod(pos, L)
    raise RuntimeError("soft-sphere relaxation did not reach the O-O minimum")


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _molecule_centres(O, R):
    """Four orbital centres (bohr) of one water with O at ``O`` rotated by R."""
    half = math.radians(THETA_HOH / 2.0)
    uh1 = np.array([math.sin(half), 0.0, math.cos(half)])
    uh2 = np.array([-math.sin(half), 0.0, math.cos(half)])
    b = np.array([0.0, 0.0, 1.0])  # bisector (towards the H atoms)
    n = np.array([0.0, 1.0, 0.0])  # plane normal
    la = math.radians(LONE_ANGLE)
    ul1 = -b * math.cos(la) + n * math.sin(la)
    ul2 = -b * math.cos(la) - n * math.sin(la)
    local = [D_BOND * uh1, D_BOND * uh2, D_LONE * ul1, D_LONE * ul2]
    return [O + ANGSTROM * (R @ v) for v in local]


def _axis_moments(coords, c, L, alpha):
    """Image-summed 1-D factors sum_n g, sum_n g d, sum_n g d^2 on one axis."""
    g0 = np.zeros_like(coords)
    g1 = np.zeros_like(coords)
    g2 = np.zeros_like(coords)
    for n in (-1, 0, 1):
        d = coords - c - n * L
        g = np.exp(-alpha * d * d)
        g0 += g
        g1 += g * d
        g2 += g * d * d
    return g0, g1, g2


def _orbital(xs, ys, zs, cell, c, alpha, A):
    """exp(-alpha|d|^2)(1 + 0.1 d^T A d) summed over images |n_a| <= 1.

    Each image term is a product of 1-D Gaussians times a quadratic, so the
    image sum factorizes into 1-D sums per axis (same value, fewer exps).
    """
    X0, X1, X2 = _axis_moments(xs, c[0], cell[0], alpha)
    Y0, Y1, Y2 = _axis_moments(ys, c[1], cell[1], alpha)
    Z0, Z1, Z2 = _axis_moments(zs, c[2], cell[2], alpha)
    o = np.einsum

    def t(z, y, x):
        return o("k,j,i->kji", z, y, x)

    f = t(Z0, Y0, X0)
    f = f + 0.1 * (A[0, 0] * t(Z0, Y0, X2) + A[1, 1] * t(Z0, Y2, X0)
                   + A[2, 2] * t(Z2, Y0, X0)
                   + 2 * A[0, 1] * t(Z0, Y1, X1) + 2 * A[0, 2] * t(Z1, Y0, X1)
                   + 2 * A[1, 2] * t(Z1, Y1, X0))
    return f


def _draw(n_mol, L_angstrom, grid, seed, alpha_range=(1.5, 3.0), centre_first=False):
    """The seeded parameters of one configuration: cell, grid, orbital
    centres, exponents, quadratic-factor matrices, oxygen positions."""
    if isinstance(grid, int):
        grid = (grid, grid, grid)
    L = L_angstrom * ANGSTROM
    cell = (L, L, L)
    rng = np.random.default_rng(seed)
    oxy = _place_oxygens(rng, n_mol, L, MIN_OO * ANGSTROM)
    if centre_first:
        oxy = np.mod(oxy - oxy[0] + 0.5 * L, L)
    rots = [_random_rotation(rng) for _ in range(n_mol)]
    centres = []
    for m in range(n_mol):
        centres.extend(_molecule_centres(oxy[m], rots[m]))
    centres = np.mod(np.array(centres), L)
    n_orb = len(centres)
    alphas = rng.uniform(alpha_range[0], alpha_range[1], size=n_orb)
    As = rng.uniform(-1.0, 1.0, size=(n_orb, 3, 3))
    As = 0.5 * (As + np.transpose(As, (0, 2, 1)))
    return cell, tuple(grid), centres, alphas, As, oxy


def make_waters(n_mol: int, L_angstrom: float, grid, seed: int,
                loewdin: bool = True, alpha_range=(1.5, 3.0),
                centre_first: bool = False) -> System:
    """Build one seeded (H2O)n-like orbital set in a cubic cell of edge L.

    ``alpha_range`` sets the Gaussian exponent interval (bohr^-2);
    ``centre_first`` moves the first oxygen to the cell centre (used for
    isolated-molecule cases that must not touch the cell boundary)."""
    cell, grid, centres, alphas, As, oxy = _draw(n_mol, L_angstrom, grid, seed, alpha_range,
                                                 centre_first)
    nx, ny, nz = grid
    n_orb = len(centres)
    xs = np.arange(nx) * (cell[0] / nx)
    ys = np.arange(ny) * (cell[1] / ny)
    zs = np.arange(nz) * (cell[2] / nz)
    phi = np.empty((n_orb, nz, ny, nx))
    for i in range(n_orb):
        phi[i] = _orbital(xs, ys, zs, cell, centres[i], alphas[i], As[i])
    dV = (cell[0] * cell[1] * cell[2]) / (nx * ny * nz)
    if loewdin:
        phi = loewdin_orthonormalize(phi, dV)
    return System(phi=phi, cell=cell, grid=(nx, ny, nz), centers=centres,
                  alphas=alphas, oxygens=oxy)


def loewdin_orthonormalize(phi: np.ndarray, dV: float) -> np.ndarray:
    """Phi <- Phi S^{-1/2} with S = Phi^T Phi dV (symmetric orthogonalization)."""
    n = phi.shape[0]
    F = phi.reshape(n, -1)
    S = (F @ F.T) * dV
    w, U = np.linalg.eigh(S)
    Sm = (U / np.sqrt(w)) @ U.T
    return (Sm.T @ F).reshape(phi.shape)


def separated_gaussians(n: int, grid: int, L: float, alpha: float = 3.0):
    """n Gaussians exp(-alpha r^2) on a simple cubic lattice of centres in a
    cubic cell of edge L (bohr) on grid^3 points, Loewdin-orthonormalized:
    a localized basis whose rotations test orbital localization.  Returns
    (phi [n][grid][grid][grid], dV)."""
    ax = np.arange(grid) * (L / grid)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    side = int(np.ceil(n ** (1 / 3)))
    phi = np.zeros((n, grid, grid, grid))
    for k in range(n):
        c = (np.array([k % side, (k // side) % side, k // (side * side)]) + 0.5) * (L / side)
        phi[k] = np.exp(-alpha * ((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2))
    dV = (L / grid) ** 3
    return loewdin_orthonormalize(phi, dV), dV


# Workload shapes (cubic cells).  Densities follow from 18.015 g/mol waters.
CONFIGS = {
    # 8 waters, 6.21 A, 48^3: the small case the oracle finishes in seconds.
    "h2o8_48": dict(n_mol=8, L=6.21, grid=48, seed=1000),
    # 64 waters at 1.0 g/cm^3, 12.42 A, 96^3: the paper-scale workload.
    "h2o64_96": dict(n_mol=64, L=12.42, grid=96, seed=1001),
    # 64 waters at 0.4 / 1.0 / 1.7 g/cm^3.
    "h2o64_d04_128": dict(n_mol=64, L=16.86, grid=128, seed=1002),
    "h2o64_d10_96": dict(n_mol=64, L=12.42, grid=96, seed=1002),
    "h2o64_d17_80": dict(n_mol=64, L=10.41, grid=80, seed=1002),
    # the 256-orbital system on a coarse 48^3 grid (h = 0.49 bohr): a
    # profiling case with the benchmark's orbital count, small enough for
    # multi-pass kernel captures, its orbital array still larger than L2.
    "h2o64_48": dict(n_mol=64, L=12.42, grid=48, seed=1001),
    # 16 waters in the benchmark's cell and grid (0.25 g/cm^3): the same grid
    # spacing, box sizes and 96 x 96 planes with 64 orbitals, for multi-pass
    # captures of the kernels whose shape follows the grid (outputs 0.45 GB).
    "h2o16_96": dict(n_mol=16, L=12.42, grid=96, seed=1003),
}


def make_config(name: str, **over) -> System:
    c = dict(CONFIGS[name])
    c.update(over)
    return make_waters(c["n_mol"], c["L"], c["grid"], c["seed"])


def random_trial_vectors(n_vec: int, grid, seed: int) -> np.ndarray:
    """Seeded dense trial vectors psi[n_vec][nz][ny][nx] for the ACE apply."""
    nx, ny, nz = grid if not isinstance(grid, int) else (grid, grid, grid)
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_vec, nz, ny, nx))


def make_waters_device(n_mol: int, L_angstrom: float, grid, seed: int, device):
    """The orbitals of ``make_waters`` (same seeded parameters) evaluated and
    Loewdin-orthonormalized with torch float64 on ``device`` -- for the large
    workloads (hundreds of orbitals on 10^6-10^7 points), whose host
    generation would take minutes.  The values agree with ``make_waters`` up
    to floating-point summation order.  Returns (phi [n][nz][ny][nx] tensor on
    the device, cell, grid)."""
    import torch
    cell, grid, centres, alphas, As, _ = _draw(n_mol, L_angstrom, grid, seed)
    nx, ny, nz = grid
    n = len(centres)
    dt = torch.float64
    c = torch.as_tensor(centres, dtype=dt, device=device)
    al = torch.as_tensor(alphas, dtype=dt, device=device)
    A = torch.as_tensor(As, dtype=dt, device=device)

    def moments(npts, axis):
        coords = torch.arange(npts, dtype=dt, device=device) * (cell[axis] / npts)
        d0 = coords[None, :] - c[:, axis:axis + 1]
        g0 = torch.zeros((n, npts), dtype=dt, device=device)
        g1 = torch.zeros_like(g0)
        g2 = torch.zeros_like(g0)
        for img in (-1, 0, 1):
            d = d0 - img * cell[axis]
            g = torch.exp(-al[:, None] * d * d)
            g0 += g
            g1 += g * d
            g2 += g * d * d
        return g0, g1, g2

    X0, X1, X2 = moments(nx, 0)
    Y0, Y1, Y2 = moments(ny, 1)
    Z0, Z1, Z2 = moments(nz, 2)
    phi = torch.empty((n, nz, ny, nx), dtype=dt, device=device)
    terms = [(None, Z0, Y0, X0), ((0, 0), Z0, Y0, X2), ((1, 1), Z0, Y2, X0), ((2, 2), Z2, Y0, X0),
             ((0, 1), Z0, Y1, X1), ((0, 2), Z1, Y0, X1), ((1, 2), Z1, Y1, X0)]
    for i0 in range(0, n, 32):
        i1 = min(n, i0 + 32)
        acc = None
        for idx, Z, Y, X in terms:
            t = Z[i0:i1, :, None, None] * Y[i0:i1, None, :, None] * X[i0:i1, None, None, :]
            if idx is not None:
                w = A[i0:i1, idx[0], idx[1]] * (0.1 if idx[0] == idx[1] else 0.2)
                t = t * w[:, None, None, None]
            acc = t if acc is None else acc + t
        phi[i0:i1] = acc
    dV = (cell[0] * cell[1] * cell[2]) / (nx * ny * nz)
    F = phi.reshape(n, -1)
    S = (F @ F.T) * dV
    w, U = torch.linalg.eigh(S)
    Sm = (U / torch.sqrt(w)[None, :]) @ U.T
    out = (Sm.T @ F).reshape(n, nz, ny, nx)
    del phi, F
    return out, cell, grid
