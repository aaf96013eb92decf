"""Free-space Poisson reference on a grid, by FFT (test infrastructure only).

The plain definition behind Eqs. exxGen and Dxx: v solves
Lap v = -4 pi rho in free space, i.e. v = rho * (1/|r|).  On a grid this is
evaluated spectrally with the Coulomb kernel truncated at a radius R_c that
covers the whole charge box, on a zero-padded periodic grid large enough that
no periodic image reaches the box:  v(G) = 4 pi rho(G) (1 - cos(G R_c)) / G^2,
with the G = 0 limit 2 pi R_c^2 rho(0).  For a charge box of diagonal D this
is exact (up to the band limit of rho) when R_c >= D and the padded edge is
at least box edge + R_c.  Used to pin the oracle; never by the product path.
"""
from __future__ import annotations

import numpy as np


def freespace_potential(rho: np.ndarray, h) -> np.ndarray:
    """Continuum free-space potential of a [z][y][x] grid density."""
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    hx, hy, hz = h
    D = np.sqrt((nx * hx) ** 2 + (ny * hy) ** 2 + (nz * hz) ** 2)
    Rc = D
    Mx = int(np.ceil((nx * hx + Rc) / hx)) + 1
    My = int(np.ceil((ny * hy + Rc) / hy)) + 1
    Mz = int(np.ceil((nz * hz + Rc) / hz)) + 1
    pad = np.zeros((Mz, My, Mx))
    pad[:nz, :ny, :nx] = rho
    kx = 2 * np.pi * np.fft.fftfreq(Mx, d=hx)
    ky = 2 * np.pi * np.fft.fftfreq(My, d=hy)
    kz = 2 * np.pi * np.fft.fftfreq(Mz, d=hz)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    G2 = KX ** 2 + KY ** 2 + KZ ** 2
    G = np.sqrt(G2)
    with np.errstate(divide="ignore", invalid="ignore"):
        ker = 4 * np.pi * (1.0 - np.cos(G * Rc)) / G2
    ker[0, 0, 0] = 2 * np.pi * Rc * Rc
    vg = np.fft.fftn(pad) * ker
    v = np.real(np.fft.ifftn(vg))
    return v[:nz, :ny, :nx]
