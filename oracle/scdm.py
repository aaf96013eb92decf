"""SCDM localization (Sec. II A, Eqs. phi_qr, nonortho_scdm, ortho_scdm,
unitary_scdm) -- CPU reference.

TEST INFRASTRUCTURE ONLY (see ``oracle.py``).

Orbitals are rows: ``phi[n][N]`` (the paper's Phi^T), orthonormal with the
grid weight dV.  Steps in the paper's order: column-pivoted QR of Phi^T
(library routine: LAPACK's pivoted QR through scipy), C = the first n
pivots, B = (Phi^T)_{:,C}, P_CC = B^T B (= X^T X dV for X = Phi B), the
symmetric inverse square root of P_CC (library eigendecomposition),
U = B P_CC^{-1/2}, Phi~ = Phi U.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def scdm(phi):
    """(C, U, phi_tilde) for phi [n][N]."""
    A = np.asarray(phi, dtype=np.float64).reshape(phi.shape[0], -1)
    n = A.shape[0]
    _, _, piv = scipy.linalg.qr(A, mode="economic", pivoting=True)
    C = np.asarray(piv[:n])
    B = A[:, C]
    P = B.T @ B
    lam, V = np.linalg.eigh(P)
    Pm = (V / np.sqrt(lam)[None, :]) @ V.T
    U = B @ Pm
    phit = U.T @ A
    return C, U, phit.reshape(phi.shape)
