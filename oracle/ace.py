"""ACE steps of the oracle (Sec. II C, Eq. Vace, Eq. exx_ace; App. A).

TEST INFRASTRUCTURE ONLY (see ``oracle.py``).

Orbitals and grid functions are rows: ``F[i, r]`` = phi_i(r), shape
[n, N_grid]; inner products carry the grid weight dV.

Sign convention.  The paper builds M from D^i = -V_xx phi_i, which makes it
positive semi-definite.  Here W = V_xx Phi (the output of the exchange
application), so M = Phi^T W dV is the paper's M with the sign flipped; the
Cholesky factor L of -Mbar is the paper's, and Xi = W L^-T equals the paper's
xi = -D L^-T.  The operator is V^ACE = -Xi Xi^T (dV), Eq. Vace.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


class NotPositiveDefinite(ArithmeticError):
    pass


def cholesky_lower(A: np.ndarray) -> np.ndarray:
    """Plain column-by-column Cholesky A = L L^T (no LAPACK); raises when a
    pivot is not positive (the case App. A's eigen fallback is for)."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        d = A[j, j] - np.dot(L[j, :j], L[j, :j])
        if not d > 0.0:
            raise NotPositiveDefinite(f"pivot {j} = {d}")
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (A[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    return L


def build_ace(F: np.ndarray, W: np.ndarray, dV: float) -> dict:
    """M = Phi^T W dV, Mbar = (M + M^T)/2 (App. A), -Mbar = L L^T,
    Xi = W L^-T (Eq. Vace).  ``F`` and ``W`` are [n, N_grid]."""
    F = np.asarray(F, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    M = (F @ W.T) * dV
    Mbar = 0.5 * (M + M.T)
    L = cholesky_lower(-Mbar)
    # rows of Xi: Xi[k] = sum_i (L^-T)_{ik} W[i]  ->  Xi = L^-1 W (row layout)
    Xi = scipy.linalg.solve_triangular(L, W, lower=True)
    return dict(M=M, Mbar=Mbar, L=L, Xi=Xi)


def apply_ace(Xi: np.ndarray, psi: np.ndarray, dV: float) -> np.ndarray:
    """V^ACE psi = -Xi (Xi^T psi dV) for row-layout psi [n_vec, N_grid]."""
    C = (Xi @ psi.T) * dV  # [n, n_vec]
    return -(C.T @ Xi)


def exx_ace(F: np.ndarray, Xi: np.ndarray, dV: float) -> float:
    """E_xx = -sum_ik <phi_i|xi_k>^2 (Eq. exx_ace)."""
    P = (F @ Xi.T) * dV
    return float(-np.sum(P * P))


def build_ace_eigen(F: np.ndarray, W: np.ndarray, dV: float, cut: float = 1e-13) -> dict:
    """App. A: -Mbar = Q Lambda Q^T (library eigensolver) and
    zeta_k = sum_i W_i (Q Lambda^-1/2)_ik, complex where lambda_k < 0
    (the paper's zeta = -D Z^-T with D = -W).  Eigenvalues within
    cut * max|lambda| of zero are dropped."""
    F = np.asarray(F, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    M = (F @ W.T) * dV
    Mbar = 0.5 * (M + M.T)
    lam, Q = np.linalg.eigh(-Mbar)
    keep = np.abs(lam) > cut * np.abs(lam).max()
    s = np.zeros(len(lam), dtype=np.complex128)
    s[keep] = 1.0 / np.sqrt(lam[keep].astype(np.complex128))
    zeta = (Q * s[None, :]).T @ W  # rows: zeta_k
    return dict(M=M, Mbar=Mbar, lam=lam, Q=Q, keep=keep, zeta=zeta[keep])


def apply_ace_eigen(zeta: np.ndarray, psi: np.ndarray, dV: float) -> np.ndarray:
    """V^ACE psi = -sum_k |zeta_k> <zeta_k|psi> dV (Eq. Vace_alter) with the
    Hermitian inner product <zeta_k|psi> = sum conj(zeta_k) psi (reading:
    the plane-wave code's products are Hermitian)."""
    C = (np.conj(zeta) @ psi.T) * dV
    Y = -(C.T @ zeta)
    return np.real(Y)
