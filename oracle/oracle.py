"""CPU oracle for the SCDM+exx+ACE exchange path (arXiv 2208.06097).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py``.  The product library
never loads it.  It shares no code with the CUDA path.

The heavy per-pair steps live in ``sea_oracle.c`` (plain C loops, FP64,
``-ffp-contract=off``); this module compiles it on first use and wraps every
entry point with numpy arrays.  The ACE steps (Eq. Vace, Eq. exx_ace, App. A
symmetrization) are in ``ace.py``; the free-space spectral Poisson reference
used to pin the oracle is in ``freespace.py``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sea_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

_i = ctypes.c_int
_d = ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)
_pi = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, OpenMP, no contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("eps", _d), ("delta", _d), ("cg_tol", _d), ("cg_tol_mode", _i),
                ("cg_max_iter", _i), ("lmax", _i), ("fd_half", _i)]


@dataclasses.dataclass
class Params:
    """Method knobs: eps (Eq. oii), delta (Eq. sij), CG tolerance, l_max and
    stencil half width (App. C: l_max = 6, O(h^12) -> 6)."""

    eps: float = 10 ** -3.5
    delta: float = 1e-3
    cg_tol: float = 1e-8
    cg_tol_mode: int = 0
    cg_max_iter: int = 5000
    lmax: int = 6
    fd_half: int = 6

    def c(self) -> _Params:
        return _Params(self.eps, self.delta, self.cg_tol, self.cg_tol_mode,
                       self.cg_max_iter, self.lmax, self.fd_half)


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(build())
        L.ora_fd_coeffs.argtypes = [_i, _pd]
        L.ora_apply_neg_lap.argtypes = [_pd, _pd, _i, _i, _i, _pd, _i]
        L.ora_solid_harmonic.argtypes = [_i, _i, _d, _d, _d]
        L.ora_solid_harmonic.restype = _d
        L.ora_solid_harmonics_all.argtypes = [_i, _d, _d, _d, _pd]
        L.ora_moments.argtypes = [_pd, _i, _i, _i, _pd, _d, _i, _pd]
        L.ora_me_eval.argtypes = [_pd, _i, _d, _d, _d]
        L.ora_me_eval.restype = _d
        L.ora_cg.argtypes = [_pd, _pd, _i, _i, _i, _pd, _i, _d, _i, _i, _pd]
        L.ora_cg.restype = _i
        L.ora_marginals.argtypes = [_pd, _pi, _d, _pd, _pd, _pd]
        L.ora_fit_interval.argtypes = [_pd, _i, _d, _pi, _pi]
        L.ora_boxes.argtypes = [_pd, _i, _pi, _d, _d, _pi]
        L.ora_intersect.argtypes = [_i, _i, _i, _i, _i, _pi, _pi, _pi]
        L.ora_intersect.restype = _i
        L.ora_overlap_abs.argtypes = [_pd, _pd, _pi, _pi, _pi, _d]
        L.ora_overlap_abs.restype = _d
        L.ora_pairs.argtypes = [_pd, _i, _pi, _d, _pi, _d, _i, _pi, _pi, _pi, _pi, _pd]
        L.ora_pairs.restype = _i
        L.ora_scale2x.argtypes = [_i, _i, _i, _pi, _pi]
        L.ora_pair_solve.argtypes = [_pd, _pd, _pi, _pd, _pi, _pi,
                                     ctypes.POINTER(_Params), _pd, _pd, _pd]
        L.ora_pair_solve.restype = _i
        L.ora_apply_vxx.argtypes = [_pd, _i, _pi, _pd, ctypes.POINTER(_Params), _pd, _pd,
                                    _pi, _i, _pi, _pi, _pi, _pi, _pi, _pd, _pi, _pd, _pd]
        L.ora_apply_vxx.restype = _i
        L.ora_pair_potential_at.argtypes = [_pd, _pd, _i, _pi, _pi, _pd, _i, _pi, _pd]
        L.ora_num_threads.restype = _i
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(_pd)


def _ip(a):
    return a.ctypes.data_as(_pi)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return lib().ora_num_threads()


# ---- stencil (App. C) ------------------------------------------------------

def fd_coeffs(p: int = 6) -> np.ndarray:
    c = np.zeros(p + 1)
    lib().ora_fd_coeffs(p, _dp(c))
    return c


def neg_laplacian(v: np.ndarray, h, p: int = 6) -> np.ndarray:
    """-Lap_h v on a [z][y][x] box with zero values outside it."""
    v = _f64(v)
    ez, ey, ex = v.shape
    out = np.empty_like(v)
    lib().ora_apply_neg_lap(_dp(v), _dp(out), ex, ey, ez, _dp(_f64(h)), p)
    return out


# ---- harmonics and multipoles (Eqs. me, mepole) ----------------------------

def solid_harmonic(l, m, x, y, z) -> float:
    return lib().ora_solid_harmonic(l, m, x, y, z)


def solid_harmonics_all(lmax: int, pts: np.ndarray) -> np.ndarray:
    pts = _f64(np.atleast_2d(pts))
    nq = (lmax + 1) ** 2
    out = np.empty((pts.shape[0], nq))
    buf = np.empty(nq)
    for t, (x, y, z) in enumerate(pts):
        lib().ora_solid_harmonics_all(lmax, x, y, z, _dp(buf))
        out[t] = buf
    return out


def moments(rho: np.ndarray, h, dV: float, lmax: int = 6) -> np.ndarray:
    rho = _f64(rho)
    ez, ey, ex = rho.shape
    Q = np.zeros((lmax + 1) ** 2)
    lib().ora_moments(_dp(rho), ex, ey, ez, _dp(_f64(h)), dV, lmax, _dp(Q))
    return Q


def me_eval(Q: np.ndarray, lmax: int, pts: np.ndarray) -> np.ndarray:
    Q = _f64(Q)
    pts = _f64(np.atleast_2d(pts))
    return np.array([lib().ora_me_eval(_dp(Q), lmax, *p) for p in pts])


# ---- CG (Eq. pe) ------------------------------------------------------------

def cg(b: np.ndarray, h, p: int = 6, tol: float = 1e-8, tol_mode: int = 0,
       max_iter: int = 5000):
    b = _f64(b)
    ez, ey, ex = b.shape
    x = np.empty_like(b)
    res = np.zeros(1)
    it = lib().ora_cg(_dp(b), _dp(x), ex, ey, ez, _dp(_f64(h)), p, tol, tol_mode,
                      max_iter, _dp(res))
    return x, it, float(res[0])


# ---- domains and pairs (Eqs. oii, sij) --------------------------------------

def marginals(f: np.ndarray, dV: float):
    f = _f64(f)
    nz, ny, nx = f.shape
    N = _i32([nx, ny, nz])
    mx, my, mz = np.empty(nx), np.empty(ny), np.empty(nz)
    lib().ora_marginals(_dp(f), _ip(N), dV, _dp(mx), _dp(my), _dp(mz))
    return mx, my, mz


def fit_interval(m: np.ndarray, tail: float):
    m = _f64(m)
    s, L = _i32([0]), _i32([0])
    lib().ora_fit_interval(_dp(m), len(m), tail, _ip(s), _ip(L))
    return int(s[0]), int(L[0])


def boxes(phi: np.ndarray, dV: float, eps: float) -> np.ndarray:
    phi = _f64(phi)
    n, nz, ny, nx = phi.shape
    box = np.zeros((n, 6), dtype=np.int32)
    lib().ora_boxes(_dp(phi), n, _ip(_i32([nx, ny, nz])), dV, eps, _ip(box))
    return box


def intersect(s1, L1, s2, L2, n):
    lo, ext, k = _i32([0]), _i32([0]), _i32([0])
    ok = lib().ora_intersect(s1, L1, s2, L2, n, _ip(lo), _ip(ext), _ip(k))
    return (int(lo[0]), int(ext[0]), int(k[0])) if ok else None


def overlap_abs(fi, fj, lo, ext, dV) -> float:
    fi, fj = _f64(fi), _f64(fj)
    nz, ny, nx = fi.shape
    return lib().ora_overlap_abs(_dp(fi), _dp(fj), _ip(_i32([nx, ny, nz])),
                                 _ip(_i32(lo)), _ip(_i32(ext)), dV)


def scale2x(s, L, n):
    ws, wl = _i32([0]), _i32([0])
    lib().ora_scale2x(s, L, n, _ip(ws), _ip(wl))
    return int(ws[0]), int(wl[0])


def pairs(phi: np.ndarray, dV: float, box: np.ndarray, delta: float):
    phi = _f64(phi)
    n, nz, ny, nx = phi.shape
    cap = n * n
    pair = np.zeros((cap, 2), np.int32)
    plo = np.zeros((cap, 3), np.int32)
    pext = np.zeros((cap, 3), np.int32)
    pk = np.zeros((cap, 3), np.int32)
    S = np.zeros(cap)
    np_ = lib().ora_pairs(_dp(phi), n, _ip(_i32([nx, ny, nz])), dV, _ip(_i32(box)), delta,
                          cap, _ip(pair), _ip(plo), _ip(pext), _ip(pk), _dp(S))
    return dict(pair=pair[:np_], lo=plo[:np_], ext=pext[:np_], k=pk[:np_], S=S[:np_])


# ---- per-pair problem -------------------------------------------------------

def pair_solve(fi, fj, cell, lo, ext, params: Params | None = None):
    """rho = phi_i phi_j on [lo, lo+ext), its Q_lm and its potential v."""
    params = params or Params()
    fi, fj = _f64(fi), _f64(fj)
    nz, ny, nx = fi.shape
    ext = _i32(ext)
    v = np.empty((ext[2], ext[1], ext[0]))
    Q = np.empty((params.lmax + 1) ** 2)
    e = np.zeros(1)
    prm = params.c()
    it = lib().ora_pair_solve(_dp(fi), _dp(fj), _ip(_i32([nx, ny, nz])), _dp(_f64(cell)),
                              _ip(_i32(lo)), _ip(ext), ctypes.byref(prm), _dp(v), _dp(Q),
                              _dp(e))
    return v, Q, float(e[0]), it


def pair_potential_at(v, Q, lmax, lo, ext, h, pts_unwrapped) -> np.ndarray:
    pts = _i32(np.atleast_2d(pts_unwrapped))
    out = np.empty(pts.shape[0])
    lib().ora_pair_potential_at(_dp(_f64(v)), _dp(_f64(Q)), lmax, _ip(_i32(lo)),
                                _ip(_i32(ext)), _dp(_f64(h)), pts.shape[0], _ip(pts),
                                _dp(out))
    return out


# ---- whole application ------------------------------------------------------

def apply_vxx(phi: np.ndarray, cell, params: Params | None = None) -> dict:
    """V_xx phi_i for every orbital and E_xx (Eqs. tDxx, DxxVxx, exxGen_mlwf).

    Returns a dict with ``vxx`` ([n][nz][ny][nx]), ``exx`` and the plan
    (boxes, pairs, per-pair S, CG iterations, pair integrals, moments)."""
    params = params or Params()
    phi = _f64(phi)
    n, nz, ny, nx = phi.shape
    vxx = np.empty_like(phi)
    exx = np.zeros(1)
    box = np.zeros((n, 6), np.int32)
    cap = n * n
    nq = (params.lmax + 1) ** 2
    npairs = _i32([0])
    pair = np.zeros((cap, 2), np.int32)
    plo = np.zeros((cap, 3), np.int32)
    pext = np.zeros((cap, 3), np.int32)
    pk = np.zeros((cap, 3), np.int32)
    S = np.zeros(cap)
    its = np.zeros(cap, np.int32)
    ep = np.zeros(cap)
    Q = np.zeros((cap, nq))
    prm = params.c()
    rc = lib().ora_apply_vxx(_dp(phi), n, _ip(_i32([nx, ny, nz])), _dp(_f64(cell)),
                             ctypes.byref(prm), _dp(vxx), _dp(exx), _ip(box), cap,
                             _ip(npairs), _ip(pair), _ip(plo), _ip(pext), _ip(pk), _dp(S),
                             _ip(its), _dp(ep), _dp(Q))
    P = int(npairs[0])
    return dict(rc=rc, vxx=vxx, exx=float(exx[0]), box=box, pair=pair[:P], lo=plo[:P],
                ext=pext[:P], k=pk[:P], S=S[:P], iters=its[:P], epair=ep[:P], Q=Q[:P])
