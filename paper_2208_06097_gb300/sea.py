"""Python binding of libsea.so (argument marshalling only).

Every step of the exchange path runs in the CUDA library; this module only
passes pointers and sizes through the C ABI declared in ``include/sea.h``.
Device buffers are torch CUDA tensors (float64, contiguous); host buffers
are numpy float64 arrays.  There is no CPU fallback: if the library is
missing the import of :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsea.so")

SEA_OK = 0
STATUS = {0: "SEA_OK", 1: "SEA_ERR_ARG", 2: "SEA_ERR_STATE", 3: "SEA_ERR_CUDA",
          4: "SEA_ERR_OOM", 5: "SEA_ERR_CG_NOT_CONVERGED", 6: "SEA_ERR_NOT_PD",
          7: "SEA_ERR_TIMEOUT", 8: "SEA_ERR_INPUT", 9: "SEA_ERR_LIMIT"}

EXPORTS = ["sea_default_params", "sea_create", "sea_set_orbitals", "sea_apply_vxx",
           "sea_build_ace", "sea_build_ace_from", "sea_apply_ace", "sea_get_ace_matrices", "sea_get_ace_vectors",
           "sea_get_plan", "sea_get_stats", "sea_last_error", "sea_destroy",
           "sea_poisson_batch", "sea_poisson_batch_noalloc", "sea_apply_vxx_batch",
           "sea_unet_create", "sea_unet_num_weights", "sea_unet_weights", "sea_unet_forward",
           "sea_unet_loss_grad", "sea_unet_collect", "sea_unet_num_samples", "sea_unet_train",
           "sea_unet_attach", "sea_unet_last_error", "sea_unet_destroy", "sea_scdm"]


class SeaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("delta", ctypes.c_double),
                ("cg_tol", ctypes.c_double), ("cg_tol_mode", ctypes.c_int),
                ("cg_max_iter", ctypes.c_int), ("lmax", ctypes.c_int),
                ("fd_order", ctypes.c_int), ("self_scale", ctypes.c_double),
                ("precision", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("timeout_ms", ctypes.c_double), ("ace_decomp", ctypes.c_int),
                ("orth_tol", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n_orb", ctypes.c_int), ("n_pairs", ctypes.c_int),
                ("n_proto_pairs", ctypes.c_int), ("n_unknowns", ctypes.c_longlong),
                ("n_window_points", ctypes.c_longlong), ("cg_iters_min", ctypes.c_int),
                ("cg_iters_max", ctypes.c_int), ("cg_iters_mean", ctypes.c_double),
                ("cg_unknown_iters", ctypes.c_longlong), ("exx", ctypes.c_double),
                ("ms_plan", ctypes.c_double), ("ms_setup", ctypes.c_double),
                ("ms_cg", ctypes.c_double), ("ms_accumulate", ctypes.c_double),
                ("ms_ace_build", ctypes.c_double), ("ms_ace_apply", ctypes.c_double),
                ("ace_support_points", ctypes.c_longlong), ("n_launches", ctypes.c_longlong),
                ("ms_gram_build", ctypes.c_double), ("ms_gram_apply", ctypes.c_double),
                ("ms_expand_apply", ctypes.c_double), ("ace_eigen", ctypes.c_int),
                ("ace_eigen_sweeps", ctypes.c_int), ("ace_negative_eigenvalues", ctypes.c_int),
                ("ace_dropped_eigenvalues", ctypes.c_int), ("batch_graph", ctypes.c_int),
                ("ace_max_tile_list", ctypes.c_int), ("batch_order", ctypes.c_int),
                ("batch_ctas_per_sm", ctypes.c_int), ("batch_ctas_per_sm_fp64", ctypes.c_int),
                ("batch_tune_ms", ctypes.c_double), ("exx_ace", ctypes.c_double)]


_LIB = None
_p = ctypes.c_void_p
_i = ctypes.c_int


def lib() -> ctypes.CDLL:
    """Load libsea.so (build it first with ``build.build()``)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        L.sea_default_params.argtypes = [ctypes.POINTER(Params)]
        L.sea_default_params.restype = None
        L.sea_create.argtypes = [_p, _p, ctypes.POINTER(Params), _p, ctypes.POINTER(_p)]
        L.sea_set_orbitals.argtypes = [_p, _p, _i, _i]
        L.sea_apply_vxx.argtypes = [_p, _p, _i, _p]
        L.sea_build_ace.argtypes = [_p]
        L.sea_build_ace_from.argtypes = [_p, _p, _i]
        L.sea_apply_ace.argtypes = [_p, _p, _i, _p, _i]
        L.sea_get_ace_matrices.argtypes = [_p, _p, _p, _i]
        L.sea_get_ace_vectors.argtypes = [_p, _p, _i]
        L.sea_get_plan.argtypes = [_p, _p, _p, _i, _p, _p, _p, _p, _p, _p]
        L.sea_get_stats.argtypes = [_p, ctypes.POINTER(Stats)]
        L.sea_last_error.argtypes = [_p]
        L.sea_last_error.restype = ctypes.c_char_p
        L.sea_poisson_batch.argtypes = [_p, _i, _p, _p, _p, ctypes.c_double, _i, _i, _p, _p]
        L.sea_poisson_batch_noalloc.argtypes = [_p, _i, _p, _p, _p, ctypes.c_double, _i, _i,
                                                _p, _p]
        L.sea_apply_vxx_batch.argtypes = [_p, _i, _p, _i, _p]
        L.sea_destroy.argtypes = [_p]
        L.sea_destroy.restype = None
        L.sea_scdm.argtypes = [_p, _p, _i, _i, _p, _p]
        L.sea_unet_create.argtypes = [_i, _i, _p, ctypes.POINTER(_p)]
        L.sea_unet_num_weights.argtypes = [_p]
        L.sea_unet_num_weights.restype = ctypes.c_longlong
        L.sea_unet_weights.argtypes = [_p, _p, _i]
        L.sea_unet_forward.argtypes = [_p, _p, _i, _p, _i]
        L.sea_unet_loss_grad.argtypes = [_p, _p, _p, _i, _p, _p, _i]
        L.sea_unet_collect.argtypes = [_p, _p]
        L.sea_unet_num_samples.argtypes = [_p]
        L.sea_unet_num_samples.restype = ctypes.c_longlong
        L.sea_unet_train.argtypes = [_p, _i, _i, ctypes.c_double, _i, _p]
        L.sea_unet_attach.argtypes = [_p, _p]
        L.sea_unet_last_error.argtypes = [_p]
        L.sea_unet_last_error.restype = ctypes.c_char_p
        L.sea_unet_destroy.argtypes = [_p]
        L.sea_unet_destroy.restype = None
        special = ("sea_default_params", "sea_last_error", "sea_destroy", "sea_unet_num_weights",
                   "sea_unet_num_samples", "sea_unet_last_error", "sea_unet_destroy")
        for f in EXPORTS:
            if f not in special:
                getattr(L, f).restype = _i
        _LIB = L
    return _LIB


def default_params(**over) -> Params:
    p = Params()
    lib().sea_default_params(ctypes.byref(p))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def _ptr(a):
    """(pointer, on_device) of a torch CUDA tensor or a numpy array."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data, 0
    if getattr(a, "is_cuda", False):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("device tensors must be contiguous float64")
        return a.data_ptr(), 1
    raise TypeError("expected a numpy array or a CUDA torch tensor")


def poisson_batch(h, ext, rhs, x, tol=1e-8, tol_mode=0, max_iter=5000, stream=None,
                  noalloc=False):
    """Solve -Lap_h x_b = rhs_b on boxes (device tensors, concatenated).

    ``noalloc=True`` calls sea_poisson_batch_noalloc (fixed internal
    scratch, no device allocation; see include/sea.h for its limits)."""
    ext = np.ascontiguousarray(np.asarray(ext, dtype=np.int32).reshape(-1, 3))
    nb = ext.shape[0]
    it = np.zeros(nb, np.int32)
    hh = (ctypes.c_double * 3)(*h)
    p1, d1 = _ptr(rhs)
    p2, d2 = _ptr(x)
    if not (d1 and d2):
        raise ValueError("rhs and x must be CUDA tensors")
    fn = lib().sea_poisson_batch_noalloc if noalloc else lib().sea_poisson_batch
    rc = fn(hh, nb, _p(ext.ctypes.data), _p(p1), _p(p2), tol, tol_mode, max_iter,
            _p(it.ctypes.data), _p(stream) if stream else None)
    if rc not in (SEA_OK, 5):
        raise SeaError(rc, "poisson_batch")
    return it, rc


def apply_vxx_batch(ctxs, outs):
    """Batched V_xx application over several contexts (same device and
    stream); outs: matching torch CUDA tensors or numpy arrays.  Returns the
    list of E_xx values."""
    n = len(ctxs)
    hs = (_p * n)(*[c.handle for c in ctxs])
    ptrs = [_ptr(o) for o in outs]
    if len({d for _, d in ptrs}) != 1:
        raise ValueError("outputs must be all host or all device")
    op = (_p * n)(*[p for p, _ in ptrs])
    ex = (ctypes.c_double * n)()
    rc = lib().sea_apply_vxx_batch(hs, n, op, ptrs[0][1], ex)
    if rc != SEA_OK:
        msgs = "; ".join(lib().sea_last_error(c.handle).decode() for c in ctxs)
        raise SeaError(rc, f"apply_vxx_batch: {msgs}")
    return list(ex)


class Context:
    """One exchange engine on the current CUDA device (see include/sea.h)."""

    def __init__(self, cell, grid, params: Params | None = None, stream=None, **over):
        self._h = _p()
        c = (ctypes.c_double * 3)(*cell)
        g = (ctypes.c_int * 3)(*grid)
        prm = params if params is not None else default_params(**over)
        self.grid = tuple(int(x) for x in grid)
        self.cell = tuple(float(x) for x in cell)
        s = _p(stream) if stream is not None else None
        self._check(lib().sea_create(c, g, ctypes.byref(prm), s, ctypes.byref(self._h)), "create")
        self.n_orb = 0

    @property
    def handle(self):
        return self._h

    def _check(self, rc, what):
        if rc != SEA_OK:
            msg = lib().sea_last_error(self._h).decode() if self._h else what
            raise SeaError(rc, f"{what}: {msg}")

    def set_orbitals(self, phi):
        ptr, dev = _ptr(phi)
        n = int(phi.shape[0])
        self._check(lib().sea_set_orbitals(self._h, _p(ptr), n, dev), "set_orbitals")
        self.n_orb = n

    def scdm(self, phi):
        """Localize the orbitals phi (SCDM, Sec. II A) into the context;
        returns (U, selected grid points)."""
        ptr, dev = _ptr(phi)
        n = int(phi.shape[0])
        U = np.zeros((n, n))
        cols = np.zeros(n, np.int32)
        self._check(lib().sea_scdm(self._h, _p(ptr), n, dev, _p(U.ctypes.data),
                                   _p(cols.ctypes.data)), "scdm")
        self.n_orb = n
        return U, cols

    def apply_vxx(self, out, allow_cap: bool = False):
        """out <- V_xx phi (same kind as out: torch CUDA tensor or numpy)."""
        ptr, dev = _ptr(out)
        e = ctypes.c_double(0.0)
        rc = lib().sea_apply_vxx(self._h, _p(ptr), dev, ctypes.byref(e))
        if not (allow_cap and rc == 5):
            self._check(rc, "apply_vxx")
        return e.value

    def build_ace(self):
        self._check(lib().sea_build_ace(self._h), "build_ace")

    def build_ace_from(self, W):
        """ACE from a caller-supplied W = V_xx Phi (treated as dense)."""
        ptr, dev = _ptr(W)
        self._check(lib().sea_build_ace_from(self._h, _p(ptr), dev), "build_ace_from")

    def apply_ace(self, psi, out):
        p1, d1 = _ptr(psi)
        p2, d2 = _ptr(out)
        if d1 != d2:
            raise ValueError("psi and out must both be host or both device")
        self._check(lib().sea_apply_ace(self._h, _p(p1), int(psi.shape[0]), _p(p2), d1),
                    "apply_ace")

    def ace_matrices(self):
        n = self.n_orb
        M = np.zeros((n, n))
        L = np.zeros((n, n))
        self._check(lib().sea_get_ace_matrices(self._h, _p(M.ctypes.data), _p(L.ctypes.data), 0),
                    "get_ace_matrices")
        return M, L

    def ace_vectors(self, out):
        ptr, dev = _ptr(out)
        self._check(lib().sea_get_ace_vectors(self._h, _p(ptr), dev), "get_ace_vectors")

    def plan(self) -> dict:
        n = self.n_orb
        np_ = ctypes.c_int(0)
        self._check(lib().sea_get_plan(self._h, None, ctypes.byref(np_), 0, None, None, None,
                                       None, None, None), "get_plan")
        P = np_.value
        box = np.zeros((n, 6), np.int32)
        pairs = np.zeros((P, 2), np.int32)
        lo = np.zeros((P, 3), np.int32)
        ext = np.zeros((P, 3), np.int32)
        S = np.zeros(P)
        it = np.zeros(P, np.int32)
        ep = np.zeros(P)
        c = lambda a: _p(a.ctypes.data)  # noqa: E731
        self._check(lib().sea_get_plan(self._h, c(box), ctypes.byref(np_), P, c(pairs), c(lo),
                                       c(ext), c(S), c(it), c(ep)), "get_plan")
        return dict(box=box, pair=pairs, lo=lo, ext=ext, S=S, iters=it, epair=ep)

    def stats(self) -> dict:
        s = Stats()
        self._check(lib().sea_get_stats(self._h, ctypes.byref(s)), "get_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def close(self):
        if self._h:
            lib().sea_destroy(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


PATCH = 32  # edge of the warm-start patches


def _fptr(a, shape=None):
    """(pointer, on_device) of a float32 numpy array or CUDA tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float32")
        return a.ctypes.data, 0
    if getattr(a, "is_cuda", False):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError("device tensors must be contiguous float32")
        return a.data_ptr(), 1
    raise TypeError("expected a numpy array or a CUDA torch tensor")


class WarmStartNet:
    """The learned warm start (sea_unet_*): a 3-level 3D U-Net on 32^3
    patches (see include/sea.h)."""

    def __init__(self, width=16, seed=0, stream=None):
        self._h = _p()
        self.width = width
        rc = lib().sea_unet_create(width, seed, _p(stream) if stream else None,
                                   ctypes.byref(self._h))
        if rc != SEA_OK:
            raise SeaError(rc, "unet_create")

    def _check(self, rc, what):
        if rc != SEA_OK:
            raise SeaError(rc, f"{what}: {lib().sea_unet_last_error(self._h).decode()}")

    @property
    def handle(self):
        return self._h

    def num_weights(self) -> int:
        return int(lib().sea_unet_num_weights(self._h))

    def get_weights(self) -> np.ndarray:
        w = np.zeros(self.num_weights(), np.float32)
        self._check(lib().sea_unet_weights(self._h, _p(w.ctypes.data), 0), "unet_weights")
        return w

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        if w.size != self.num_weights():
            raise ValueError("weight count mismatch")
        self._check(lib().sea_unet_weights(self._h, _p(w.ctypes.data), 1), "unet_weights")

    def forward(self, x, out):
        p1, d1 = _fptr(x)
        p2, d2 = _fptr(out)
        if d1 != d2:
            raise ValueError("in and out must both be host or both device")
        self._check(lib().sea_unet_forward(self._h, _p(p1), int(x.shape[0]), _p(p2), d1),
                    "unet_forward")

    def loss_grad(self, x, target, want_grad=True):
        p1, d1 = _fptr(x)
        p2, d2 = _fptr(target)
        if d1 != d2:
            raise ValueError("in and target must both be host or both device")
        loss = ctypes.c_double(0.0)
        g = np.zeros(self.num_weights(), np.float32) if want_grad else None
        self._check(lib().sea_unet_loss_grad(self._h, _p(p1), _p(p2), int(x.shape[0]),
                                             ctypes.byref(loss),
                                             _p(g.ctypes.data) if want_grad else None, d1),
                    "unet_loss_grad")
        return loss.value, g

    def collect(self, ctx):
        self._check(lib().sea_unet_collect(self._h, ctx.handle), "unet_collect")
        return int(lib().sea_unet_num_samples(self._h))

    def train(self, steps, batch=8, lr=1e-3, seed=0) -> float:
        loss = ctypes.c_double(0.0)
        self._check(lib().sea_unet_train(self._h, steps, batch, lr, seed, ctypes.byref(loss)),
                    "unet_train")
        return loss.value

    def attach(self, ctx):
        rc = lib().sea_unet_attach(ctx.handle, self._h)
        if rc != SEA_OK:
            raise SeaError(rc, "unet_attach")

    @staticmethod
    def detach(ctx):
        lib().sea_unet_attach(ctx.handle, None)

    def close(self):
        if self._h:
            lib().sea_unet_destroy(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
