"""GB300-native low-rank eigenmode integration (LREI) for the q-LL / q-LLG equations.

Thin Python binding of the C ABI declared in include/lrei.h.  It only
marshals arguments: every step of the computation runs in the CUDA kernels
of liblrei.so.  PyTorch supplies device memory and the CUDA stream.  There
is no CPU fallback: if the compiled library is missing, import of the
binding raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, ensure_built

__all__ = ["Lrei", "LreiError", "load_library", "QLL", "QLLG", "FP64", "MIXED_C64", "SCHEMES"]

QLL, QLLG = 0, 1
FP64, MIXED_C64 = 0, 1
C128, C64 = 0, 1
SCHEMES = {"rk1": 0, "rk2": 1, "rk3": 2, "rk4": 3, "ab2": 4, "ab3": 5, "ab4": 6}


class LreiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lrei error {code}: {msg}")
        self.code = code


class _Bonds(ctypes.Structure):
    _fields_ = [("nbonds", ctypes.c_int),
                ("site_i", ctypes.POINTER(ctypes.c_int)), ("site_j", ctypes.POINTER(ctypes.c_int)),
                ("jxy", ctypes.POINTER(ctypes.c_double)), ("jz", ctypes.POINTER(ctypes.c_double))]


class Obs(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("energy", ctypes.c_double), ("mx", ctypes.c_double),
                ("my", ctypes.c_double), ("mz", ctypes.c_double), ("purity", ctypes.c_double),
                ("trace", ctypes.c_double), ("orth_err", ctypes.c_double), ("herm_err", ctypes.c_double),
                ("comm_norm", ctypes.c_double), ("r", ctypes.c_int),
                ("ritz", ctypes.c_double * 64), ("lambda0", ctypes.c_double * 64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("ritz", "lambda0")}
        d["ritz"] = np.array(self.ritz[: self.r])
        d["lambda0"] = np.array(self.lambda0[: self.r])
        return d


_lib = None


def load_library(path: str | None = None):
    """Load liblrei.so (building it first when the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = ensure_built() if os.environ.get("LREI_NO_BUILD") is None else LIB
    if not os.path.exists(path):
        raise OSError(f"liblrei.so not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "lrei_create": (I, [I, ctypes.POINTER(_Bonds), ctypes.POINTER(D), D, I, I, I, P, ctypes.POINTER(P)]),
        "lrei_set_state": (I, [P, P, I, I, I, ctypes.POINTER(D)]),
        "lrei_get_state": (I, [P, P, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "lrei_step": (I, [P, D, I, I]),
        "lrei_step_adaptive": (I, [P, D, D, I]),
        "lrei_observables": (I, [P, ctypes.POINTER(Obs)]),
        "lrei_destroy": (I, [P]),
        "lrei_error_string": (ctypes.c_char_p, [I]),
        "lrei_apply_h": (I, [P, P, P, I]),
        "lrei_rhs": (I, [P, P, P, ctypes.POINTER(D), I]),
        "lrei_kernel_launches": (L, [P]),
        "lrei_last_status": (I, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code, h=None):
    if code != 0:
        extra = f" (status bits {_lib.lrei_last_status(h)})" if h is not None else ""
        raise LreiError(code, _lib.lrei_error_string(code).decode() + extra)


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


class Lrei:
    """One LREI context (owns its device memory).  Methods mirror include/lrei.h."""

    def __init__(self, n, bonds, B=(0.0, 0.0, 0.0), kappa=0.1, model="qll", precision="fp64", r_max=16,
                 stream=None):
        lib = load_library()
        self._lib = lib
        self.n, self.N, self.r_max = n, 1 << n, r_max
        self.precision = FP64 if precision == "fp64" else MIXED_C64
        self._arrays = (np.ascontiguousarray(bonds.site_i, dtype=np.int32),
                        np.ascontiguousarray(bonds.site_j, dtype=np.int32),
                        np.ascontiguousarray(bonds.jxy, dtype=np.float64),
                        np.ascontiguousarray(bonds.jz, dtype=np.float64))
        si, sj, jxy, jz = self._arrays
        b = _Bonds(len(si), si.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                   sj.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                   jxy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                   jz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        Bv = (ctypes.c_double * 3)(*[float(x) for x in B])
        m = QLLG if model == "qllg" else QLL
        h = ctypes.c_void_p()
        self._stream = stream
        _check(lib.lrei_create(n, ctypes.byref(b), Bv, float(kappa), m, self.precision, r_max,
                               _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.r = None

    @property
    def torch_dtype(self):
        import torch
        return torch.complex128 if self.precision == FP64 else torch.complex64

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lrei_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, V, lam):
        """V: torch complex128/complex64 CUDA tensor (N x r, row stride >= r); lam: r weights."""
        import torch
        assert V.is_cuda and V.dim() == 2
        if V.shape[1] > 1 and V.stride(1) != 1:
            V = V.contiguous()
        ld = max(V.stride(0), V.shape[1])
        dtype = C128 if V.dtype == torch.complex128 else C64
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        self.r = V.shape[1]
        _check(self._lib.lrei_set_state(self._h, ctypes.c_void_p(V.data_ptr()), V.shape[1], ld, dtype,
                                        lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self._h)

    def get_state(self):
        import torch
        V = torch.empty((self.N, self.r), dtype=self.torch_dtype, device="cuda")
        lam = np.zeros(self.r)
        t = ctypes.c_double()
        _check(self._lib.lrei_get_state(self._h, ctypes.c_void_p(V.data_ptr()),
                                        lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(t)))
        return V, lam, t.value

    def step(self, dt, scheme="rk4", nsteps=1):
        _check(self._lib.lrei_step(self._h, float(dt), SCHEMES[scheme], int(nsteps)), self._h)

    def step_adaptive(self, t_end, tol, controller=0):
        _check(self._lib.lrei_step_adaptive(self._h, float(t_end), float(tol), int(controller)))

    def observables(self):
        o = Obs()
        _check(self._lib.lrei_observables(self._h, ctypes.byref(o)))
        return o.as_dict()

    def apply_h(self, V, Y):
        assert V.is_contiguous() and Y.is_contiguous()
        _check(self._lib.lrei_apply_h(self._h, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                      V.shape[1]))

    def rhs(self, complement=0):
        import torch
        Z = torch.empty((self.N, self.r), dtype=self.torch_dtype, device="cuda")
        W = torch.empty_like(Z)
        G = np.zeros(2 * self.r * self.r)
        _check(self._lib.lrei_rhs(self._h, ctypes.c_void_p(Z.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                                  G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(complement)))
        Gc = (G[0::2] + 1j * G[1::2]).reshape(self.r, self.r).T  # column-major -> row-major
        return Z, W, Gc

    def kernel_launches(self):
        return int(self._lib.lrei_kernel_launches(self._h))
