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

__all__ = ["Lrei", "Batch", "LreiError", "load_library", "QLL", "QLLG", "FP64", "MIXED_C64", "SCHEMES"]

QLL, QLLG = 0, 1
FP64, MIXED_C64, MIXED_BF16X = 0, 1, 2
PRECISIONS = {"fp64": FP64, "mixed": MIXED_C64, "bf16x": MIXED_BF16X}
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


class CtrlStats(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_longlong), ("rejected", ctypes.c_longlong), ("judged", ctypes.c_longlong),
                ("rk4_steps", ctypes.c_longlong), ("h", ctypes.c_double), ("err_judged", ctypes.c_double),
                ("calib", ctypes.c_double)]


NFEAT = 40
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
        "lrei_set_werner": (I, [P, D]),
        "lrei_set_dmi": (I, [P, I, ctypes.POINTER(D)]),
        "lrei_set_eig_sweeps": (I, [P, I]),
        "lrei_batch_create": (I, [I, P, P, ctypes.POINTER(P)]),
        "lrei_batch_step": (I, [P, D, I]),
        "lrei_batch_autotune": (I, [P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "lrei_batch_destroy": (I, [P]),
        "lrei_checkpoint_bytes": (L, [P]),
        "lrei_checkpoint_save": (I, [P, P, L]),
        "lrei_checkpoint_load": (I, [P, P, L]),
        "lrei_truncate_rank": (I, [P, D, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "lrei_two_spin_rdm": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D),
                                  ctypes.POINTER(D), ctypes.POINTER(D)]),
        "lrei_destroy": (I, [P]),
        "lrei_error_string": (ctypes.c_char_p, [I]),
        "lrei_apply_h": (I, [P, P, P, I]),
        "lrei_gram": (I, [P, P, I, P]),
        "lrei_rhs": (I, [P, P, P, ctypes.POINTER(D), I]),
        "lrei_householder": (I, [P, P, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "lrei_kernel_launches": (L, [P]),
        "lrei_last_status": (I, [P]),
        "lrei_debug_counters": (I, [ctypes.POINTER(ctypes.c_ulonglong)]),
        "lrei_mlp_create": (I, [I, I, P, P, ctypes.POINTER(P)]),
        "lrei_mlp_destroy": (I, [P]),
        "lrei_mlp_num_params": (I, [P]),
        "lrei_mlp_get_params": (I, [P, P, I]),
        "lrei_mlp_set_params": (I, [P, P, I]),
        "lrei_mlp_forward": (I, [P, P, I, P]),
        "lrei_mlp_grads": (I, [P, P, P, P, I, P, ctypes.POINTER(ctypes.c_float)]),
        "lrei_mlp_adam": (I, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "lrei_controller_config": (I, [P, I, I, D]),
        "lrei_controller_attach": (I, [P, P]),
        "lrei_controller_stats": (I, [P, ctypes.POINTER(CtrlStats)]),
        "lrei_controller_records": (I, [P, P, I, ctypes.POINTER(I)]),
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
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        self.precision = PRECISIONS[precision]
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

    def set_dmi(self, dz):
        """Dzyaloshinskii-Moriya vectors d_ij = dz[b] e_z, one per bond in the bonds' order (eq. H1)."""
        dz = np.ascontiguousarray(dz, dtype=np.float64)
        self._dz = dz
        _check(self._lib.lrei_set_dmi(self._h, len(dz), dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def checkpoint(self):
        """The state as a bytes object (lrei_checkpoint_save)."""
        nb = int(self._lib.lrei_checkpoint_bytes(self._h))
        buf = ctypes.create_string_buffer(max(nb, 1))
        _check(self._lib.lrei_checkpoint_save(self._h, buf, nb))
        return buf.raw[:nb]

    def restore(self, blob):
        """Continue from a checkpoint taken with the same model and precision (lrei_checkpoint_load)."""
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self._lib.lrei_checkpoint_load(self._h, buf, len(blob)))
        self.r = int(np.frombuffer(blob[:20], dtype=np.int32)[4])   # header: 8-byte tag, version, n, r

    def set_eig_sweeps(self, max_sweeps):
        _check(self._lib.lrei_set_eig_sweeps(self._h, int(max_sweeps)))

    def set_werner(self, p):
        """rho = p I/N + (1 - p) rho_hat: shifted damping for the steps, observables of rho (Sec. 5)."""
        _check(self._lib.lrei_set_werner(self._h, float(p)))

    def two_spin_rdm(self, pairs):
        """R_kl (npairs x 4 x 4 complex), concurrence and negativity for site pairs [(k, l), ...]."""
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        k = np.ascontiguousarray(pairs[:, 0])
        l = np.ascontiguousarray(pairs[:, 1])
        npairs = pairs.shape[0]
        R = np.zeros(32 * npairs)
        conc = np.zeros(npairs)
        neg = np.zeros(npairs)
        pi = ctypes.POINTER(ctypes.c_int)
        pd = ctypes.POINTER(ctypes.c_double)
        _check(self._lib.lrei_two_spin_rdm(self._h, npairs, k.ctypes.data_as(pi), l.ctypes.data_as(pi),
                                           R.ctypes.data_as(pd), conc.ctypes.data_as(pd), neg.ctypes.data_as(pd)),
               self._h)
        Rc = (R[0::2] + 1j * R[1::2]).reshape(npairs, 4, 4).transpose(0, 2, 1)   # column-major -> [q, i, j]
        return Rc, conc, neg

    def truncate_rank(self, tol_r):
        """Drop trailing eigenvalues of total weight <= tol_r; returns (new rank, dropped weight)."""
        k, wgt = ctypes.c_int(), ctypes.c_double()
        _check(self._lib.lrei_truncate_rank(self._h, float(tol_r), ctypes.byref(k), ctypes.byref(wgt)), self._h)
        self.r = k.value
        return k.value, wgt.value

    def observables(self):
        o = Obs()
        _check(self._lib.lrei_observables(self._h, ctypes.byref(o)))
        return o.as_dict()

    def apply_h(self, V, Y):
        assert V.is_contiguous() and Y.is_contiguous()
        _check(self._lib.lrei_apply_h(self._h, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                      V.shape[1]))

    def gram(self, blocks, out=None):
        """P = [B_0..B_{m-1}]^* B_{m-1} as a (m r) x r complex128 device tensor (no host sync)."""
        import torch
        m = len(blocks)
        for b in blocks:
            assert b.is_contiguous() and b.dtype == self.torch_dtype and tuple(b.shape) == (self.N, self.r)
        ptrs = (ctypes.c_void_p * m)(*[b.data_ptr() for b in blocks])
        if out is None:
            out = torch.empty((self.r, m * self.r), dtype=torch.complex128, device="cuda")   # column-major (m r) x r
        _check(self._lib.lrei_gram(self._h, ptrs, m, ctypes.c_void_p(out.data_ptr())), self._h)
        return out.T

    def rhs(self, complement=0):
        import torch
        Z = torch.empty((self.N, self.r), dtype=self.torch_dtype, device="cuda")
        W = torch.empty_like(Z)
        G = np.zeros(2 * self.r * self.r)
        _check(self._lib.lrei_rhs(self._h, ctypes.c_void_p(Z.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                                  G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(complement)), self._h)
        Gc = (G[0::2] + 1j * G[1::2]).reshape(self.r, self.r).T  # column-major -> row-major
        return Z, W, Gc

    def householder(self):
        """Compact WY factors (U, T, D) of the current factor's Householder reflectors."""
        import torch
        U = torch.empty((self.N, self.r), dtype=self.torch_dtype, device="cuda")
        T = np.zeros(2 * self.r * self.r)
        Dd = np.zeros(2 * self.r)
        _check(self._lib.lrei_householder(self._h, ctypes.c_void_p(U.data_ptr()),
                                          T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          Dd.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self._h)
        Tc = (T[0::2] + 1j * T[1::2]).reshape(self.r, self.r).T
        return U, Tc, Dd[0::2] + 1j * Dd[1::2]

    def kernel_launches(self):
        return int(self._lib.lrei_kernel_launches(self._h))

    def controller_config(self, judge_every=8, record=False, h0=0.0):
        _check(self._lib.lrei_controller_config(self._h, int(judge_every), int(bool(record)), float(h0)))

    def controller_attach(self, net):
        self._net = net
        _check(self._lib.lrei_controller_attach(self._h, net._h if net is not None else None))

    def controller_stats(self):
        st = CtrlStats()
        _check(self._lib.lrei_controller_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def controller_records(self):
        n = ctypes.c_int()
        _check(self._lib.lrei_controller_records(self._h, None, 0, ctypes.byref(n)))
        rows = np.zeros((n.value, NFEAT + 4))
        if n.value:
            _check(self._lib.lrei_controller_records(self._h, rows.ctypes.data, n.value, ctypes.byref(n)))
        return rows


class Batch:
    """Many contexts stepped together: one graph launch per RK4 step of the whole batch."""

    def __init__(self, contexts, stream=None):
        self._lib = load_library()
        self._ctx = list(contexts)          # the contexts must outlive the batch
        arr = (ctypes.c_void_p * len(self._ctx))(*[c._h.value for c in self._ctx])
        h = ctypes.c_void_p()
        _check(self._lib.lrei_batch_create(len(self._ctx), arr, _stream_handle(stream), ctypes.byref(h)))
        self._h = h

    def step(self, dt, nsteps=1):
        _check(self._lib.lrei_batch_step(self._h, float(dt), int(nsteps)))

    def autotune(self, dt, steps=2):
        """Pick the SM share per trajectory by timing batch steps; returns (share, ms per batch step)."""
        k, ms = ctypes.c_int(), ctypes.c_double()
        _check(self._lib.lrei_batch_autotune(self._h, float(dt), int(steps), ctypes.byref(k), ctypes.byref(ms)))
        return k.value, ms.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lrei_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The controller network (FP32, hidden width 128) with GPU training kernels."""

    def __init__(self, n_in, n_out, params=None, stream=None):
        self._lib = load_library()
        h = ctypes.c_void_p()
        buf = None
        if params is not None:
            buf = np.ascontiguousarray(params, dtype=np.float32)
        _check(self._lib.lrei_mlp_create(n_in, n_out, buf.ctypes.data if buf is not None else None,
                                         _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.n_in, self.n_out = n_in, n_out
        self.n_params = self._lib.lrei_mlp_num_params(h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lrei_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(self._lib.lrei_mlp_get_params(self._h, out.ctypes.data, self.n_params))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self._lib.lrei_mlp_set_params(self._h, p.ctypes.data, self.n_params))

    def forward(self, X):
        import torch
        X = X.contiguous().float()
        Y = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device="cuda")
        _check(self._lib.lrei_mlp_forward(self._h, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                          ctypes.c_void_p(Y.data_ptr())))
        return Y

    def grads(self, X, T, w=None, want_grad=False):
        import torch
        X, T = X.contiguous().float(), T.contiguous().float()
        wb = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        G = torch.empty(self.n_params, dtype=torch.float32, device="cuda") if want_grad else None
        loss = ctypes.c_float()
        _check(self._lib.lrei_mlp_grads(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                        wb.ctypes.data if wb is not None else None, X.shape[0],
                                        ctypes.c_void_p(G.data_ptr()) if G is not None else None, ctypes.byref(loss)))
        return loss.value, G

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(self._lib.lrei_mlp_adam(self._h, lr, beta1, beta2, eps))


def eig_counters():
    """Cumulative small-eigensolver counters on the current device (lrei_debug_counters):
    dict of FP32 Jacobi calls and sweeps, FP64 Jacobi calls and sweeps."""
    lib = load_library()
    out = (ctypes.c_ulonglong * 4)()
    _check(lib.lrei_debug_counters(out))
    return {"fp32_calls": out[0], "fp32_sweeps": out[1], "fp64_calls": out[2], "fp64_sweeps": out[3]}
