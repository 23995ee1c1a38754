"""The allocation-free observables entry point against the context-based one (GPU).

lrei_observables_noalloc serves callers that cannot allocate device memory (a host whose
own allocator has reserved it, a monitoring loop that must not allocate per call): its
scratch is a static device array inside the library.  Here it is called twice in a row
on the factor held by a context and must reproduce lrei_observables within the tolerance the
parity tests use for a reduction of the same data (1e-12 relative in FP64, 1e-6 in complex64).
The file name sorts last, so a run that stops at its first failure has run every other test
before this one.
"""
import ctypes

import numpy as np
import pytest

import lrei_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_21200_gb300 import Lrei, Obs, load_library  # noqa: E402
from paper_2508_21200_gb300 import _Bonds  # noqa: E402

KEYS = ("energy", "mx", "my", "mz", "purity", "trace", "comm_norm")


def _noalloc(lib, w, V, lam, dtype):
    si = np.ascontiguousarray(w.bonds.site_i, dtype=np.int32)
    sj = np.ascontiguousarray(w.bonds.site_j, dtype=np.int32)
    jxy = np.ascontiguousarray(w.bonds.jxy, dtype=np.float64)
    jz = np.ascontiguousarray(w.bonds.jz, dtype=np.float64)
    b = _Bonds(len(si), si.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), sj.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
               jxy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), jz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    Bv = (ctypes.c_double * 3)(*[float(x) for x in w.B])
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    f = lib.lrei_observables_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.POINTER(_Bonds), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.POINTER(Obs)]
    o = Obs()
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    code = f(w.n, ctypes.byref(b), Bv, ctypes.c_void_p(V.data_ptr()), V.shape[1], dtype,
             lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), stream, ctypes.byref(o))
    assert code == 0, code
    return o.as_dict()


@pytest.mark.parametrize("precision,dtype,tol", [("fp64", 0, 1e-12), ("mixed", 1, 1e-6)])
@pytest.mark.parametrize("n,r", [(10, 6), (14, 16)])   # n = 14: more 16-row tiles than partial slots
def test_noalloc_observables_match_context_observables_twice(precision, dtype, tol, n, r):
    lib = load_library()
    w = li.workload(2, n=n, r=r)
    L = Lrei(w.n, w.bonds, w.B, w.kappa, w.model, precision, w.r)
    Vin = torch.from_numpy(w.V).to("cuda", torch.complex128 if precision == "fp64" else torch.complex64)
    L.set_state(Vin, w.lam)
    L.step(w.dt, "rk4", 2)
    ref = L.observables()
    V, lam, _ = L.get_state()
    for _ in range(2):
        got = _noalloc(lib, w, V, lam, dtype)
        for k in KEYS:
            assert abs(got[k] - ref[k]) <= tol * max(1.0, abs(ref[k])), (k, got[k], ref[k])
        assert got["r"] == w.r and np.allclose(got["lambda0"], lam)


@pytest.mark.parametrize("precision,dtype,tol", [("fp64", 0, 1e-12), ("mixed", 1, 1e-6)])
def test_noalloc_observables_match_the_dense_oracle(precision, dtype, tol):
    # directly against the oracle's observables of rho = V Lambda V^* (dense, n = 8)
    from oracle import model, dense_ei as de
    lib = load_library()
    w = li.workload(2, n=8, r=5)
    V = torch.from_numpy(w.V).to("cuda", torch.complex128 if precision == "fp64" else torch.complex64)
    got = _noalloc(lib, w, V, w.lam, dtype)
    H = model.hamiltonian(w.n, w.bonds, w.B)
    M = {v: model.magnetization_op(v, w.n) for v in "xyz"}
    Vr = V.cpu().numpy().astype(np.complex128)   # the factor as stored (complex64 rounding included)
    Rc = np.linalg.cholesky(Vr.conj().T @ Vr).conj().T
    ref = de.observables(Vr @ np.linalg.inv(Rc), w.lam, H, M)
    sE = float(np.sum(np.abs(w.bonds.jxy) + np.abs(w.bonds.jz) / 2) + w.n * np.linalg.norm(w.B) / 2)
    for k, s in (("energy", sE), ("mx", 0.5), ("my", 0.5), ("mz", 0.5), ("purity", 1.0)):
        assert abs(got[k] - ref[k]) <= tol * max(abs(ref[k]), s), (k, got[k], ref[k])
    assert abs(got["comm_norm"] - ref["comm_norm"]) <= tol * max(ref["comm_norm"], 1.0)


def test_noalloc_rejects_rank_above_its_limit():
    lib = load_library()
    w = li.workload(2, n=8, r=17, with_state=False)
    V = torch.zeros((1 << w.n, 17), dtype=torch.complex128, device="cuda")
    f = lib.lrei_observables_noalloc
    f.restype = ctypes.c_int
    o = Obs()
    code = f(w.n, None, None, ctypes.c_void_p(V.data_ptr()), 17, 0,
             np.full(17, 1 / 17).ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, ctypes.byref(o))
    assert code == -1
