"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/lrei.h declares (no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lrei.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lrei_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2508_21200_gb300 import build
    try:
        return build.ensure_built()
    except (RuntimeError, FileNotFoundError) as e:  # no nvcc in this environment
        pytest.skip(f"cannot build: {e}")


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("lrei_create", "lrei_set_state", "lrei_step", "lrei_observables", "lrei_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    for s in declared_symbols():
        assert re.search(rf"\bT {s}$", out, flags=re.M), s


def test_error_strings_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.lrei_error_string.restype = ctypes.c_char_p
    assert lib.lrei_error_string(0) == b"ok"
    assert b"argument" in lib.lrei_error_string(-1)
    # every status the header declares has its own message
    hdr = open(os.path.join(ROOT, "include", "lrei.h")).read()
    codes = [int(v) for v in re.findall(r"LREI_(?:OK|ERR_\w+) = (-?\d+)", hdr)]
    assert len(codes) >= 12 and 0 in codes
    msgs = [lib.lrei_error_string(c) for c in codes]
    assert len(set(msgs)) == len(codes) and b"unknown error" not in msgs
    assert lib.lrei_error_string(-99) == b"unknown error"


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    h = ctypes.c_void_p()
    B = (ctypes.c_double * 3)(0.0, 0.0, 0.5)
    assert lib.lrei_create(0, None, B, ctypes.c_double(0.1), 0, 0, 4, None, ctypes.byref(h)) == -1   # n < 1
    assert lib.lrei_create(8, None, B, ctypes.c_double(-1.0), 0, 0, 4, None, ctypes.byref(h)) == -1  # kappa < 0
    assert lib.lrei_create(8, None, B, ctypes.c_double(0.1), 0, 0, 64, None, ctypes.byref(h)) == -1  # r_max > 32
    Bn = (ctypes.c_double * 3)(0.3, float("nan"), 0.5)
    assert lib.lrei_create(8, None, Bn, ctypes.c_double(0.1), 0, 0, 4, None, ctypes.byref(h)) == -3  # non-finite field


def test_nonfinite_model_gives_the_same_code_from_both_entry_points(lib_path):
    # lrei_create and lrei_observables_noalloc share one validation of n, the bonds and the field
    lib = ctypes.CDLL(lib_path)

    class Bonds(ctypes.Structure):
        _fields_ = [("nbonds", ctypes.c_int), ("site_i", ctypes.POINTER(ctypes.c_int)),
                    ("site_j", ctypes.POINTER(ctypes.c_int)), ("jxy", ctypes.POINTER(ctypes.c_double)),
                    ("jz", ctypes.POINTER(ctypes.c_double))]
    si, sj = (ctypes.c_int * 1)(0), (ctypes.c_int * 1)(1)
    lam = (ctypes.c_double * 1)(1.0)
    out = (ctypes.c_char * 4096)()
    h = ctypes.c_void_p()
    lib.lrei_create.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.lrei_observables_noalloc.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]
    cases = [((1.0, float("nan")), (0.0, 0.0, 0.5), -3),   # non-finite jz
             ((float("inf"), 1.0), (0.0, 0.0, 0.5), -3),   # non-finite jxy
             ((1.0, 1.0), (0.0, 0.0, float("nan")), -3)]   # non-finite field
    for (jxy, jz), B, code in cases:
        b = Bonds(1, si, sj, (ctypes.c_double * 1)(jxy), (ctypes.c_double * 1)(jz))
        Bv = (ctypes.c_double * 3)(*B)
        a = lib.lrei_create(4, ctypes.byref(b), Bv, 0.1, 0, 0, 1, None, ctypes.byref(h))
        # a dummy non-NULL device pointer: the call must fail in its argument checks first
        c = lib.lrei_observables_noalloc(4, ctypes.byref(b), Bv, ctypes.c_void_p(256), 1, 0, lam, None, out)
        assert a == c == code, (jxy, jz, B, a, c)
