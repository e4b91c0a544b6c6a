"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
exports every entry point include/qr.h declares, validates arguments on the
host before touching a GPU, and the product path never reaches the oracle."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_21084_b300 import _lib, build

    build.build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "qr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qr_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    from paper_2407_21084_b300 import _lib

    assert _declared() == sorted(_lib.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_checked_build_exports_the_same_symbols():
    import ctypes as C

    from paper_2407_21084_b300 import build

    if not os.path.exists(build.LIB_CHECKED):
        pytest.skip("libqrmc_checked.so not built")
    lc = C.CDLL(build.LIB_CHECKED)
    for name in _declared():
        assert hasattr(lc, name), name


def test_sm103a_code_object(lib):
    from paper_2407_21084_b300 import build

    assert any("compute_103a" in a for a in build.ARCH)
    data = open(build.LIB, "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data


def _init(lib, d=2, N=4, T=1.0, gamma=(1, 2), M=64, prec=0, fkind=0, gkind=0, nu=(0, 3.0), lattice=0, kern=0):
    from paper_2407_21084_b300 import _lib as L

    b = np.zeros(max(d, 1))
    sig = np.eye(max(d, 1)).ravel()
    par = np.ones(16)
    ctx = C.c_void_p()
    st = lib.qr_init(C.byref(ctx), d, N, T, C.byref(L.QrNu(*nu)), C.byref(L.QrGamma(*gamma)),
                     b.ctypes.data_as(C.POINTER(C.c_double)), sig.ctypes.data_as(C.POINTER(C.c_double)),
                     C.byref(L.QrFn(fkind, par.ctypes.data_as(C.POINTER(C.c_double)), 16)),
                     C.byref(L.QrFn(gkind, par.ctypes.data_as(C.POINTER(C.c_double)), 16)),
                     C.byref(L.QrOpts(M, 1, prec, 0.0, None, 1 if lattice else 0, lattice, 0, kern)))
    msg = lib.qr_last_error(ctx).decode() if ctx else ""
    lib.qr_destroy(ctx)
    return st, msg


@pytest.mark.parametrize("kw,frag", [
    (dict(d=0), "d must"), (dict(d=13), "d must"), (dict(d=9), "Z^d need d <= 8"),
    (dict(d=9, gamma=(5, 1), kern=1), "unfolded cosine route needs d <= 8"), (dict(N=0), "N must"), (dict(N=257), "N must"),
    (dict(T=-1.0), "T must"), (dict(M=0), "M must"), (dict(prec=7), "precision"),
    (dict(gamma=(6, 2)), "index set"), (dict(gamma=(5, 0)), "index set"), (dict(d=5, gamma=(2, 128)), "|k_l| <= 127"),
    (dict(d=1, gamma=(0, 40000)), "|k_l| <= 32767"),
    (dict(d=1, gamma=(3, 120), kern=1), "unfolded set"), (dict(d=1, gamma=(3, 70000)), "direct cosine kernels"),
    (dict(kern=2), "needs a cosine index set"), (dict(kern=5), "unknown path kernel"), (dict(nu=(0, -1.0)), "mu"),
    (dict(fkind=9), "driver"), (dict(gkind=9), "terminal"), (dict(lattice=3, M=10), "lattice"),
])
def test_host_validation_rejects_before_any_device_work(lib, kw, frag):
    st, msg = _init(lib, **kw)
    assert st in (1, 6), (st, msg)
    assert frag in msg


def test_fault_injection_validates_without_a_device(lib):
    import ctypes as C

    from paper_2407_21084_b300 import _lib as L

    assert lib.qr_inject_fault(None, L.QR_FAULT_ALLOC) == L.QR_EINVAL
    # a context kept for its message by a refused qr_init still takes a fault kind
    st, ctx = _init_keep(lib, d=0)
    try:
        assert st == L.QR_EINVAL and ctx
        assert lib.qr_inject_fault(ctx, 9) == L.QR_EINVAL
        assert lib.qr_inject_fault(ctx, L.QR_FAULT_NAN) == L.QR_OK
        assert lib.qr_inject_fault(ctx, L.QR_FAULT_NONE) == L.QR_OK
    finally:
        lib.qr_destroy(ctx)


def _init_keep(lib, d):
    import ctypes as C

    from paper_2407_21084_b300 import _lib as L

    b = np.zeros(1)
    sig = np.eye(1).ravel()
    par = np.ones(4)
    ctx = C.c_void_p()
    st = lib.qr_init(C.byref(ctx), d, 4, 1.0, C.byref(L.QrNu(0, 3.0)), C.byref(L.QrGamma(1, 2)),
                     b.ctypes.data_as(C.POINTER(C.c_double)), sig.ctypes.data_as(C.POINTER(C.c_double)),
                     C.byref(L.QrFn(0, par.ctypes.data_as(C.POINTER(C.c_double)), 4)),
                     C.byref(L.QrFn(0, par.ctypes.data_as(C.POINTER(C.c_double)), 4)),
                     C.byref(L.QrOpts(64, 1, 0, 0.0, None, 0, 0, 0, 0)))
    return st, ctx


def test_status_strings(lib):
    assert lib.qr_status_string(0) == b"ok"
    assert lib.qr_status_string(4) == b"device wait timed out"


def test_product_never_imports_the_oracle():
    pat = re.compile(r"(^\s*(import|from)\s+oracle\b)|liboracle|qr_oracle|ora_[a-z]", re.M)
    pkg = os.path.join(ROOT, "paper_2407_21084_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                assert not pat.search(open(os.path.join(dirpath, f)).read()), f
