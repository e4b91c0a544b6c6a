"""FP64 CPU oracle of the QRMC Picard iteration (arXiv 2407.21084).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
(``paper_2407_21084_b300``) never imports it, and this package imports nothing
from the product path: the two share no code.

The arithmetic lives in ``qr_oracle.c`` (plain C, double precision, OpenMP
over path chunks); this module only compiles it and marshals numpy arrays.
See ``qr_oracle.h`` for the per-function citations and pins.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qr_oracle.c")
_HDR = os.path.join(_HERE, "qr_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

# enums of qr_oracle.h
G_LINF_Z, G_L1_Z, G_HYP_Z, G_FULL_N, G_TOTAL_N, G_HYP_N = range(6)
TAG_START, TAG_INCR, TAG_TEST, TAG_PARAM = range(4)
NU_LOMAX, NU_STUDENT2, NU_CAUCHY = range(3)
F_ZERO, F_LINEAR, F_CUBIC_MANUF, F_PAPER_MIN = range(4)
GT_COS, GT_TRIGPOLY, GT_PAPER_SIN = range(3)
BASIS_FOURIER, BASIS_COS = range(2)


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (plain gcc, no -ffast-math)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("d", C.c_int),
        ("N", C.c_int),
        ("T", C.c_double),
        ("nu_kind", C.c_int),
        ("mu", C.c_double),
        ("nG", C.c_int),
        ("k", C.POINTER(C.c_int)),
        ("kmax", C.c_int),
        ("b", C.POINTER(C.c_double)),
        ("sigma", C.POINTER(C.c_double)),
        ("f_kind", C.c_int),
        ("f_par", C.POINTER(C.c_double)),
        ("g_kind", C.c_int),
        ("g_par", C.POINTER(C.c_double)),
        ("M", C.c_longlong),
        ("seed", C.c_uint64),
        ("instance", C.c_int),
        ("clamp_L", C.c_double),
        ("lattice_n", C.c_int),
        ("basis", C.c_int),
        ("q_damp", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        dp = C.POINTER(C.c_double)
        L.ora_gamma_count.restype = C.c_longlong
        L.ora_gamma_count.argtypes = [C.c_int, C.c_int, C.c_int]
        L.ora_gamma_list.restype = C.c_longlong
        L.ora_gamma_list.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_longlong]
        L.ora_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.ora_u01.restype = C.c_double
        L.ora_u01.argtypes = [C.c_uint32, C.c_uint32]
        for nm in ("ora_start_uniforms", "ora_test_uniforms"):
            getattr(L, nm).argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_uint32, C.c_int, dp]
        L.ora_normals.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_uint32, C.c_int, C.c_int, dp]
        for nm in ("ora_nu_pdf", "ora_nu_cdf", "ora_nu_icdf"):
            getattr(L, nm).restype = C.c_double
            getattr(L, nm).argtypes = [C.c_int, C.c_double, C.c_double]
        pp = C.POINTER(_Problem)
        L.ora_series.restype = C.c_double
        L.ora_series.argtypes = [pp, dp, dp]
        L.ora_g.restype = C.c_double
        L.ora_g.argtypes = [pp, dp]
        L.ora_f.restype = C.c_double
        L.ora_f.argtypes = [pp, C.c_double, dp, C.c_double]
        L.ora_response.restype = C.c_double
        L.ora_response.argtypes = [pp, dp, C.c_int, C.c_longlong, dp, C.POINTER(C.c_longlong)]
        L.ora_picard_iter.restype = C.c_int
        L.ora_picard_iter.argtypes = [
            pp, dp, dp, C.c_int, C.c_int, C.c_longlong, C.c_longlong, C.c_int,
            C.POINTER(C.c_longlong),
        ]
        L.ora_backward_sweep.restype = C.c_int
        L.ora_backward_sweep.argtypes = [
            pp, dp, C.c_longlong, C.c_longlong, C.c_int, C.POINTER(C.c_longlong),
        ]
        L.ora_responses.restype = C.c_int
        L.ora_responses.argtypes = [pp, dp, C.c_int, C.c_longlong, C.c_longlong, dp, C.c_int]
        L.ora_max_threads.restype = C.c_int
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ------------------------------------------------------------------ helpers

def gamma_count(kind: int, d: int, n: int) -> int:
    return int(lib().ora_gamma_count(kind, d, n))


def gamma_list(kind: int, d: int, n: int) -> np.ndarray:
    cnt = gamma_count(kind, d, n)
    if cnt < 0:
        raise ValueError("bad Gamma arguments")
    out = np.zeros((cnt, d), dtype=np.int32)
    got = lib().ora_gamma_list(kind, d, n, out.ctypes.data_as(C.POINTER(C.c_int)), cnt)
    assert got == cnt
    return out


def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def u01(a: int, b: int) -> float:
    return float(lib().ora_u01(a, b))


def start_uniforms(seed, instance, i, m, d) -> np.ndarray:
    u = np.zeros(d)
    lib().ora_start_uniforms(seed, instance, i, m, d, _dp(u))
    return u


def test_uniforms(seed, instance, i, p, d) -> np.ndarray:
    u = np.zeros(d)
    lib().ora_test_uniforms(seed, instance, i, p, d, _dp(u))
    return u


def normals(seed, instance, i, m, j, d) -> np.ndarray:
    z = np.zeros(d)
    lib().ora_normals(seed, instance, i, m, j, d, _dp(z))
    return z


def nu_pdf(kind, mu, x):
    return float(lib().ora_nu_pdf(kind, mu, x))


def nu_cdf(kind, mu, x):
    return float(lib().ora_nu_cdf(kind, mu, x))


def nu_icdf(kind, mu, u):
    return float(lib().ora_nu_icdf(kind, mu, u))


@dataclass
class Problem:
    """Plain description of one QRMC problem (mirrors ``ora_problem``)."""

    d: int
    N: int
    T: float
    k: np.ndarray  # |Gamma| x d int32, canonical order
    b: np.ndarray
    sigma: np.ndarray  # d x d
    f_kind: int
    f_par: np.ndarray
    g_kind: int
    g_par: np.ndarray
    M: int
    seed: int
    nu_kind: int = NU_LOMAX
    mu: float = 3.0
    instance: int = 0
    clamp_L: float = 0.0
    lattice_n: int = 0
    basis: int = 0  # BASIS_FOURIER (k in Z^d) or BASIS_COS (k in N^d, real coefficients)
    q_damp: float = 0.0  # damping exponent q of eq. (yqi)
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _Problem:
        k = np.ascontiguousarray(self.k, dtype=np.int32)
        b = np.ascontiguousarray(self.b, dtype=np.float64)
        s = np.ascontiguousarray(self.sigma, dtype=np.float64).reshape(-1)
        fp = np.ascontiguousarray(np.atleast_1d(self.f_par), dtype=np.float64)
        gp = np.ascontiguousarray(np.atleast_1d(self.g_par), dtype=np.float64)
        if k.ndim != 2 or k.shape[1] != self.d or b.size != self.d or s.size != self.d * self.d:
            raise ValueError("k needs d columns, b d and sigma d*d entries (d = %d)" % self.d)
        self._keep = [k, b, s, fp, gp]
        return _Problem(
            self.d, self.N, self.T, self.nu_kind, self.mu, k.shape[0],
            k.ctypes.data_as(C.POINTER(C.c_int)), int(np.abs(k).max()) if k.size else 0,
            _dp(b), _dp(s), self.f_kind, _dp(fp), self.g_kind, _dp(gp), self.M,
            self.seed, self.instance, self.clamp_L, self.lattice_n, self.basis, self.q_damp,
        )

    @property
    def nG(self) -> int:
        return int(self.k.shape[0])

    def zeros(self) -> np.ndarray:
        """alpha array (N, nG) complex128 of zeros (y == 0 start)."""
        return np.zeros((self.N, self.nG), dtype=np.complex128)


def _as_inter(alpha: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(alpha, dtype=np.complex128).view(np.float64)


def picard_iter(p: Problem, alpha_in: np.ndarray, i_range=None, m_range=None,
                nthreads: int = 0, alpha_out: np.ndarray | None = None):
    """One Jacobi-Picard iteration. Returns (alpha_out (N,nG) complex, clamp_hits)."""
    pc = p.c()
    ai = _as_inter(alpha_in)
    ao = np.array(alpha_in if alpha_out is None else alpha_out, dtype=np.complex128, copy=True)
    aov = ao.view(np.float64)
    i_lo, i_hi = i_range if i_range else (0, p.N)
    m_lo, m_hi = m_range if m_range else (0, p.M)
    hits = C.c_longlong(0)
    rc = lib().ora_picard_iter(C.byref(pc), _dp(ai), _dp(aov), i_lo, i_hi, m_lo, m_hi,
                               nthreads, C.byref(hits))
    if rc:
        raise RuntimeError("ora_picard_iter failed: %d" % rc)
    return ao, int(hits.value)


def picard(p: Problem, n_iter: int, alpha0: np.ndarray | None = None, nthreads: int = 0,
           m_range=None):
    a = p.zeros() if alpha0 is None else np.array(alpha0, dtype=np.complex128)
    hits = 0
    for _ in range(n_iter):
        a, h = picard_iter(p, a, m_range=m_range, nthreads=nthreads)
        hits += h
    return a, hits


def backward_sweep(p: Problem, m_range=None, nthreads: int = 0):
    pc = p.c()
    a = p.zeros()
    av = a.view(np.float64)
    m_lo, m_hi = m_range if m_range else (0, p.M)
    hits = C.c_longlong(0)
    rc = lib().ora_backward_sweep(C.byref(pc), _dp(av), m_lo, m_hi, nthreads, C.byref(hits))
    if rc:
        raise RuntimeError("ora_backward_sweep failed: %d" % rc)
    return a, int(hits.value)


def responses(p: Problem, alpha_in: np.ndarray, i: int, m_range, nthreads: int = 0):
    pc = p.c()
    ai = _as_inter(alpha_in)
    m_lo, m_hi = m_range
    S = np.zeros(m_hi - m_lo)
    rc = lib().ora_responses(C.byref(pc), _dp(ai), i, m_lo, m_hi, _dp(S), nthreads)
    if rc:
        raise RuntimeError("ora_responses failed")
    return S


def series(p: Problem, alpha_row: np.ndarray, x: np.ndarray) -> np.ndarray:
    """ybar(x) for each row of x (n x d) with one coefficient row (nG complex)."""
    pc = p.c()
    a = _as_inter(alpha_row)
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    return np.array([lib().ora_series(C.byref(pc), _dp(a), _dp(row)) for row in x])


def g(p: Problem, x: np.ndarray) -> np.ndarray:
    pc = p.c()
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    return np.array([lib().ora_g(C.byref(pc), _dp(row)) for row in x])


def f(p: Problem, t: float, x: np.ndarray, y: float) -> float:
    pc = p.c()
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().ora_f(C.byref(pc), t, _dp(x), y))


def test_points(p: Problem, i: int, n: int) -> np.ndarray:
    """n nu-distributed test points (TEST tag) at time index i, shape (n, d)."""
    out = np.zeros((n, p.d))
    for q in range(n):
        u = test_uniforms(p.seed, p.instance, i, q, p.d)
        out[q] = [nu_icdf(p.nu_kind, p.mu, v) for v in u]
    return out


def max_threads() -> int:
    return int(lib().ora_max_threads())
