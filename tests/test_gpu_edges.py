"""Degenerate and extreme cases of the CUDA path against the FP64 oracle: one
time step (no series, only g), one path, the index set {0}, the largest
dimension (d = 8, table and tree kernels), the largest number of time steps
(N = 256), and the bounded-wait mechanism: a wait that cannot complete is
reported as QR_ETIMEOUT and the context stays usable."""
import numpy as np
import pytest

from paper_2407_21084_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import build, solver

    build.build()
    return solver


def _ref(ora, w, n_iter):
    K = ora.gamma_list(w.gamma_kind, w.d, w.gamma_n)
    p = ora.Problem(d=w.d, N=w.N, T=w.T, k=K, b=w.b, sigma=w.sigma, f_kind=ora.F_CUBIC_MANUF, f_par=w.f_par,
                    g_kind=ora.GT_COS, g_par=w.g_par, M=w.M, seed=w.seed, clamp_L=w.clamp_L)
    a, _ = ora.picard(p, n_iter)
    return a


def _check(solver, ora, w, n_iter=2, kernels=(0, 1), precs=((0, 1e-10), (1, 1e-4))):
    ref = _ref(ora, w, n_iter)
    scale = max(np.abs(ref).max(), 1e-300)
    for kern in kernels:
        for prec, tol in precs:
            with solver.Solver.from_workload(w, precision=prec, path_kernel=kern) as s:
                s.picard_step(n_iter)
                a = s.coefs()
            assert np.abs(a - ref).max() / scale < tol, (kern, prec)


def test_one_time_step(mods, ora):
    _check(mods, ora, W.c1().with_(N=1, M=1500), n_iter=1)


def test_one_path(mods, ora):
    _check(mods, ora, W.c1().with_(N=3, M=1), n_iter=2)


def test_index_set_of_the_constant_only(mods, ora):
    _check(mods, ora, W.c1().with_(gamma_n=0, N=3, M=777), n_iter=2, kernels=(1,))


@pytest.mark.parametrize("n,kernels", [(2, (1,)), (3, (0, 1))])
def test_largest_dimension(mods, ora, n, kernels):
    rng = np.random.default_rng(8)
    w = W.c1().with_(d=8, gamma_kind=W.G_L1_Z, gamma_n=n, s=rng.uniform(-1, 1, size=8), sigma0=0.3, N=3, M=513)
    _check(mods, ora, w, n_iter=2, kernels=kernels)


def test_largest_number_of_time_steps(mods, ora):
    w = W.c1().with_(d=1, gamma_kind=W.G_LINF_Z, gamma_n=3, s=np.array([0.8]), N=256, M=64)
    _check(mods, ora, w, n_iter=1, precs=((0, 1e-10),))


def test_bounded_wait_timeout_is_reported_and_context_survives(mods):
    solver = mods
    from paper_2407_21084_b300 import _lib as L

    w = W.c1().with_(N=4, M=2048)
    with solver.Solver.from_workload(w, precision=0) as s:
        st = s._L.qr_selftest_wait_timeout(s._ctx)
        assert st == L.QR_ETIMEOUT
        assert b"timed out" in s._L.qr_last_error(s._ctx) or b"ran out" in s._L.qr_last_error(s._ctx)
        s.picard_step(2)
        a = s.coefs()
    with solver.Solver.from_workload(w, precision=0) as s2:
        s2.picard_step(2)
        assert np.array_equal(a.view(np.float64), s2.coefs().view(np.float64))
