"""The direct cosine kernels (path_kernel 2: real per-lane tables of
C_a(u) = sqrt(2) cos(a pi u), runs of Gamma over the last coordinate, groups
of 4 packed positions) against the FP64 oracle on the sets the unfolded
route cannot take (the paper's d = 5 and d = 7 hyperbolic-cross sets of
Sec. 5), at the edges of the group layout (d = 1 with a single entry, d = 8,
prefix bytes of both words), above d = 8 (the paper's d = 9 and d = 11
hyperbolic-cross sets with their damping exponents, d = 12), through qr_eval, against the unfolded route,
and at the full size of the paper's d = 5, Delta = 0.2, DEG = 16 row
(M = 2 10^6) on sampled responses."""
import numpy as np
import pytest

from paper_2407_21084_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import _lib, build, solver

    build.build()
    return solver, _lib


def _oracle_problem(ora, p: W.Sec5Problem, M=None):
    K = ora.gamma_list(p.gamma_kind, p.d, p.gamma_n)
    op = ora.Problem(d=p.d, N=p.N, T=p.T, k=K, b=p.b, sigma=p.sigma, f_kind=ora.F_PAPER_MIN, f_par=p.f_par,
                     g_kind=ora.GT_PAPER_SIN, g_par=p.g_par, M=p.M if M is None else M, seed=p.seed,
                     nu_kind=p.nu_kind, mu=p.mu, basis=ora.BASIS_COS)
    op.q_damp = p.q
    return op


@pytest.mark.parametrize("d,kind,n,N,M,q,precs,nu", [
    (9, W.G_HYP_N, 5, 2, 110, 17.6, (0,), W.NU_CAUCHY),    # the paper's d = 9 row with mixed-derivative damping
    (11, W.G_HYP_N, 2, 2, 130, 21.6, (0,), W.NU_CAUCHY),   # and its d = 11 row (Cauchy nu, FP64)
    (3, W.G_HYP_N, 6, 3, 500, 5.1, (0, 1), W.NU_CAUCHY),
])
def test_direct_picard_cauchy_matches_oracle(mods, ora, d, kind, n, N, M, q, precs, nu):
    test_direct_picard_matches_oracle(mods, ora, d, kind, n, N, M, q, precs, nu)


@pytest.mark.parametrize("d,kind,n,N,M,q,precs", [
    (1, W.G_FULL_N, 0, 1, 1, 0.0, (0, 1)),       # Gamma = {0}: one group, M = 1, N = 1
    (1, W.G_FULL_N, 9, 3, 257, 2.1, (0, 1)),     # one run of 10 entries (3 groups, the last ragged)
    (4, W.G_TOTAL_N, 6, 3, 611, 0.0, (0, 1)),    # prefixes in the first word only
    (5, W.G_HYP_N, 16, 3, 700, 5.1, (0, 1)),     # the paper's d = 5 set Gamma_H(16), 3042 entries
    (6, W.G_HYP_N, 9, 2, 333, 0.0, (0, 1)),      # prefix bytes in both words
    (8, W.G_TOTAL_N, 3, 3, 400, 5.1, (0, 1)),    # d = 8: seven prefix coordinates
    (7, W.G_HYP_N, 36, 2, 300, 5.1, (0, 1)),     # the paper's d = 7 set, 94460 entries: rows from global memory
    (9, W.G_HYP_N, 2, 3, 300, 17.6, (0, 1)),     # d = 9: a prefix coordinate in the third word
    (9, W.G_HYP_N, 5, 2, 120, 17.6, (0,)),       # the paper's d = 9 set Gamma_H(5), 14336 entries, its q
    (10, W.G_TOTAL_N, 3, 2, 257, 0.0, (0, 1)),
    (11, W.G_HYP_N, 2, 2, 150, 21.6, (0,)),      # the paper's d = 11 set Gamma_H(2), 13312 entries, its q
    (11, W.G_HYP_N, 1, 3, 200, 2.1, (0, 1)),     # {0,1}^11
    (12, W.G_TOTAL_N, 2, 3, 333, 5.1, (0, 1)),   # d = 12, the largest: eleven prefix coordinates
])
def test_direct_picard_matches_oracle(mods, ora, d, kind, n, N, M, q, precs, nu=W.NU_STUDENT2):
    solver, L = mods
    p = W.Sec5Problem(d=d, N=N, gamma_kind=kind, gamma_n=n, M=M, seed=21, q=q, nu_kind=nu)
    ref, _ = ora.picard(_oracle_problem(ora, p), 2)
    ref = ref.real
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        if prec not in precs:
            continue
        with solver.Solver.from_sec5(p, precision=prec, path_kernel=2) as s:
            s.picard_step(2)
            k, a = s.cosine_coefs()
        assert np.array_equal(k, ora.gamma_list(kind, d, n))
        err = np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300)
        assert err < tol, (prec, err)


@pytest.mark.parametrize("d,kind,n", [(5, W.G_HYP_N, 16), (3, W.G_TOTAL_N, 22), (5, W.G_TOTAL_N, 20)])
def test_auto_route_takes_the_paper_sets(mods, d, kind, n):
    """path_kernel 0 runs the direct kernels where no compile-time tree covers
    the unfolded set, including the paper's d = 5 total-degree set Gamma_T(20)
    (53130 entries, 2.2 10^6 unfolded), which the unfolded route refuses."""
    solver, L = mods
    p = W.Sec5Problem(d=d, N=2, gamma_kind=kind, gamma_n=n, M=256, seed=3)
    with solver.Solver.from_sec5(p, precision=1) as s:
        s.backward_sweep()
        assert s.nG == len(s.gamma_list())
    if d == 5 and kind == W.G_TOTAL_N:
        with pytest.raises(L.QrError):
            solver.Solver.from_sec5(p, precision=1, path_kernel=1)


def test_direct_backward_sweep_matches_oracle(mods, ora):
    solver, L = mods
    p = W.Sec5Problem(d=5, N=4, gamma_kind=W.G_HYP_N, gamma_n=8, M=900, seed=5, q=5.1)
    ref, _ = ora.backward_sweep(_oracle_problem(ora, p))
    with solver.Solver.from_sec5(p, precision=0, path_kernel=2) as s:
        s.backward_sweep()
        _, a = s.cosine_coefs()
    assert np.abs(a - ref.real).max() / np.abs(ref.real).max() < 1e-10


def test_direct_agrees_with_unfolded_route(mods):
    """The same estimator by the two routes (FP64): the unfolded Z^d set with
    sign-orbit averages and the direct real kernels give the same coefficients
    up to rounding."""
    solver, L = mods
    p = W.Sec5Problem(d=3, N=4, gamma_kind=W.G_HYP_N, gamma_n=6, M=1500, seed=8, q=2.1)
    out = []
    for kern in (1, 2):
        with solver.Solver.from_sec5(p, precision=0, path_kernel=kern) as s:
            s.picard_step(3)
            out.append(s.cosine_coefs()[1])
    assert np.abs(out[0] - out[1]).max() / np.abs(out[0]).max() < 1e-12


@pytest.mark.parametrize("d,kind,n", [(1, W.G_FULL_N, 60), (5, W.G_HYP_N, 16), (8, W.G_TOTAL_N, 3)])
def test_direct_eval_matches_oracle_series(mods, ora, d, kind, n):
    """qr_eval on set coefficients (decaying, random signs) at Student points,
    against the oracle's series; the bound B = sum |a_k| 2^{d'(k)/2} scales
    the tolerance."""
    solver, L = mods
    rng = np.random.default_rng(d)
    p = W.Sec5Problem(d=d, N=2, gamma_kind=kind, gamma_n=n, M=64, seed=2)
    op = _oracle_problem(ora, p)
    K = ora.gamma_list(kind, d, n)
    a = rng.normal(size=(2, len(K))) / (1.0 + (K ** 2).sum(axis=1))[None, :]
    x = rng.standard_t(2, size=(300, d)) / np.sqrt(2.0)
    B = (np.abs(a) * 2.0 ** (0.5 * (K != 0).sum(axis=1))[None, :]).sum(axis=1).max()
    for prec, tol in ((0, 1e-13), (1, 1e-5)):
        with solver.Solver.from_sec5(p, precision=prec, path_kernel=2) as s:
            s.set_coefs(a.astype(complex))
            assert np.array_equal(s.coefs().real, a)
            for i in (0, 1):
                got = s.eval(i, x)
                want = ora.series(op, a[i].astype(complex), x)
                assert np.abs(got - want).max() < tol * B, (prec, i)


@pytest.mark.parametrize("d", [9, 12])
def test_routes_above_d8(mods, d):
    """Above d = 8 the direct route is the only one: the automatic choice
    takes it, the unfolded route and the Z^d (Fourier) sets are refused."""
    solver, L = mods
    p = W.Sec5Problem(d=d, N=2, gamma_kind=W.G_HYP_N, gamma_n=1, M=128, seed=4)
    with solver.Solver.from_sec5(p, precision=1) as s:
        s.picard_step(1)
        assert s.nG == 2 ** d
    with pytest.raises(L.QrError) as e:
        solver.Solver.from_sec5(p, precision=1, path_kernel=1)
    assert e.value.status == L.QR_ENOTIMPL
    with pytest.raises(L.QrError):
        solver.Solver(d, 2, 1.0, L.QR_NU_STUDENT2, 2.0, L.QR_G_L1, 1, np.zeros(d), np.eye(d), L.QR_F_ZERO, [0.0],
                      L.QR_GT_COS, np.ones(d), 64, 1, precision=1)


def test_direct_rejects_fourier_sets(mods):
    solver, L = mods
    with pytest.raises(L.QrError):
        solver.Solver.from_workload(W.c1(), path_kernel=2)


def test_paper_d5_row_full_size_sampled_responses(mods, ora):
    """The paper's d = 5 row Delta = 0.2, Gamma_H(16), M = 2 10^6, FP32, in
    the launch geometry of `sec5.py`: after one Picard iteration from
    ybar = 0, the responses of the second iteration are checked path by path
    against the oracle from the coefficients the first one produced."""
    solver, L = mods
    p = W.Sec5Problem(d=5, N=5, gamma_kind=W.G_HYP_N, gamma_n=16, M=2 * 10 ** 6, seed=1, q=5.1)
    op = _oracle_problem(ora, p)
    rng = np.random.default_rng(55)
    with solver.Solver.from_sec5(p, precision=1) as s:
        assert s.nG == 3042
        s.picard_step(1)
        a1 = s.coefs()
        s.picard_step(1)
        for i in (0, 2, 4):
            S = s.responses(i)
            for m in list(rng.integers(0, p.M, size=6)) + [p.M - 1]:
                So = ora.responses(op, a1, i, (int(m), int(m) + 1))[0]
                assert abs(S[m] - So) < 1e-4 * max(1.0, abs(So)), (i, int(m), S[m], So)
