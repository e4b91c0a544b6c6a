"""GPU parity of libqrmc against the FP64 CPU oracle, through the C-ABI.

Bars: bit-exact for the Philox words, the start uniforms and the Gamma order;
relative 1e-10 (normwise over alpha) for the FP64 path; relative 1e-4 for the
FP32 precision form. Sizes span several tiles and a ragged tail.
"""
import os

import numpy as np
import pytest

from paper_2407_21084_b300 import workloads as W

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1
TOL = {FP64: 1e-10, FP32: 1e-4}


@pytest.fixture(scope="module")
def qr():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import build, solver

    build.build()
    return solver


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def ora_problem(ora, w, M=None, clamp=True, K=None):
    K = ora.gamma_list(w.gamma_kind, w.d, w.gamma_n) if K is None else K
    return ora.Problem(d=w.d, N=w.N, T=w.T, k=K, b=w.b, sigma=w.sigma, f_kind=ora.F_CUBIC_MANUF, f_par=w.f_par,
                       g_kind=ora.GT_COS, g_par=w.g_par, M=w.M if M is None else M, seed=w.seed,
                       clamp_L=w.clamp_L if clamp else 0.0)


# ------------------------------------------------------------- generator
def test_philox_bit_exact(qr, ora):
    rng = np.random.default_rng(0)
    ck = rng.integers(0, 2 ** 32, size=(20000, 6), dtype=np.uint64).astype(np.uint32)
    gpu = qr.philox_words(ck)
    for t in range(0, 20000, 97):
        assert list(gpu[t]) == list(ora.philox(ck[t, :4], ck[t, 4:]))
    kat = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    for line in open(kat):
        if line.strip() and not line.startswith("#"):
            w = [int(x, 16) for x in line.split()]
            assert list(qr.philox_words(np.array([w[:6]], dtype=np.uint32))[0]) == w[6:]


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_sampler(qr, ora, prec):
    d, seed, inst, i, m0, n, j = 5, 0xDEADBEEF12345, 3, 9, 1000, 777, 4
    u, x, z = qr.sample(d, 0, 3.0, seed, inst, i, m0, n, j, prec)
    tol = 1e-14 if prec == FP64 else 3e-6
    for t in range(0, n, 37):
        uo = ora.start_uniforms(seed, inst, i, m0 + t, d)
        assert np.array_equal(u[t], uo)  # exact
        xo = np.array([ora.nu_icdf(0, 3.0, v) for v in uo])
        assert np.all(np.abs(x[t] - xo) <= tol * (1 + np.abs(xo)))
        zo = ora.normals(seed, inst, i, m0 + t, j, d)
        assert np.all(np.abs(z[t] - zo) <= tol * (1 + np.abs(zo)))


@pytest.mark.parametrize("d", [1, 5, 6, 8])
def test_tree_kernel_normals(qr, ora, d):
    """The normals the FP32 tree path kernels draw (their own branch-free
    Box-Muller logarithm) against the oracle's, at the FP32 sampler bound,
    on both sides of u = 1/2 and deep in the tails (many paths)."""
    seed, inst, i, m0, n, j = 0x5EED0F7EE, 2, 7, 12345, 20000, 3
    z = qr.sample_normals_tree(d, seed, inst, i, m0, n, j)
    for t in range(0, n, 7):
        zo = ora.normals(seed, inst, i, m0 + t, j, d)
        assert np.all(np.abs(z[t] - zo) <= 3e-6 * (1 + np.abs(zo))), (t, z[t], zo)


# ------------------------------------------------------------- iteration
def _solver(qr, w, prec, M=None, clamp=True, kern=0):
    return qr.Solver.from_workload(w, precision=prec, M=M, clamp=clamp, path_kernel=kern)


TREE, TABLE = 0, 1  # path kernels: compile-time tree (default) / table-driven


@pytest.mark.parametrize("kern", [TREE, TABLE])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_c1_picard_matches_oracle(qr, ora, prec, kern):
    w = W.c1()
    p = ora_problem(ora, w)
    a_ref, hits_ref = ora.picard(p, w.n_iter)
    with _solver(qr, w, prec, kern=kern) as s:
        assert np.array_equal(s.gamma_list(), p.k)
        for _ in range(w.n_iter):
            s.picard_step(1)
        a = s.coefs()
        assert relerr(a, a_ref) < TOL[prec]
        if prec == FP64:
            assert s.stats()["clamp_hits"] == hits_ref


@pytest.mark.parametrize("kern", [TREE, TABLE])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_responses_match_oracle(qr, ora, prec, kern):
    w = W.c1().with_(N=5)
    M = 3000  # ragged: not a multiple of the block or chunk size
    p = ora_problem(ora, w, M=M)
    a1, _ = ora.picard(p, 1)
    with _solver(qr, w, prec, M=M, kern=kern) as s:
        s.set_coefs(a1)
        s.picard_step(1)
        for i in (0, 2, 4):
            S = s.responses(i)
            So = ora.responses(p, a1, i, (0, M))
            tol = 1e-12 if prec == FP64 else 2e-5
            assert np.abs(S - So).max() < tol * max(1.0, np.abs(So).max())


@pytest.mark.parametrize("kern", [TREE, TABLE])
@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("M", [4096, 5000, 1, 33])
def test_c2_prefix_matches_oracle(qr, ora, prec, M, kern):
    """C2 (d=4, N=16, |k|_1<=4) on the first M paths, 5 iterations."""
    w = W.c2()
    n_iter = w.n_iter if M >= 4096 else 2
    p = ora_problem(ora, w, M=M)
    a_ref, _ = ora.picard(p, n_iter)
    with _solver(qr, w, prec, M=M, kern=kern) as s:
        s.picard_step(n_iter)
        assert relerr(s.coefs(), a_ref) < TOL[prec]


@pytest.mark.slow
def test_c2_full_size_matches_oracle(qr, ora):
    """C2 exactly as stated: d=4, N=16, M=2^20, |k|_1<=4 (321 coefficients),
    5 Picard iterations from y == 0, every alpha_{i,k} against the FP64
    oracle: relative 1e-10 in FP64 and 1e-4 in FP32, tree and table path
    kernels (the projection runs its full 256-chunk geometry)."""
    w = W.c2()
    assert w.M == 2 ** 20 and w.n_iter == 5
    p = ora_problem(ora, w)
    a_ref, hits_ref = ora.picard(p, w.n_iter)
    for kern in (TREE, TABLE):
        for prec in (FP64, FP32):
            with _solver(qr, w, prec, kern=kern) as s:
                s.picard_step(w.n_iter)
                err = relerr(s.coefs(), a_ref)
                assert err < TOL[prec], (kern, prec, err)
                if prec == FP64:
                    assert s.stats()["clamp_hits"] == hits_ref


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_truncation_TL_on_lattice_matches_oracle(qr, ora, prec):
    """The truncation T_L (eq. TL:2) binding on a lattice case whose oracle
    iterates are pinned by a numpy recursion (standing paths, f = lam*y,
    a planted g with L at 0.6 max|g|): GPU iterates against the oracle's,
    clamp hits > 0 and, in FP64, the same count."""
    d, kind, n, lat, N, lam = 2, 0, 2, 5, 4, 0.7
    K = ora.gamma_list(kind, d, n)
    c = _planted(ora, d, kind, n, 31)[1] * 0.25
    m = np.arange(lat ** d)
    U = np.stack([((m // lat ** l) % lat + 0.5) / lat for l in range(d)], axis=1)
    L = 0.6 * np.abs((np.exp(2j * np.pi * (U @ K.T)) @ c).real).max()
    p = ora.Problem(d=d, N=N, T=1.0, k=K, b=np.zeros(d), sigma=np.zeros((d, d)), f_kind=ora.F_LINEAR,
                    f_par=[lam], g_kind=ora.GT_TRIGPOLY, g_par=c.view(np.float64), M=lat ** d, seed=1,
                    lattice_n=lat, clamp_L=L)
    a_ref, hits_ref = ora.picard(p, N)
    assert hits_ref > 0
    with qr.Solver(d, N, 1.0, 0, 3.0, kind, n, np.zeros(d), np.zeros((d, d)), 1, [lam], 1, c.view(np.float64),
                   lat ** d, 1, precision=prec, lattice_n=lat, clamp_L=L) as s:
        s.picard_step(N)
        assert relerr(s.coefs(), a_ref) < TOL[prec]
        hits = s.stats()["clamp_hits"]
        assert hits > 0
        if prec == FP64:
            assert hits == hits_ref


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_c2_ragged_projection_chunks_match_oracle(qr, ora, prec):
    """C2 at M = 270000: the projection's chunk of paths (256 * ceil(M / 65536)
    = 1280 in FP32, 128 * ceil(M / 32768) = 1152 in FP64) is not a multiple
    of the tiled kernel's block of paths, so every chunk ends with a partly
    empty block. Two iterations, rows N-3 .. N-1 against the oracle."""
    w = W.c2()
    M = 270000
    p = ora_problem(ora, w, M=M)
    rows = (w.N - 3, w.N)
    a1, _ = ora.picard_iter(p, p.zeros(), i_range=rows)
    a2, _ = ora.picard_iter(p, a1, i_range=rows)
    with _solver(qr, w, prec, M=M, kern=TREE) as s:
        s.picard_step(2)
        a = s.coefs()
    assert relerr(a[rows[0]:], a2[rows[0]:]) < TOL[prec]


def test_picard_N_equals_backward_sweep_and_is_deterministic(qr, ora):
    w = W.c1().with_(N=4)
    with _solver(qr, w, FP64, M=2048) as s:
        s.picard_step(w.N)
        aq = s.coefs()
    with _solver(qr, w, FP64, M=2048) as s:
        s.backward_sweep()
        ab = s.coefs()
    assert np.array_equal(aq.view(np.float64), ab.view(np.float64))
    with _solver(qr, w, FP64, M=2048) as s:
        s.picard_step(w.N)
        assert np.array_equal(s.coefs().view(np.float64), aq.view(np.float64))
    p = ora_problem(ora, w, M=2048)
    ref, _ = ora.backward_sweep(p)
    assert relerr(ab, ref) < 1e-10


def _planted(ora, d, kind, n, seed):
    rng = np.random.default_rng(seed)
    K = ora.gamma_list(kind, d, n)
    idx = {tuple(k): e for e, k in enumerate(K)}
    c = rng.normal(size=len(K)) + 1j * rng.normal(size=len(K))
    for e, k in enumerate(K):
        e2 = idx[tuple(-k)]
        if e2 == e:
            c[e] = c[e].real
        elif e2 < e:
            c[e] = np.conj(c[e2])
    return K, c


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("d,kind,n", [(2, 0, 2), (3, 1, 2), (3, 0, 1), (2, 1, 3)])
def test_planted_polynomial_and_linear_driver_on_lattice(qr, ora, prec, d, kind, n):
    K, c = _planted(ora, d, kind, n, 10 + d)
    lat, N, lam = 2 * n + 1, 4, 0.7
    gp = c.view(np.float64)
    with qr.Solver(d, N, 1.0, 0, 3.0, kind, n, np.zeros(d), np.zeros((d, d)), 1, [lam], 1, gp, lat ** d, 1,
                   precision=prec, lattice_n=lat) as s:
        s.picard_step(N)
        a = s.coefs()
    tol = 1e-11 if prec == FP64 else 1e-5
    for i in range(N):
        assert np.abs(a[i] - (1 + lam / N) ** (N - i) * c).max() < tol * np.abs(c).max()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_eval_matches_oracle_series(qr, ora, prec):
    import torch

    w = W.c2()
    p = ora_problem(ora, w, M=1024)
    a, _ = ora.picard(p, 2)
    x = ora.test_points(p, 3, 300)
    with _solver(qr, w, prec, M=1024) as s:
        s.set_coefs(a)
        for i in (0, 3, w.N - 1):
            yo = ora.series(p, a[i], x)
            y = s.eval(i, x)
            tol = 1e-12 if prec == FP64 else 3e-6
            assert np.abs(y - yo).max() < tol * max(1, np.abs(yo).max())
            yd = s.eval(i, torch.from_numpy(x).cuda()).cpu().numpy()
            assert np.array_equal(yd, y)
        assert np.allclose(s.eval(w.N, x), ora.g(p, x), rtol=0, atol=1e-12 if prec == FP64 else 1e-6)
        assert s.eval(0, np.zeros((0, w.d))).shape == (0,)


@pytest.mark.parametrize("kern", [TREE, TABLE])
def test_c3_full_launch_sampled_responses(qr, ora, kern):
    """C3 at its full size (d=6, N=32, M=2^22, |Gamma|=3653, FP32): the launch
    geometry the benchmark times. Responses are checked path by path against
    the oracle on a sample of (i, m), from a nonzero previous iterate."""
    w = W.c3()
    K = ora.gamma_list(w.gamma_kind, w.d, w.gamma_n)
    p = ora_problem(ora, w, K=K)
    rng = np.random.default_rng(3)
    # a smooth nonzero previous iterate: the exact projection scale ~ |k|^-2
    amp = 0.05 / (1.0 + np.abs(K).sum(1)) ** 2
    a0 = np.zeros((w.N, len(K)), dtype=complex)
    half = rng.normal(size=(w.N, len(K))) + 1j * rng.normal(size=(w.N, len(K)))
    z = len(K) // 2
    a0[:, z:] = half[:, z:] * amp[z:]
    a0[:, :z] = np.conj(a0[:, z:][:, ::-1][:, : z])
    a0[:, z] = a0[:, z].real + 0.5
    with _solver(qr, w, FP32, kern=kern) as s:
        s.set_coefs(a0)
        s.picard_step(1)
        for i in (0, 13, w.N - 1):
            S = s.responses(i)
            ms = rng.integers(0, w.M, size=24)
            for m in ms:
                So = ora.responses(p, a0, i, (int(m), int(m) + 1))[0]
                assert abs(S[m] - So) < 1e-4 * max(1.0, abs(So))
        a = s.coefs()
        assert np.all(np.isfinite(a))
        st = s.stats()
        assert st["nonfinite"] == 0


def test_tree_and_table_kernels_agree_on_c3_prefix(qr):
    """The two path kernels order the series sum differently; on the d=6,
    |k|_1<=5 set they must agree to FP32 rounding."""
    w = W.c3()
    a = []
    for kern in (TREE, TABLE):
        with _solver(qr, w, FP32, M=8192, kern=kern) as s:
            s.picard_step(2)
            a.append(s.coefs())
    assert relerr(a[0], a[1]) < 1e-5


def test_test_points_match_oracle(qr, ora):
    w = W.c2()
    p = ora_problem(ora, w, M=64)
    with _solver(qr, w, FP64, M=64) as s:
        for i in (0, 7):
            x = s.test_points(i, 257)
            xo = ora.test_points(p, i, 257)
            assert np.all(np.abs(x - xo) <= 1e-14 * (1 + np.abs(xo)))
