"""GPU tests of the multi-instance engine: a batch of mixed instances gives
exactly the coefficients of the same instances run one by one (same
kernels per item, fixed reduction order), and a class it adds is checked
against the FP64 oracle."""
import numpy as np
import pytest

from paper_2407_21084_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import batch, build, solver

    build.build()
    return batch, solver, torch


def test_batch_equals_single_runs(mods):
    batch, solver, torch = mods
    ws = W.c4(n_instances=10, n_shared=3, M=3000)  # ragged M: partial tiles and chunks
    st = torch.cuda.Stream()
    sol = batch.solvers_for(ws, st.cuda_stream)
    b = batch.Batch(sol)
    b.picard_step(1)
    b.picard_step(2)
    for w, s in zip(ws, sol):
        with solver.Solver.from_workload(w, precision=1, stream=st.cuda_stream) as one:
            one.picard_step(3)
            assert np.array_equal(one.coefs().view(np.float64), s.coefs().view(np.float64)), w.name
    info = b.info()
    assert info["tiles_per_item"] in (1, 4, 16) and info["grid"] > 0
    b.close()
    for s in sol:
        s.close()


@pytest.mark.parametrize("d,n", [(5, 4), (7, 3)])
def test_new_classes_match_oracle(mods, ora, d, n):
    _, solver, _ = mods
    rng = np.random.default_rng(d)
    w = W.c1().with_(d=d, N=6, gamma_kind=W.G_L1_Z, gamma_n=n, s=rng.uniform(-1, 1, size=d), sigma0=0.35, M=2048)
    K = ora.gamma_list(w.gamma_kind, w.d, w.gamma_n)
    p = ora.Problem(d=w.d, N=w.N, T=w.T, k=K, b=w.b, sigma=w.sigma, f_kind=ora.F_CUBIC_MANUF, f_par=w.f_par,
                    g_kind=ora.GT_COS, g_par=w.g_par, M=w.M, seed=w.seed, clamp_L=w.clamp_L)
    ref, _ = ora.picard(p, 2)
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        with solver.Solver.from_workload(w, precision=prec) as s:
            s.picard_step(2)
            a = s.coefs()
        assert np.abs(a - ref).max() / np.abs(ref).max() < tol


def test_c4_full_size_sampled_responses(mods, ora):
    """The multi-instance workload at its full size (256 instances of uneven
    d, |Gamma| and N, M = 2^18 each, 64 of them sharing their points and run
    by the tensor-core path), in the launch geometry `batch.py` times: after
    one batch iteration from y == 0, the responses of the second iteration
    are checked path by path against the oracle, from the coefficients the
    first one produced, on a sample of instances, rows and paths."""
    batch, solver, torch = mods
    ws = W.c4()
    st = torch.cuda.Stream()
    sol = batch.solvers_for(ws, st.cuda_stream)
    b = batch.Batch(sol)
    assert b.info()["grouped_instances"] == 64
    b.picard_step(1)
    rng = np.random.default_rng(44)
    picks = sorted(set([0, 1] + list(rng.choice(len(ws) - 64, 3, replace=False)) + [len(ws) - 64, len(ws) - 1]))
    a1 = {q: sol[q].coefs() for q in picks}
    b.picard_step(1)
    for q in picks:
        w, s = ws[q], sol[q]
        K = ora.gamma_list(w.gamma_kind, w.d, w.gamma_n)
        p = ora.Problem(d=w.d, N=w.N, T=w.T, k=K, b=w.b, sigma=w.sigma, f_kind=ora.F_CUBIC_MANUF, f_par=w.f_par,
                        g_kind=ora.GT_COS, g_par=w.g_par, M=w.M, seed=w.seed, clamp_L=w.clamp_L)
        for i in (0, w.N // 2, w.N - 1):
            S = s.responses(i)
            for m in rng.integers(0, w.M, size=6):
                So = ora.responses(p, a1[q], i, (int(m), int(m) + 1))[0]
                assert abs(S[m] - So) < 1e-4 * max(1.0, abs(So)), (w.name, i, int(m))
    b.close()
    for s in sol:
        s.close()
