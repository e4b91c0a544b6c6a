"""GPU tests of the shared-point tensor-core path of the multi-instance
engine: instances that share their sample points, run as one group (series
as a BF16 split-operand product), give the coefficients of the same
instances run one by one with the FP32 tree kernel within the FP32 tolerance
(relative 1e-4 of the largest coefficient); instances outside the group stay
bit-identical; groups with a ragged last block of instances and a ragged
last tile of paths are covered."""
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


def _shared_d2(n, M, seed=7):
    rng = np.random.default_rng(seed)
    base = W.c1().with_(d=2, N=8, gamma_kind=W.G_LINF_Z, gamma_n=4, sigma0=0.4, M=M, seed=77)
    return [base.with_(a=float(rng.uniform(0, 0.5)), s=rng.uniform(-1, 1, size=2)) for _ in range(n)]


@pytest.mark.parametrize("case", ["d6_l1_3", "d2_linf_4"])
def test_group_matches_single_runs(mods, case):
    batch, solver, torch = mods
    if case == "d6_l1_3":
        ws = W.c4(n_instances=42, n_shared=40, M=3000)  # 2 persistent-kernel instances + 40 shared
        n_group = 40
    else:
        ws = W.c4(n_instances=2, n_shared=0, M=3000) + _shared_d2(33, 3000)
        n_group = 33
    st = torch.cuda.Stream()
    sol = batch.solvers_for(ws, st.cuda_stream)
    b = batch.Batch(sol, group_min=16)
    info = b.info()
    assert info["shared_groups"] == 1 and info["grouped_instances"] == n_group
    b.picard_step(1)
    b.picard_step(2)
    worst = 0.0
    for q, (w, s) in enumerate(zip(ws, sol)):
        with solver.Solver.from_workload(w, precision=1, stream=st.cuda_stream) as one:
            one.picard_step(3)
            a, c = one.coefs(), s.coefs()
        if q < len(ws) - n_group:
            assert np.array_equal(a.view(np.float64), c.view(np.float64)), w.name
        else:
            rel = np.abs(a - c).max() / np.abs(a).max()
            worst = max(worst, rel)
            assert rel < 1e-4, (w.name, rel)
    assert worst > 0.0  # the group really ran a different kernel
    with pytest.raises(Exception):
        b_set = b._L.qr_batch_set_grouping(b._b, 0)
        if b_set != 0:
            raise RuntimeError(b_set)
    b.close()
    for s in sol:
        s.close()


def test_grouping_off_is_bit_identical(mods):
    batch, solver, torch = mods
    ws = W.c4(n_instances=20, n_shared=20, M=1000)
    st = torch.cuda.Stream()
    sol = batch.solvers_for(ws, st.cuda_stream)
    b = batch.Batch(sol, group_min=0)
    assert b.info()["grouped_instances"] == 0
    b.picard_step(2)
    for w, s in zip(ws, sol):
        with solver.Solver.from_workload(w, precision=1, stream=st.cuda_stream) as one:
            one.picard_step(2)
            assert np.array_equal(one.coefs().view(np.float64), s.coefs().view(np.float64)), w.name
    b.close()
    for s in sol:
        s.close()


def test_set_coefs_between_batch_steps_reaches_the_group_kernel(mods):
    """Coefficients set from the host on grouped instances between batch
    iterations (a warm start, a resume) are the ones the next shared-point
    iteration uses: the batch continues exactly as single runs started from
    the same coefficients (within the BF16 split tolerance)."""
    batch, solver, torch = mods
    ws = W.c4(n_instances=18, n_shared=16, M=2048)
    st = torch.cuda.Stream()
    sol = batch.solvers_for(ws, st.cuda_stream)
    b = batch.Batch(sol, group_min=16)
    assert b.info()["grouped_instances"] == 16
    b.picard_step(1)
    rng = np.random.default_rng(5)
    starts = []
    for s in sol:
        a = s.coefs()
        a = a * (1.0 + 0.3 * rng.uniform(-1, 1))  # a different, still conjugate-symmetric iterate
        s.set_coefs(a)
        starts.append(a)
    b.picard_step(1)
    for q, (w, s) in enumerate(zip(ws, sol)):
        with solver.Solver.from_workload(w, precision=1, stream=st.cuda_stream) as one:
            one.set_coefs(starts[q])
            one.picard_step(1)
            a, c = one.coefs(), s.coefs()
        if q < 2:
            assert np.array_equal(a.view(np.float64), c.view(np.float64)), w.name
        else:
            assert np.abs(a - c).max() / np.abs(a).max() < 1e-4, w.name
    b.close()
    for s in sol:
        s.close()
