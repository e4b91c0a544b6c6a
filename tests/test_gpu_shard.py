"""One problem sharded over ranks by path chunks (Sec. 4's multi-GPU split of
the Monte-Carlo sum), emulated on one GPU: the W shards of a problem run one
after another, each simulating and projecting only its own chunks of paths;
their group sums are exchanged by device copies (what an all-gather does
between GPUs) and every shard finishes with the common reduction. The
coefficients must equal the unsharded iteration's bit for bit, and the
shards' clamp counts must add up to the unsharded count."""
import numpy as np
import pytest

from paper_2407_21084_b300 import workloads as W

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1
TREE, TABLE = 0, 1


@pytest.fixture(scope="module")
def qr():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import build, solver

    build.build()
    return solver


CASES = [
    ("c1", FP64, TREE, 2 ** 14, 2),
    ("c1", FP32, TABLE, 3000, 4),
    ("c2", FP32, TREE, 70000, 2),   # 137 chunks: groups of 17 and 18, ragged last chunk
    ("c2", FP64, TREE, 70000, 4),
    ("c2", FP32, TREE, 700, 8),     # fewer chunks than groups: some shards own none
]


@pytest.mark.parametrize("wl,prec,kern,M,world", CASES)
def test_sharded_iterations_equal_one_gpu_bit_for_bit(qr, wl, prec, kern, M, world):
    import torch

    w = getattr(W, wl)()
    n_iter = 2
    with qr.Solver.from_workload(w, precision=prec, M=M, path_kernel=kern) as one:
        one.picard_step(n_iter)
        ref = one.coefs()
        hits_ref = one.stats()["clamp_hits"]
    shards = [qr.Solver.from_workload(w, precision=prec, M=M, path_kernel=kern) for _ in range(world)]
    try:
        for r, s in enumerate(shards):
            s.shard(r, world)
        for _ in range(n_iter):
            bufs = []
            for s in shards:
                s.picard_begin()
                bufs.append(s.shard_groups())
            torch.cuda.synchronize()
            # the exchange: every shard receives every other shard's groups
            for buf, _, _ in bufs:
                for src, gl, gh in bufs:
                    if src.data_ptr() != buf.data_ptr():
                        buf[gl:gh].copy_(src[gl:gh])
            torch.cuda.synchronize()
            res = [s.picard_finish() for s in shards]
            assert len(set(res)) == 1
        for s in shards:
            a = s.coefs()
            assert np.array_equal(a.view(np.float64), ref.view(np.float64))
        assert sum(s.stats()["clamp_hits"] for s in shards) == hits_ref
    finally:
        for s in shards:
            s.close()


def test_sharded_context_refuses_the_one_gpu_calls(qr):
    w = W.c1()
    with qr.Solver.from_workload(w, precision=FP64, M=4096) as s:
        s.shard(1, 2)
        with pytest.raises(Exception):
            s.picard_step(1)
        with pytest.raises(Exception):
            s.backward_sweep()
        s.shard(0, 1)  # back to the whole problem
        s.picard_step(1)
