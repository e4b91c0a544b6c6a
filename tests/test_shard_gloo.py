"""Host logic of one problem sharded over ranks (no GPU): the library's
partition of the projection chunks (qr_shard_plan) and the group-sum
exchange (solver.exchange_group_sums) over two gloo ranks on CPU. Each rank
forms the two-level sums of its own groups from the same chunk partials;
after the exchange both ranks' fixed-order totals equal the one-rank total
bit for bit."""
import os

import numpy as np
import pytest


def _two_level(partials, n_chunks, groups):
    """Chunks in order within each group, then the groups in order."""
    out = np.zeros((8,) + partials.shape[1:])
    for g in groups:
        lo = (g * n_chunks) // 8
        hi = ((g + 1) * n_chunks) // 8
        acc = np.zeros(partials.shape[1:])
        for c in range(lo, hi):
            acc = acc + partials[c]
        out[g] = acc
    return out


def _total(gs):
    t = np.zeros(gs.shape[1:])
    for g in range(8):
        t = t + gs[g]
    return t


@pytest.mark.parametrize("n_chunks", [1, 5, 8, 137, 256])
def test_plan_partitions_chunks_into_whole_groups(n_chunks):
    from paper_2407_21084_b300 import _lib as L

    for world in (1, 2, 4, 8):
        seen = []
        for r in range(world):
            p = L.shard_plan(n_chunks, r, world)
            assert p["g_hi"] - p["g_lo"] == 8 // world
            assert p["c_lo"] == (p["g_lo"] * n_chunks) // 8 and p["c_hi"] == (p["g_hi"] * n_chunks) // 8
            seen += list(range(p["c_lo"], p["c_hi"]))
        assert seen == list(range(n_chunks))
    for bad in ((n_chunks, 0, 3), (n_chunks, 2, 2), (n_chunks, -1, 2), (0, 0, 1)):
        with pytest.raises(Exception):
            L.shard_plan(*bad)


def _rank(rank, world, port, n_chunks, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2407_21084_b300 import _lib as L
        from paper_2407_21084_b300.solver import exchange_group_sums

        rng = np.random.default_rng(11)
        partials = rng.normal(size=(n_chunks, 3, 5, 2)) * 10.0 ** rng.integers(-8, 8, size=(n_chunks, 1, 1, 1))
        p = L.shard_plan(n_chunks, rank, world)
        mine = _two_level(partials, n_chunks, range(p["g_lo"], p["g_hi"]))
        buf = torch.from_numpy(mine)
        exchange_group_sums(buf, p["g_lo"], p["g_hi"], world)
        got = _total(buf.numpy())
        ref = _total(_two_level(partials, n_chunks, range(8)))
        q.put((rank, bool(np.array_equal(got, ref))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_chunks", [137, 6])
def test_exchange_over_two_gloo_ranks_is_bit_identical(n_chunks):
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, n_chunks, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: True, 1: True}
