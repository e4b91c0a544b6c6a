"""Host logic of the replica runs of bench.py (one independent problem per
rank, no data-path collective): two gloo ranks on the CPU agree on the job
time (the slowest rank's), and the whole-job throughput counts every
rank's work. Each rank's problem uses its rank as the Philox instance, so
the ranks' clouds differ (checked on the oracle's generator)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    ms = 100.0 + 37.0 * rank
    out[rank] = (bench.max_over_ranks(ms, ws), bench.job_value(1e12, bench.max_over_ranks(ms, ws), ws))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_job_time():
    ws = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == (137.0, 2 * 1e12 / 0.137)


def test_replica_instances_draw_different_clouds(ora):
    u0 = ora.start_uniforms(7, 0, 3, 11, 4)
    u1 = ora.start_uniforms(7, 1, 3, 11, 4)
    assert not np.allclose(u0, u1)
