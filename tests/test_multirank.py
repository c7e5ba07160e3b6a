"""The multi-rank benchmark path on CPU (gloo, world size 2): the job's batch (world x 8 sources)
is dealt over the ranks by the library's length-balanced partition (weak scaling, no data-path
collective), and the job throughput is the sum of all ranks' samples over the slowest rank's time,
identical on every rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    lens, srcs = bench.workload(rank, ws, 8)
    samples = int(lens.sum())
    ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
    value, ms, total = bench.job_throughput(samples, ms_local)
    out[rank] = (value, ms, total, samples, sorted(float(s.f) for s in srcs))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_job_throughput():
    ws, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    r0, r1 = out[0], out[1]
    # every rank reports the same job figures
    assert r0[:3] == r1[:3]
    value, ms, total = r0[:3]
    assert ms == 150.0                          # max over ranks
    assert total == r0[3] + r1[3]               # sum over ranks
    assert np.isclose(value, 6.0 * total / 0.150)
    # the ranks' shares are disjoint and together the whole batch, balanced within one source
    glens, gsrcs = bench.workload(0, 1, 2 * 8)
    assert sorted(r0[4] + r1[4]) == sorted(float(s.f) for s in gsrcs)
    assert total == glens.sum()
    assert abs(r0[3] - r1[3]) <= glens.max()


def test_single_process_identity():
    value, ms, total = bench.job_throughput(1000, 20.0)
    assert (ms, total) == (20.0, 1000.0) and np.isclose(value, 6000 / 0.02)
