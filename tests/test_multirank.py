"""The N-GPU bench runs independent replicas (weak scaling: rank r steps its
own chamber, seeded 1 + r; no data-path collective).  Its whole-job figures
come from one reduction: the slowest rank's timed region and the work of all
ranks.  Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = 100.0 + 50.0 * rank                       # rank 1 is the slower one
        counts = [1000.0 * (rank + 1), 2000.0 * (rank + 1), 1e12 * (rank + 1)]
        out[rank] = bench.reduce_over_ranks(ms, counts, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        ms, tot = res[r]
        assert ms == 150.0                              # max over ranks
        assert tot == [3000.0, 6000.0, 3e12]            # summed work


def test_replicas_get_their_own_workloads():
    """Rank r's workload is seeded 1 + r: different charges, same shapes."""
    sys.path.insert(0, ROOT)
    import bench
    a = bench._workload(1, 2000, 2000)
    b = bench._workload(2, 2000, 2000)
    assert a[2].pos_q.shape == b[2].pos_q.shape
    assert not (a[2].pos_q == b[2].pos_q).all()
