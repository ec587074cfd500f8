"""The exchanges of the sharded step (all-gather of the shards' charges,
all-reduce(MIN) of the recombination keys, all-gather of spawn counts and
status with the exclusive scan of the spawn ids), run over two gloo ranks on
the CPU and compared with the same exchanges among shards in one process;
and the all-or-nothing commit plan."""
import os
import socket
import sys

import numpy as np
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2110_09214_gb300 import obem, shard  # noqa: E402

INT64_MAX = (1 << 63) - 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _parts(rank):
    """Rank r's local shard data: uneven row counts, keys with 'none'."""
    g = torch.Generator().manual_seed(10 + rank)
    n = [5, 3][rank]
    pos = torch.randn(n, 4, generator=g)
    ids = torch.arange(100 * rank, 100 * rank + n, dtype=torch.int32)
    keys = torch.randint(0, 1 << 40, (9,), generator=g, dtype=torch.int64)
    keys[torch.arange(9) % (2 + rank) == 0] = INT64_MAX
    row = [7 + 4 * rank, obem.OBEM_OK if rank == 0 else obem.OBEM_ERR_CAPACITY]
    return pos, ids, keys, row


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ex = shard.DistExchange()
        pos, ids, keys, row = _parts(rank)
        out[rank] = (ex.gather([pos]).numpy(), ex.gather([ids]).numpy(), ex.allmin([keys]).numpy(),
                     ex.gather_ints([row]), ex.first_index)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_exchanges_match_in_process_shards():
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
    loc = shard.LocalExchange()
    parts = [_parts(r) for r in range(2)]
    g_pos = loc.gather([p[0] for p in parts]).numpy()
    g_ids = loc.gather([p[1] for p in parts]).numpy()
    g_keys = loc.allmin([p[2] for p in parts]).numpy()
    g_rows = loc.gather_ints([p[3] for p in parts])
    assert g_pos.shape == (8, 4) and list(g_ids) == [0, 1, 2, 3, 4, 100, 101, 102]
    for r in range(2):
        pos, ids, keys, rows, first = res[r]
        assert first == r
        assert np.array_equal(pos, g_pos) and np.array_equal(ids, g_ids)
        assert np.array_equal(keys, g_keys)
        assert rows == g_rows
    want = np.minimum(parts[0][2].numpy(), parts[1][2].numpy())
    assert np.array_equal(g_keys, want)


def test_commit_plan_scan_and_all_or_nothing():
    rows = [[3, 0], [0, 0], [5, 0], [2, 0]]
    st, commit, bases, nxt = shard.commit_plan(1000, rows, 1, 2)
    assert st == obem.OBEM_OK and commit
    assert bases == [1006, 1006]                  # shards 1 and 2: 3 pairs before, then 0 more
    assert nxt == 1000 + 2 * 10
    st, commit, bases, nxt = shard.commit_plan(1000, [[3, 0], [1, obem.OBEM_ERR_CAPACITY], [2, 0]], 0, 3)
    assert st == obem.OBEM_ERR_CAPACITY and not commit and nxt == 1000
    assert bases == [1000, 1006, 1008]


def test_split_charges_contiguous_ranges():
    from paper_2110_09214_gb300 import inputs
    rng = np.random.default_rng(0)
    ch = inputs.make_charges(rng.normal(size=(10, 3)), rng.normal(size=(10, 3)), np.zeros(10, np.uint8))
    parts = shard.split_charges(ch, 3)
    assert [len(p.id) for p in parts] == [3, 3, 4]
    assert np.array_equal(np.concatenate([p.id for p in parts]), ch.id)


class _FakeState:
    """CPU stand-in for a shard's DeviceState (the rebalancing only moves
    rows between the arrays)."""

    def __init__(self, ids, cap):
        import torch
        n = len(ids)
        self.capacity = cap
        self.pos_q = torch.zeros((cap, 4))
        self.pos_q[:n, 0] = torch.tensor(ids, dtype=torch.float32)
        self.vel = self.pos_q.clone()
        self.id = torch.zeros(cap, dtype=torch.int32)
        self.id[:n] = torch.tensor(ids, dtype=torch.int32)
        self.birth = torch.zeros(cap, dtype=torch.int32)
        self.species = torch.zeros(cap, dtype=torch.uint8)
        self.scalars = torch.tensor([n, 0], dtype=torch.int32)


def test_rebalance_restores_contiguous_id_ranges():
    """After a step shard j holds its survivors, then its spawns (ids above
    every survivor, numbered shard by shard).  Rebalancing gives each shard an
    equal consecutive slice of the id order again."""
    from types import SimpleNamespace
    survivors = [[0, 2, 3], [5, 6], [8, 9, 11, 12]]
    spawns = [[20, 21], [], [22, 23, 24, 25]]
    shards = [SimpleNamespace(state=_FakeState(a + b, 16)) for a, b in zip(survivors, spawns)]
    shard.rebalance(shards, shard.LocalExchange(), 3, [len(a) for a in survivors],
                    [len(a) + len(b) for a, b in zip(survivors, spawns)])
    got = [sh.state.id[:int(sh.state.scalars[0])].tolist() for sh in shards]
    allids = sorted(sum(survivors, []) + sum(spawns, []))
    assert sum(got, []) == allids
    assert [len(g) for g in got] == [5, 5, 5]
    for sh in shards:                              # the rows moved with their ids
        n = int(sh.state.scalars[0])
        assert sh.state.pos_q[:n, 0].tolist() == [float(i) for i in sh.state.id[:n].tolist()]
