"""Sharded tracking step: the charges partitioned among shards, each shard
evaluating the field at its own charges only -- the division of the field
work among GPUs of the paper's multi-GPU runs (Sec. 2.4, Sec. 3.2.4).

This module only orders the library's calls (obem_shard_field / _propose /
_count / _commit, see include/obem.h) and moves data between shards; every
step of the method runs in the library's kernels.  Per step:

  1. all-gather of the live charges of every shard (positions and charges,
     ids, births, species), in shard order;
  2. per shard: field at its own charges from the gathered charges;
     recombination proposals of its electrons into a per-cation key array;
  3. all-reduce(MIN) of the key arrays;
  4. per shard: recombination outcome and the flight / collision pass;
     all-gather of the shards' spawned pairs and status;
  5. per shard: commit with spawn ids after those of the shards before it
     (an exclusive scan of the spawned pairs), or no commit at all when any
     shard failed (capacity, trials): the step is all-or-nothing;
  6. rebalance: the shards take equal consecutive slices of the union in
     id order again (contiguous id ranges), moving the spawned charges.

Two ways to exchange: LocalExchange for several shards in one process (one
GPU, "virtual" shards: the collectives are plain tensor operations) and
DistExchange for one shard per rank over torch.distributed (NCCL between
GPUs, gloo on CPU tensors)."""
from __future__ import annotations

import dataclasses

import numpy as np

from . import obem

INT64_MAX = (1 << 63) - 1


class LocalExchange:
    """Exchanges among the shards held by this process."""

    first_index = 0

    def gather(self, parts):
        import torch
        return torch.cat(parts) if len(parts) > 1 else parts[0].clone()

    def allmin(self, keys):
        import torch
        out = keys[0].clone()
        for k in keys[1:]:
            torch.minimum(out, k, out=out)
        return out

    def gather_ints(self, rows):
        return [list(r) for r in rows]


class DistExchange:
    """One shard per rank of a torch.distributed process group; tensors on
    the group's device (CUDA for NCCL, CPU for gloo)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        self.first_index = self.rank

    def gather(self, parts):
        """Concatenation in rank order of every rank's (rows, ...) tensor; the
        row counts may differ (padded to the largest for the collective)."""
        import torch
        (x,) = parts
        n = torch.tensor([x.shape[0]], dtype=torch.int64, device=x.device)
        ns = [torch.zeros_like(n) for _ in range(self.size)]
        self.dist.all_gather(ns, n, group=self.group)
        ns = [int(v.item()) for v in ns]
        m = max(ns) if ns else 0
        pad = torch.zeros((m,) + tuple(x.shape[1:]), dtype=x.dtype, device=x.device)
        pad[:x.shape[0]] = x
        bufs = [torch.empty_like(pad) for _ in range(self.size)]
        self.dist.all_gather(bufs, pad, group=self.group)
        return torch.cat([b[:k] for b, k in zip(bufs, ns)])

    def allmin(self, keys):
        (k,) = keys
        out = k.clone()
        self.dist.all_reduce(out, op=self.dist.ReduceOp.MIN, group=self.group)
        return out

    def gather_ints(self, rows):
        import torch
        (r,) = rows
        t = torch.tensor(list(r), dtype=torch.int64)
        if self.dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        out = [torch.zeros_like(t) for _ in range(self.size)]
        self.dist.all_gather(out, t, group=self.group)
        return [[int(v) for v in o.cpu().tolist()] for o in out]


@dataclasses.dataclass
class Shard:
    """A shard held by this process: its context, charges, stats and field."""
    ctx: object
    state: object            # obem.DeviceState
    stats: object            # obem.new_stats()
    E: object                # CUDA float [capacity, 4]


class _View:
    """An obem_state over gathered arrays (velocities unused: the positions
    stand in for them)."""

    def __init__(self, pos_q, ids, birth, species, n_dev):
        self.pos_q, self.id, self.birth, self.species, self.scalars = pos_q, ids, birth, species, n_dev
        self.capacity = int(pos_q.shape[0])

    def c_struct(self):
        return obem.obem_state(pos_q=self.pos_q.data_ptr(), vel=self.pos_q.data_ptr(), id=self.id.data_ptr(),
                               birth=self.birth.data_ptr(), species=self.species.data_ptr(),
                               n=self.scalars.data_ptr(), next_id=self.scalars.data_ptr() + 4,
                               capacity=self.capacity)


def split_charges(ch, k):
    """Initial partition: k contiguous id ranges of a host charge set
    (sorted by id), as equal as the count allows."""
    from types import SimpleNamespace
    n = ch.pos_q.shape[0]
    cuts = [n * i // k for i in range(k + 1)]
    return [SimpleNamespace(pos_q=ch.pos_q[a:b], vel=ch.vel[a:b], id=ch.id[a:b], birth=ch.birth[a:b],
                            species=ch.species[a:b]) for a, b in zip(cuts[:-1], cuts[1:])]


def commit_plan(next_id, rows, first_index, k):
    """From every shard's (spawned pairs, status) in shard order: the step's
    status (OBEM_OK, else the first failing shard's code), whether to commit
    (all shards OK), the spawn-id base of this process's k shards starting at
    shard first_index (the global next id plus twice the spawned pairs of the
    shards before each: an exclusive scan), and the next id after the step."""
    status = next((int(r[1]) for r in rows if int(r[1]) != obem.OBEM_OK), obem.OBEM_OK)
    commit = status == obem.OBEM_OK
    before = np.concatenate([[0], np.cumsum([int(r[0]) for r in rows])]).astype(np.int64)
    bases = [(next_id + 2 * int(before[first_index + j])) & 0xFFFFFFFF for j in range(k)]
    new_next = (next_id + 2 * int(before[-1])) & 0xFFFFFFFF if commit else next_id
    return status, commit, bases, new_next


def sharded_step(shards, ex, step, next_id, E_given=None):
    """One tracking step of every shard (this process's shards; all ranks
    call it together).  next_id: the global next unused id.  E_given: None to
    evaluate the field, else one CUDA float [capacity, 4] field per local
    shard (its charges' field, in its order).  Returns (status, next_id after
    the step, per-local-shard stats dicts); status is OBEM_OK or the first
    failing shard's code, and nothing is committed unless every shard is OK."""
    import torch
    ns = [int(sh.state.scalars[0].item()) for sh in shards]
    counts = [c[0] for c in ex.gather_ints([[n] for n in ns])]
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    total = int(offs[-1])
    me = [ex.first_index + k for k in range(len(shards))]      # global shard indices
    # 1. gathered charges (every shard's live charges, shard order)
    G_pos = ex.gather([sh.state.pos_q[:n] for sh, n in zip(shards, ns)])
    G_id = ex.gather([sh.state.id[:n] for sh, n in zip(shards, ns)])
    G_birth = ex.gather([sh.state.birth[:n] for sh, n in zip(shards, ns)])
    G_sp = ex.gather([sh.state.species[:n] for sh, n in zip(shards, ns)])
    dev = G_pos.device
    if total == 0:
        G_pos = torch.zeros((1, 4), dtype=torch.float32, device=dev)
        G_id = torch.zeros(1, dtype=torch.int32, device=dev)
        G_birth = torch.zeros(1, dtype=torch.int32, device=dev)
        G_sp = torch.zeros(1, dtype=torch.uint8, device=dev)
    G = _View(G_pos, G_id, G_birth, G_sp, torch.tensor([total, 0], dtype=torch.int32, device=dev))
    # 2. field and proposals
    keys = []
    for k, sh in enumerate(shards):
        if E_given is None:
            obem.obem_shard_field(sh.ctx, sh.state, G_pos, total, int(offs[me[k]]), sh.E)
        E = sh.E if E_given is None else E_given[k]
        sh.E_used = E
        kk = torch.empty(G.capacity, dtype=torch.int64, device=dev)
        obem.obem_shard_propose(sh.ctx, sh.state, G, step, kk)
        keys.append(kk)
    # 3. recombination keys reduced over every shard
    red = ex.allmin(keys)
    # 4. outcome and flight; spawned pairs and status of every shard
    rows = []
    for k, sh in enumerate(shards):
        obem.obem_shard_count(sh.ctx, sh.state, sh.E_used, step, red, int(offs[me[k]]), sh.stats)
        s = obem.read_stats(sh.stats)
        rows.append([s["spawned_pairs"], s["status"]])
    status, commit, bases, new_next = commit_plan(next_id, ex.gather_ints(rows), ex.first_index, len(shards))
    # 5. commit with ids after the shards before this one (exclusive scan)
    out = []
    for k, sh in enumerate(shards):
        obem.obem_shard_commit(sh.ctx, sh.state, sh.E_used, step, bases[k], commit, sh.stats)
        out.append(obem.read_stats(sh.stats))
    if commit:
        rebalance(shards, ex, len(counts), [int(o["n_after"]) - 2 * int(o["spawned_pairs"]) for o in out],
                  [int(o["n_after"]) for o in out])
    for sh in shards:
        sh.state.scalars[1:2].fill_(int(np.uint32(new_next).view(np.int32)))
    return status, new_next, out


FIELDS = ("pos_q", "vel", "id", "birth", "species")


def rebalance(shards, ex, n_shards, keep, n_after):
    """Restore the partition into contiguous id ranges after a committed step.
    Shard j then holds its survivors (its first keep[j] charges) and the
    charges it spawned, whose ids follow every survivor's; in id order the
    union is every shard's survivors in shard order, then every shard's spawns
    in shard order (the exclusive scan gave them their ids in that order).
    The shards take equal consecutive slices of that order again, so that the
    next step's spawns, numbered shard by shard, are numbered in parent id
    order as the unsharded step numbers them."""
    import torch
    g = {f: torch.cat([ex.gather([getattr(sh.state, f)[:k] for sh, k in zip(shards, keep)]),
                       ex.gather([getattr(sh.state, f)[k:m] for sh, k, m in zip(shards, keep, n_after)])])
         for f in FIELDS}
    tot = int(g["id"].shape[0])
    cuts = [tot * i // n_shards for i in range(n_shards + 1)]
    for k, sh in enumerate(shards):
        j = ex.first_index + k
        a, b = cuts[j], cuts[j + 1]
        if b - a > sh.state.capacity:
            raise RuntimeError("shard %d: %d charges after rebalancing exceed its capacity %d"
                               % (j, b - a, sh.state.capacity))
        for f in FIELDS:
            getattr(sh.state, f)[:b - a].copy_(g[f][a:b])
        sh.state.scalars[0:1].fill_(b - a)
