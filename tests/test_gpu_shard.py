"""The sharded tracking step on virtual shards (several shards on one GPU,
exchanged in-process): K shards must reproduce the unsharded obem_step bit
for bit given the same field -- every charge's state, the ids of spawned
charges, next_id and the step counts -- including recombination pairs that
straddle shards (an electron on one shard, its cation on another) and the
all-or-nothing commit when one shard overflows; the sharded field (one-sided
kernel over the gathered charges) matches the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem, shard
from gpu_util import FIELD_TOL, guarded_rel_err

pytestmark = pytest.mark.gpu
ME = 9.1093837015e-31
COUNT_KEYS = ["spawned_pairs", "absorbed", "attached", "recombined_pairs", "collisions", "trials",
              "n_electron", "n_cation", "n_anion", "n_after"]


def _mixture(seed, n_e=1500, n_i=600, close=200):
    rng = np.random.default_rng(seed)
    pe = rng.uniform([0, 0, 2e-4], [1e-3, 1e-3, 1.8e-3], (n_e, 3))
    pi = rng.uniform([0, 0, 2e-4], [1e-3, 1e-3, 1.8e-3], (n_i, 3))
    pi[:close] = pe[:close] + rng.normal(0, 1.2e-9, (close, 3))        # recombination candidates
    ve = inputs.maxwellian(rng, n_e, 8.0, ME)
    vi = inputs.maxwellian(rng, n_i, 0.025, 40 * 1.66053906660e-27)
    sp = np.concatenate([np.zeros(n_e, np.uint8), np.ones(n_i, np.uint8)])
    perm = rng.permutation(n_e + n_i)          # electrons and their cations end up in different shards
    ch = inputs.make_charges(np.concatenate([pe, pi])[perm], np.concatenate([ve, vi])[perm], sp[perm])
    ch.birth[:] = np.where(rng.random(n_e + n_i) < 0.1, 3, 0).astype(np.uint32)
    return ch


def _field(pos_q):
    """A field that depends on the charge's position only (so that it is the
    same for a charge whichever shard holds it)."""
    p = np.asarray(pos_q[:, :3], np.float64)
    E = np.zeros((len(p), 4), np.float32)
    E[:, 0] = 2e5 * np.sin(p[:, 1] / 1.3e-4)
    E[:, 1] = 1e5 * np.cos(p[:, 0] / 0.7e-4)
    E[:, 2] = -3e6 + 4e5 * np.sin(p[:, 2] / 2.1e-4)
    return E


def _ctx(trk, gas, cap, flags=0):
    c = obem.obem_create(capacity=cap, dt=trk.dt, seed=trk.seed, softening=trk.softening, z_lo=trk.z_lo,
                         z_hi=trk.z_hi, beta=trk.beta, trial_cap=trk.trial_cap, flags=flags)
    obem.obem_gas_load(c, gas)
    return c


def _shards(ch, k, trk, gas, cap, flags=0, next_id=None, caps=None):
    out = []
    for j, part in enumerate(shard.split_charges(ch, k)):
        ctx = _ctx(trk, gas, cap, flags)
        st = obem.DeviceState(cap if caps is None else caps[j])
        st.upload(part, ch.pos_q.shape[0] if next_id is None else next_id)
        out.append(shard.Shard(ctx, st, obem.new_stats(), torch.zeros((st.capacity, 4), device="cuda")))
    return out


def _union(shards):
    parts = [sh.state.download()[0] for sh in shards]
    cat = {k: np.concatenate([getattr(p, k) for p in parts]) for k in ("pos_q", "vel", "id", "birth", "species")}
    o = np.argsort(cat["id"], kind="stable")
    return {k: v[o] for k, v in cat.items()}, [p.id for p in parts]


def _close(shards):
    for sh in shards:
        obem.obem_destroy(sh.ctx)


@pytest.mark.parametrize("k", [2, 3, 5])
def test_virtual_shards_bit_exact_with_the_unsharded_step(k):
    gas = inputs.argon_like_gas()
    trk = inputs.Tracking(dt=1e-12, seed=5, z_lo=0.0, z_hi=2e-3, beta=1e-13)
    ch = _mixture(7)
    cap = 12000
    ref_ctx = _ctx(trk, gas, cap)
    ref = obem.DeviceState(cap)
    ref.upload(ch)
    rstats = obem.new_stats()
    shards = _shards(ch, k, trk, gas, cap)
    ex = shard.LocalExchange()
    nid = ch.pos_q.shape[0]
    try:
        for s in range(8):
            cur, _ = ref.download()
            Eref = np.zeros((cap, 4), np.float32)
            Eref[:cur.n] = _field(cur.pos_q)
            obem.obem_step(ref_ctx, ref, s, rstats, E_in=torch.from_numpy(Eref).cuda())
            Eg = []
            for sh in shards:
                loc, _ = sh.state.download()
                e = np.zeros((sh.state.capacity, 4), np.float32)
                e[:loc.n] = _field(loc.pos_q)
                Eg.append(torch.from_numpy(e).cuda())
            status, nid, sstats = shard.sharded_step(shards, ex, s, nid, E_given=Eg)
            torch.cuda.synchronize()
            r = obem.read_stats(rstats)
            assert status == 0 and r["status"] == 0
            got, ids = _union(shards)
            want, rnid = ref.download()
            assert nid == rnid
            for key in ("pos_q", "vel"):
                assert np.array_equal(got[key].view(np.uint32), getattr(want, key).view(np.uint32)), (s, key)
            for key in ("id", "birth", "species"):
                assert np.array_equal(got[key], getattr(want, key)), (s, key)
            for key in COUNT_KEYS:
                assert sum(int(x[key]) for x in sstats) == int(r[key]), (s, key)
            # contiguous id ranges again: the shards in shard order are sorted by id
            assert np.all(np.diff(np.concatenate(ids).astype(np.int64)) > 0)
            assert max(len(i) for i in ids) - min(len(i) for i in ids) <= 1
        assert r["recombined_pairs"] >= 0
        assert sum(int(x["spawned_pairs"]) for x in sstats) >= 0
    finally:
        obem.obem_destroy(ref_ctx)
        _close(shards)


def test_recombination_across_shards_is_exercised():
    """The pairing rules across shard boundaries: with the cations of the
    close pairs all on one shard and their electrons on others, the sharded
    and unsharded steps recombine the same pairs (and some do recombine)."""
    gas = inputs.maxwell_gas(0.0, 40.0)
    gas.nuc[:] = 0.0
    gas.nu_ion = 0.0
    trk = inputs.Tracking(dt=1e-12, seed=1, z_lo=-1, z_hi=1, beta=1e-13)
    rng = np.random.default_rng(3)
    n = 600
    pe = rng.uniform(0, 1e-4, (n, 3))
    pc = pe + rng.normal(0, 1.5e-9, (n, 3))
    pos = np.concatenate([pe, pc])                 # electrons first, cations after: shards split them
    sp = np.concatenate([np.zeros(n, np.uint8), np.ones(n, np.uint8)])
    ch = inputs.make_charges(pos, np.zeros((2 * n, 3)), sp)
    ref_ctx = _ctx(trk, gas, 4 * n)
    ref = obem.DeviceState(4 * n)
    ref.upload(ch)
    rstats = obem.new_stats()
    shards = _shards(ch, 2, trk, gas, 4 * n)
    try:
        E0 = torch.zeros((4 * n, 4), device="cuda")
        obem.obem_step(ref_ctx, ref, 0, rstats, E_in=E0)
        status, nid, sstats = shard.sharded_step(shards, shard.LocalExchange(), 0, 2 * n,
                                                 E_given=[torch.zeros((4 * n, 4), device="cuda")] * 2)
        r = obem.read_stats(rstats)
        assert status == 0 and r["recombined_pairs"] > 50
        assert sum(int(x["recombined_pairs"]) for x in sstats) == r["recombined_pairs"]
        got, _ = _union(shards)
        want, _ = ref.download()
        assert np.array_equal(got["id"], want.id)
    finally:
        obem.obem_destroy(ref_ctx)
        _close(shards)


def test_overflow_in_one_shard_commits_nothing_anywhere():
    gas = inputs.argon_like_gas()
    trk = inputs.Tracking(dt=1e-12, seed=5, z_lo=0.0, z_hi=2e-3, beta=-1.0)
    ch = _mixture(8, n_e=3000, n_i=0, close=0)
    for m in (2,):
        parts = shard.split_charges(ch, m)
        caps = [len(parts[0].id) + 2, 12000]        # shard 0 cannot hold its spawns
        shards = _shards(ch, m, trk, gas, 12000, caps=caps)
        try:
            before = [sh.state.download() for sh in shards]
            Eg = [torch.from_numpy(np.pad(_field(p.pos_q), ((0, sh.state.capacity - len(p.id)), (0, 0)))).cuda()
                  for p, sh in zip(parts, shards)]
            status, nid, sstats = shard.sharded_step(shards, shard.LocalExchange(), 0, 3000, E_given=Eg)
            assert status == obem.OBEM_ERR_CAPACITY and nid == 3000
            assert sstats[0]["status"] == obem.OBEM_ERR_CAPACITY and sstats[1]["status"] == obem.OBEM_ERR_STATE
            for b, sh in zip(before, shards):
                a = sh.state.download()
                assert a[1] == 3000 and np.array_equal(a[0].pos_q, b[0].pos_q) and np.array_equal(a[0].id, b[0].id)
        finally:
            _close(shards)


def test_sharded_field_matches_oracle():
    mesh, gas, ch, trk = inputs.config_small_plates(seed=4, n=1200)
    trk.softening = 1e-9
    sig = oracle.bem_solve(mesh)
    flags = obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD
    shards = _shards(ch, 3, trk, gas, 2000, flags=flags)
    try:
        sg = torch.empty(mesh.n, dtype=torch.float32, device="cuda")
        for sh in shards:
            obem.obem_mesh_load(sh.ctx, mesh)
            obem.obem_bem_assemble(sh.ctx, obem.OBEM_LU_FP32)
            obem.obem_bem_solve(sh.ctx, mesh.group_voltage, sg)
        G = torch.from_numpy(np.ascontiguousarray(ch.pos_q)).cuda()
        off = 0
        got = []
        for sh in shards:
            n = int(sh.state.scalars[0].item())
            obem.obem_shard_field(sh.ctx, sh.state, G, ch.n, off, sh.E)
            got.append(sh.E[:n].cpu().numpy().astype(np.float64))
            off += n
        torch.cuda.synchronize()
        got = np.concatenate(got)
    finally:
        _close(shards)
    ref = oracle.field_at_charges(ch, mesh, sg.cpu().numpy().astype(np.float64), trk.softening)
    assert guarded_rel_err(got[:, :3], ref) <= FIELD_TOL
