"""Batch of chambers (obem_batch_*, CUDA through the C ABI) against the
oracle, chamber by chamber: the field at every live charge (its chamber's
cells, Eq. (BEM3), plus the other charges of its chamber, Eq. (nbody)) within
the field tolerance; the tracking step given the oracle's field bit-exact
(states, ids, counts) in every chamber, over several steps; the captured CUDA
graph replaying the fused step exactly as the plain calls; the all-or-nothing
commit; the autotuner; and the swarm parameters of each chamber (Eqs. (vd),
(diffusion), (townsend)) from the batched run against the oracle's run."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem, swarm
from gpu_util import FIELD_TOL, guarded_rel_err, to_dev

pytestmark = pytest.mark.gpu
E = 1.602176634e-19
ME = 9.1093837015e-31
SOFT = 1e-9
COUNT_KEYS = ["spawned_pairs", "absorbed", "attached", "recombined_pairs", "collisions", "trials",
              "n_electron", "n_cation", "n_anion"]


def _chamber(rng, n, gap, e_kv_cm, n_plate, seed, hot=False, electrons=False):
    mesh = inputs.parallel_plates(1e-2, gap, n_plate, 0.0, e_kv_cm * 1e5 * gap)
    ch = inputs.avalanche_snapshot(rng, n, gap=gap)
    if electrons:
        ch = inputs.make_charges(ch.pos_q[:, :3].astype(np.float64), np.zeros((n, 3)), np.zeros(n, np.uint8))
    ch.pos_q[:, 2] = np.clip(ch.pos_q[:, 2], 0.05 * gap, 0.95 * gap).astype(np.float32)
    if hot:                                  # 50 eV electrons: ionisations in the first step
        e = ch.species == 0
        d = rng.normal(size=(int(e.sum()), 3))
        d /= np.linalg.norm(d, axis=1)[:, None]
        ch.vel[e, :3] = (d * np.sqrt(2 * 50 * E / ME)).astype(np.float32)
    trk = inputs.Tracking(dt=1e-12, seed=seed, z_lo=0.0, z_hi=gap, beta=1e-13, softening=SOFT)
    sigma = oracle.bem_solve(mesh)
    return mesh, ch, trk, sigma


def _setup(sizes, seed=5, caps=None, hot=(), electrons=()):
    rng = np.random.default_rng(seed)
    chs = []
    for k, n in enumerate(sizes):
        gap = rng.uniform(0.5e-3, 3e-3)
        e = 10 ** rng.uniform(np.log10(1.0), np.log10(30.0))
        chs.append(_chamber(rng, n, gap, e, int(rng.integers(3, 6)), 1 + k, hot=k in hot, electrons=k in electrons))
    gas = inputs.argon_like_gas()
    ctx = obem.obem_create(capacity=16, dt=1e-12, softening=SOFT, beta=1e-13,
                           flags=obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD)
    obem.obem_gas_load(ctx, gas)
    caps = caps or [max(4 * n, 64) for n in sizes]
    b = obem.Batch(ctx, caps, [0.0] * len(sizes), [c[2].z_hi for c in chs], [c[2].seed for c in chs])
    for k, (mesh, ch, trk, sigma) in enumerate(chs):
        b.cells(k, mesh.tri, sigma.astype(np.float32))
    st = b.state()
    st.upload([c[1] for c in chs])
    return ctx, b, st, chs, gas


def _close(ctx, b):
    b.destroy()
    obem.obem_destroy(ctx)


def _oracle_field(mesh, sigma, ch):
    pts = ch.pos_q[:, :3].astype(np.float64)
    Ep, _ = oracle.panel_field(mesh.tri, sigma.astype(np.float32).astype(np.float64), pts)
    En, _ = oracle.nbody_field(pts, ch.pos_q.astype(np.float64), True, SOFT)
    return Ep + En


def _gpu_field(b, st):
    out = torch.full((st.capacity, 4), float("nan"), device="cuda")
    b.field_eval(st, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_batch_field_matches_oracle_per_chamber():
    """Chambers of 0, 1, 700, 1500 and 2600 charges (1..3 tiles of 1024, ragged
    tails, an empty and a single-charge chamber), each with its own cells."""
    sizes = [0, 1, 700, 1500, 2600]
    ctx, b, st, chs, _ = _setup(sizes)
    try:
        got = _gpu_field(b, st)
    finally:
        _close(ctx, b)
    for k, (mesh, ch, trk, sigma) in enumerate(chs):
        o, n = int(b.seg_off[k]), sizes[k]
        if n == 0:
            continue
        ref = _oracle_field(mesh, sigma, ch)
        assert np.all(np.isfinite(got[o:o + n])), k
        assert guarded_rel_err(got[o:o + n, :3], ref) <= FIELD_TOL, k


def _assert_same(a, b, k):
    assert a.pos_q.shape == b.pos_q.shape, (k, a.pos_q.shape, b.pos_q.shape)
    for f in ("pos_q", "vel"):
        assert np.array_equal(getattr(a, f).view(np.uint32), getattr(b, f).view(np.uint32)), (k, f)
    for f in ("id", "birth", "species"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), (k, f)


def test_batch_step_bit_exact_vs_oracle():
    """Given the oracle's field (rounded to binary32), three batched steps
    equal the oracle's steps in every chamber: states, next ids, counts
    (argon-like gas, recombination on, hot electrons spawning)."""
    sizes = [300, 1, 1200, 0, 800]
    ctx, b, st, chs, gas = _setup(sizes, seed=7, caps=[16384, 64, 65536, 64, 3200], hot=(0, 2))
    cur = [c[1] for c in chs]
    nid = [c[1].n for c in chs]
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    stats = obem.new_batch_stats(len(sizes))
    try:
        for s in range(3):
            Ein = np.zeros((st.capacity, 4), np.float32)
            for k, (mesh, _, trk, sigma) in enumerate(chs):
                if cur[k].n:
                    o = int(b.seg_off[k])
                    Ein[o:o + cur[k].n, :3] = _oracle_field(mesh, sigma, cur[k]).astype(np.float32)
            b.step(st, step, stats, E_in=to_dev(Ein))
            torch.cuda.synchronize()
            gs = obem.read_batch_stats(stats, len(sizes))
            got = st.download()
            for k, (mesh, _, trk, sigma) in enumerate(chs):
                if cur[k].n == 0:
                    assert got[k][0].n == 0 and gs[k]["status"] == 0 and gs[k]["n_after"] == 0
                    continue
                cap = int(b.seg_off[k + 1] - b.seg_off[k])
                Ek = Ein[int(b.seg_off[k]):int(b.seg_off[k]) + cur[k].n, :3]
                rc, cur[k], nid[k], os_ = oracle.step(cur[k], Ek, s, nid[k], gas, trk, capacity=cap)
                assert rc == 0 and gs[k]["status"] == 0, (k, rc, gs[k]["status"])
                _assert_same(got[k][0], cur[k], k)
                assert got[k][1] == nid[k], k
                for key in COUNT_KEYS:
                    assert int(gs[k][key]) == int(os_[key]), (s, k, key, gs[k][key], os_[key])
            assert int(step.item()) == s + 1
        assert cur[0].n > sizes[0] and cur[2].n > sizes[2]          # the hot chambers spawned
    finally:
        _close(ctx, b)


def test_batch_graph_replays_the_fused_step():
    """The fused step captured once in a CUDA graph and replayed four times
    leaves the same bits as four plain calls (the step index advances on the
    device)."""
    sizes = [500, 1300, 90]
    ctx, b, st, chs, _ = _setup(sizes, seed=9, caps=[4096, 65536, 1024], hot=(1,))
    st2 = b.state()
    st2.upload([c[1] for c in chs])
    s1 = torch.zeros(1, dtype=torch.int32, device="cuda")
    s2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    stats1, stats2 = obem.new_batch_stats(3), obem.new_batch_stats(3)
    try:
        for _ in range(4):
            b.step(st, s1, stats1)
            b.step_graph(st2, s2, stats2)
        torch.cuda.synchronize()
        a, c = st.download(), st2.download()
        g1, g2 = obem.read_batch_stats(stats1, 3), obem.read_batch_stats(stats2, 3)
    finally:
        _close(ctx, b)
    assert int(s1.item()) == 4 and int(s2.item()) == 4
    for k in range(3):
        _assert_same(a[k][0], c[k][0], k)
        assert a[k][1] == c[k][1]
        assert g1[k]["status"] == 0 and g2[k]["status"] == 0
        for key in COUNT_KEYS:
            assert g1[k][key] == g2[k][key], (k, key)


def test_batch_all_or_nothing():
    """A chamber whose step would overflow its segment (1024 hot electrons in a
    1024-slot segment) stops the whole batch: no state changes, the step index
    stays, the failing chamber reports OBEM_ERR_CAPACITY with the capacity it
    needed, the others OBEM_ERR_STATE."""
    sizes = [200, 1024, 50]
    ctx, b, st, chs, _ = _setup(sizes, seed=11, caps=[400, 1024, 100], hot=(1,), electrons=(1,))
    before = [x[0] for x in st.download()]
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    stats = obem.new_batch_stats(3)
    try:
        b.step(st, step, stats)
        torch.cuda.synchronize()
        gs = obem.read_batch_stats(stats, 3)
        after = [x[0] for x in st.download()]
    finally:
        _close(ctx, b)
    assert gs[1]["status"] == obem.OBEM_ERR_CAPACITY and gs[1]["required_capacity"] > 1024
    assert gs[0]["status"] == obem.OBEM_ERR_STATE and gs[2]["status"] == obem.OBEM_ERR_STATE
    assert int(step.item()) == 0
    for k in range(3):
        _assert_same(before[k], after[k], k)
        assert gs[k]["n_after"] == gs[k]["n_before"] == sizes[k]


def test_batch_autotune_and_block_sizes():
    """The autotuner keeps one of 128 / 256 / 512 targets per cell block; every
    block size gives the field within tolerance."""
    sizes = [900, 2100]
    ctx, b, st, chs, _ = _setup(sizes, seed=13)
    try:
        r = b.autotune(st, reps=2)
        assert r["cells_per_block"] in (128, 256, 512) and r["ms"] > 0
        fields = {}
        for cut in (64, 128, 512):
            b.set_block(cut)
            fields[cut] = _gpu_field(b, st)
        with pytest.raises(obem.ObemError):
            b.set_block(16)
    finally:
        _close(ctx, b)
    for k, (mesh, ch, trk, sigma) in enumerate(chs):
        o, n = int(b.seg_off[k]), sizes[k]
        ref = _oracle_field(mesh, sigma, ch)
        for cut, got in fields.items():
            assert guarded_rel_err(got[o:o + n, :3], ref) <= FIELD_TOL, (k, cut)


def test_batch_swarm_parameters_vs_oracle():
    """Per chamber, drift velocity, longitudinal diffusion and Townsend
    coefficient from the batched run's step statistics against the oracle's
    run of the same chamber (its own FP64 field every step): within three
    statistical sigma (the runs draw the same numbers).  Plummer length
    0.1 um: with 1 nm, the pair an ionisation places ~1 nm apart (Eq.
    (distIoni)) holds its electron in a ~1e9 V/m step-start field for the whole
    1 ps step and the avalanche runs away (in the oracle as on the GPU)."""
    SOFT = 1e-7
    rng = np.random.default_rng(21)
    chs, gaps = [], [1.0e-3, 2.0e-3]
    for k, (gap, e) in enumerate(zip(gaps, [15.0, 25.0])):
        mesh = inputs.parallel_plates(1e-2, gap, 4, 0.0, e * 1e5 * gap)
        # a 50 um cloud: its own field (~1 kV/cm) stays small against the applied one
        pos = inputs.gaussian_ball(rng, 200, (5e-3, 5e-3, 0.3 * gap), 50e-6)
        ch = inputs.make_charges(pos, inputs.maxwellian(rng, 200, 1.0, ME), np.zeros(200, np.uint8))
        trk = inputs.Tracking(dt=1e-12, seed=1 + k, z_lo=0.0, z_hi=gap, beta=1e-13, softening=SOFT)
        chs.append((mesh, ch, trk, oracle.bem_solve(mesh)))
    gas = inputs.argon_like_gas()
    ctx = obem.obem_create(capacity=16, dt=1e-12, softening=SOFT, beta=1e-13,
                           flags=obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD)
    obem.obem_gas_load(ctx, gas)
    steps = 60
    b = obem.Batch(ctx, [16384, 16384], [0.0, 0.0], gaps, [1, 2])
    try:
        for k, c in enumerate(chs):
            b.cells(k, c[0].tri, c[3].astype(np.float32))
        st = b.state()
        st.upload([c[1] for c in chs])
        step = torch.zeros(1, dtype=torch.int32, device="cuda")
        stats = obem.new_batch_stats(2)
        hist = [[], []]
        for _ in range(steps):
            b.step_graph(st, step, stats)
            for k, g in enumerate(obem.read_batch_stats(stats, 2)):
                assert g["status"] == 0
                hist[k].append(g)
    finally:
        _close(ctx, b)
    for k, (mesh, ch, trk, sigma) in enumerate(chs):
        _, _, ohist = oracle.run(ch, gas, trk, steps, mesh=mesh, sigma=sigma.astype(np.float32).astype(np.float64),
                                 capacity=16384)
        t = trk.dt * (1.0 + np.arange(steps))
        n_o, mean_o, var_o = oracle.cloud_moments(ohist)
        vd_o = oracle.drift_velocity(t, mean_o[:, 2])
        dl_o = oracle.diffusion_coefficient(t, var_o[:, 2])
        al_o = oracle.townsend_alpha(t, n_o, vd_o)
        vd, dl, al = swarm.swarm_params(hist[k], trk.dt)
        n_g, mean_g, var_g = swarm.electron_moments(hist[k])
        # statistical scale of each fit: spread of the cloud over the run
        T = t[-1] - t[0]
        s_vd = np.sqrt(var_o[-1, 2] / n_o[-1]) / T
        s_dl = var_o[-1, 2] * np.sqrt(2.0 / n_o[-1]) / T
        s_al = 1.0 / (np.sqrt(n_o.min()) * T * abs(vd_o))
        assert vd > 0 and abs(vd - vd_o) <= 3 * s_vd, (k, vd, vd_o, s_vd)
        assert abs(dl - dl_o) <= 3 * s_dl, (k, dl, dl_o, s_dl)
        assert abs(al - al_o) <= 3 * s_al, (k, al, al_o, s_al)
