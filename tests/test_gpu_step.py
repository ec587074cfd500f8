"""obem_step (CUDA, through the C ABI) against the oracle's binary32 step.

Given the same field, every decision and every bit of the new state must
match: positions, velocities, ids, births, species, spawn/absorb/attach/
recombination counts, trial counts.  The fused path (field evaluated inside
obem_step) is compared with tolerance, and swarm parameters of independent
seeds within 3 statistical sigma."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem
from gpu_util import pts4, to_dev

pytestmark = pytest.mark.gpu
E = 1.602176634e-19
ME = 9.1093837015e-31
COUNT_KEYS = ["n_after", "spawned_pairs", "absorbed", "attached", "recombined_pairs",
              "collisions", "trials", "n_electron", "n_cation", "n_anion"]


class GpuRun:
    def __init__(self, gas, trk, capacity, flags=0, mesh=None, e_ext=(0.0, 0.0, 0.0)):
        self.ctx = obem.obem_create(capacity=capacity, dt=trk.dt, seed=trk.seed,
                                    softening=trk.softening, z_lo=trk.z_lo, z_hi=trk.z_hi,
                                    beta=trk.beta, trial_cap=trk.trial_cap, flags=flags,
                                    e_ext=e_ext)
        obem.obem_gas_load(self.ctx, gas)
        self.mesh = mesh
        if mesh is not None:
            obem.obem_mesh_load(self.ctx, mesh)
        self.st = obem.DeviceState(capacity)
        self.stats = obem.new_stats()
        self.cap = capacity

    def solve(self):
        sig = torch.empty(self.mesh.n, dtype=torch.float32, device="cuda")
        obem.obem_bem_assemble(self.ctx, obem.OBEM_LU_FP32)
        rep = obem.obem_bem_solve(self.ctx, self.mesh.group_voltage, sig)
        return sig.cpu().numpy(), rep

    def upload(self, ch, next_id=None):
        self.st.upload(ch, next_id)

    def step(self, s, E_in=None):
        Ed = None
        if E_in is not None:
            buf = np.zeros((self.cap, 4), np.float32)
            buf[:len(E_in), :3] = E_in[:, :3]
            Ed = to_dev(buf)
        obem.obem_step(self.ctx, self.st, s, self.stats, E_in=Ed)
        torch.cuda.synchronize()
        return obem.read_stats(self.stats)

    def state(self):
        return self.st.download()

    def close(self):
        obem.obem_destroy(self.ctx)


def _assert_same_state(a, b):
    assert a.pos_q.shape == b.pos_q.shape, (a.pos_q.shape, b.pos_q.shape)
    for k in ("pos_q", "vel"):
        x, y = getattr(a, k), getattr(b, k)
        bad = np.flatnonzero(~np.all(x.view(np.uint32) == y.view(np.uint32), axis=1))
        assert bad.size == 0, "%s differs at %s: %s vs %s" % (k, bad[:5], x[bad[:2]], y[bad[:2]])
    for k in ("id", "birth", "species"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k


def _assert_same_counts(gs, os_):
    for k in COUNT_KEYS:
        assert int(gs[k]) == int(os_[k]), (k, gs[k], os_[k])
    assert gs["status"] == 0


MOMENT_KEYS = [("sum_e", "sum_%s_e", False), ("sum2_e", "sum_%s2_e", True),
               ("sum_i", "sum_%s_i", False), ("sum2_i", "sum_%s2_i", True)]


def _assert_same_moments(gs, os_, cur):
    """The FP64 observables of the step (Sec. 4.1: the cloud moments that the
    swarm parameters are fitted to) against the oracle's, per species and
    axis.  Both sum the same binary32 values in FP64, in different orders, so
    they agree to FP64 rounding of the sum of the terms' magnitudes."""
    pos = np.asarray(cur.pos_q[:, :3], np.float64)
    el = cur.species == 0
    for gk, ok, sq in MOMENT_KEYS:
        sel = el if gk.endswith("_e") else ~el
        terms = pos[sel] ** 2 if sq else np.abs(pos[sel])
        for a, ax in enumerate("xyz"):
            scale = terms[:, a].sum() + 1e-300
            assert abs(gs[gk][a] - os_[ok % ax]) <= 1e-12 * scale, (gk, ax, gs[gk][a], os_[ok % ax])
    v = np.asarray(cur.vel[el, :3], np.float64)
    en = (0.5 * ME * (v ** 2).sum(1) / E).sum() + 1e-300
    assert abs(gs["sum_energy_e"] - os_["sum_energy_e"]) <= 1e-12 * en


def _run_pair(ch, gas, trk, E_fn, steps, capacity, next_id=None, flags=0):
    g = GpuRun(gas, trk, capacity, flags=flags)
    try:
        g.upload(ch, next_id)
        cur, nid = ch, (ch.pos_q.shape[0] if next_id is None else next_id)
        for s in range(steps):
            Ef = E_fn(cur).astype(np.float32)
            gs = g.step(s, Ef)
            st, cur, nid, os_ = oracle.step(cur, Ef, s, nid, gas, trk, capacity)
            assert st == 0
            gst, gnid = g.state()
            _assert_same_state(gst, cur)
            assert gnid == nid
            _assert_same_counts(gs, os_)
            _assert_same_moments(gs, os_, cur)
        return cur
    finally:
        g.close()


def test_maxwell_plates_bit_exact_20_steps():
    """The small plain-method chamber: oracle field (cells + charges) fed to
    both sides, 20 steps, identical states."""
    mesh, gas, ch, trk = inputs.config_small_plates(seed=1, n=1000)
    sig = oracle.bem_solve(mesh)
    trk.softening = 1e-9
    E_fn = lambda c: oracle.field_at_charges(c, mesh, sig, trk.softening)
    _run_pair(ch, gas, trk, E_fn, 20, 1200)


def _hot_mixture(seed, n_e=1500, n_i=600, close_pairs=150):
    rng = np.random.default_rng(seed)
    pe = rng.uniform([0, 0, 2e-4], [1e-3, 1e-3, 1.8e-3], (n_e, 3))
    pi = rng.uniform([0, 0, 2e-4], [1e-3, 1e-3, 1.8e-3], (n_i, 3))
    pi[:close_pairs] = pe[:close_pairs] + rng.normal(0, 1.2e-9, (close_pairs, 3))
    ve = inputs.maxwellian(rng, n_e, 8.0, ME)
    vi = inputs.maxwellian(rng, n_i, 0.025, 40 * 1.66053906660e-27)
    sp = np.concatenate([np.zeros(n_e, np.uint8), np.ones(n_i, np.uint8)])
    perm = rng.permutation(n_e + n_i)
    ch = inputs.make_charges(np.concatenate([pe, pi])[perm], np.concatenate([ve, vi])[perm], sp[perm])
    ch.birth[:] = np.where(rng.random(n_e + n_i) < 0.1, 3, 0).astype(np.uint32)
    return ch


def test_argon_like_ionisation_attachment_recombination_bit_exact():
    """Hot electrons in the synthetic argon-like gas at 30 kV/cm: elastic,
    excitation, ionisation (spawns), attachment (anions), recombination with
    close cations (some exempt as fresh), absorption at the planes."""
    gas = inputs.argon_like_gas()
    trk = inputs.Tracking(dt=1e-12, seed=5, z_lo=0.0, z_hi=2e-3, beta=1e-13)
    ch = _hot_mixture(5)
    rng = np.random.default_rng(9)
    base = np.array([0.0, 0.0, -3e6])
    E_fn = lambda c: base[None, :] + rng.normal(0, 2e5, (c.pos_q.shape[0], 3))
    fin = _run_pair(ch, gas, trk, E_fn, 8, 8000, next_id=ch.n + 100)
    assert fin.pos_q.shape[0] > 0


@pytest.mark.parametrize("gas_kind", ["maxwell", "argon"])
def test_per_step_probability_scheme_bit_exact(gas_kind):
    """OBEM_STEP_PROB_COLLISION (the paper's own collision sampling, one
    interaction test per step) against the oracle's same scheme: identical
    states, decisions and counts."""
    if gas_kind == "maxwell":
        mesh, gas, ch, trk = inputs.config_small_plates(seed=2, n=1000)
        trk.softening = 1e-9
        trk.coll_mode = 1
        sig = oracle.bem_solve(mesh)
        E_fn = lambda c: oracle.field_at_charges(c, mesh, sig, trk.softening)
        _run_pair(ch, gas, trk, E_fn, 15, 1200, flags=obem.OBEM_STEP_PROB_COLLISION)
    else:
        gas = inputs.argon_like_gas()
        trk = inputs.Tracking(dt=1e-13, seed=7, z_lo=0.0, z_hi=2e-3, beta=1e-13, coll_mode=1)
        ch = _hot_mixture(7)
        rng = np.random.default_rng(11)
        base = np.array([0.0, 0.0, -3e6])
        E_fn = lambda c: base[None, :] + rng.normal(0, 2e5, (c.pos_q.shape[0], 3))
        fin = _run_pair(ch, gas, trk, E_fn, 8, 8000, next_id=ch.n + 100, flags=obem.OBEM_STEP_PROB_COLLISION)
        assert fin.pos_q.shape[0] > 0


def test_exempt_and_tie_rules_on_gpu():
    gas = inputs.maxwell_gas(0.0, 40.0)
    gas.nuc[:] = 0.0
    gas.nu_ion = 0.0
    trk = inputs.Tracking(dt=1e-12, seed=1, z_lo=-1, z_hi=1, beta=1e-13)
    rc = (3 * 1e-13 * 1e-12 / (4 * math.pi)) ** (1 / 3)
    x = np.float32(1e-3)
    pos = np.array([[x, 0, 0], [x + 0.5 * rc, 0, 0], [x - 0.3 * rc, 0, 0], [x - 0.5 * rc, 0, 0],
                    [0, 1e-3, 0], [0.4 * rc, 1e-3, 0], [-0.4 * rc, 1e-3, 0], [0, 0, 1e-3],
                    [0.1 * rc, 0, 1e-3]], np.float64)
    sp = np.array([0, 1, 0, 1, 0, 1, 1, 0, 1], np.uint8)
    ch = inputs.make_charges(pos, np.zeros((9, 3)), sp)
    ch.birth[8] = 5
    g = GpuRun(gas, trk, 16)
    try:
        g.upload(ch)
        gs = g.step(5, np.zeros((9, 3), np.float32))
        out, _ = g.state()
    finally:
        g.close()
    assert gs["recombined_pairs"] == 3
    assert sorted(out.id.tolist()) == [6, 7, 8]


@pytest.mark.parametrize("n", [9, 1500, 5000])
def test_fused_partner_search_matches_oracle(n):
    """Recombination partners proposed inside the fused all-pairs kernel (the
    symmetric one: each pair once, both directions of the partner rule):
    binary32 positions alone decide them, so the charges removed must be
    exactly the oracle's, whatever the field."""
    gas = inputs.maxwell_gas(0.0, 40.0)
    gas.nuc[:] = 0.0
    gas.nu_ion = 0.0
    trk = inputs.Tracking(dt=1e-12, seed=1, z_lo=-1, z_hi=1, beta=1e-13)
    trk.softening = 1e-9
    rc = (3 * 1e-13 * 1e-12 / (4 * math.pi)) ** (1 / 3)
    rng = np.random.default_rng(n)
    ne = (n + 1) // 2
    pe = rng.uniform(0, 5e-5, (ne, 3))
    pc = rng.uniform(0, 5e-5, (n - ne, 3))
    k = (n - ne) // 2
    near = rng.integers(0, ne, k)
    off = rng.normal(0, 1.0, (k, 3))
    off *= (rng.uniform(0.2, 1.3, k) * rc / np.linalg.norm(off, axis=1))[:, None]
    pc[:k] = pe[near] + off
    pos = np.concatenate([pe, pc])
    perm = rng.permutation(n)                  # electrons and cations interleaved in memory
    sp = np.concatenate([np.zeros(ne, np.uint8), np.ones(n - ne, np.uint8)])[perm]
    ch = inputs.make_charges(pos[perm], np.zeros((n, 3)), sp)
    cap = n + 16
    g = GpuRun(gas, trk, cap, flags=obem.OBEM_STEP_SPACE_CHARGE)
    try:
        g.upload(ch)
        gs = g.step(5)
        out, _ = g.state()
    finally:
        g.close()
    p64 = ch.pos_q.astype(np.float64)
    Eo = oracle.nbody_field(p64[:, :3], p64, True, trk.softening)[0].astype(np.float32)
    st, cur, _, os_ = oracle.step(ch, Eo, 5, n, gas, trk, cap)
    assert st == 0 and gs["status"] == 0
    assert gs["recombined_pairs"] == os_["recombined_pairs"] > 0
    assert np.array_equal(np.sort(out.id), np.sort(cur.id))


def test_capacity_overflow_is_all_or_nothing():
    gas = inputs.maxwell_gas(1e12, 40.0)
    gas.kind = np.array([inputs.P_IONISATION], np.int32)
    gas.nuc = np.array([5e11], np.float32)
    gas.T = 0.0
    trk = inputs.Tracking(dt=1e-12, seed=2, z_lo=-1, z_hi=1, beta=-1)
    rng = np.random.default_rng(0)
    n = 100
    ch = inputs.make_charges(rng.uniform(0, 1e-3, (n, 3)), inputs.maxwellian(rng, n, 5.0, ME),
                             np.zeros(n, np.uint8))
    g = GpuRun(gas, trk, n + 4)
    try:
        g.upload(ch)
        before = g.state()[0]
        gs = g.step(0, np.zeros((n, 3), np.float32))
        after = g.state()[0]
    finally:
        g.close()
    st, _, _, os_ = oracle.step(ch, np.zeros((n, 3), np.float32), 0, n, gas, trk, n + 4)
    assert st == oracle.ST_CAPACITY
    assert gs["status"] == obem.OBEM_ERR_CAPACITY
    assert gs["required_capacity"] == int(os_["required_capacity"]) > n + 4
    _assert_same_state(after, before)


def test_trial_cap_overflow_reports_and_commits_nothing():
    gas = inputs.maxwell_gas(1e14, 0.0)
    trk = inputs.Tracking(dt=1e-12, seed=2, z_lo=-1, z_hi=1, beta=-1, trial_cap=20)
    rng = np.random.default_rng(1)
    ch = inputs.make_charges(rng.uniform(0, 1e-3, (50, 3)), inputs.maxwellian(rng, 50, 1.0, ME),
                             np.zeros(50, np.uint8))
    g = GpuRun(gas, trk, 64)
    try:
        g.upload(ch)
        gs = g.step(0, np.zeros((50, 3), np.float32))
        after = g.state()[0]
    finally:
        g.close()
    assert gs["status"] == obem.OBEM_ERR_TRIALS
    _assert_same_state(after, ch)


def test_empty_state_step():
    gas = inputs.maxwell_gas(1e12, 0.0)
    trk = inputs.Tracking()
    g = GpuRun(gas, trk, 8)
    try:
        ch = inputs.make_charges(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.uint8))
        g.upload(ch)
        gs = g.step(0)
        out, nid = g.state()
    finally:
        g.close()
    assert gs["status"] == 0 and out.n == 0 and nid == 0


def test_uniform_field_many_steps_bit_exact():
    """Field-free of charges: the uniform external field is the whole field on
    both sides, so 120 steps of an avalanche stay identical."""
    gas = inputs.argon_like_gas()
    trk = inputs.Tracking(dt=1e-12, seed=3, z_lo=-1.0, z_hi=1.0, beta=-1.0)
    rng = np.random.default_rng(4)
    n = 300
    ch = inputs.make_charges(np.zeros((n, 3)) + [0, 0, 1e-4], inputs.maxwellian(rng, n, 0.1, ME),
                             np.zeros(n, np.uint8))
    Eext = (0.0, 0.0, -3e6)
    g = GpuRun(gas, trk, 40000, flags=0, e_ext=Eext)
    try:
        g.upload(ch)
        cur, nid = ch, n
        Ef = np.array(Eext, np.float32)
        for s in range(120):
            gs = g.step(s)
            st, cur, nid, os_ = oracle.step(cur, np.tile(Ef, (cur.pos_q.shape[0], 1)), s, nid, gas, trk, 40000)
            assert st == 0
            _assert_same_counts(gs, os_)
            _assert_same_moments(gs, os_, cur)
        gst, gnid = g.state()
        _assert_same_state(gst, cur)
        assert gnid == nid and cur.pos_q.shape[0] > n
    finally:
        g.close()


def test_fused_field_step_matches_oracle_run():
    """obem_step evaluating the field itself (BEM cells with the GPU-solved
    sigma + softened all-pairs field): after 5 steps the states agree within
    the field tolerance (decisions are identical for almost all charges)."""
    mesh, gas, ch, trk = inputs.config_small_plates(seed=3, n=1000)
    trk.softening = 1e-9
    g = GpuRun(gas, trk, 1200, flags=obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD, mesh=mesh)
    try:
        sig_gpu, rep = g.solve()
        g.upload(ch)
        for s in range(5):
            g.step(s)
        gst, _ = g.state()
    finally:
        g.close()
    sig = oracle.bem_solve(mesh)
    fin, _, _ = oracle.run(ch, gas, trk, 5, mesh, sig)
    common, ia, ib = np.intersect1d(gst.id, fin.id, return_indices=True)
    assert len(common) >= 0.99 * max(len(gst.id), len(fin.id))
    assert (gst.species[ia] == fin.species[ib]).mean() >= 0.99
    # the two fields differ at the 1e-6 level, so velocities differ in their
    # last bits; a charge whose collision decisions were the same has a
    # velocity within ~1e-4 relative, one with a flipped decision a random one
    vg = gst.vel[ia, :3].astype(float)
    vo = fin.vel[ib, :3].astype(float)
    rel = np.linalg.norm(vg - vo, axis=1) / np.maximum(np.linalg.norm(vo, axis=1), 1.0)
    same = rel < 1e-3
    assert same.mean() > 0.97
    d = np.abs(gst.pos_q[ia, :3].astype(float) - fin.pos_q[ib, :3].astype(float)).max(axis=1)
    assert np.quantile(d[same], 0.99) < 1e-9


def _swarm(run_fn, seeds):
    vd, dl, dt, alpha = [], [], [], []
    for sd in seeds:
        hist = run_fn(sd)
        n = np.array([h["n_electron"] for h in hist], float)
        mean = np.array([h["sum_e"] for h in hist]) / n[:, None]
        var = np.array([h["sum2_e"] for h in hist]) / n[:, None] - mean ** 2
        t = (np.arange(len(hist)) + 1) * 1e-12
        sl = slice(len(hist) // 3, None)
        v = oracle.drift_velocity(t[sl], mean[sl, 2])
        vd.append(v)
        dl.append(oracle.diffusion_coefficient(t[sl], var[sl, 2]))
        dt.append(oracle.diffusion_coefficient(t[sl], 0.5 * (var[sl, 0] + var[sl, 1])))
        alpha.append(oracle.townsend_alpha(t[sl], n[sl], v))
    return [np.array(x) for x in (vd, dl, dt, alpha)]


def test_swarm_parameters_agree_within_3_sigma():
    """Drift velocity, longitudinal / transverse diffusion and the effective
    Townsend coefficient (Eqs. (vd), (diffusion), (townsend)) from independent
    seeds on the GPU and in the oracle (16 per side): means agree within
    3 sigma."""
    gas = inputs.argon_like_gas()
    Ez = -6e6
    steps, n0 = 150, 400

    def cloud(sd):
        rng = np.random.default_rng(sd)
        return inputs.make_charges(np.zeros((n0, 3)), inputs.maxwellian(rng, n0, 0.5, ME),
                                   np.zeros(n0, np.uint8))

    def gpu(sd):
        trk = inputs.Tracking(dt=1e-12, seed=sd, z_lo=-1.0, z_hi=1.0, beta=-1.0)
        g = GpuRun(gas, trk, 200000, flags=0, e_ext=(0, 0, Ez))
        try:
            g.upload(cloud(sd))
            return [g.step(s) for s in range(steps)]
        finally:
            g.close()

    def ora(sd):
        trk = inputs.Tracking(dt=1e-12, seed=sd, z_lo=-1.0, z_hi=1.0, beta=-1.0)
        hist = oracle.run(cloud(sd), gas, trk, steps, space_charge=False, e_ext=np.array([0, 0, Ez]),
                          capacity=200000)[2]
        return [{"n_electron": h["n_electron"], "sum_e": [h["sum_x_e"], h["sum_y_e"], h["sum_z_e"]],
                 "sum2_e": [h["sum_x2_e"], h["sum_y2_e"], h["sum_z2_e"]]} for h in hist]

    G = _swarm(gpu, list(range(101, 117)))
    O = _swarm(ora, list(range(201, 217)))
    for g_, o_ in zip(G, O):
        se = math.sqrt(g_.var(ddof=1) / len(g_) + o_.var(ddof=1) / len(o_))
        assert abs(g_.mean() - o_.mean()) <= 3 * se + 1e-12 * abs(o_.mean()), (g_, o_)
    assert np.all(G[0] > 0)


def test_checkpoint_resume_bit_identical():
    """Checkpoint / resume: the charge arrays, next_id and the step index are
    the whole state (draws are keyed by id and step).  Six fused steps (cells
    + all-pairs field evaluated inside obem_step, ionisation, recombination)
    equal three steps, a host copy of the state, a new context loaded with it,
    and three more steps -- bit for bit."""
    mesh, gas, _, trk = inputs.config_avalanche(seed=4, e_kv_cm=30.0, n_seed=100, n_plate=8)
    ch = _hot_mixture(4)
    trk.softening = 1e-7
    flags = obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD

    def run(steps, start, state, nid):
        g = GpuRun(gas, trk, 16384, flags=flags, mesh=mesh)
        try:
            g.solve()
            g.upload(state, nid)
            for s in range(start, start + steps):
                last = g.step(s)
                assert last["status"] == 0
            return g.state(), last
        finally:
            g.close()

    (full, nid_full), st_full = run(6, 0, ch, ch.n)
    (half, nid_half), _ = run(3, 0, ch, ch.n)
    (resumed, nid_res), st_res = run(3, 3, half, nid_half)
    _assert_same_state(full, resumed)
    assert nid_full == nid_res and full.n > ch.n
    # the step's observables too: FP64 moments are folded in block order
    for k in ("sum_e", "sum2_e", "sum_i", "sum2_i"):
        assert st_full[k] == st_res[k], k
    assert st_full["sum_energy_e"] == st_res["sum_energy_e"]


def test_batch_checkpoint_resume_bit_identical():
    """The same for a batch of chambers: the concatenated arrays, per-chamber
    n / next_id and the device step index, saved to the host after two steps
    and loaded into a new batch, continue exactly as the uninterrupted run."""
    gas = inputs.argon_like_gas()
    chs = []
    for k, gap in enumerate([1e-3, 2e-3, 1.5e-3]):
        mesh = inputs.parallel_plates(1e-2, gap, 4, 0.0, 25.0 * 1e5 * gap)
        rng = np.random.default_rng(30 + k)
        c = inputs.avalanche_snapshot(rng, [300, 1200, 50][k], gap=gap)
        c.pos_q[:, 2] = np.clip(c.pos_q[:, 2], 0.05 * gap, 0.95 * gap).astype(np.float32)
        chs.append((mesh, c, gap, oracle.bem_solve(mesh).astype(np.float32)))
    ctx = obem.obem_create(capacity=16, dt=1e-12, softening=1e-7, beta=1e-13,
                           flags=obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD)
    obem.obem_gas_load(ctx, gas)

    def batch():
        b = obem.Batch(ctx, [4096] * 3, [0.0] * 3, [c[2] for c in chs], [11, 12, 13])
        for k, c in enumerate(chs):
            b.cells(k, c[0].tri, c[3])
        return b

    def steps(b, st, step, n):
        stats = obem.new_batch_stats(3)
        for _ in range(n):
            b.step_graph(st, step, stats)
        torch.cuda.synchronize()
        assert all(g["status"] == 0 for g in obem.read_batch_stats(stats, 3))

    try:
        b1 = batch()
        st1 = b1.state()
        st1.upload([c[1] for c in chs])
        s1 = torch.zeros(1, dtype=torch.int32, device="cuda")
        steps(b1, st1, s1, 4)
        full = st1.download()
        b1.destroy()
        b2 = batch()
        st2 = b2.state()
        st2.upload([c[1] for c in chs])
        s2 = torch.zeros(1, dtype=torch.int32, device="cuda")
        steps(b2, st2, s2, 2)
        ckpt = st2.download(), int(s2.item())                 # host checkpoint
        b2.destroy()
        b3 = batch()
        st3 = b3.state()
        st3.upload([x[0] for x in ckpt[0]], next_ids=[x[1] for x in ckpt[0]])
        s3 = torch.full((1,), ckpt[1], dtype=torch.int32, device="cuda")
        steps(b3, st3, s3, 2)
        res = st3.download()
        b3.destroy()
    finally:
        obem.obem_destroy(ctx)
    assert int(s3.item()) == 4
    for k in range(3):
        _assert_same_state(full[k][0], res[k][0])
        assert full[k][1] == res[k][1]
