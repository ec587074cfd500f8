"""Pins of the oracle's tabulated cross-section path (Sec. 3.3.1, 3.3.3):
table lookup and linear interpolation in energy, thresholds, the null-collision
majorant, and the energetics of excitation and ionisation.

Every expectation here is computed in FP64 from the gas definition itself
(numpy interpolation, closed-form rates of a Poisson process, the energy
balance of Sec. 3.3.3), never from the oracle's own arithmetic, so that a
wrong grid segment, a wrong interpolation weight, a threshold compared the
wrong way, a majorant taken at the wrong end of a segment or a wrong energy
loss each fails one of them.  CPU only."""
import math

import numpy as np

import oracle
from paper_2110_09214_gb300 import inputs

E = 1.602176634e-19
ME = 9.1093837015e-31
KB = 1.380649e-23
AMU = 1.66053906660e-27
KC = 8.9875517923e9
N_GAS = 2.4143e25


def _table_gas(egrid, rows, kinds, thr, T=0.0, M_amu=0.0):
    n_p = len(rows)
    return inputs.Gas(np.asarray(egrid, np.float32), np.asarray(rows, np.float32),
                      np.asarray(kinds, np.int32), np.full(n_p, inputs.MODE_TABLE, np.int32),
                      np.asarray(thr, np.float32), np.zeros(n_p, np.float32), N=N_GAS, T=T,
                      M_amu=M_amu, nu_ion=0.0)


def _open(dt, seed):
    return inputs.Tracking(dt=dt, seed=seed, z_lo=-1.0, z_hi=1.0, beta=-1.0)


def _speed(eps_eV):
    return np.sqrt(2.0 * np.asarray(eps_eV, np.float64) * E / ME)


def _iso(rng, n):
    d = rng.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1)[:, None]


def _electrons_at(eps_eV, rng, spread=1e-4):
    eps = np.asarray(eps_eV, np.float64)
    n = len(eps)
    vel = _speed(eps)[:, None] * _iso(rng, n)
    pos = rng.uniform(-spread, spread, (n, 3))
    return inputs.make_charges(pos, vel, np.zeros(n, np.uint8))


def _energy_eV(vel):
    v = np.asarray(vel, np.float64)[:, :3]
    return 0.5 * ME * (v ** 2).sum(1) / E


def _energy32(vel, K_e):
    """The binary32 energy K_e (vx^2 + vy^2 + vz^2) that the step's decisions
    are taken on (one rounding per operation, left to right)."""
    v = np.asarray(vel, np.float32)[:, :3]
    v2 = (v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2]
    return (np.float32(K_e) * v2).astype(np.float64)


def _sigma_interp(gas, j, eps):
    """sigma_j at energy eps: linear in energy between grid points, held at the
    end values outside the grid, zero below the process threshold."""
    eg = gas.egrid.astype(np.float64)
    s = np.interp(eps, eg, gas.xs[j].astype(np.float64))
    return np.where(eps < float(gas.thr[j]), 0.0, s)


def _majorant_dense(gas, samples_per_segment=400):
    """max over the grid of N sigma_tot(E) v(E), sampled densely (FP64)."""
    eg = gas.egrid.astype(np.float64)
    t = np.linspace(0.0, 1.0, samples_per_segment)
    Es = (eg[:-1, None] + t[None, :] * (eg[1:] - eg[:-1])[:, None]).ravel()
    tot = sum(_sigma_interp(gas, j, Es) for j in range(gas.n_proc))
    return float((N_GAS * tot * _speed(Es)).max())


# ----------------------------------------------------------------------------
# 1. a table that makes nu constant reproduces the Maxwell model
# ----------------------------------------------------------------------------
def _const_nu_table_gas(nu0, n_e=2000):
    eg = (1e-6 * 10.0 ** (9.0 * np.arange(n_e) / (n_e - 1))).astype(np.float32)   # 1 ueV .. 1 keV
    sig = nu0 / (N_GAS * _speed(eg.astype(np.float64)))
    return _table_gas(eg, [sig], [inputs.P_ELASTIC], [0.0])


def test_table_with_sigma_nu0_over_Nv_gives_the_maxwell_drift():
    """sigma(E) = nu0 / (N v(E)) tabulated: the interpolated collision
    frequency is nu0 (to the interpolation error of E^-1/2 on the grid,
    < 1e-5), so with isotropic speed-keeping scattering the mean velocity
    obeys d<v_z>/dt = a - nu0 <v_z>: <v_z>(t) = (a/nu0)(1 - exp(-nu0 t))
    for a cloud with <v_z>(0) = 0."""
    nu0, Ez, n = 1e12, -1e6, 20000
    gas = _const_nu_table_gas(nu0)
    rng = np.random.default_rng(21)
    ch = inputs.make_charges(rng.uniform(-1e-4, 1e-4, (n, 3)), inputs.maxwellian(rng, n, 0.1, ME),
                             np.zeros(n, np.uint8))
    ch.vel[:, :3] -= ch.vel[:, :3].mean(0)                  # <v>(0) = 0 exactly
    trk = _open(1e-12, 17)
    a = E * -Ez / ME
    nid = n
    for s in range(6):
        field = np.tile(np.array([0, 0, Ez], np.float32), (ch.n, 1))
        st, ch, nid, stats = oracle.step(ch, field, s, nid, gas, trk)
        assert st == 0
        vz = ch.vel[:, 2].astype(np.float64)
        want = a / nu0 * (1 - math.exp(-nu0 * (s + 1) * 1e-12))
        assert abs(vz.mean() - want) < 4 * vz.std() / math.sqrt(n) + 1e-3 * want, (s, vz.mean(), want)


def test_table_constant_nu_trials_and_real_collisions():
    """Same table: trials per step ~ Poisson(nu_max dt) with nu_max the bound
    of the grid segments, nu0 sqrt(E_i+1 / E_i) (sigma_i v_i = nu0 / N on the
    grid); the real-collision share of the trials is nu0 / nu_max."""
    nu0, n = 1e12, 20000
    gas = _const_nu_table_gas(nu0)
    eg = gas.egrid.astype(np.float64)
    nu_max_expect = nu0 * math.sqrt((eg[1:] / eg[:-1]).max())
    trk = _open(2e-12, 5)
    nu_max = oracle.gas_constants(gas, trk)["nu_max_e"]
    assert abs(nu_max / nu_max_expect - 1) < 2e-6
    rng = np.random.default_rng(3)
    ch = inputs.make_charges(rng.uniform(-1e-4, 1e-4, (n, 3)), inputs.maxwellian(rng, n, 0.5, ME),
                             np.zeros(n, np.uint8))
    _, _, hist = oracle.run(ch, gas, trk, 10, space_charge=False)
    tr = np.array([h["trials"] for h in hist], np.float64)
    co = np.array([h["collisions"] for h in hist], np.float64)
    lam = n * nu_max * 2e-12
    assert abs(tr.mean() - lam) < 4 * math.sqrt(lam / len(tr))
    p = nu0 / nu_max
    assert abs(co.sum() / tr.sum() - p) < 5 * math.sqrt(p * (1 - p) / tr.sum())


# ----------------------------------------------------------------------------
# 2. lookup and interpolation at fixed energies on a coarse table
# ----------------------------------------------------------------------------
def test_interpolation_segment_and_weight_on_a_coarse_table():
    """A coarse, non-monotone elastic table; electrons held at one energy
    (no field, infinite gas mass: elastic scattering keeps the speed).  Every
    trial is then taken at that energy, so the share of real collisions among
    the trials is N v sigma(eps) / nu_max with sigma linear in energy inside
    the segment holding eps (np.interp).  A wrong segment or a weight taken
    from the wrong end changes the share by far more than its sampling error.
    Energies outside the grid take the end values."""
    eg = [0.01, 0.1, 1.0, 10.0, 100.0]
    sig = np.array([1.0, 5.0, 2.0, 8.0, 3.0]) * 1e-20
    gas = _table_gas(eg, [sig], [inputs.P_ELASTIC], [0.0])
    trk = _open(3e-13, 8)
    nu_max = oracle.gas_constants(gas, trk)["nu_max_e"]
    rng = np.random.default_rng(11)
    for eps0 in (0.004, 0.03, 0.077, 0.5, 3.0, 9.0, 40.0, 250.0):
        n = 20000
        ch = _electrons_at(np.full(n, eps0), rng)
        st, out, _, stats = oracle.step(ch, np.zeros((n, 3), np.float32), 0, n, gas, trk, n + 16)
        assert st == 0
        p = N_GAS * _speed(eps0) * float(_sigma_interp(gas, 0, np.array([eps0]))[0]) / nu_max
        tr = stats["trials"]
        got = stats["collisions"] / tr
        assert abs(got - p) < 5 * math.sqrt(p * (1 - p) / tr) + 1e-6, (eps0, got, p)
        # speed kept by every collision (infinite mass): energy unchanged
        assert np.allclose(_energy_eV(out.vel), eps0, rtol=2e-6)


def test_majorant_bounds_the_table_and_is_tight_for_a_monotone_table():
    """nu_max of the null-collision method must bound N sigma_tot(E) v(E)
    everywhere on the grid (dense FP64 scan of a random piecewise-linear,
    non-monotone table with thresholds); for a table increasing with energy the
    bound is attained at the last grid point: nu_max = N sigma_tot(E_n) v(E_n).
    Constant-frequency rows add their frequency."""
    rng = np.random.default_rng(5)
    eg = np.sort(rng.uniform(0.01, 50.0, 40)).astype(np.float32)
    rows = rng.uniform(0.0, 3e-20, (3, 40))
    thr = [0.0, 7.3, 12.1]
    gas = _table_gas(eg, rows, [inputs.P_ELASTIC, inputs.P_EXCITATION, inputs.P_IONISATION], thr)
    trk = _open(1e-12, 1)
    nu_max = oracle.gas_constants(gas, trk)["nu_max_e"]
    dense = _majorant_dense(gas)
    assert nu_max >= dense * (1 - 1e-6)
    # tight within one segment's speed ratio
    assert nu_max <= dense * math.sqrt((eg[1:] / eg[:-1]).max()) * (1 + 1e-6)
    # monotone increasing table: attained at the top of the grid
    inc = np.cumsum(rng.uniform(0.0, 1e-21, (2, 40)), axis=1)
    gas2 = _table_gas(eg, inc, [inputs.P_ELASTIC, inputs.P_EXCITATION], [0.0, 0.0])
    top = N_GAS * float(inc[:, -1].astype(np.float32).astype(np.float64).sum()) * float(_speed(float(eg[-1])))
    assert abs(oracle.gas_constants(gas2, trk)["nu_max_e"] / top - 1) < 1e-6
    # plus a constant-frequency row
    gas3 = _table_gas(eg, np.vstack([inc, np.zeros(40)]), [inputs.P_ELASTIC, inputs.P_EXCITATION,
                                                           inputs.P_ATTACHMENT], [0.0, 0.0, 0.0])
    gas3.mode[2] = inputs.MODE_CONST
    gas3.nuc[2] = 3e11
    assert abs(oracle.gas_constants(gas3, trk)["nu_max_e"] / (top + 3e11) - 1) < 1e-6


# ----------------------------------------------------------------------------
# 3. thresholds and the energy loss of excitation
# ----------------------------------------------------------------------------
def test_excitation_threshold_and_energy_loss():
    """Two excitations, T1 = 10 eV and T2 = 14 eV, listed in the order (T2, T1),
    with tables that are non-zero below their thresholds (the threshold alone
    must zero them).  No field, infinite gas mass, energies 5 .. 19.9 eV, so
    an electron is excited at most once per step (eps - T1 < T1).
      - below T1 nothing changes, bit for bit;
      - an excited electron ends at eps - T1, or eps - T2 if eps >= T2, and at
        eps - T1 if T1 <= eps < T2;
      - the number excited is sum over electrons of 1 - exp(-N v sigma(eps) dt)
        (the real collisions of a Poisson process at a fixed energy);
      - electrons exactly at the threshold (eps == T1 in binary32) can be
        excited: sigma is zero only below the threshold, and they stop."""
    s1, s2 = 2e-20, 1e-20
    eg = [0.1, 1.0, 10.0, 14.0, 100.0]
    gas = _table_gas(eg, [np.full(5, s2), np.full(5, s1)], [inputs.P_EXCITATION, inputs.P_EXCITATION],
                     [14.0, 10.0])
    trk = _open(2e-13, 23)
    K_e = np.float32(oracle.gas_constants(gas, trk)["K_e"])
    # a speed whose binary32 energy K_e * v^2 is exactly the threshold T1
    vz = np.float32(math.sqrt(10.0 / float(K_e)))
    while np.float32(K_e * np.float32(vz * vz)) < np.float32(10.0):
        vz = np.nextafter(vz, np.float32(np.inf))
    T1 = float(np.float32(K_e * np.float32(vz * vz)))
    gas.thr[1] = np.float32(T1)
    gas.egrid[2] = np.float32(T1)
    rng = np.random.default_rng(2)
    n, n_at = 30000, 2000
    eps0 = rng.uniform(5.0, 19.9, n)
    ch = _electrons_at(eps0, rng)
    at = inputs.make_charges(rng.uniform(-1e-4, 1e-4, (n_at, 3)), np.zeros((n_at, 3)), np.zeros(n_at, np.uint8))
    at.vel[:, 2] = vz
    both = inputs.make_charges(np.concatenate([ch.pos_q[:, :3], at.pos_q[:, :3]]),
                               np.concatenate([ch.vel[:, :3], at.vel[:, :3]]), np.zeros(n + n_at, np.uint8))
    e_in = _energy32(both.vel, K_e)
    st, out, _, stats = oracle.step(both, np.zeros((n + n_at, 3), np.float32), 0, n + n_at, gas, trk,
                                    n + n_at + 16)
    assert st == 0 and out.n == n + n_at
    changed = ~np.all(out.vel.view(np.uint32) == both.vel.view(np.uint32), axis=1)
    e_out = _energy_eV(out.vel)
    below = e_in < T1
    assert not changed[below].any()
    assert stats["collisions"] == changed.sum()
    mid = (e_in >= T1) & (e_in < 14.0) & changed
    assert np.allclose(e_out[mid], e_in[mid] - T1, atol=2e-5 * 14.0)
    hi = (e_in >= 14.0) & changed
    d1 = np.abs(e_out[hi] - (e_in[hi] - T1))
    d2 = np.abs(e_out[hi] - (e_in[hi] - 14.0))
    assert np.all(np.minimum(d1, d2) < 2e-5 * 14.0)
    # both excitations occur above T2, in the ratio of their cross sections
    k2 = (d2 < d1).sum()
    assert abs(k2 / hi.sum() - s2 / (s1 + s2)) < 5 * math.sqrt(2 / 9 / hi.sum())
    # count of excited electrons: 1 - exp(-nu dt) summed over the electrons
    nu = N_GAS * _speed(e_in) * (np.where(e_in >= T1, s1, 0.0) + np.where(e_in >= 14.0, s2, 0.0))
    p = 1.0 - np.exp(-nu * trk.dt)
    free = np.arange(n + n_at) < n
    assert abs(changed[free].sum() - p[free].sum()) < 5 * math.sqrt((p[free] * (1 - p[free])).sum())
    # exactly at the threshold: excited at the rate of sigma(T1), and stopped
    ex_at = changed[n:]
    pa = 1.0 - math.exp(-N_GAS * float(_speed(T1)) * s1 * trk.dt)
    assert abs(ex_at.sum() - pa * n_at) < 5 * math.sqrt(n_at * pa * (1 - pa))
    assert np.all(e_out[n:][ex_at] == 0.0)


# ----------------------------------------------------------------------------
# 4. ionisation energetics (Sec. 3.3.3, Eq. (distIoni))
# ----------------------------------------------------------------------------
def test_ionisation_energy_split_spawn_distance_and_cation_speed():
    """One tabulated ionisation, I = 15.8 eV, gas at T = 300 K with M = 40 amu.
    E_res = eps - I - (3/2) k T: electrons with E_res <= 0 never ionise; for the
    others both electrons leave with E_res / 2 and opposite velocities, sit
    k_C e / E_res apart (each r = k_C e / (2 E_res) from the cation, Eq.
    (distIoni)), and the cation starts at the parent's position with the
    thermal speed sqrt(3 k T / M).  eps < 3 I keeps both electrons below I, so
    each parent ionises at most once per step."""
    I, T, M_amu = 15.8, 300.0, 40.0
    Eth = 1.5 * KB * T / E
    si = 3e-20
    gas = _table_gas([0.1, 1.0, I, 1000.0], [np.full(4, si)], [inputs.P_IONISATION], [I], T=T, M_amu=M_amu)
    trk = _open(3e-13, 31)
    rng = np.random.default_rng(7)
    n, n_gap = 12000, 600
    eps0 = np.concatenate([rng.uniform(1.05 * I, 2.9 * I, n), np.full(n_gap, I + 0.5 * Eth)])
    ch = _electrons_at(eps0, rng, spread=0.0)          # at the origin: fine binary32 resolution
    K_e = oracle.gas_constants(gas, trk)["K_e"]
    e_in = _energy32(ch.vel, K_e)
    N0 = n + n_gap
    st, out, nid, stats = oracle.step(ch, np.zeros((N0, 3), np.float32), 0, N0, gas, trk, 3 * N0)
    assert st == 0
    ns = int(stats["spawned_pairs"])
    assert ns > 0 and nid == N0 + 2 * ns and out.n == N0 + 2 * ns
    par = {int(i): k for k, i in enumerate(out.id)}
    # spawns: ids N0.. in (parent, trial) order, electron then cation
    spawn_e = out.id >= N0
    assert np.array_equal(out.species[spawn_e], np.tile(np.array([0, 1], np.uint8), ns))
    new_e = np.flatnonzero(spawn_e & (out.species == 0))
    new_i = np.flatnonzero(spawn_e & (out.species == 1))
    # which parent: the one whose velocity is the exact negative of the new electron's
    pv = {tuple(out.vel[par[p], :3].view(np.uint32)): p for p in range(N0)}
    parents = []
    for k in new_e:
        key = tuple((-out.vel[k, :3]).view(np.uint32))
        assert key in pv, "new electron without an opposite parent"
        parents.append(pv[key])
    parents = np.array(parents)
    assert len(set(parents.tolist())) == ns and np.all(np.diff(parents) > 0)
    er = e_in[parents] - I - Eth
    assert np.all(er > 0)
    assert not np.isin(np.arange(n, N0), parents).any()            # E_res <= 0: null
    e_par = _energy_eV(out.vel[[par[p] for p in parents]])
    e_new = _energy_eV(out.vel[new_e])
    assert np.allclose(e_par, er / 2, rtol=3e-6, atol=1e-6)
    assert np.allclose(e_new, er / 2, rtol=3e-6, atol=1e-6)
    # the new electron sits r = k_C e / (2 E_res) from the cation along its own
    # direction of motion (it starts moving next step; the parent flies on)
    pn = out.pos_q[new_e, :3].astype(np.float64)
    pc = out.pos_q[new_i, :3].astype(np.float64)
    r = KC * E / (2 * er)
    off = pn - pc
    res = np.sqrt((np.spacing(np.abs(out.pos_q[new_e, :3])).astype(np.float64) ** 2).sum(1))
    assert np.all(np.abs(np.linalg.norm(off, axis=1) - r) < 1e-5 * r + res)
    vdir = out.vel[new_e, :3].astype(np.float64)
    vdir /= np.linalg.norm(vdir, axis=1)[:, None]
    assert np.all(np.linalg.norm(off - r[:, None] * vdir, axis=1) < 1e-5 * r + 2 * res)
    vth = math.sqrt(3 * KB * T / (M_amu * AMU))
    assert np.allclose(np.linalg.norm(out.vel[new_i, :3].astype(np.float64), axis=1), vth, rtol=2e-6)
    # ionisation count: 1 - exp(-N v sigma_i dt) per electron with E_res > 0
    p = np.where(e_in - I - Eth > 0, 1.0 - np.exp(-N_GAS * _speed(e_in) * si * trk.dt), 0.0)
    assert abs(ns - p.sum()) < 5 * math.sqrt((p * (1 - p)).sum())
    assert stats["n_electron"] - stats["n_cation"] == N0
