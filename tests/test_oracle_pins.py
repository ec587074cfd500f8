"""Pins of the CPU oracle against things other than itself: closed forms,
brute-force quadrature, conservation laws, published known-answer vectors and
exact statistics of the step's stochastic model.  All CPU-only."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2110_09214_gb300 import inputs

EPS0 = 8.8541878128e-12
E = 1.602176634e-19
ME = 9.1093837015e-31
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

TRI = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.3, 0.9, 0.05]])


# ----------------------------------------------------------------------------
# independent brute-force quadrature of the cell integrals
# ----------------------------------------------------------------------------
_GX, _GW = np.polynomial.legendre.leggauss(8)
_GX = 0.5 * (_GX + 1.0)
_GW = 0.5 * _GW


def _duffy_rule(a, b, c):
    """Quadrature points/weights on triangle (a, b, c), collapsed at a."""
    u, w = np.meshgrid(_GX, _GX, indexing="ij")
    wu, ww = np.meshgrid(_GW, _GW, indexing="ij")
    pts = a + u[..., None] * (b - a) + (u * w)[..., None] * (c - b)
    jac = np.linalg.norm(np.cross(b - a, c - b)) * u
    return pts.reshape(-1, 3), (wu * ww * jac).reshape(-1)


def brute(v, r, depth=18):
    """Adaptive subdivision: a sub-triangle is integrated with a 64-point rule
    once its diameter is below 0.15 x its distance to r, else split in 4."""
    r = np.asarray(r, float)
    stack = [(np.asarray(v, float), 0)]
    phi = 0.0
    F = np.zeros(3)
    while stack:
        t, d = stack.pop()
        cen = t.mean(axis=0)
        diam = max(np.linalg.norm(t[0] - t[1]), np.linalg.norm(t[1] - t[2]),
                   np.linalg.norm(t[2] - t[0]))
        dist = np.linalg.norm(r - cen)
        if diam < 0.15 * dist or d >= depth:
            p, w = _duffy_rule(t[0], t[1], t[2])
            dv = r - p
            R = np.linalg.norm(dv, axis=1)
            phi += (w / R).sum()
            F += ((w / R ** 3)[:, None] * dv).sum(axis=0)
        else:
            a, b, c = t
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            stack += [(np.array([a, ab, ca]), d + 1), (np.array([ab, b, bc]), d + 1),
                      (np.array([ca, bc, c]), d + 1), (np.array([ab, bc, ca]), d + 1)]
    return phi, F


def _geom(v):
    e1, e2 = v[1] - v[0], v[2] - v[0]
    nn = np.cross(e1, e2)
    return v.mean(axis=0), nn / np.linalg.norm(nn), 0.5 * np.linalg.norm(nn)


@pytest.mark.parametrize("dist", [1e-2, 0.1, 0.5, 1.0, 3.0, 10.0, 100.0, 1000.0])
def test_tri_integrals_vs_brute_force_off_plane(dist):
    c, n, _ = _geom(TRI)
    rng = np.random.default_rng(int(dist * 1000))
    for _ in range(3):
        d = rng.normal(size=3)
        d += 2.0 * n * np.sign(d @ n)
        d /= np.linalg.norm(d)
        r = c + dist * d
        phi, F = oracle.tri_integrals(TRI, r)
        pb, Fb = brute(TRI, r)
        assert abs(phi - pb) <= 1e-9 * abs(pb)
        assert np.linalg.norm(F - Fb) <= 1e-8 * np.linalg.norm(Fb)


@pytest.mark.parametrize("where", ["edge", "vertex", "inplane_out", "below"])
def test_tri_integrals_near_singular(where):
    c, n, _ = _geom(TRI)
    if where == "edge":
        mid = 0.5 * (TRI[0] + TRI[1])
        r = mid + 1e-3 * n + 1e-3 * (mid - c)
    elif where == "vertex":
        r = TRI[2] + 2e-3 * n + 1e-3 * (TRI[2] - c)
    elif where == "inplane_out":
        r = TRI[1] + 0.3 * (TRI[1] - c)
        r = r - ((r - TRI[0]) @ n) * n
    else:
        r = c - 0.02 * n + 0.1 * (TRI[0] - c)
    phi, F = oracle.tri_integrals(TRI, r)
    pb, Fb = brute(TRI, r, depth=22)
    assert abs(phi - pb) <= 1e-8 * abs(pb)
    assert np.linalg.norm(F - Fb) <= 1e-6 * np.linalg.norm(Fb)


def test_tri_potential_in_plane_inside():
    """Target inside the cell, in its plane: split at the target into three
    triangles collapsed there (Duffy), where the integrand is regular."""
    c, n, _ = _geom(TRI)
    r = c + 0.1 * (TRI[0] - c)
    r = r - ((r - TRI[0]) @ n) * n
    xs, ws = np.polynomial.legendre.leggauss(60)
    xs = 0.5 * (xs + 1)
    ws = 0.5 * ws
    ref = 0.0
    for i in range(3):
        a, b = TRI[i], TRI[(i + 1) % 3]
        cr = np.linalg.norm(np.cross(a - r, b - a))
        ref += sum(wj * cr / np.linalg.norm((a - r) + xj * (b - a)) for xj, wj in zip(xs, ws))
    phi, F = oracle.tri_integrals(TRI, r)
    assert abs(phi - ref) <= 1e-10 * ref
    # principal value of the normal component in the plane, and the jump of
    # Eqs. (fldinterf1/2): F.n -> +-2 pi on either side
    assert abs(F @ n) < 1e-12
    _, Fp = oracle.tri_integrals(TRI, r + 1e-10 * n)
    _, Fm = oracle.tri_integrals(TRI, r - 1e-10 * n)
    assert abs(Fp @ n - 2 * math.pi) < 1e-6
    assert abs(Fm @ n + 2 * math.pi) < 1e-6
    # tangential part continuous across the cell
    tp = Fp - (Fp @ n) * n
    tm = Fm - (Fm @ n) * n
    assert np.linalg.norm(tp - tm) < 1e-6 * np.linalg.norm(tp)
    # potential continuous
    assert abs(oracle.tri_integrals(TRI, r + 1e-10 * n)[0] - phi) < 1e-8


def test_far_field_point_charge_limit():
    """Far away a cell acts as a point charge of its area: error O((h/d)^2)."""
    c, n, A = _geom(TRI)
    d = np.array([0.3, -0.5, 0.8])
    d /= np.linalg.norm(d)
    errs = []
    for dist in (10.0, 100.0):
        r = c + dist * d
        phi, F = oracle.tri_integrals(TRI, r)
        Fp = A * (r - c) / dist ** 3
        errs.append(np.linalg.norm(F - Fp) / np.linalg.norm(Fp))
        assert abs(phi - A / dist) <= 0.1 / dist ** 2 * (A / dist)
    assert errs[0] < 2e-3
    assert 50 < errs[0] / errs[1] < 200


# ----------------------------------------------------------------------------
# BEM pins
# ----------------------------------------------------------------------------
def _areas(mesh):
    e1 = mesh.tri[:, 1] - mesh.tri[:, 0]
    e2 = mesh.tri[:, 2] - mesh.tri[:, 0]
    return 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)


def test_conducting_sphere_capacitance_and_field():
    """Sphere at potential V: sigma = eps0 V / R, C = 4 pi eps0 R,
    E(r) = V R / r^2 outside; discretisation error O(h^2)."""
    R, V = 1e-3, 1.0
    errs = []
    for lev in (2, 3):
        m = inputs.conducting_sphere(R, lev, V)
        sig = oracle.bem_solve(m)
        Q = (sig * _areas(m)).sum()
        errs.append(abs(Q / (4 * math.pi * EPS0 * R * V) - 1))
        Ef, Vf = oracle.panel_field(m.tri, sig, np.array([[0, 0, 3 * R], [2 * R, 2 * R, 0]]))
        r2 = np.array([3 * R, 2 * math.sqrt(2) * R])
        assert np.allclose(np.linalg.norm(Ef, axis=1), V * R / r2 ** 2 * (Q / (4 * math.pi * EPS0 * R * V)), rtol=1e-3)
        assert np.allclose(np.abs(sig).mean(), EPS0 * V / R, rtol=0.03)
    assert errs[0] < 0.02 and errs[1] < 0.005
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_dielectric_sphere_in_uniform_field():
    """Dielectric sphere (eps_r) in a uniform field E0 given through the
    right-hand side of Eq. (BEMfldpart): interior field 3 E0 / (eps_r + 2),
    surface density 3 eps0 E0 cos(theta) (eps_r - 1)/(eps_r + 2).  Flat cells
    on a curved second-kind surface converge at first order in h, so the pin
    is the first-order convergence and its Richardson extrapolation."""
    R, er = 1e-3, 4.0
    E0 = np.array([0.0, 0.0, 1e5])
    want_in = 3 * E0[2] / (er + 2)
    vals = []
    for lev in (2, 3):
        tri = inputs.icosphere(R, lev)
        n = len(tri)
        m = inputs.Mesh(tri, np.ones(n, np.int32), -np.ones(n, np.int32), np.full(n, er),
                        np.ones(n), np.zeros(0))
        nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
        nrm /= np.linalg.norm(nrm, axis=1)[:, None]
        drhs = -(m.eps_plus - m.eps_minus) * EPS0 * (nrm @ E0)
        sig = oracle.solve(oracle.assemble(m), drhs)
        Ein, _ = oracle.panel_field(tri, sig, np.array([[0, 0, 0], [0.3 * R, 0.1 * R, -0.2 * R]]))
        Ein = Ein + E0
        assert abs(Ein[0, 2] - Ein[1, 2]) < 1e-3 * want_in       # uniform inside
        assert np.all(np.abs(Ein[:, :2]) < 1e-3 * E0[2])
        cen = tri.mean(axis=1)
        cos = cen[:, 2] / np.linalg.norm(cen, axis=1)
        want = 3 * EPS0 * E0[2] * cos * (er - 1) / (er + 2)
        assert np.abs(sig - want).max() < 0.1 * np.abs(want).max()
        vals.append(Ein[0, 2])
    e2, e3 = vals[0] - want_in, vals[1] - want_in
    assert 0 < e3 < e2 < 0.08 * want_in
    assert 1.6 < e2 / e3 < 2.4
    assert abs((2 * vals[1] - vals[0]) / want_in - 1) < 0.01


def test_parallel_plates_field_and_collocation():
    m = inputs.parallel_plates(1e-2, 1e-3, 16, 0.0, 100.0)
    sig = oracle.bem_solve(m)
    cen = m.tri.mean(axis=1)
    _, Vc = oracle.panel_field(m.tri, sig, cen)
    want = m.group_voltage[m.group]
    assert np.abs(Vc - want).max() < 1e-9 * 100.0
    Ec, _ = oracle.panel_field(m.tri, sig, np.array([[5e-3, 5e-3, 5e-4]]))
    assert abs(Ec[0, 0]) < 1e-6 * abs(Ec[0, 2]) and abs(Ec[0, 1]) < 1e-6 * abs(Ec[0, 2])
    # infinite-plate closed form V/d; the fringe correction at the centre of
    # L/d = 10 plates is exponentially small (~exp(-5 pi))
    assert abs(-Ec[0, 2] / 1e5 - 1) < 2e-4
    # a zero-thickness plate carries the charge of both faces: the net charge
    # of the two plates is opposite (capacitor) up to the outer-face share
    q = sig * _areas(m)
    assert q[m.group == 0].sum() < 0 < q[m.group == 1].sum()


def _sphere_flux(fn, centre, radius, n_th=48, n_ph=96):
    x, w = np.polynomial.legendre.leggauss(n_th)
    ph = (np.arange(n_ph) + 0.5) * 2 * math.pi / n_ph
    ct, P = np.meshgrid(x, ph, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    nrm = np.stack([st * np.cos(P), st * np.sin(P), ct], -1).reshape(-1, 3)
    pts = np.asarray(centre) + radius * nrm
    Ev = fn(pts)
    wt = (np.repeat(w, n_ph) * (2 * math.pi / n_ph) * radius ** 2)
    return float(((Ev * nrm).sum(1) * wt).sum())


def test_gauss_law_panels_and_charges():
    """Flux of E through a closed surface equals Q_enc / eps0 (cells: Eq. (BEM3);
    charges: Eq. (nbody))."""
    m = inputs.conducting_sphere(1e-3, 2, 1.0)
    sig = oracle.bem_solve(m)
    Q = (sig * _areas(m)).sum()
    flux = _sphere_flux(lambda p: oracle.panel_field(m.tri, sig, p)[0], (1e-4, -2e-4, 5e-5), 2.5e-3)
    assert abs(flux - Q / EPS0) < 2e-6 * abs(Q / EPS0)
    # part of a plate inside the surface: enclosed charge = sum over cells
    # fully inside (cells cut by the surface are avoided by the geometry)
    pl = inputs.rect_plate(-1e-3, 1e-3, -1e-3, 1e-3, 0.0, 4, 4)
    sg = np.linspace(1.0, 2.0, len(pl)) * 1e-6
    flux = _sphere_flux(lambda p: oracle.panel_field(pl, sg, p)[0], (0, 0, 0), 3e-3)
    Qp = (sg * _areas(inputs.Mesh(pl, None, None, None, None, None))).sum()
    assert abs(flux - Qp / EPS0) < 2e-6 * abs(Qp / EPS0)
    rng = np.random.default_rng(5)
    src = np.zeros((20, 4))
    src[:, :3] = rng.uniform(-2e-3, 2e-3, (20, 3))
    src[:, 3] = rng.choice([-E, E], 20)
    inside = np.linalg.norm(src[:, :3] - np.array([5e-4, 0, 0]), axis=1) < 1.5e-3
    flux = _sphere_flux(lambda p: oracle.nbody_field(p, src)[0], (5e-4, 0, 0), 1.5e-3, 96, 192)
    want = src[inside, 3].sum() / EPS0
    assert abs(flux - want) < 1e-2 * E / EPS0


def test_nbody_antisymmetry_and_softening():
    rng = np.random.default_rng(2)
    src = np.zeros((50, 4))
    src[:, :3] = rng.uniform(0, 1e-4, (50, 3))
    src[:, 3] = rng.choice([-E, E], 50)
    Ef, _ = oracle.nbody_field(src[:, :3], src, self_exclude=True)
    F = (src[:, 3:4] * Ef).sum(axis=0)
    scale = np.abs(src[:, 3:4] * Ef).sum()
    assert np.linalg.norm(F) < 1e-12 * scale
    # Plummer softening -> paper's sum as soft -> 0
    Es, _ = oracle.nbody_field(src[:, :3], src, True, 1e-12)
    assert np.abs(Es - Ef).max() < 1e-5 * np.abs(Ef).max()


def test_influence_rhs_closed_form():
    """A point charge far from a small cell: mean potential on the cell ->
    k q / d (Eq. (potpart)); dd rows take -(e+ - e-) eps0 Ebar.n (Eq. (fldpart))."""
    tri = np.array([[[0, 0, 0], [1e-5, 0, 0], [0, 1e-5, 0]]], float)
    src = np.array([[0.3e-5, 0.3e-5, 1e-2, E]])
    m = inputs.Mesh(tri, np.zeros(1, np.int32), np.zeros(1, np.int32), np.ones(1), np.ones(1),
                    np.zeros(1))
    d = oracle.influence_rhs(m, src)
    kq = E / (4 * math.pi * EPS0)
    assert abs(-d[0] - kq / 1e-2) < 1e-6 * kq / 1e-2
    m2 = inputs.Mesh(tri, np.ones(1, np.int32), -np.ones(1, np.int32), np.full(1, 3.0),
                     np.ones(1), np.zeros(0))
    d2 = oracle.influence_rhs(m2, src)
    # field of the charge at the cell points -z (charge above): Ebar.n = -kq/d^2
    want = -(1.0 - 3.0) * EPS0 * (-kq / 1e-4)
    assert abs(d2[0] - want) < 1e-5 * abs(want)


def test_gepp_matches_lapack():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(200, 200)) + 10 * np.eye(200)
    b = rng.normal(size=200)
    assert np.allclose(oracle.solve(A, b, force_gepp=True), np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


# ----------------------------------------------------------------------------
# RNG and sampling helpers of the step
# ----------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        out = oracle.philox(vals[:4], vals[4:6])
        assert out.tolist() == vals[6:10]


def test_neg_log_and_iso_dir():
    rng = np.random.default_rng(1)
    us = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64)
    for u in us[:2000]:
        U = ((int(u) >> 8) + 1) * 2.0 ** -24
        assert abs(oracle.neg_log_u(int(u)) - (-math.log(U))) < 2e-6 * max(1.0, -math.log(U))
    d = np.array([oracle.iso_dir(int(a), int(b)) for a, b in us.reshape(-1, 2)])
    assert np.abs(np.linalg.norm(d, axis=1) - 1).max() < 1e-6
    n = len(d)
    assert np.abs(d.mean(axis=0)).max() < 5 / math.sqrt(3 * n)
    assert np.abs((d ** 2).mean(axis=0) - 1 / 3).max() < 5 * math.sqrt(4 / 45 / n)


# ----------------------------------------------------------------------------
# step: exact statistics of the Maxwell model and the step's bookkeeping
# ----------------------------------------------------------------------------
def _cloud(n, kT=0.1, seed=0, at_rest=False):
    rng = np.random.default_rng(seed)
    vel = np.zeros((n, 3)) if at_rest else inputs.maxwellian(rng, n, kT, ME)
    return inputs.make_charges(np.zeros((n, 3)), vel, np.zeros(n, np.uint8))


def _open_trk(seed=7, dt=1e-12):
    return inputs.Tracking(dt=dt, seed=seed, z_lo=-1.0, z_hi=1.0, beta=-1.0)


def test_maxwell_mean_velocity():
    """Constant nu, isotropic scattering: <v_z>(t) = (qE/m nu)(1 - exp(-nu t))
    for a cloud starting at rest."""
    nu, Ez, n = 1e12, -1e5, 20000
    gas = inputs.maxwell_gas(nu, 0.0)
    trk = _open_trk()
    ch = _cloud(n, at_rest=True)
    vd = E * 1e5 / (ME * nu)
    nid = n
    for s in range(6):
        Eg = np.tile(np.array([0, 0, Ez], np.float32), (ch.n, 1))
        st, ch, nid, _ = oracle.step(ch, Eg, s, nid, gas, trk)
        assert st == 0
        t = (s + 1) * 1e-12
        vz = ch.vel[:, 2].astype(float)
        want = vd * (1 - math.exp(-nu * t))
        assert abs(vz.mean() - want) < 4 * vz.std() / math.sqrt(n) + 1e-3 * vd


def test_maxwell_zero_field_diffusion():
    """E = 0, M = inf: <x^2> = (2<v^2>/3nu)(t - (1 - exp(-nu t))/nu)."""
    nu, n = 1e12, 20000
    gas = inputs.maxwell_gas(nu, 0.0)
    trk = _open_trk(seed=11)
    ch = _cloud(n, kT=0.1, seed=3)
    v2 = (ch.vel[:, :3].astype(float) ** 2).sum(1).mean()
    _, _, hist = oracle.run(ch, gas, trk, 20, space_charge=False)
    for s in (1, 4, 19):
        h = hist[s]
        x2 = (h["sum_x2_e"] + h["sum_y2_e"] + h["sum_z2_e"]) / (3 * h["n_electron"])
        t = (s + 1) * 1e-12
        want = 2 * v2 / (3 * nu) * (t - (1 - math.exp(-nu * t)) / nu)
        assert abs(x2 / want - 1) < 0.04


def test_trial_counts_are_poisson():
    nu, n = 1e12, 5000
    gas = inputs.maxwell_gas(nu, 0.0)
    ch = _cloud(n)
    _, _, hist = oracle.run(ch, gas, _open_trk(seed=5, dt=2e-12), 30, space_charge=False)
    tr = np.array([h["trials"] for h in hist])
    lam = n * nu * 2e-12
    assert abs(tr.mean() - lam) < 4 * math.sqrt(lam / len(tr))
    assert 0.5 * lam < tr.var() < 1.8 * lam


def _gas_with(extra_kind, extra_nu, T=0.0):
    g = inputs.maxwell_gas(1e12, 0.0)
    g.kind = np.array([inputs.P_ELASTIC, extra_kind], np.int32)
    g.mode = np.array([inputs.MODE_CONST, inputs.MODE_CONST], np.int32)
    g.thr = np.zeros(2, np.float32)
    g.nuc = np.array([1e12, extra_nu], np.float32)
    g.xs = np.zeros((2, 2), np.float32)
    g.T = T
    g.M_amu = 40.0
    g.nu_ion = 0.0
    return g


def test_constant_ionisation_growth_and_conservation():
    """Constant ionisation frequency nu_i (threshold 0, T = 0): each charge
    present at step start ionises Poisson(nu_i dt) times and the spawned
    electron starts moving next step, so E[N_e(s)] = N0 (1 + nu_i dt)^s;
    every ionisation adds one electron and one cation."""
    n0, nui = 20000, 1e10
    gas = _gas_with(inputs.P_IONISATION, nui)
    ch = _cloud(n0, kT=1.0, seed=4)
    fin, nid, hist = oracle.run(ch, gas, _open_trk(seed=9), 60, space_charge=False)
    ne = np.array([h["n_electron"] for h in hist])
    want = n0 * (1 + nui * 1e-12) ** 60
    sd = math.sqrt(n0 * want / n0 * (want / n0 - 1))
    assert abs(ne[-1] - want) < 4 * sd
    assert all(h["n_electron"] - h["n_cation"] == n0 for h in hist)
    assert np.all(np.diff(fin.id.astype(np.int64)) > 0)
    assert nid == n0 + 2 * int(sum(h["spawned_pairs"] for h in hist))


def test_constant_attachment_decay():
    n0, nua = 20000, 2e10
    gas = _gas_with(inputs.P_ATTACHMENT, nua, T=300.0)
    ch = _cloud(n0, seed=6)
    _, _, hist = oracle.run(ch, gas, _open_trk(seed=13), 40, space_charge=False)
    p = math.exp(-nua * 40e-12)
    ne = hist[-1]["n_electron"]
    assert abs(ne - n0 * p) < 4 * math.sqrt(n0 * p * (1 - p))
    assert hist[-1]["n_anion"] == n0 - ne


def test_absorption_on_electrode_planes():
    gas = inputs.maxwell_gas(1e12, 0.0)
    trk = inputs.Tracking(dt=1e-12, seed=1, z_lo=0.0, z_hi=1e-6, beta=-1.0)
    n = 200
    rng = np.random.default_rng(0)
    pos = np.column_stack([rng.uniform(0, 1e-3, n), rng.uniform(0, 1e-3, n), np.full(n, 5e-7)])
    ch = inputs.make_charges(pos, inputs.maxwellian(rng, n, 0.1, ME), np.zeros(n, np.uint8))
    fin, _, hist = oracle.run(ch, gas, trk, 400, space_charge=False)
    absorbed = sum(h["absorbed"] for h in hist)
    assert absorbed + fin.pos_q.shape[0] == n and absorbed > 0.9 * n
    assert np.all((fin.pos_q[:, 2] > 0) & (fin.pos_q[:, 2] < 1e-6))


def test_recombination_pairing_rules():
    """Each electron proposes its nearest cation within R_c (ties: lower id),
    each cation accepts the proposer with the smallest (d^2, id); cations
    created in the previous step are exempt (Eq. (distRecomb) with the
    capture radius of the rate coefficient)."""
    gas = inputs.maxwell_gas(0.0, 40.0)
    gas.nuc[:] = 0.0
    gas.nu_ion = 0.0
    trk = inputs.Tracking(dt=1e-12, seed=1, z_lo=-1, z_hi=1, beta=1e-13)
    rc = (3 * 1e-13 * 1e-12 / (4 * math.pi)) ** (1 / 3)
    x = np.float32(1e-3)
    # e0 <-> c0 at 0.5 rc; e1 at 0.3 rc from c0 but 0.2 rc from c1;
    # e2 equidistant from c2 and c3 (tie -> lower id c2); c4 fresh (exempt)
    pos = np.array([
        [x, 0, 0], [x + 0.5 * rc, 0, 0],                 # e0 (id0), c0 (id1)
        [x - 0.3 * rc, 0, 0], [x - 0.5 * rc, 0, 0],       # e1 (id2), c1 (id3)
        [0, 1e-3, 0], [0.4 * rc, 1e-3, 0], [-0.4 * rc, 1e-3, 0],  # e2, c2, c3
        [0, 0, 1e-3], [0.1 * rc, 0, 1e-3],               # e3, c4 (fresh)
    ], np.float64)
    sp = np.array([0, 1, 0, 1, 0, 1, 1, 0, 1], np.uint8)
    ch = inputs.make_charges(pos, np.zeros((9, 3)), sp)
    ch.birth[8] = 5
    st, out, _, stats = oracle.step(ch, np.zeros((9, 3), np.float32), 5, 9, gas, trk)
    assert st == 0
    # e1 proposes c1 (0.2 rc) not c0 (0.3 rc); e0 proposes c0; e2 -> c2 (tie);
    # c4 is exempt, so e3 survives
    assert stats["recombined_pairs"] == 3
    assert sorted(out.id.tolist()) == [6, 7, 8]


def test_resume_is_bit_identical():
    mesh, gas, ch, trk = inputs.config_small_plates(seed=2, n=200)
    sig = oracle.bem_solve(mesh)
    a, nida, _ = oracle.run(ch, gas, trk, 10, mesh, sig)
    b1, nidb, _ = oracle.run(ch, gas, trk, 6, mesh, sig)
    b, nidb, _ = oracle.run(b1, gas, trk, 4, mesh, sig, start_step=6, next_id=nidb)
    assert nida == nidb
    for k in ("pos_q", "vel", "id", "birth", "species"):
        assert np.array_equal(getattr(a, k), getattr(b, k))


def test_capacity_overflow_commits_nothing():
    n0 = 100
    gas = _gas_with(inputs.P_IONISATION, 5e11)
    ch = _cloud(n0, kT=5.0, seed=1)
    st, out, nid, stats = oracle.step(ch, np.zeros((n0, 3), np.float32), 0, n0, gas,
                                      _open_trk(), capacity=n0 + 2)
    assert st == oracle.ST_CAPACITY and out.pos_q.shape[0] == 0 and nid == n0
    assert stats["required_capacity"] > n0 + 2


def test_swarm_fits_exact():
    t = np.linspace(0, 1e-9, 50)
    assert abs(oracle.drift_velocity(t, 3e4 * t + 1e-6) - 3e4) < 1e-6
    assert abs(oracle.diffusion_coefficient(t, 2 * 0.05 * t) - 0.05) < 1e-12
    assert abs(oracle.townsend_alpha(t, 10 * np.exp(2e10 * t), 4e4) - 5e5) < 1e-3


# ----------------------------------------------------------------------------
# the paper's per-step collision probability (Sec. 3.3.1), coll_mode = 1
# ----------------------------------------------------------------------------
def test_per_step_scheme_collision_fraction_and_drift():
    """Maxwell model (constant nu, isotropic elastic, infinite gas mass: the
    speed is kept and the mean velocity after a collision is zero).  One step:
    a charge collides with probability P = 1 - exp(-nu dt) and exactly one
    test is made per charge.  Steady state: <v_z> at the start of a step
    obeys v = (1 - P)(v + a dt), i.e. v = (1 - P) a dt / P."""
    nu, dt = 1e12, 3e-13
    P = 1.0 - math.exp(-nu * dt)
    gas = inputs.maxwell_gas(nu, 0.0)
    trk = inputs.Tracking(dt=dt, seed=3, z_lo=-1.0, z_hi=1.0, beta=-1.0, coll_mode=1)
    n = 20000
    rng = np.random.default_rng(1)
    ch = inputs.make_charges(rng.uniform(-1e-4, 1e-4, (n, 3)), inputs.maxwellian(rng, n, 0.1, ME),
                             np.zeros(n, np.uint8))
    st, out, _, stats = oracle.step(ch, np.zeros((n, 3), np.float32), 0, n, gas, trk, n + 16)
    assert st == 0 and stats["trials"] == n
    frac = stats["collisions"] / n
    assert abs(frac - P) <= 5 * math.sqrt(P * (1 - P) / n)
    # drift to the steady state under a uniform field
    Ez = -1e5
    a = E * -Ez / ME                     # electron acceleration along z: -e E_z / m
    field = np.tile(np.array([[0.0, 0.0, Ez]], np.float32), (n, 1))
    cur = ch
    for s_ in range(60):
        st, cur, _, _ = oracle.step(cur, field, s_, n, gas, trk, n + 16)
    vz = cur.vel[:, 2].astype(np.float64)
    expect = (1 - P) * np.float32(a) * dt / P
    assert abs(vz.mean() - expect) <= 5 * vz.std() / math.sqrt(n)


# ----------------------------------------------------------------------------
# approximate N-body (Sec. 3.2.4 nearest-neighbour option)
# ----------------------------------------------------------------------------
def _nn_cloud(n, seed):
    rng = np.random.default_rng(seed)
    p = np.concatenate([rng.normal(0, 1e-5, (n // 2, 3)), rng.normal([4e-5, 0, 1e-4], 1e-5, (n - n // 2, 3))])
    q = rng.choice([-E, E], n)
    return np.column_stack([p, q]).astype(np.float32).astype(np.float64)


def test_nn_with_one_or_two_cells_per_axis_is_exact():
    """With 1 or 2 cells per axis every cell is a neighbour of every other:
    the approximation reduces to the exact sum of Eq. (nbody)."""
    src = _nn_cloud(700, 1)
    ref = oracle.nbody_field(src[:, :3], src, True, 1e-9)[0]
    for G in (1, 2):
        got = oracle.nbody_nn(src, G, 1e-9)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_nn_far_cells_are_exact_for_point_like_cells():
    """Charges on a lattice of spacing two cells (no two in neighbouring
    cells; one lattice site holds two equal charges at the same point): every
    far cell's charge centre is exactly its charge, so the approximation must
    equal the exact sum of Eq. (nbody) -- a check of the cell assignment, the
    neighbour exclusion and the per-sign aggregation."""
    K, h = 5, 1e-5
    rng = np.random.default_rng(4)
    g = np.arange(K) * 2 * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    p = np.column_stack([X.ravel(), Y.ravel(), Z.ravel()])
    q = rng.choice([-E, E], len(p))
    p = np.concatenate([p, p[7:8]])
    q = np.concatenate([q, q[7:8]])
    src = np.column_stack([p, q]).astype(np.float32).astype(np.float64)
    exact = oracle.nbody_field(src[:, :3], src, True, 0.0)[0]
    nn = oracle.nbody_nn(src, 2 * K - 1, 0.0)      # cell edge 8h/9: site i in cell floor(2.25 i)
    assert np.abs(nn - exact).max() <= 1e-12 * np.abs(exact).max()


# ----------------------------------------------------------------------------
# charging-up: cells absorb the charges crossing them (Eq. (charge-up))
# ----------------------------------------------------------------------------
def test_surface_hits_absorb_at_the_crossed_cell_and_count_deposits():
    """Two dielectric cells forming the square [0, 1 mm]^2 at z = 0, no field,
    no collisions: a charge whose step carries it through the square is
    absorbed by the cell that contains the exact (FP64) crossing point; one
    that stops short, or passes beside the square, survives; deposits count
    e per charge with its sign."""
    L = 1e-3
    tri = np.array([[[0, 0, 0], [L, 0, 0], [L, L, 0]], [[0, 0, 0], [L, L, 0], [0, L, 0]]], np.float64)
    mesh = inputs.Mesh(tri, np.array([1, 1], np.int32), np.array([-1, -1], np.int32), np.ones(2), np.full(2, 3.5),
                       np.zeros(0))
    gas = inputs.maxwell_gas(0.0, 40.0)
    gas.nuc[:] = 0.0
    gas.nu_ion = 0.0
    trk = inputs.Tracking(dt=1e-12, seed=1, z_lo=-1.0, z_hi=1.0, beta=-1.0, surface_hits=True)
    rng = np.random.default_rng(3)
    n = 400
    xy = rng.uniform(-0.2 * L, 1.2 * L, (n, 2))
    z0 = rng.uniform(1e-7, 3e-6, n)
    vz = -rng.uniform(1e5, 2e6, n)                 # displacement 1e-7 .. 2e-6 m in one step
    pos = np.column_stack([xy, z0])
    vel = np.column_stack([np.zeros((n, 2)), vz])
    sp = rng.integers(0, 2, n).astype(np.uint8)
    ch = inputs.make_charges(pos, vel, sp)
    dep = np.zeros(2, np.int64)
    st, out, _, stats = oracle.step(ch, np.zeros((n, 3), np.float32), 0, n, gas, trk, n + 16, mesh=mesh, deposits=dep)
    assert st == 0
    p32 = ch.pos_q[:, :3].astype(np.float64)
    v32 = ch.vel[:, :3].astype(np.float64)
    z_end = p32[:, 2] + v32[:, 2] * trk.dt
    inside = (p32[:, 0] >= 0) & (p32[:, 0] <= L) & (p32[:, 1] >= 0) & (p32[:, 1] <= L)
    reach = z_end <= 0.0
    margin = (np.minimum.reduce([p32[:, 0], L - p32[:, 0], p32[:, 1], L - p32[:, 1]]) > 1e-9) & \
             (np.abs(z_end) > 1e-12)
    absorbed = ~np.isin(ch.id, out.id)
    sure = margin & (np.abs(p32[:, 0] - p32[:, 1]) > 1e-9)
    assert np.array_equal(absorbed[sure], (inside & reach)[sure])
    assert stats["absorbed"] == absorbed.sum()
    # which cell: x > y lies in cell 0, x < y in cell 1
    q = np.where(sp == 1, 1, -1)
    hit = absorbed & sure
    exp0 = q[hit & (p32[:, 0] > p32[:, 1])].sum()
    exp1 = q[hit & (p32[:, 0] < p32[:, 1])].sum()
    on_edge = absorbed & ~sure
    assert dep.sum() == q[absorbed].sum()
    assert abs(dep[0] - exp0) + abs(dep[1] - exp1) <= np.abs(q[on_edge]).sum()
