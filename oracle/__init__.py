"""CPU oracle for the OuroborosBEM field + tracking-step method (arXiv 2110.09214).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product path never imports it and
shares no code with it.  The arithmetic lives in ``obem_oracle.c`` (FP64 for
geometry, integrals, fields and the BEM system; IEEE binary32 with one rounding
per operation for the tracking step, whose integer decisions must be taken in
the kernel's precision).  This module only marshals numpy arrays, plus the
swarm-parameter fits of Sec. 4.1 (Eqs. (vd), (diffusion), (townsend)).

Parity status of each function (see the test-suite for the pins):
  tri_integrals, panel_field, nbody_field, assemble, bem_solve, influence_rhs,
  philox, step, swarm fits, tri_jacobian, field_jacobian, field_backward,
  bem_solve_adjoint, grid_nodes, trilinear, nbody_nn: pinned.
  gas_constants and the step on tabulated cross sections (grid lookup,
  interpolation, thresholds, majorant, excitation and ionisation energetics):
  pinned by tests/test_oracle_gas_pins.py.
  No function here is unpinned.  The swarm parameters of the synthetic
  argon-like gas are not a function of their own: they are the pinned fits
  applied to the moments of many pinned steps.  That gas has no closed form
  for them, so their GPU-vs-oracle agreement (16 seeds per side, 3 sigma) is
  a consistency check, not a pin.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from .build import build as _build

KC = 1.0 / (4.0 * math.pi * 8.8541878128e-12)
E_CHARGE = 1.602176634e-19
M_ELECTRON = 9.1093837015e-31
EPS0 = 8.8541878128e-12
N_STATS = 25
STATS_NAMES = ["n_before", "n_after", "n_electron", "n_cation", "n_anion", "spawned_pairs",
               "absorbed", "attached", "recombined_pairs", "collisions", "trials",
               "required_capacity", "sum_x_e", "sum_y_e", "sum_z_e", "sum_x2_e", "sum_y2_e",
               "sum_z2_e", "sum_x_i", "sum_y_i", "sum_z_i", "sum_x2_i", "sum_y2_i", "sum_z2_i",
               "sum_energy_e"]
ST_OK, ST_CAPACITY, ST_TRIALS = 0, -6, -8

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build())
        P = C.c_void_p
        I = C.c_int
        U = C.c_uint32
        _lib.or_tri_integrals.argtypes = [P, P, P, P]
        _lib.or_tri_geometry.argtypes = [P, P, P, P]
        _lib.or_panel_field.argtypes = [I, P, P, I, P, P, P]
        _lib.or_nbody_field.argtypes = [I, P, I, P, I, C.c_double, P, P]
        _lib.or_tri_jacobian.argtypes = [P, P, P]
        _lib.or_trilinear.argtypes = [I, I, I, P, P, I, P, I, P, P]
        _lib.or_nbody_nn.argtypes = [I, P, I, C.c_double, P]
        _lib.or_field_jacobian.argtypes = [I, P, P, I, P, I, P, I, P]
        _lib.or_field_backward.argtypes = [I, P, P, I, P, I, P, I, P, P, P, P]
        _lib.or_assemble.argtypes = [I, P, P, P, P, P]
        _lib.or_solve_gepp.argtypes = [I, P, P]
        _lib.or_solve_gepp.restype = I
        _lib.or_influence_rhs.argtypes = [I, P, P, P, P, I, P, P]
        _lib.or_philox4x32_10.argtypes = [P, P, P]
        _lib.or_gas_constants.argtypes = [P, I, I, P, P, P, P, P, P, P]
        _lib.or_step.argtypes = [I, P, P, P, P, P, P, U, U, P, I, I, P, P, P, P, P, P,
                                 I, P, P, P, P, P, P, P, P, I, P, P]
        _lib.or_step.restype = I
        _lib.or_neg_log_u.argtypes = [U]
        _lib.or_neg_log_u.restype = C.c_float
        _lib.or_iso_dir.argtypes = [U, U, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- geometry / BEM
def tri_integrals(v, r):
    """phi = int_T dA'/|r-r'| and F = int_T (r-r')/|r-r'|^3 dA' (unit density)."""
    v = _c(v, np.float64).reshape(9)
    r = _c(r, np.float64).reshape(3)
    phi = np.zeros(1)
    F = np.zeros(3)
    lib().or_tri_integrals(_p(v), _p(r), _p(phi), _p(F))
    return float(phi[0]), F


def tri_geometry(v):
    v = _c(v, np.float64).reshape(9)
    c, n, a = np.zeros(3), np.zeros(3), np.zeros(1)
    lib().or_tri_geometry(_p(v), _p(c), _p(n), _p(a))
    return c, n, float(a[0])


def panel_field(tri, sigma, pts):
    """E and V of the cells with densities sigma at pts, Eqs. (BEM2), (BEM3)."""
    tri = _c(tri, np.float64)
    sigma = _c(sigma, np.float64)
    pts = _c(pts, np.float64).reshape(-1, 3)
    E = np.zeros((len(pts), 3))
    V = np.zeros(len(pts))
    lib().or_panel_field(len(sigma), _p(tri), _p(sigma), len(pts), _p(pts), _p(E), _p(V))
    return E, V


def nbody_field(pts, src, self_exclude=False, soft=0.0):
    """Coulomb field of point charges src[:, :3] with charges src[:, 3], Eq. (nbody)."""
    pts = _c(pts, np.float64).reshape(-1, 3)
    src = _c(src, np.float64).reshape(-1, 4)
    E = np.zeros((len(pts), 3))
    V = np.zeros(len(pts))
    lib().or_nbody_field(len(pts), _p(pts), len(src), _p(src), int(self_exclude),
                         float(soft), _p(E), _p(V))
    return E, V


def tri_jacobian(v, r):
    """J[a, b] = dF_a/dr_b of the unit-density cell field F (closed form)."""
    v = _c(v, np.float64).reshape(9)
    r = _c(r, np.float64).reshape(3)
    J = np.zeros(9)
    lib().or_tri_jacobian(_p(v), _p(r), _p(J))
    return J.reshape(3, 3)


def _field_inputs(tri, sigma, pts, src):
    tri = _c(np.zeros((0, 3, 3)) if tri is None else tri, np.float64).reshape(-1, 9)
    sigma = _c(np.zeros(0) if sigma is None else sigma, np.float64).reshape(-1)
    if len(sigma) == 0:
        tri = tri[:0]
    pts = _c(pts, np.float64).reshape(-1, 3)
    src = _c(np.zeros((0, 4)) if src is None else src, np.float64).reshape(-1, 4)
    return tri, sigma, pts, src


def field_jacobian(tri, sigma, pts, src=None, self_exclude=False):
    """dE/dr at pts (nt x 3 x 3) of cells with densities sigma plus point
    charges src (derivatives of Eqs. (BEM3), (nbody))."""
    tri, sigma, pts, src = _field_inputs(tri, sigma, pts, src)
    J = np.zeros((len(pts), 9))
    lib().or_field_jacobian(len(sigma), _p(tri), _p(sigma), len(pts), _p(pts), len(src), _p(src),
                            int(self_exclude), _p(J))
    return J.reshape(-1, 3, 3)


def field_backward(tri, sigma, pts, src, self_exclude, g):
    """Vector-Jacobian product of the field evaluation (E, V) at pts for the
    upstream gradient g (nt x 4): returns dL/dsigma (np), dL/dpts (nt x 3)
    and dL/dsrc (ns x 4: position, charge)."""
    tri, sigma, pts, src = _field_inputs(tri, sigma, pts, src)
    g = _c(g, np.float64).reshape(-1, 4)
    ds = np.zeros(len(sigma))
    dp = np.zeros((len(pts), 3))
    dq = np.zeros((len(src), 4))
    lib().or_field_backward(len(sigma), _p(tri), _p(sigma), len(pts), _p(pts), len(src), _p(src),
                            int(self_exclude), _p(g), _p(ds), _p(dp), _p(dq))
    return ds, dp, dq


def grid_nodes(lo, hi, dims):
    """Nodes lo + (i, j, k) (hi - lo) / (dims - 1) of a regular grid, x fastest
    ([nz * ny * nx, 3]) -- the static field map's nodes (Sec. 2.4)."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    step = (hi - lo) / (np.asarray(dims) - 1)
    k, j, i = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    return np.column_stack([lo[0] + i.ravel() * step[0], lo[1] + j.ravel() * step[1], lo[2] + k.ravel() * step[2]])


def trilinear(values, lo, hi, dims, pts):
    """Trilinear interpolation of node values ([n_nodes, nc], x fastest) at
    pts; points outside the box are moved to the nearest point of the box."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    step = (hi - lo) / (np.asarray(dims) - 1)
    values = _c(values, np.float64)
    nc = values.shape[1] if values.ndim == 2 else 1
    pts = _c(pts, np.float64).reshape(-1, 3)
    out = np.zeros((len(pts), nc))
    lib().or_trilinear(int(dims[0]), int(dims[1]), int(dims[2]), _p(_c(lo, np.float64)), _p(_c(step, np.float64)),
                       nc, _p(values), len(pts), _p(pts), _p(out))
    return out


def nbody_nn(src, grid, soft=0.0):
    """Approximate N-body field at the charges (Sec. 3.2.4 nearest-neighbour
    option): exact over the 27 cells around each charge, per-sign charge
    centres of the other cells (grid^3 cells over the bounding box)."""
    src = _c(src, np.float64).reshape(-1, 4)
    E = np.zeros((len(src), 3))
    lib().or_nbody_nn(len(src), _p(src), int(grid), float(soft), _p(E))
    return E


def assemble(mesh):
    """Dense matrix of Eq. (matrixBEM): Q rows for electrode cells, W rows for
    dielectric cells (Eqs. (BEMpot), (BEMfld))."""
    n = mesh.n
    A = np.zeros((n, n))
    lib().or_assemble(n, _p(_c(mesh.tri, np.float64)), _p(_c(mesh.kind, np.int32)),
                      _p(_c(mesh.eps_minus, np.float64)), _p(_c(mesh.eps_plus, np.float64)),
                      _p(A))
    return A


def bem_rhs(mesh, sigma_free=None, drhs=None, group_voltage=None):
    """Left-hand side vector of Eq. (matrixBEM): V_k on electrode cells, the
    free density on dielectric cells, plus an optional influence correction."""
    gv = mesh.group_voltage if group_voltage is None else np.asarray(group_voltage)
    b = np.where(mesh.kind == 0, gv[np.maximum(mesh.group, 0)], 0.0).astype(np.float64)
    if sigma_free is not None:
        b = b + np.where(mesh.kind == 1, sigma_free, 0.0)
    if drhs is not None:
        b = b + drhs
    return b


def solve(A, b, force_gepp=False):
    """Direct solve: the oracle's own Gaussian elimination with partial
    pivoting for n <= 3000, LAPACK's (numpy) above."""
    n = len(b)
    if n <= 3000 or force_gepp:
        A2 = np.array(A, np.float64, order="C", copy=True)
        x = np.array(b, np.float64, copy=True)
        if lib().or_solve_gepp(n, _p(A2), _p(x)) != 0:
            raise np.linalg.LinAlgError("singular BEM matrix")
        return x
    return np.linalg.solve(A, b)


def bem_solve(mesh, sigma_free=None, drhs=None, group_voltage=None):
    A = assemble(mesh)
    return solve(A, bem_rhs(mesh, sigma_free, drhs, group_voltage))


def bem_solve_adjoint(mesh, g_sigma):
    """Adjoint of bem_solve for L with dL/dsigma = g_sigma: mu = A^-T g_sigma
    is dL/db for the right-hand side b of Eq. (matrixBEM) (so it is dL/d
    sigma_free on dielectric cells and dL/d drhs everywhere), and dL/dV_k is
    the sum of mu over the electrode cells of group k.  Returns (mu, dL/dV)."""
    A = assemble(mesh)
    mu = solve(np.ascontiguousarray(A.T), np.asarray(g_sigma, np.float64))
    ed = mesh.kind == 0
    dV = np.zeros(len(mesh.group_voltage))
    np.add.at(dV, mesh.group[ed], mu[ed])
    return mu, dV


def influence_rhs(mesh, src):
    """RHS correction of Eqs. (BEMpotpart), (BEMfldpart) from charges src."""
    src = _c(src, np.float64).reshape(-1, 4)
    d = np.zeros(mesh.n)
    lib().or_influence_rhs(mesh.n, _p(_c(mesh.tri, np.float64)), _p(_c(mesh.kind, np.int32)),
                           _p(_c(mesh.eps_minus, np.float64)), _p(_c(mesh.eps_plus, np.float64)),
                           len(src), _p(src), _p(d))
    return d


# ---------------------------------------------------------------- RNG
def philox(ctr, key):
    ctr = _c(ctr, np.uint32).reshape(4)
    key = _c(key, np.uint32).reshape(2)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(ctr), _p(key), _p(out))
    return out


# ---------------------------------------------------------------- step
def neg_log_u(u):
    """-ln(((u >> 8) + 1) 2^-24) as computed inside the step (binary32)."""
    return float(lib().or_neg_log_u(int(u)))


def iso_dir(ua, ub):
    d = np.zeros(3, np.float32)
    lib().or_iso_dir(int(ua), int(ub), _p(d))
    return d


def _prm(gas, trk):
    seed = int(trk.seed)
    return np.array([trk.dt, gas.T, gas.N, gas.M_amu, gas.nu_ion, trk.z_lo, trk.z_hi,
                     trk.beta, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF, trk.trial_cap,
                     getattr(trk, "coll_mode", 0), 1 if getattr(trk, "surface_hits", False) else 0],
                    np.float64)


def _gas_arrays(gas):
    return (_c(gas.egrid, np.float32), _c(gas.xs, np.float32), _c(gas.kind, np.int32),
            _c(gas.mode, np.int32), _c(gas.thr, np.float32), _c(gas.nuc, np.float32))


def gas_constants(gas, trk):
    eg, xs, kind, mode, thr, nuc = _gas_arrays(gas)
    out = np.zeros(8, np.float32)
    prm = _prm(gas, trk)
    lib().or_gas_constants(_p(prm), gas.n_proc, len(eg), _p(eg), _p(xs), _p(kind), _p(mode),
                           _p(thr), _p(nuc), _p(out))
    keys = ["nu_max_e", "E_therm", "v_th_ion", "rc2", "KCE", "K_e", "two_m_over_M", "recomb_on"]
    return dict(zip(keys, out.tolist()))


def step(ch, E, step_index, next_id, gas, trk, capacity=None, mesh=None, deposits=None):
    """One tracking step (binary32 decisions).  Returns (status, charges_out,
    next_id_out, stats dict).  With trk.surface_hits and a mesh, charges whose
    sub-flight chords cross a cell are absorbed there and counted (in units
    of e, by sign) into deposits (int64 [n_cells], updated in place when the
    step commits)."""
    from types import SimpleNamespace
    n = ch.pos_q.shape[0]
    cap = int(capacity if capacity is not None else max(4 * n + 64, 64))
    E = _c(np.asarray(E)[:, :3], np.float32)
    eg, xs, kind, mode, thr, nuc = _gas_arrays(gas)
    prm = _prm(gas, trk)
    o_pos = np.zeros((cap, 4), np.float32)
    o_vel = np.zeros((cap, 4), np.float32)
    o_id = np.zeros(cap, np.uint32)
    o_birth = np.zeros(cap, np.uint32)
    o_sp = np.zeros(cap, np.uint8)
    o_n = np.zeros(1, np.int32)
    o_next = np.zeros(1, np.uint32)
    stats = np.zeros(N_STATS)
    pos = _c(ch.pos_q, np.float32)
    vel = _c(ch.vel, np.float32)
    ids = _c(ch.id, np.uint32)
    birth = _c(ch.birth, np.uint32)
    sp = _c(ch.species, np.uint8)
    tri9 = _c(np.zeros((0, 9)) if mesh is None else np.asarray(mesh.tri).reshape(-1, 9), np.float32)
    if deposits is None:
        deposits = np.zeros(len(tri9), np.int64)
    assert deposits.dtype == np.int64 and deposits.flags.c_contiguous and len(deposits) == len(tri9)
    st = lib().or_step(n, _p(pos), _p(vel), _p(ids), _p(birth), _p(sp), _p(E),
                       int(step_index), int(next_id), _p(prm), gas.n_proc, len(eg), _p(eg),
                       _p(xs), _p(kind), _p(mode), _p(thr), _p(nuc), cap, _p(o_pos), _p(o_vel),
                       _p(o_id), _p(o_birth), _p(o_sp), _p(o_n), _p(o_next), _p(stats),
                       len(tri9), _p(tri9), _p(deposits))
    m = int(o_n[0]) if st == ST_OK else 0
    out = SimpleNamespace(pos_q=o_pos[:m].copy(), vel=o_vel[:m].copy(), id=o_id[:m].copy(),
                          birth=o_birth[:m].copy(), species=o_sp[:m].copy(), n=m)
    return st, out, int(o_next[0]) if st == ST_OK else int(next_id), dict(zip(STATS_NAMES, stats))


def field_at_charges(ch, mesh=None, sigma=None, soft=0.0, e_ext=None):
    """Total field at every charge: cells (Eq. (BEM3)) + all other charges
    (Eq. (nbody)), FP64."""
    pts = np.asarray(ch.pos_q[:, :3], np.float64)
    src = np.asarray(ch.pos_q, np.float64)
    E, _ = nbody_field(pts, src, self_exclude=True, soft=soft)
    if mesh is not None and sigma is not None:
        Ep, _ = panel_field(mesh.tri, sigma, pts)
        E = E + Ep
    if e_ext is not None:
        E = E + np.asarray(e_ext)[None, :]
    return E


def run(ch, gas, trk, n_steps, mesh=None, sigma=None, space_charge=True, e_ext=None,
        capacity=None, start_step=0, next_id=None):
    """Multi-step oracle run: field in FP64 at step start, rounded to binary32,
    then the binary32 step.  Returns (final charges, next_id, list of stats)."""
    hist = []
    nid = int(ch.pos_q.shape[0]) if next_id is None else int(next_id)
    cur = ch
    for s in range(start_step, start_step + n_steps):
        if cur.pos_q.shape[0] == 0:
            break
        if space_charge:
            E = field_at_charges(cur, mesh, sigma, trk.softening, e_ext)
        else:
            pts = np.asarray(cur.pos_q[:, :3], np.float64)
            E = np.zeros_like(pts)
            if mesh is not None and sigma is not None:
                E = panel_field(mesh.tri, sigma, pts)[0]
            if e_ext is not None:
                E = E + np.asarray(e_ext)[None, :]
        st, cur, nid, stats = step(cur, E.astype(np.float32), s, nid, gas, trk, capacity)
        if st != ST_OK:
            raise RuntimeError("oracle step status %d" % st)
        hist.append(stats)
    return cur, nid, hist


# ---------------------------------------------------------------- swarm fits
def cloud_moments(hist, species="e"):
    """Mean and variance per axis from the per-step sums."""
    suf = "_e" if species == "e" else "_i"
    nk = "n_electron" if species == "e" else "n_cation"
    n = np.array([h[nk] + (h["n_anion"] if species != "e" else 0) for h in hist], np.float64)
    mean = np.array([[h["sum_%s%s" % (a, suf)] for a in "xyz"] for h in hist]) / n[:, None]
    m2 = np.array([[h["sum_%s2%s" % (a, suf)] for a in "xyz"] for h in hist]) / n[:, None]
    return n, mean, m2 - mean ** 2


def drift_velocity(t, zmean):
    """Eq. (vd): slope of the cloud centroid along the field (least squares)."""
    return float(np.polyfit(t, zmean, 1)[0])


def diffusion_coefficient(t, var):
    """Eq. (diffusion): sigma^2 = 2 D t, D from the slope of the variance."""
    return float(np.polyfit(t, var, 1)[0] / 2.0)


def townsend_alpha(t, n_e, v_d):
    """Eq. (townsend) with G = exp(alpha d), d = V_d t: alpha = d ln N / (V_d dt)."""
    return float(np.polyfit(t, np.log(n_e), 1)[0] / v_d)
