"""Seeded synthetic inputs: meshes, charge clouds and gas tables.

This module only *describes* workloads (geometry, initial charges, cross-section
shapes); it contains none of the method's arithmetic (no panel integrals, no
field, no collision physics).  Both the CUDA path and the CPU oracle consume
its output, which is why it depends on nothing but numpy.

Units are SI (metres, volts, seconds, m^2 for cross sections, eV for energies
on the cross-section grid).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

E_CHARGE = 1.602176634e-19
M_ELECTRON = 9.1093837015e-31
K_BOLTZMANN = 1.380649e-23

KIND_ELECTRODE = 0      # ed-interface cell (Dirichlet row)
KIND_DIELECTRIC = 1     # dd-interface cell (Neumann row)

P_ELASTIC, P_EXCITATION, P_IONISATION, P_ATTACHMENT = 0, 1, 2, 3
MODE_TABLE, MODE_CONST = 0, 1

SP_ELECTRON, SP_CATION, SP_ANION = 0, 1, 2


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Mesh:
    """Flat triangular cells.  tri[i] = (v0, v1, v2), the cell normal is
    (v1-v0) x (v2-v0) and points from the eps_minus side to the eps_plus side."""
    tri: np.ndarray            # float64 [n, 3, 3]
    kind: np.ndarray           # int32 [n]  KIND_ELECTRODE / KIND_DIELECTRIC
    group: np.ndarray          # int32 [n]  electrode group (ed cells), -1 for dd
    eps_minus: np.ndarray      # float64 [n] relative permittivity, negative side
    eps_plus: np.ndarray       # float64 [n] relative permittivity, positive side
    group_voltage: np.ndarray  # float64 [n_groups]

    @property
    def n(self) -> int:
        return int(self.tri.shape[0])

    @property
    def n_groups(self) -> int:
        return int(self.group_voltage.shape[0])


def _concat(parts):
    tri = np.concatenate([p[0] for p in parts], axis=0)
    kind = np.concatenate([np.full(len(p[0]), p[1], np.int32) for p in parts])
    group = np.concatenate([np.full(len(p[0]), p[2], np.int32) for p in parts])
    em = np.concatenate([np.full(len(p[0]), p[3], np.float64) for p in parts])
    ep = np.concatenate([np.full(len(p[0]), p[4], np.float64) for p in parts])
    return tri, kind, group, em, ep


def rect_plate(x0, x1, y0, y1, z, nx, ny, up=True):
    """Square grid of nx*ny quads on the plane z, each split into 2 triangles,
    normal +z (up) or -z."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    tris = []
    for i in range(nx):
        for j in range(ny):
            a = (xs[i], ys[j], z)
            b = (xs[i + 1], ys[j], z)
            c = (xs[i + 1], ys[j + 1], z)
            d = (xs[i], ys[j + 1], z)
            if up:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, c, b), (a, d, c)]
    return np.asarray(tris, np.float64)


def parallel_plates(side=1e-2, gap=1e-3, n=16, v_low=0.0, v_high=100.0, ny=None) -> Mesh:
    """Two side x side plates at z=0 (v_low) and z=gap (v_high), n*ny*2
    triangles each (ny = n by default; the Sec. 2.4 timing set-up and the
    swarm chambers of Sec. 4.1)."""
    ny = n if ny is None else ny
    lo = rect_plate(0, side, 0, side, 0.0, n, ny, up=True)
    hi = rect_plate(0, side, 0, side, gap, n, ny, up=False)
    tri, kind, group, em, ep = _concat([(lo, KIND_ELECTRODE, 0, 1.0, 1.0),
                                        (hi, KIND_ELECTRODE, 1, 1.0, 1.0)])
    return Mesh(tri, kind, group, em, ep, np.array([v_low, v_high], np.float64))


def icosphere(radius=1.0, level=2, center=(0.0, 0.0, 0.0)):
    """Subdivided icosahedron projected on a sphere; outward normals."""
    t = (1.0 + 5 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
             (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9),
             (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2),
             (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
             (8, 6, 7), (9, 8, 1)]
    v = [np.asarray(p, np.float64) / np.linalg.norm(p) for p in verts]
    for _ in range(level):
        cache = {}
        nf = []

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = v[i] + v[j]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.asarray(v) * radius + np.asarray(center, np.float64)
    tri = V[np.asarray(faces)]
    # orient outward
    cen = tri.mean(axis=1) - np.asarray(center)
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    flip = (nrm * cen).sum(axis=1) < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return tri


def conducting_sphere(radius=1e-3, level=3, voltage=1.0) -> Mesh:
    tri = icosphere(radius, level)
    n = len(tri)
    return Mesh(tri, np.zeros(n, np.int32), np.zeros(n, np.int32), np.ones(n), np.ones(n),
                np.array([voltage], np.float64))


def dielectric_sphere_in_plates(radius=1e-3, level=3, eps_r=4.0, side=2e-2, gap=1e-2,
                                n_plate=24, v=1000.0) -> Mesh:
    """Dielectric sphere (eps_r inside, vacuum outside) centred between two
    large plates that make an approximately uniform field."""
    c = (side / 2, side / 2, gap / 2)
    sph = icosphere(radius, level, c)
    lo = rect_plate(0, side, 0, side, 0.0, n_plate, n_plate, up=True)
    hi = rect_plate(0, side, 0, side, gap, n_plate, n_plate, up=False)
    tri, kind, group, em, ep = _concat([(lo, KIND_ELECTRODE, 0, 1.0, 1.0),
                                        (hi, KIND_ELECTRODE, 1, 1.0, 1.0),
                                        (sph, KIND_DIELECTRIC, -1, eps_r, 1.0)])
    return Mesh(tri, kind, group, em, ep, np.array([0.0, v], np.float64))


# --------------------------------------------------------------------------
# GEM unit patch
# --------------------------------------------------------------------------
@dataclasses.dataclass
class GemGeometry:
    pitch: float = 140e-6
    d_outer: float = 70e-6        # hole diameter at the kapton surfaces and in the copper
    d_inner: float = 50e-6        # hole diameter at the foil mid-plane
    t_kapton: float = 50e-6
    t_copper: float = 5e-6
    eps_kapton: float = 3.5
    gap_drift: float = 300e-6
    gap_induction: float = 300e-6
    dv_gem: float = 400.0
    e_drift: float = 2e5          # V/m (2 kV/cm)
    e_induction: float = 3e5      # V/m (3 kV/cm)
    rings: int = 2                # hexagonal patch: 1 + 3 rings (rings + 1) holes

    def hole_centres(self):
        p = self.pitch
        out = []
        R = self.rings
        for q in range(-R, R + 1):
            for r in range(-R, R + 1):
                s = -q - r
                if max(abs(q), abs(r), abs(s)) > R:
                    continue
                out.append((p * (q + r / 2.0), p * (r * math.sqrt(3) / 2.0)))
        return np.asarray(out, np.float64)

    def voltages(self):
        """Groups: 0 drift plane, 1 top copper, 2 bottom copper, 3 anode."""
        v_anode = 0.0
        v_bot = v_anode - self.e_induction * self.gap_induction
        v_top = v_bot - self.dv_gem
        v_drift = v_top - self.e_drift * self.gap_drift
        return np.array([v_drift, v_top, v_bot, v_anode], np.float64)

    @property
    def z_top(self):
        return self.t_kapton / 2 + self.t_copper

    @property
    def z_drift(self):
        return self.z_top + self.gap_drift

    @property
    def z_anode(self):
        return -self.z_top - self.gap_induction


def _hex_radius(theta, apothem):
    # Voronoi cell of the hexagonal lattice whose neighbours lie at 0, 60, ... deg
    k = np.round(theta / (np.pi / 3.0))
    return apothem / np.cos(theta - k * np.pi / 3.0)


def _ring_face(cx, cy, z, r_in, apothem, n_th, n_r, up):
    th = np.arange(n_th + 1) * (2 * np.pi / n_th)
    s = (np.arange(n_r + 1) / n_r) ** 1.5          # finer near the hole edge
    tris = []
    for i in range(n_th):
        for j in range(n_r):
            pts = []
            for (a, b) in ((i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)):
                R = _hex_radius(th[a], apothem)
                rr = r_in + s[b] * (R - r_in)
                pts.append((cx + rr * np.cos(th[a]), cy + rr * np.sin(th[a]), z))
            A, B, C, D = pts
            if up:
                tris += [(A, B, C), (A, C, D)]
            else:
                tris += [(A, C, B), (A, D, C)]
    return tris


def _wall(cx, cy, z0, z1, r0, r1, n_th, n_z, inward):
    """Surface of revolution between (r0 at z0) and (r1 at z1); normals point
    toward the axis if inward."""
    th = np.arange(n_th + 1) * (2 * np.pi / n_th)
    zs = np.linspace(z0, z1, n_z + 1)
    rs = np.linspace(r0, r1, n_z + 1)
    tris = []
    for i in range(n_th):
        for j in range(n_z):
            A = (cx + rs[j] * np.cos(th[i]), cy + rs[j] * np.sin(th[i]), zs[j])
            B = (cx + rs[j] * np.cos(th[i + 1]), cy + rs[j] * np.sin(th[i + 1]), zs[j])
            C = (cx + rs[j + 1] * np.cos(th[i + 1]), cy + rs[j + 1] * np.sin(th[i + 1]), zs[j + 1])
            D = (cx + rs[j + 1] * np.cos(th[i]), cy + rs[j + 1] * np.sin(th[i]), zs[j + 1])
            tris += [(A, B, C), (A, C, D)]
    tri = np.asarray(tris, np.float64)
    cen = tri.mean(axis=1)
    radial = cen[:, :2] - np.array([cx, cy])
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    outward = (nrm[:, :2] * radial).sum(axis=1) > 0
    flip = outward if inward else ~outward
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return tri


def _gem_foil(g: GemGeometry, z0, n_theta, n_r, n_zc, n_zk):
    """Cells of one GEM foil centred at z = z0: the copper of its top and
    bottom layers (faces and hole walls) and the biconical kapton hole walls."""
    ap = g.pitch / 2.0
    r_out, r_in = g.d_outer / 2, g.d_inner / 2
    zk = g.t_kapton / 2
    zc = zk + g.t_copper
    top, bot, kap = [], [], []
    for cx, cy in g.hole_centres():
        top += _ring_face(cx, cy, z0 + zc, r_out, ap, n_theta, n_r, up=True)
        top += _ring_face(cx, cy, z0 + zk, r_out, ap, n_theta, n_r, up=False)
        bot += _ring_face(cx, cy, z0 - zk, r_out, ap, n_theta, n_r, up=True)
        bot += _ring_face(cx, cy, z0 - zc, r_out, ap, n_theta, n_r, up=False)
        top += list(_wall(cx, cy, z0 + zk, z0 + zc, r_out, r_out, n_theta, n_zc, inward=True))
        bot += list(_wall(cx, cy, z0 - zc, z0 - zk, r_out, r_out, n_theta, n_zc, inward=True))
        half = n_zk // 2
        kap += list(_wall(cx, cy, z0 - zk, z0, r_out, r_in, n_theta, half, inward=True))
        kap += list(_wall(cx, cy, z0, z0 + zk, r_in, r_out, n_theta, n_zk - half, inward=True))
    return np.asarray(top, np.float64), np.asarray(bot, np.float64), np.asarray(kap, np.float64)


def _plane_half_width(g: GemGeometry):
    cen = g.hole_centres()
    ext = np.abs(cen).max(axis=0) + g.pitch
    return float(ext.max())


def gem_mesh(geo: GemGeometry | None = None, n_theta=48, n_r=4, n_zc=2, n_zk=12,
             n_plane=20) -> Mesh:
    """Single-GEM patch: copper (top/bottom faces and hole walls of both
    layers), biconical kapton hole walls (dd cells, kapton on the negative
    side), and the drift and induction planes (Sec. 4.2 geometry; sizes of the
    CERN design).  Electrode groups as in GemGeometry.voltages()."""
    g = geo or GemGeometry()
    top, bot, kap = _gem_foil(g, 0.0, n_theta, n_r, n_zc, n_zk)
    L = _plane_half_width(g)
    drift = rect_plate(-L, L, -L, L, g.z_drift, n_plane, n_plane, up=False)
    anode = rect_plate(-L, L, -L, L, g.z_anode, n_plane, n_plane, up=True)
    parts = [(drift, KIND_ELECTRODE, 0, 1.0, 1.0),
             (top, KIND_ELECTRODE, 1, 1.0, 1.0),
             (bot, KIND_ELECTRODE, 2, 1.0, 1.0),
             (anode, KIND_ELECTRODE, 3, 1.0, 1.0),
             (kap, KIND_DIELECTRIC, -1, g.eps_kapton, 1.0)]
    tri, kind, group, em, ep = _concat(parts)
    return Mesh(tri, kind, group, em, ep, g.voltages())


def gem_triangle_count(holes, n_theta, n_r, n_zc, n_zk, n_plane):
    return holes * (4 * n_theta * n_r * 2 + 2 * n_theta * n_zc * 2 + n_theta * n_zk * 2) \
        + 2 * n_plane * n_plane * 2


def _resolution_search(target, count, tol):
    """(n_theta, n_r, n_zk, n_plane) whose triangle count(n_theta, n_r, n_zc=2,
    n_zk, n_plane) is within tol of target, hole walls as square as possible."""
    best = None
    for n_theta in range(24, 145, 12):
        for n_r in range(2, 9):
            for n_zk in range(4, 25, 2):
                for n_plane in range(8, 41, 2):
                    c = count(n_theta, n_r, 2, n_zk, n_plane)
                    err = abs(c - target) / target
                    score = (err > tol, abs(n_theta / (4 * n_zk) - 1.0), err)
                    if best is None or score < best[0]:
                        best = (score, (n_theta, n_r, n_zk, n_plane))
    return best[1]


def gem_mesh_target(target=60000, geo: GemGeometry | None = None, tol=0.01) -> Mesh:
    """GEM patch with a triangle count within tol of target (mesh resolution
    chosen by a small search over the angular / radial / plane divisions)."""
    g = geo or GemGeometry()
    holes = len(g.hole_centres())
    n_theta, n_r, n_zk, n_plane = _resolution_search(
        target, lambda *a: gem_triangle_count(holes, *a), tol)
    return gem_mesh(g, n_theta=n_theta, n_r=n_r, n_zc=2, n_zk=n_zk, n_plane=n_plane)


def gem_inside_solid(geo: GemGeometry, pts):
    """True where a point lies inside copper or kapton of the GEM foil."""
    pts = np.asarray(pts)
    zk = geo.t_kapton / 2
    zc = zk + geo.t_copper
    cen = geo.hole_centres()
    d2 = ((pts[:, None, :2] - cen[None, :, :]) ** 2).sum(-1)
    r = np.sqrt(d2.min(axis=1))
    z = pts[:, 2]
    r_out, r_in = geo.d_outer / 2, geo.d_inner / 2
    in_foil = np.abs(z) < zc
    wall = np.where(np.abs(z) < zk, r_in + (r_out - r_in) * np.abs(z) / zk, r_out)
    return in_foil & (r >= wall)


@dataclasses.dataclass
class DoubleGemGeometry:
    """Two foils of the single-GEM design stacked along z, their mid-planes
    `spacing` apart (upper foil at +spacing/2), the drift plane gap_drift above
    the upper foil's copper, the anode gap_induction below the lower foil's,
    and a transfer field e_transfer between the foils."""
    foil: GemGeometry = dataclasses.field(default_factory=GemGeometry)
    spacing: float = 2e-3
    e_transfer: float = 3e5       # V/m (3 kV/cm)

    @property
    def z_upper(self):
        return self.spacing / 2

    @property
    def z_lower(self):
        return -self.spacing / 2

    @property
    def z_drift(self):
        return self.z_upper + self.foil.z_top + self.foil.gap_drift

    @property
    def z_anode(self):
        return self.z_lower - self.foil.z_top - self.foil.gap_induction

    def voltages(self):
        """Groups: 0 drift plane, 1 / 2 upper foil top / bottom copper, 3 / 4
        lower foil top / bottom copper, 5 anode (0 V)."""
        f = self.foil
        v5 = 0.0
        v4 = v5 - f.e_induction * f.gap_induction
        v3 = v4 - f.dv_gem
        v2 = v3 - self.e_transfer * (self.spacing - 2 * f.z_top)
        v1 = v2 - f.dv_gem
        v0 = v1 - f.e_drift * f.gap_drift
        return np.array([v0, v1, v2, v3, v4, v5], np.float64)


def double_gem_mesh(geo: DoubleGemGeometry | None = None, n_theta=48, n_r=4, n_zc=2, n_zk=12,
                    n_plane=20) -> Mesh:
    """Double-GEM stack: both foils meshed as in gem_mesh (copper electrodes,
    kapton hole walls as dd cells), the drift plane and the anode.  Electrode
    groups as in DoubleGemGeometry.voltages()."""
    d = geo or DoubleGemGeometry()
    g = d.foil
    t1, b1, k1 = _gem_foil(g, d.z_upper, n_theta, n_r, n_zc, n_zk)
    t2, b2, k2 = _gem_foil(g, d.z_lower, n_theta, n_r, n_zc, n_zk)
    L = _plane_half_width(g)
    drift = rect_plate(-L, L, -L, L, d.z_drift, n_plane, n_plane, up=False)
    anode = rect_plate(-L, L, -L, L, d.z_anode, n_plane, n_plane, up=True)
    parts = [(drift, KIND_ELECTRODE, 0, 1.0, 1.0),
             (t1, KIND_ELECTRODE, 1, 1.0, 1.0),
             (b1, KIND_ELECTRODE, 2, 1.0, 1.0),
             (t2, KIND_ELECTRODE, 3, 1.0, 1.0),
             (b2, KIND_ELECTRODE, 4, 1.0, 1.0),
             (anode, KIND_ELECTRODE, 5, 1.0, 1.0),
             (np.concatenate([k1, k2]), KIND_DIELECTRIC, -1, g.eps_kapton, 1.0)]
    tri, kind, group, em, ep = _concat(parts)
    return Mesh(tri, kind, group, em, ep, d.voltages())


def double_gem_triangle_count(holes, n_theta, n_r, n_zc, n_zk, n_plane):
    return 2 * (gem_triangle_count(holes, n_theta, n_r, n_zc, n_zk, n_plane) - 2 * n_plane * n_plane * 2) \
        + 2 * n_plane * n_plane * 2


def double_gem_mesh_target(target=120000, geo: DoubleGemGeometry | None = None, tol=0.01) -> Mesh:
    """Double-GEM stack with a triangle count within tol of target."""
    d = geo or DoubleGemGeometry()
    holes = len(d.foil.hole_centres())
    n_theta, n_r, n_zk, n_plane = _resolution_search(
        target, lambda *a: double_gem_triangle_count(holes, *a), tol)
    return double_gem_mesh(d, n_theta=n_theta, n_r=n_r, n_zc=2, n_zk=n_zk, n_plane=n_plane)


def double_gem_inside_solid(geo: DoubleGemGeometry, pts):
    """True where a point lies inside copper or kapton of either foil."""
    pts = np.asarray(pts, np.float64)
    up = pts - np.array([0.0, 0.0, geo.z_upper])
    lo = pts - np.array([0.0, 0.0, geo.z_lower])
    return gem_inside_solid(geo.foil, up) | gem_inside_solid(geo.foil, lo)


def probe_line(geo: DoubleGemGeometry, n=4096, centre=(0.0, 0.0)):
    """n points on the axis of the hole at `centre`, at the midpoints of n
    equal steps from the anode to the drift plane (none on a plane; the axis
    runs through the holes, so none inside a solid)."""
    z = geo.z_anode + (np.arange(n) + 0.5) * ((geo.z_drift - geo.z_anode) / n)
    return np.column_stack([np.full(n, centre[0]), np.full(n, centre[1]), z])


# --------------------------------------------------------------------------
# charges
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Charges:
    pos_q: np.ndarray      # float32 [n, 4]  x, y, z (m), q (C)
    vel: np.ndarray        # float32 [n, 4]  vx, vy, vz (m/s), 0
    id: np.ndarray         # uint32 [n]
    birth: np.ndarray      # uint32 [n]     0 for initial charges
    species: np.ndarray    # uint8 [n]

    @property
    def n(self) -> int:
        return int(self.pos_q.shape[0])


def make_charges(pos, vel, species) -> Charges:
    n = len(pos)
    pos_q = np.zeros((n, 4), np.float32)
    pos_q[:, :3] = pos
    q = np.where(np.asarray(species) == SP_CATION, E_CHARGE, -E_CHARGE)
    pos_q[:, 3] = q.astype(np.float32)
    vel4 = np.zeros((n, 4), np.float32)
    vel4[:, :3] = vel
    return Charges(pos_q, vel4, np.arange(n, dtype=np.uint32), np.zeros(n, np.uint32),
                   np.asarray(species, np.uint8))


def maxwellian(rng, n, kT_eV, mass):
    s = math.sqrt(kT_eV * E_CHARGE / mass)
    return rng.normal(0.0, s, size=(n, 3))


def uniform_box(rng, n, lo, hi):
    return rng.uniform(np.asarray(lo), np.asarray(hi), size=(n, 3))


def gaussian_ball(rng, n, centre, sigma):
    return np.asarray(centre) + rng.normal(0.0, sigma, size=(n, 3))


# --------------------------------------------------------------------------
# gases
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Gas:
    egrid: np.ndarray      # float32 [n_e] eV, increasing
    xs: np.ndarray         # float32 [n_proc, n_e] m^2 (rows of MODE_CONST ignored)
    kind: np.ndarray       # int32 [n_proc]
    mode: np.ndarray       # int32 [n_proc]
    thr: np.ndarray        # float32 [n_proc] eV
    nuc: np.ndarray        # float32 [n_proc] 1/s for MODE_CONST
    N: float = 2.4143e25   # gas number density (m^-3), 1 bar 300 K
    T: float = 300.0       # K
    M_amu: float = 40.0    # gas / ion mass; <= 0: infinite
    nu_ion: float = 1.6e10  # constant ion collision frequency (1/s)

    @property
    def n_proc(self):
        return int(self.kind.shape[0])


def maxwell_gas(nu=1e12, M_amu=0.0) -> Gas:
    """Constant collision frequency, isotropic elastic only (Maxwell model)."""
    eg = np.asarray([0.01, 1000.0], np.float32)
    return Gas(eg, np.zeros((1, 2), np.float32), np.array([P_ELASTIC], np.int32),
               np.array([MODE_CONST], np.int32), np.zeros(1, np.float32),
               np.array([nu], np.float32), M_amu=M_amu)


def argon_like_gas(n_e=2000) -> Gas:
    """Synthetic argon-like cross sections on a log grid 0.01 .. 1000 eV:
    1 elastic with a Ramsauer-like minimum near 0.25 eV, 10 excitations with
    thresholds 11.5 .. 14 eV, 1 Born-like ionisation at 15.8 eV, 1 attachment
    resonance near 6 eV.  Shapes invented for testing; not measured data."""
    i = np.arange(n_e, dtype=np.float64)
    E = 0.01 * 10.0 ** (5.0 * i / (n_e - 1))
    L = np.log(E / 0.25)
    rows, kinds, thr = [], [], []
    rows.append(1.5e-19 * L * L / (L * L + 1.0) / (1.0 + E / 50.0) + 1e-21)
    kinds.append(P_ELASTIC); thr.append(0.0)
    for j in range(10):
        T = 11.5 + j * 2.5 / 9.0
        x = E / T
        rows.append(np.where(E > T, 2.7e-21 * np.log(np.maximum(x, 1.0)) / x, 0.0))
        kinds.append(P_EXCITATION); thr.append(T)
    I = 15.8
    x = E / I
    rows.append(np.where(E > I, 8e-20 * np.log(np.maximum(x, 1.0)) / x, 0.0))
    kinds.append(P_IONISATION); thr.append(I)
    rows.append(1e-22 * np.exp(-((E - 6.0) / 1.0) ** 2))
    kinds.append(P_ATTACHMENT); thr.append(0.0)
    n_p = len(rows)
    return Gas(E.astype(np.float32), np.asarray(rows).astype(np.float32),
               np.asarray(kinds, np.int32), np.zeros(n_p, np.int32),
               np.asarray(thr, np.float32), np.zeros(n_p, np.float32))


# --------------------------------------------------------------------------
# tracking parameters
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Tracking:
    dt: float = 1e-12
    seed: int = 1
    z_lo: float = 0.0           # absorbing planes (electrodes)
    z_hi: float = 1e-3
    beta: float = -1.0          # recombination rate coefficient (m^3/s); <0 off, 0 -> Eq. distRecomb
    trial_cap: int = 256
    softening: float = 1e-9     # Plummer length for the N-body field in the dynamics
    coll_mode: int = 0          # 0: null-collision trials; 1: the paper's per-step probability
    surface_hits: bool = False  # cells absorb the charges crossing them (charging-up)


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------
def config_small_plates(seed=1, n=1000):
    """Plain method, small size: 1 cm x 1 cm plates 1 mm apart (0 V / 100 V),
    16x16x2 triangles each; Maxwell-model gas, 1e12 /s isotropic elastic;
    n electrons uniform in the gap, Maxwellian at kT = 0.1 eV; dt = 1 ps."""
    rng = np.random.default_rng(seed)
    mesh = parallel_plates(1e-2, 1e-3, 16, 0.0, 100.0)
    pos = uniform_box(rng, n, (0, 0, 0), (1e-2, 1e-2, 1e-3))
    vel = maxwellian(rng, n, 0.1, M_ELECTRON)
    ch = make_charges(pos, vel, np.zeros(n, np.uint8))
    trk = Tracking(dt=1e-12, seed=seed, z_lo=0.0, z_hi=1e-3, beta=-1.0)
    return mesh, maxwell_gas(1e12, 0.0), ch, trk


def config_avalanche(seed=1, e_kv_cm=10.0, n_seed=100, n_plate=32):
    """Parallel-plate avalanche counter: 2 mm gap, 1 cm plates, n_plate^2*2
    triangles each, argon-like gas, seed electrons in a 5 um Gaussian ball
    300 um from the cathode (Sec. 4.1 set-up); beta = 1e-7 cm^3/s."""
    rng = np.random.default_rng(seed)
    gap = 2e-3
    mesh = parallel_plates(1e-2, gap, n_plate, 0.0, e_kv_cm * 1e5 * gap)
    pos = gaussian_ball(rng, n_seed, (5e-3, 5e-3, 300e-6), 5e-6)
    vel = maxwellian(rng, n_seed, 0.1, M_ELECTRON)
    ch = make_charges(pos, vel, np.zeros(n_seed, np.uint8))
    trk = Tracking(dt=1e-12, seed=seed, z_lo=0.0, z_hi=gap, beta=1e-13)
    return mesh, argon_like_gas(), ch, trk


def avalanche_snapshot(rng, n, gap=2e-3, side=1e-2):
    """Avalanche-shaped cloud of n charges (half electrons, half cations): a
    drop-shaped Gaussian cloud with the electrons ahead of the cations."""
    ne = n // 2
    ni = n - ne
    c = np.array([side / 2, side / 2, 0.6 * gap])
    pe = c + rng.normal(0, 1.0, (ne, 3)) * np.array([40e-6, 40e-6, 60e-6]) + [0, 0, 50e-6]
    pi = c + rng.normal(0, 1.0, (ni, 3)) * np.array([40e-6, 40e-6, 120e-6])
    pos = np.concatenate([pe, pi])
    vel = np.concatenate([maxwellian(rng, ne, 1.0, M_ELECTRON), np.zeros((ni, 3))])
    sp = np.concatenate([np.zeros(ne, np.uint8), np.ones(ni, np.uint8)])
    perm = rng.permutation(n)
    return make_charges(pos[perm], vel[perm], sp[perm])


@dataclasses.dataclass
class Chamber:
    """One chamber of the batched sweep."""
    mesh: Mesh
    charges: Charges
    trk: Tracking
    e_kv_cm: float
    n_plate: int


def config_batch(seed=1, n_chambers=256, n_min=100, n_max=100_000, n_plate=(16, 32), side=1e-2):
    """Batched sweep of independent parallel-plate chambers, uneven sizes.
    Chamber i draws from its own generator (seed + i): gap ~ U(0.5, 3) mm,
    field ~ logU(0.1, 30) kV/cm (lower plate 0 V, upper plate E * gap),
    charges ~ logU(n_min, n_max) as an avalanche-shaped cloud (half electrons,
    half cations) with z kept inside (2 %, 98 %) of the gap, plates of
    n x n x 2 triangles each with n ~ U{n_plate}; Philox key 1 + i; argon-like
    gas (config 2), beta = 1e-7 cm^3/s, dt = 1 ps."""
    out = []
    for i in range(n_chambers):
        rng = np.random.default_rng(seed + i)
        gap = rng.uniform(0.5e-3, 3e-3)
        e = 10.0 ** rng.uniform(np.log10(0.1), np.log10(30.0))
        n = int(round(10.0 ** rng.uniform(np.log10(n_min), np.log10(n_max))))
        npl = int(rng.integers(n_plate[0], n_plate[1] + 1))
        mesh = parallel_plates(side, gap, npl, 0.0, e * 1e5 * gap)
        ch = avalanche_snapshot(rng, n, gap=gap, side=side)
        ch.pos_q[:, 2] = np.clip(ch.pos_q[:, 2], 0.02 * gap, 0.98 * gap).astype(np.float32)
        trk = Tracking(dt=1e-12, seed=1 + i, z_lo=0.0, z_hi=gap, beta=1e-13)
        out.append(Chamber(mesh=mesh, charges=ch, trk=trk, e_kv_cm=e, n_plate=npl))
    return out


def config_gem(seed=1, n=1_000_000, target_panels=60000, geo: GemGeometry | None = None):
    """Single-GEM unit patch meshed into target_panels triangles; n charges
    (half electrons, half cations) in Gaussian clouds (sigma 20 um) on the
    hole axes, points inside copper or kapton rejected."""
    g = geo or GemGeometry()
    mesh = gem_mesh_target(target_panels, g)
    rng = np.random.default_rng(seed)
    cen = g.hole_centres()
    pts = np.empty((0, 3))
    while len(pts) < n:
        m = int((n - len(pts)) * 1.3) + 16
        h = rng.integers(0, len(cen), m)
        p = np.column_stack([cen[h, 0], cen[h, 1], np.zeros(m)]) + rng.normal(0, 20e-6, (m, 3))
        p = p[~gem_inside_solid(g, p)]
        pts = np.concatenate([pts, p])
    pts = pts[:n]
    ne = n // 2
    sp = np.concatenate([np.zeros(ne, np.uint8), np.ones(n - ne, np.uint8)])
    sp = sp[rng.permutation(n)]
    vel = np.where((sp == SP_ELECTRON)[:, None], maxwellian(rng, n, 1.0, M_ELECTRON), 0.0)
    ch = make_charges(pts, vel, sp)
    trk = Tracking(dt=1e-12, seed=seed, z_lo=g.z_anode, z_hi=g.z_drift, beta=1e-13)
    return mesh, argon_like_gas(), ch, trk, g


def config_double_gem(seed=1, n=100_000, target_panels=120_000, n_probe=4096,
                      geo: DoubleGemGeometry | None = None):
    """Double-GEM stack (two single-GEM foils 2 mm apart) meshed into
    target_panels triangles; n charges (half electrons, half cations) in
    Gaussian clouds (sigma 20 um) on the hole axes of either foil, points
    inside copper or kapton rejected; a probe line of n_probe points through
    the central hole's axis from the anode to the drift plane."""
    d = geo or DoubleGemGeometry()
    mesh = double_gem_mesh_target(target_panels, d)
    rng = np.random.default_rng(seed)
    cen = d.foil.hole_centres()
    zf = np.array([d.z_upper, d.z_lower])
    pts = np.empty((0, 3))
    while len(pts) < n:
        m = int((n - len(pts)) * 1.3) + 16
        h = rng.integers(0, len(cen), m)
        f = rng.integers(0, 2, m)
        p = np.column_stack([cen[h, 0], cen[h, 1], zf[f]]) + rng.normal(0, 20e-6, (m, 3))
        p = p[~double_gem_inside_solid(d, p)]
        pts = np.concatenate([pts, p])
    pts = pts[:n]
    ne = n // 2
    sp = np.concatenate([np.zeros(ne, np.uint8), np.ones(n - ne, np.uint8)])
    sp = sp[rng.permutation(n)]
    vel = np.where((sp == SP_ELECTRON)[:, None], maxwellian(rng, n, 1.0, M_ELECTRON), 0.0)
    ch = make_charges(pts, vel, sp)
    trk = Tracking(dt=1e-12, seed=seed, z_lo=d.z_anode, z_hi=d.z_drift, beta=1e-13)
    return mesh, argon_like_gas(), ch, trk, d, probe_line(d, n_probe)
