"""Pins of the oracle's field derivatives (backward evaluation) against things
other than their own formulas: central finite differences of the independently
pinned forward field, Laplace's equation (trace 0), the curl-free field
(symmetric Jacobian), the point-charge limit far from a cell, and
finite differences of the scalar L = sum_t g_t . (E_t, V_t).  All CPU-only."""
import numpy as np
import pytest

import oracle
from paper_2110_09214_gb300 import inputs

TRI = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.3, 0.9, 0.05]])


def _fd_jac(v, r, h):
    J = np.zeros((3, 3))
    for b in range(3):
        e = np.zeros(3)
        e[b] = h
        J[:, b] = (oracle.tri_integrals(v, r + e)[1] - oracle.tri_integrals(v, r - e)[1]) / (2 * h)
    return J


def _probe_points():
    """Off-cell points of every kind the edge formulas distinguish: above and
    below, in the cell's plane outside it, next to an edge (foot on the
    edge), on an edge's line beyond either vertex (foot past / before the
    edge), near a vertex, and far away."""
    c, n, _ = oracle.tri_geometry(TRI)
    v0, v1, v2 = TRI
    t01 = (v1 - v0) / np.linalg.norm(v1 - v0)
    out = (np.cross(t01, n))
    pts = [c + 0.4 * n, c - 0.25 * n, c + 0.01 * n,
           v0 + 1.7 * (v1 - v0),                        # in plane, past v1 on edge 0-1's line
           v0 - 0.6 * (v1 - v0) + 1e-4 * n,             # before v0 on the same line, just off the plane
           0.5 * (v0 + v1) + 0.05 * out,                # in plane, beside edge 0-1, outside
           0.5 * (v0 + v1) + 2e-3 * out + 2e-3 * n,     # close to the edge
           v2 + 0.02 * (v2 - c) + 0.01 * n,             # near a vertex
           c + np.array([30.0, -20.0, 45.0])]           # far
    return pts


def _dist_to_tri(r, m=400):
    """Distance from r to the closed triangle, by a dense barycentric grid."""
    u, w = np.meshgrid(np.linspace(0, 1, m), np.linspace(0, 1, m), indexing="ij")
    keep = u + w <= 1.0
    P = TRI[0] + u[keep, None] * (TRI[1] - TRI[0]) + w[keep, None] * (TRI[2] - TRI[0])
    return float(np.linalg.norm(P - r, axis=1).min())


@pytest.mark.parametrize("k", range(9))
def test_tri_jacobian_matches_central_differences(k):
    r = _probe_points()[k]
    d = min(_dist_to_tri(r), 1.0)
    J = oracle.tri_jacobian(TRI, r)
    Jf = _fd_jac(TRI, r, 1e-4 * d)
    assert np.abs(J - Jf).max() <= 1e-6 * np.abs(Jf).max()


def test_tri_jacobian_traceless_and_symmetric():
    rng = np.random.default_rng(1)
    for _ in range(200):
        r = rng.normal(0.3, 1.0, 3)
        J = oracle.tri_jacobian(TRI, r)
        s = np.abs(J).max()
        assert abs(np.trace(J)) <= 1e-12 * s          # div E = 0 off the cell
        assert np.abs(J - J.T).max() <= 1e-12 * s      # curl E = 0


def test_tri_jacobian_far_limit_is_point_charge():
    c, n, area = oracle.tri_geometry(TRI)
    for dirn in ([1.0, 2.0, 3.0], [0.0, 0.0, 1.0], [1.0, -1.0, 0.0]):
        d = np.asarray(dirn) / np.linalg.norm(dirn) * 2000.0
        J = oracle.tri_jacobian(TRI, c + d)
        r = np.linalg.norm(d)
        T = area * (np.eye(3) / r ** 3 - 3 * np.outer(d, d) / r ** 5)
        # the cell's quadrupole moment enters at relative order (size/r)^2
        assert np.abs(J - T).max() <= 1e-5 * np.abs(T).max()


def test_point_charge_jacobian_matches_central_differences():
    rng = np.random.default_rng(2)
    src = np.column_stack([rng.uniform(0, 1e-3, (12, 3)), rng.choice([-1.6e-19, 1.6e-19], 12)])
    pts = rng.uniform(-2e-4, 1.2e-3, (6, 3))
    J = oracle.field_jacobian(None, None, pts, src)
    h = 1e-9
    for t in range(len(pts)):
        for b in range(3):
            e = np.zeros(3)
            e[b] = h
            fd = (oracle.nbody_field(pts[t] + e, src)[0][0] - oracle.nbody_field(pts[t] - e, src)[0][0]) / (2 * h)
            assert np.abs(J[t][:, b] - fd).max() <= 1e-6 * np.abs(J[t]).max()


def _case(seed=4):
    mesh = inputs.parallel_plates(1e-2, 1e-3, 4, 0.0, 100.0)
    rng = np.random.default_rng(seed)
    sigma = rng.normal(0, 1e-6, mesh.n)
    pts = np.column_stack([rng.uniform(0, 1e-2, (10, 2)), rng.uniform(1e-4, 9e-4, 10)])
    src = np.column_stack([rng.uniform(0, 1e-2, (8, 2)), rng.uniform(1e-4, 9e-4, 8),
                           rng.choice([-1.6e-19, 1.6e-19], 8)])
    g = rng.normal(0, 1.0, (len(pts), 4))
    g[:, 3] *= 1e3                                     # V and E gradients on comparable scales
    return mesh, sigma, pts, src, g


def _loss(mesh, sigma, pts, src, g, self_exclude=False):
    E1, V1 = oracle.panel_field(mesh.tri, sigma, pts)
    E2, V2 = oracle.nbody_field(pts, src, self_exclude)
    return float((g[:, :3] * (E1 + E2)).sum() + (g[:, 3] * (V1 + V2)).sum())


def test_field_backward_matches_finite_differences():
    mesh, sigma, pts, src, g = _case()
    ds, dp, dq = oracle.field_backward(mesh.tri, sigma, pts, src, False, g)
    # sigma: L is linear in sigma, so a unit step is exact up to rounding
    for j in (0, 7, 19, 31):
        e = np.zeros(mesh.n)
        e[j] = 1e-6
        fd = (_loss(mesh, sigma + e, pts, src, g) - _loss(mesh, sigma - e, pts, src, g)) / 2e-6
        assert abs(ds[j] - fd) <= 1e-9 * max(abs(fd), np.abs(ds).max())
    h = 1e-8
    for t in (0, 3, 9):
        for b in range(3):
            p1, p2 = pts.copy(), pts.copy()
            p1[t, b] += h
            p2[t, b] -= h
            fd = (_loss(mesh, sigma, p1, src, g) - _loss(mesh, sigma, p2, src, g)) / (2 * h)
            assert abs(dp[t, b] - fd) <= 1e-5 * np.abs(dp).max()
    zero = np.zeros(mesh.n)   # the cell part does not depend on the charges
    for p in (0, 5):
        for b in range(3):
            s1, s2 = src.copy(), src.copy()
            s1[p, b] += h
            s2[p, b] -= h
            fd = (_loss(mesh, zero, pts, s1, g) - _loss(mesh, zero, pts, s2, g)) / (2 * h)
            assert abs(dq[p, b] - fd) <= 1e-5 * np.abs(dq[:, :3]).max()
        s1, s2 = src.copy(), src.copy()   # L is linear in q_p: a whole step is exact
        s1[p, 3] *= 2.0
        s2[p, 3] = 0.0
        fd = (_loss(mesh, zero, pts, s1, g) - _loss(mesh, zero, pts, s2, g)) / (2.0 * src[p, 3])
        assert abs(dq[p, 3] - fd) <= 1e-9 * np.abs(dq[:, 3]).max()


def test_field_backward_self_exclusion():
    """Targets that are the sources: the pair t == p is skipped in both roles,
    and the two gradients are the target-role and source-role parts."""
    rng = np.random.default_rng(5)
    src = np.column_stack([rng.uniform(0, 1e-3, (9, 3)), rng.choice([-1.6e-19, 1.6e-19], 9)])
    pts = src[:, :3].copy()
    g = rng.normal(0, 1.0, (9, 4))
    _, dp, dq = oracle.field_backward(None, None, pts, src, True, g)
    h = 1e-10
    for t in (0, 4):
        for b in range(3):
            p1, p2 = pts.copy(), pts.copy()
            p1[t, b] += h
            p2[t, b] -= h
            l1 = float((g[:, :3] * oracle.nbody_field(p1, src, True)[0]).sum() + (g[:, 3] * oracle.nbody_field(p1, src, True)[1]).sum())
            l2 = float((g[:, :3] * oracle.nbody_field(p2, src, True)[0]).sum() + (g[:, 3] * oracle.nbody_field(p2, src, True)[1]).sum())
            assert abs(dp[t, b] - (l1 - l2) / (2 * h)) <= 1e-5 * np.abs(dp).max()
    # translation invariance: moving every charge (both roles) by the same
    # vector leaves the pair sum unchanged, so the gradients add up to zero
    tot = dp.sum(axis=0) + dq[:, :3].sum(axis=0)
    assert np.abs(tot).max() <= 1e-9 * np.abs(dp).max()


# ----------------------------------------------------------------------------
# adjoint of the BEM solve: sigma depends linearly on (V, sigma_free, drhs),
# so the gradient of L = g . sigma is exact from solves with unit inputs
# ----------------------------------------------------------------------------
def _sphere_mesh():
    return inputs.dielectric_sphere_in_plates(radius=1e-3, level=1, eps_r=4.0, side=2e-2, gap=1e-2, n_plate=4)


def test_bem_adjoint_voltage_gradient_is_exact_by_linearity():
    mesh = _sphere_mesh()
    rng = np.random.default_rng(6)
    g = rng.normal(0, 1.0, mesh.n)
    mu, dV = oracle.bem_solve_adjoint(mesh, g)
    ng = len(mesh.group_voltage)
    assert ng >= 2
    for k in range(ng):
        e = np.zeros(ng)
        e[k] = 1.0
        ref = float(g @ oracle.bem_solve(mesh, group_voltage=e))
        assert abs(dV[k] - ref) <= 1e-9 * max(abs(ref), np.abs(dV).max())


def test_bem_adjoint_free_density_and_rhs_gradient():
    mesh = _sphere_mesh()
    rng = np.random.default_rng(7)
    g = rng.normal(0, 1.0, mesh.n)
    mu, _ = oracle.bem_solve_adjoint(mesh, g)
    zero_v = np.zeros(len(mesh.group_voltage))
    dd = np.flatnonzero(mesh.kind == 1)
    ed = np.flatnonzero(mesh.kind == 0)
    assert len(dd) > 0 and len(ed) > 0
    for i in (dd[0], dd[len(dd) // 2], ed[3]):
        e = np.zeros(mesh.n)
        e[i] = 1.0
        # a unit free density on a dielectric cell, or a unit rhs correction
        if mesh.kind[i] == 1:
            ref = float(g @ oracle.bem_solve(mesh, sigma_free=e, group_voltage=zero_v))
            assert abs(mu[i] - ref) <= 1e-9 * np.abs(mu).max()
        ref = float(g @ oracle.bem_solve(mesh, drhs=e, group_voltage=zero_v))
        assert abs(mu[i] - ref) <= 1e-9 * np.abs(mu).max()


def _probe_line(mesh, n=64):
    """Probe points on a line across the sphere-in-plates chamber, off every
    surface (the loss of the differentiable-field workload: mean |E|^2)."""
    c = np.array([1e-2, 1e-2, 5e-3])
    t = np.linspace(-1.0, 1.0, n)
    return c + np.column_stack([4e-3 * t, 1.5e-3 + 0 * t, 4e-3 * t])


def _probe_loss(mesh, V, pts):
    sigma = oracle.bem_solve(mesh, group_voltage=V)
    E, _ = oracle.panel_field(mesh.tri, sigma, pts)
    return float((E ** 2).sum(axis=1).mean()), sigma, E


def test_probe_loss_voltage_gradient_matches_central_differences():
    """dL/dV of L = mean |E|^2 at probes, E from sigma = solve(V): the
    oracle's chain (field backward, then the adjoint solve) against FP64
    central differences with h = 1e-4 relative.  L is quadratic in V, so the
    central difference is exact up to rounding."""
    mesh = _sphere_mesh()
    pts = _probe_line(mesh)
    V = np.array([-300.0, 1000.0])
    L, sigma, E = _probe_loss(mesh, V, pts)
    g = np.column_stack([2.0 * E / len(pts), np.zeros(len(pts))])
    dsig, _, _ = oracle.field_backward(mesh.tri, sigma, pts, None, False, g)
    _, dV = oracle.bem_solve_adjoint(mesh, dsig)
    for k in range(2):
        h = 1e-4 * abs(V[k])
        Vp, Vm = V.copy(), V.copy()
        Vp[k] += h
        Vm[k] -= h
        fd = (_probe_loss(mesh, Vp, pts)[0] - _probe_loss(mesh, Vm, pts)[0]) / (2 * h)
        assert abs(dV[k] - fd) <= 1e-7 * np.abs(dV).max()


# ----------------------------------------------------------------------------
# static field map: trilinear interpolation
# ----------------------------------------------------------------------------
def test_trilinear_is_exact_for_trilinear_functions_and_nodes():
    lo, hi, dims = np.array([-1.0, 0.5, 2.0]), np.array([3.0, 1.5, 2.7]), (7, 4, 5)
    nodes = oracle.grid_nodes(lo, hi, dims)
    assert nodes.shape == (7 * 4 * 5, 3)
    assert np.allclose(nodes[0], lo) and np.allclose(nodes[-1], hi)
    c = np.array([0.3, -1.2, 2.5, 0.7, -0.4, 1.1, 0.9, -2.0])

    def f(p):
        x, y, z = p[:, 0], p[:, 1], p[:, 2]
        return c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * y * z + c[6] * x * z + c[7] * x * y * z
    vals = np.column_stack([f(nodes), 2.0 * f(nodes)])
    rng = np.random.default_rng(8)
    pts = rng.uniform(lo, hi, (500, 3))
    got = oracle.trilinear(vals, lo, hi, dims, pts)
    assert np.abs(got[:, 0] - f(pts)).max() <= 1e-12 * np.abs(f(pts)).max()
    assert np.abs(got[:, 1] - 2 * f(pts)).max() <= 1e-12 * np.abs(f(pts)).max()
    assert np.abs(oracle.trilinear(vals, lo, hi, dims, nodes) - vals).max() <= 1e-12 * np.abs(vals).max()
    # outside the box: the value at the nearest point of the box
    out = np.array([[-5.0, 1.0, 2.3], [10.0, 10.0, 10.0]])
    near = np.clip(out, lo, hi)
    assert np.allclose(oracle.trilinear(vals, lo, hi, dims, out), oracle.trilinear(vals, lo, hi, dims, near))


# ----------------------------------------------------------------------------
# the double-GEM stack (coarse, one hole per foil): six electrode voltages
# ----------------------------------------------------------------------------
def _coarse_double_gem():
    d = inputs.DoubleGemGeometry(foil=inputs.GemGeometry(rings=0))
    return d, inputs.double_gem_mesh(d, n_theta=12, n_r=2, n_zc=1, n_zk=4, n_plane=6)


def test_double_gem_axis_field_is_axial():
    """The coarse stack is symmetric under a half turn about the hole axis
    (hexagonal cells, square planes, 12 angular divisions), so on the axis
    the transverse field of the solved stack vanishes up to rounding."""
    d, mesh = _coarse_double_gem()
    sigma = oracle.bem_solve(mesh)
    pts = inputs.probe_line(d, 64)
    E, V = oracle.panel_field(mesh.tri, sigma, pts)
    assert np.abs(E[:, :2]).max() <= 1e-9 * np.abs(E[:, 2]).max()
    # maximum principle (charge-free gas, potential 0 at infinity, anode at
    # 0 V): the potential stays within the electrodes' range
    v = mesh.group_voltage
    assert np.all(V >= v.min() * (1 + 1e-9)) and np.all(V <= max(v.max(), 0.0) + 1e-9 * np.abs(v).max())


def test_double_gem_probe_loss_gradient_in_all_six_voltages():
    """dL/dV_k (k = drift, two copper layers per foil, anode) of the probe
    loss on the axis, the oracle's chain against central differences (L is
    quadratic in V: exact up to rounding)."""
    d, mesh = _coarse_double_gem()
    pts = inputs.probe_line(d, 64)
    V = mesh.group_voltage.copy()
    L, sigma, E = _probe_loss(mesh, V, pts)
    g = np.column_stack([2.0 * E / len(pts), np.zeros(len(pts))])
    dsig, _, _ = oracle.field_backward(mesh.tri, sigma, pts, None, False, g)
    _, dV = oracle.bem_solve_adjoint(mesh, dsig)
    assert dV.shape == (6,)
    h = 1e-4 * np.abs(V).max()
    for k in range(6):
        Vp, Vm = V.copy(), V.copy()
        Vp[k] += h
        Vm[k] -= h
        fd = (_probe_loss(mesh, Vp, pts)[0] - _probe_loss(mesh, Vm, pts)[0]) / (2 * h)
        assert abs(dV[k] - fd) <= 1e-7 * np.abs(dV).max(), (k, dV[k], fd)
