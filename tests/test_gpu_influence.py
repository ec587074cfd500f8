"""obem_influence_rhs (CUDA, through the C ABI): the influence of free charges
on the cells (Sec. 3.2.2, Eqs. (potpart), (fldpart)), i.e. the right-hand-side
correction of Eqs. (BEMpotpart), (BEMfldpart), against the oracle's FP64
closed-form cell integrals, and the dynamic re-solve of the cell charges with
it against the oracle's solve of the same system.

Each entry is a sum of signed terms over the charges, so it is gated like the
potential: the error relative to max(|ref|, 1e-2 rms|ref|, 0.1 A) with A the
sum of the terms' magnitudes (charges taken as points at distance d from the
cell centroid: k |q| / d for electrode rows, (eps+ - eps-) eps0 k |q| / d^2
for dielectric rows)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem
from gpu_util import FIELD_TOL, to_dev

pytestmark = pytest.mark.gpu
E = 1.602176634e-19
KC = 8.9875517923e9
EPS0 = 8.8541878128e-12


def _gem_case(n=2500, seed=3):
    g = inputs.GemGeometry(rings=1)
    mesh = inputs.gem_mesh(g, n_theta=24, n_r=3, n_zc=1, n_zk=6, n_plane=10)
    rng = np.random.default_rng(seed)
    hc = g.hole_centres()
    h = rng.integers(0, len(hc), 3 * n)
    p = np.column_stack([hc[h], np.zeros(3 * n)]) + rng.normal(0, 25e-6, (3 * n, 3))
    p = p[~inputs.gem_inside_solid(g, p)][:n]
    src = np.zeros((len(p), 4), np.float32)
    src[:, :3] = p
    src[:, 3] = rng.choice([-E, E], len(p))
    return mesh, src


def _abs_scale(mesh, src):
    cen = mesh.tri.mean(axis=1)
    d = np.linalg.norm(cen[:, None, :] - src[None, :, :3].astype(np.float64), axis=-1)
    aq = np.abs(src[:, 3]).astype(np.float64)
    sv = KC * (aq[None, :] / d).sum(1)
    sf = KC * (aq[None, :] / d ** 2).sum(1)
    epsd = np.where(mesh.kind == 1, mesh.eps_plus - mesh.eps_minus, 0.0)
    return np.where(mesh.kind == 0, sv, np.abs(epsd) * EPS0 * sf)


def _err(got, ref, scale):
    rms = np.sqrt((ref ** 2).mean())
    den = np.maximum(np.maximum(np.abs(ref), 1e-2 * rms), 0.1 * scale)
    return float((np.abs(got - ref) / den).max())


def _gpu_influence(ctx, mesh, src):
    out = torch.full((mesh.n,), float("nan"), dtype=torch.float32, device="cuda")
    obem.obem_influence_rhs(ctx, to_dev(src) if len(src) else None, out)
    torch.cuda.synchronize()
    return out


def test_influence_matches_oracle_on_gem_patch():
    mesh, src = _gem_case()
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        got = _gpu_influence(ctx, mesh, src).cpu().numpy().astype(np.float64)
        again = _gpu_influence(ctx, mesh, src).cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)
    ref = oracle.influence_rhs(mesh, src.astype(np.float64))
    assert np.all(np.isfinite(got))
    assert np.array_equal(got, again)                 # deterministic
    for kind in (0, 1):
        sel = mesh.kind == kind
        assert sel.any()
        assert _err(got[sel], ref[sel], _abs_scale(mesh, src)[sel]) <= FIELD_TOL, kind


def test_distant_charge_gives_minus_kq_over_d_on_plates():
    """A charge far from a pair of small electrode plates: every cell sees the
    point-charge potential k q / d averaged over the cell, so drhs = -k q / d
    to O((h/d)^2)."""
    mesh = inputs.parallel_plates(1e-3, 1e-3, 8, 0.0, 100.0)
    src = np.array([[0.5e-3, 0.5e-3, 0.25, 3 * E]], np.float32)
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        got = _gpu_influence(ctx, mesh, src).cpu().numpy().astype(np.float64)
        none = _gpu_influence(ctx, mesh, np.zeros((0, 4), np.float32)).cpu().numpy()
    finally:
        obem.obem_destroy(ctx)
    cen = mesh.tri.mean(axis=1)
    d = np.linalg.norm(cen - src[0, :3].astype(np.float64), axis=1)
    want = -KC * float(src[0, 3]) / d
    assert np.abs(got / want - 1).max() < 1e-5
    assert np.all(none == 0.0)


def test_dynamic_resolve_with_the_influence_matches_oracle():
    """The dynamic option of Sec. 3.2.2: the cell charges re-solved with the
    influence of the free charges (Eqs. (BEMpotpart), (BEMfldpart)) through
    obem_bem_solve's drhs, against the oracle's solve with its own
    right-hand side."""
    from test_gpu_bem import _check
    mesh, src = _gem_case(n=1500, seed=5)
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        obem.obem_bem_assemble(ctx, obem.OBEM_LU_BF16)
        drhs = _gpu_influence(ctx, mesh, src)
        sig = torch.empty(mesh.n, dtype=torch.float32, device="cuda")
        rep = obem.obem_bem_solve(ctx, mesh.group_voltage, sig, drhs=drhs)
        assert rep["status"] == 0
        sig0 = torch.empty_like(sig)
        obem.obem_bem_solve(ctx, mesh.group_voltage, sig0)
        got = sig.cpu().numpy().astype(np.float64)
        got0 = sig0.cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)
    A = oracle.assemble(mesh)
    dref = oracle.influence_rhs(mesh, src.astype(np.float64))
    b = oracle.bem_rhs(mesh, drhs=dref)
    ref = oracle.solve(A, b)
    _check(mesh, got, A, b, ref)
    # the charges' induced part of sigma itself, not only the total: to 1e-3
    # of its largest value plus a few binary32 ulps of the total sigma (in
    # which both solutions are returned)
    ind, ind_ref = got - got0, ref - oracle.solve(A, oracle.bem_rhs(mesh))
    ulp = np.spacing(np.abs(got0).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(ind - ind_ref) <= 1e-3 * np.abs(ind_ref).max() + 4 * ulp)


def test_influence_at_full_size_sampled_cells():
    """The headline workload (59,968 cells of a GEM patch, 1e6 signed charges
    in clouds on the hole axes) through the binned kernel: every cell on the
    GPU, the oracle at 16 cells with a charge closer than one cell size (the
    per-pair tiers and the closed form) and 16 random cells, with the charges'
    sum-of-magnitudes scale of each sampled cell."""
    from types import SimpleNamespace
    from scipy.spatial import cKDTree
    mesh, _, ch, _, _ = inputs.config_gem(seed=2)
    src = np.ascontiguousarray(ch.pos_q.astype(np.float32))
    src[:, 3] = np.where(ch.species == 0, -E, E)
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        got = _gpu_influence(ctx, mesh, src).cpu().numpy().astype(np.float64)
        again = _gpu_influence(ctx, mesh, src).cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)
    assert np.all(np.isfinite(got)) and np.array_equal(got, again)
    tri = np.asarray(mesh.tri, np.float64)
    cen = tri.mean(axis=1)
    h = np.max(np.linalg.norm(tri - np.roll(tri, 1, axis=1), axis=2), axis=1)
    d, _ = cKDTree(src[:, :3].astype(np.float64)).query(cen, k=1)
    rng = np.random.default_rng(7)
    close = np.flatnonzero(d < h)
    assert len(close) >= 16
    sel = np.unique(np.concatenate([rng.choice(close, 16, replace=False), rng.choice(mesh.n, 16, replace=False)]))
    sub = SimpleNamespace(n=len(sel), tri=tri[sel], kind=mesh.kind[sel], eps_minus=mesh.eps_minus[sel],
                          eps_plus=mesh.eps_plus[sel])
    ref = oracle.influence_rhs(sub, src.astype(np.float64))
    p = src[:, :3].astype(np.float64)
    aq = np.abs(src[:, 3]).astype(np.float64)
    scale = np.empty(len(sel))
    for i, j in enumerate(sel):
        r = np.linalg.norm(p - cen[j], axis=1)
        if mesh.kind[j] == 0:
            scale[i] = KC * (aq / r).sum()
        else:
            scale[i] = abs(mesh.eps_plus[j] - mesh.eps_minus[j]) * EPS0 * KC * (aq / r ** 2).sum()
    g = got[sel]
    err = np.abs(g - ref) / np.maximum(np.abs(ref), 0.1 * scale)
    assert err.max() <= FIELD_TOL, (err.max(), sel[int(np.argmax(err))])
