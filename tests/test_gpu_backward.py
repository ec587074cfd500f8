"""obem_field_eval_backward (CUDA, through the C ABI) against the FP64 oracle's
vector-Jacobian product of the field evaluation, and the autograd wrapper.
Tolerance: 1e-5 of max(|ref|, 1e-2 rms|ref|, 0.1 A) per element, A the sum of
the magnitudes of the element's terms (gpu_util.grad_err): the gradients are
sums of terms whose signs come from the upstream gradient, which binary32
arithmetic fixes only to a few ulps of A -- the reading the potential's
tolerance already uses."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem
from gpu_util import FIELD_TOL, grad_abs_scales, grad_err, pts4, to_dev

pytestmark = pytest.mark.gpu
E = 1.602176634e-19


def _charges(rng, n, box=1e-3, pairs=0):
    p = rng.uniform(0, box, (n, 3))
    if pairs:
        k = min(pairs, n // 2)
        p[n - k:] = p[:k] + rng.normal(0, 1e-8, (k, 3))
    q = rng.choice([-E, E], n)
    return np.column_stack([p, q]).astype(np.float32)


def _grad_in(rng, n, escale=1.0, vscale=1e3):
    g = rng.normal(0, 1.0, (n, 4))
    g[:, :3] *= escale
    g[:, 3] *= vscale
    return g.astype(np.float32)


def _gpu_backward(ctx, tgt, g, src=None, self_exclude=False, sigma=None, n_panels=0):
    t = to_dev(pts4(tgt))
    s = to_dev(src) if src is not None else None
    sg = to_dev(np.asarray(sigma, np.float32)) if sigma is not None else None
    gd = to_dev(g)
    dt = torch.full((len(tgt), 4), float("nan"), device="cuda")
    ds = torch.full((len(src), 4), float("nan"), device="cuda") if src is not None else None
    dsg = torch.full((n_panels,), float("nan"), device="cuda") if n_panels else None
    obem.obem_field_eval_backward(ctx, t, gd, sources=s, self_exclude=self_exclude, sigma=sg,
                                  dL_dsigma=dsg, dL_dtargets=dt, dL_dsources=ds)
    torch.cuda.synchronize()
    f = lambda x: None if x is None else x.cpu().numpy().astype(np.float64)
    return f(dsg), f(dt), f(ds)


def _ctx(mesh=None, cap=16):
    ctx = obem.obem_create(capacity=cap, dt=1e-12)
    if mesh is not None:
        obem.obem_mesh_load(ctx, mesh)
    return ctx


@pytest.mark.parametrize("nt,ns", [(700, 1500), (1, 300), (257, 1)])
def test_backward_charges(nt, ns):
    rng = np.random.default_rng(nt + 7 * ns)
    src = _charges(rng, ns)
    tgt = rng.uniform(-2e-4, 1.2e-3, (nt, 3)).astype(np.float32)
    g = _grad_in(rng, nt)
    ctx = _ctx()
    try:
        _, dt, ds = _gpu_backward(ctx, tgt, g, src)
    finally:
        obem.obem_destroy(ctx)
    _, rt, rs = oracle.field_backward(None, None, tgt.astype(np.float64), src.astype(np.float64), False,
                                      g.astype(np.float64))
    _, at, ap, aq = grad_abs_scales(tgt, g, src)
    assert np.all(dt[:, 3] == 0.0)
    assert grad_err(dt[:, :3], rt, at) <= FIELD_TOL
    assert grad_err(ds[:, :3], rs[:, :3], ap) <= FIELD_TOL
    assert grad_err(ds[:, 3], rs[:, 3], aq) <= FIELD_TOL


@pytest.mark.parametrize("n", [2, 129, 1000])
def test_backward_self_exclude(n):
    rng = np.random.default_rng(n)
    src = _charges(rng, n, pairs=n // 10)
    g = _grad_in(rng, n)
    ctx = _ctx()
    try:
        _, dt, ds = _gpu_backward(ctx, src, g, src, self_exclude=True)
    finally:
        obem.obem_destroy(ctx)
    s64 = src.astype(np.float64)
    _, rt, rs = oracle.field_backward(None, None, s64[:, :3], s64, True, g.astype(np.float64))
    _, at, ap, aq = grad_abs_scales(s64, g, s64, self_exclude=True)
    assert grad_err(dt[:, :3], rt, at) <= FIELD_TOL
    assert grad_err(ds[:, :3], rs[:, :3], ap) <= FIELD_TOL
    assert grad_err(ds[:, 3], rs[:, 3], aq) <= FIELD_TOL


def _plate_targets(rng):
    inner = rng.uniform([0, 0, 2e-6], [1e-2, 1e-2, 1e-3 - 2e-6], (400, 3))
    near = np.column_stack([rng.uniform(0, 1e-2, (200, 2)), rng.choice([2e-6, 3e-5, 9.9e-4], 200)])
    far = np.array([[5e-3, 5e-3, 5e-2], [0.3, -0.2, 0.4], [5e-3, 5e-3, -1.5e-3], [2e-2, 5e-3, 5e-4]])
    return np.concatenate([inner, near, far]).astype(np.float32)


def test_backward_cells_parallel_plates_all_tiers():
    rng = np.random.default_rng(17)
    mesh = inputs.parallel_plates(1e-2, 1e-3, 16, 0.0, 100.0)
    sigma = oracle.bem_solve(mesh).astype(np.float32)
    tgt = _plate_targets(rng)
    src = _charges(rng, 300, box=1e-3)
    src[:, :2] *= 10.0
    src[:, 2] = rng.uniform(1e-4, 9e-4, 300)
    g = _grad_in(rng, len(tgt), 1.0, 1e3)
    ctx = _ctx(mesh)
    try:
        dsg, dt, ds = _gpu_backward(ctx, tgt, g, src, sigma=sigma, n_panels=mesh.n)
    finally:
        obem.obem_destroy(ctx)
    rsg, rt, rs = oracle.field_backward(mesh.tri, sigma.astype(np.float64), tgt.astype(np.float64),
                                        src.astype(np.float64), False, g.astype(np.float64))
    asg, at, ap, aq = grad_abs_scales(tgt, g, src, mesh.tri, sigma)
    assert grad_err(dsg, rsg, asg) <= FIELD_TOL
    assert grad_err(dt[:, :3], rt, at) <= FIELD_TOL
    assert grad_err(ds[:, :3], rs[:, :3], ap) <= FIELD_TOL
    assert grad_err(ds[:, 3], rs[:, 3], aq) <= FIELD_TOL


def test_backward_cells_gem_patch():
    """Small GEM patch (7 holes) with electrode and dielectric cells, targets
    in Gaussian clouds on the hole axes (many within a few cell sizes of the
    hole walls)."""
    g_ = inputs.GemGeometry(rings=1)
    mesh = inputs.gem_mesh(g_, n_theta=24, n_r=3, n_zc=1, n_zk=6, n_plane=10)
    cen = mesh.tri.mean(axis=1)
    sigma = (1e-6 * (1.0 + 0.5 * np.sin(cen[:, 0] / 1e-4))
             * np.where(mesh.group % 2 == 0, 1.0, -1.0)).astype(np.float32)
    rng = np.random.default_rng(3)
    hc = g_.hole_centres()
    h = rng.integers(0, len(hc), 2000)
    p = np.column_stack([hc[h], np.zeros(2000)]) + rng.normal(0, 20e-6, (2000, 3))
    p = p[~inputs.gem_inside_solid(g_, p)][:600].astype(np.float32)
    g = _grad_in(rng, len(p), 1.0, 1e4)
    ctx = _ctx(mesh)
    try:
        dsg, dt, _ = _gpu_backward(ctx, p, g, sigma=sigma, n_panels=mesh.n)
    finally:
        obem.obem_destroy(ctx)
    rsg, rt, _ = oracle.field_backward(mesh.tri, sigma.astype(np.float64), p.astype(np.float64), None,
                                       False, g.astype(np.float64))
    asg, at, _, _ = grad_abs_scales(p, g, None, mesh.tri, sigma)
    assert grad_err(dsg, rsg, asg) <= FIELD_TOL
    assert grad_err(dt[:, :3], rt, at) <= FIELD_TOL


def test_autograd_field_eval_matches_oracle():
    """loss = sum |E|^2 + sum V over the targets, through torch.autograd: the
    gradients reaching targets, sources (position and charge) and sigma are
    the oracle's vector-Jacobian products for g = (2E, 1)."""
    rng = np.random.default_rng(23)
    mesh = inputs.parallel_plates(1e-2, 1e-3, 8, 0.0, 100.0)
    sigma = oracle.bem_solve(mesh).astype(np.float32)
    tgt = pts4(np.column_stack([rng.uniform(0, 1e-2, (300, 2)), rng.uniform(5e-5, 9.5e-4, 300)]))
    src = _charges(rng, 200)
    src[:, :2] *= 10.0
    src[:, 2] = rng.uniform(1e-4, 9e-4, 200)
    ctx = _ctx(mesh)
    try:
        t = to_dev(tgt).requires_grad_(True)
        s = to_dev(src).requires_grad_(True)
        sg = to_dev(sigma).requires_grad_(True)
        out = obem.field_eval(ctx, t, s, sg)
        loss = (out[:, :3] ** 2).sum() + out[:, 3].sum()
        loss.backward()
        torch.cuda.synchronize()
        E_gpu = out.detach().cpu().numpy().astype(np.float64)
        gt, gs, gsg = (x.grad.cpu().numpy().astype(np.float64) for x in (t, s, sg))
    finally:
        obem.obem_destroy(ctx)
    g = np.column_stack([2.0 * E_gpu[:, :3], np.ones(len(tgt))])
    rsg, rt, rs = oracle.field_backward(mesh.tri, sigma.astype(np.float64), tgt[:, :3].astype(np.float64),
                                        src.astype(np.float64), False, g)
    asg, at, ap, aq = grad_abs_scales(tgt, g, src, mesh.tri, sigma)
    assert np.all(gt[:, 3] == 0.0)
    assert grad_err(gt[:, :3], rt, at) <= FIELD_TOL
    assert grad_err(gs[:, :3], rs[:, :3], ap) <= FIELD_TOL
    assert grad_err(gs[:, 3], rs[:, 3], aq) <= FIELD_TOL
    assert grad_err(gsg, rsg, asg) <= FIELD_TOL


def test_backward_empty_and_bad_arguments():
    mesh = inputs.parallel_plates(1e-2, 1e-3, 4, 0.0, 100.0)
    ctx = _ctx(mesh)
    try:
        dsg = torch.full((mesh.n,), 7.0, device="cuda")
        src = to_dev(_charges(np.random.default_rng(0), 5))
        dsr = torch.full((5, 4), 7.0, device="cuda")
        empty = torch.empty((0, 4), device="cuda")
        obem.obem_field_eval_backward(ctx, empty, empty, sources=src, dL_dsigma=dsg, dL_dsources=dsr)
        torch.cuda.synchronize()
        assert torch.all(dsg == 0) and torch.all(dsr == 0)     # sums over no targets
        t = torch.zeros((4, 4), device="cuda")
        with pytest.raises(obem.ObemError) as e:
            obem.obem_field_eval_backward(ctx, t, t, sources=torch.zeros((3, 4), device="cuda"),
                                          self_exclude=True, dL_dtargets=torch.empty_like(t))
        assert e.value.code == obem.OBEM_ERR_ARG
        with pytest.raises(obem.ObemError) as e:
            obem.obem_field_eval_backward(ctx, t, t, dL_dsources=torch.empty_like(t))
        assert e.value.code == obem.OBEM_ERR_ARG
    finally:
        obem.obem_destroy(ctx)
    ctx = _ctx()
    try:
        t = torch.zeros((4, 4), device="cuda")
        with pytest.raises(obem.ObemError) as e:
            obem.obem_field_eval_backward(ctx, t, t, dL_dsigma=torch.empty(10, device="cuda"))
        assert e.value.code == obem.OBEM_ERR_STATE
    finally:
        obem.obem_destroy(ctx)
