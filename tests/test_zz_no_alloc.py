"""obem_field_eval_noalloc: the field entry point for callers that cannot
allocate device memory (a fixed device-memory budget owned by a host
application, loops that cannot take an allocation's latency) and therefore
have no obem_ctx.  It must give what obem_field_eval gives, call after call,
although every call reuses the same fixed scratch array inside the library,
and it must leave the device's free memory unchanged."""
import numpy as np
import pytest
import torch

from paper_2110_09214_gb300 import inputs, obem
from gpu_util import FIELD_TOL, guarded_rel_err, potential_err

pytestmark = pytest.mark.gpu
E = 1.602176634e-19


def _case(seed=3, n=3000):
    g = inputs.GemGeometry(rings=1)
    mesh = inputs.gem_mesh(g, n_theta=24, n_r=3, n_zc=1, n_zk=6, n_plane=10)
    cen = mesh.tri.mean(axis=1)
    sigma = (1e-6 * (1.0 + 0.5 * np.sin(cen[:, 0] / 1e-4))
             * np.where(mesh.group % 2 == 0, 1.0, -1.0)).astype(np.float32)
    rng = np.random.default_rng(seed)
    hc = g.hole_centres()
    h = rng.integers(0, len(hc), 2 * n)
    p = np.column_stack([hc[h], np.zeros(2 * n)]) + rng.normal(0, 20e-6, (2 * n, 3))
    p = p[~inputs.gem_inside_solid(g, p)][:n]
    src = np.zeros((len(p), 4), np.float32)
    src[:, :3] = p
    src[:, 3] = rng.choice([-E, E], len(p))
    return mesh, sigma, src


def _existing(mesh, sigma, src, absolute=False):
    ctx = obem.obem_create(capacity=len(src), dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        s = torch.from_numpy(np.abs(src) if absolute else src).cuda()
        t = torch.from_numpy(src).cuda()
        sg = torch.from_numpy(np.abs(sigma) if absolute else sigma).cuda()
        out = torch.empty((len(src), 4), dtype=torch.float32, device="cuda")
        obem.obem_field_eval(ctx, t, out, sources=s, self_exclude=True, sigma=sg)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)


def test_noalloc_matches_field_eval_on_two_calls_in_a_row():
    mesh, sigma, src = _case()
    ref = _existing(mesh, sigma, src)
    vabs = _existing(mesh, sigma, src, absolute=True)[:, 3]
    t = torch.from_numpy(src).cuda()
    cells = torch.from_numpy(np.ascontiguousarray(mesh.tri, np.float64)).cuda()
    sg = torch.from_numpy(sigma).cuda()
    for k in range(2):
        out = torch.full((len(src), 4), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        obem.obem_field_eval_noalloc(t, out, sources=t, self_exclude=True, cell_xyz=cells, sigma=sg)
        torch.cuda.synchronize()
        if k == 1:                     # the first call may load the kernels' code
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        assert guarded_rel_err(got[:, :3], ref[:, :3]) <= FIELD_TOL
        assert potential_err(got[:, 3], ref[:, 3], vabs) <= FIELD_TOL


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    big = torch.zeros((obem.NOALLOC_MAX_TARGETS + 1, 4), dtype=torch.float32, device="cuda")
    out = torch.empty_like(big)
    with pytest.raises(obem.ObemError) as e:
        obem.obem_field_eval_noalloc(big, out)
    assert e.value.code == obem.OBEM_ERR_ARG and "262144" in str(e.value)
