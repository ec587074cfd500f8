"""Static field map (obem_fieldmap_build / obem_fieldmap_eval, CUDA, through
the C ABI): node values against the oracle's cell field (1e-5, the field
tolerance), interpolation against the oracle's trilinear interpolation of the
same node values, and the step's map mode against a step given the
interpolated field (bit-exact)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem
from gpu_util import FIELD_TOL, guarded_rel_err, potential_err, pts4, to_dev

pytestmark = pytest.mark.gpu
LO = np.array([0.0, 0.0, 5e-5])
HI = np.array([1e-2, 1e-2, 9.5e-4])
DIMS = (21, 17, 11)


def _plates():
    mesh = inputs.parallel_plates(1e-2, 1e-3, 16, 0.0, 100.0)
    return mesh, oracle.bem_solve(mesh).astype(np.float32)


def _ctx(mesh, sigma, **kw):
    ctx = obem.obem_create(capacity=kw.pop("capacity", 16), dt=1e-12, **kw)
    obem.obem_mesh_load(ctx, mesh)
    obem.obem_fieldmap_build(ctx, LO, HI, DIMS, to_dev(sigma))
    return ctx


def _eval(ctx, pts):
    out = torch.full((len(pts), 4), float("nan"), device="cuda")
    obem.obem_fieldmap_eval(ctx, to_dev(pts4(pts)), out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_map_nodes_match_oracle_cell_field():
    mesh, sigma = _plates()
    nodes = oracle.grid_nodes(LO, HI, DIMS).astype(np.float32)
    ctx = _ctx(mesh, sigma)
    try:
        got = _eval(ctx, nodes)
    finally:
        obem.obem_destroy(ctx)
    p = nodes.astype(np.float64)
    Eref, Vref = oracle.panel_field(mesh.tri, sigma.astype(np.float64), p)
    Vabs = oracle.panel_field(mesh.tri, np.abs(sigma.astype(np.float64)), p)[1]
    assert guarded_rel_err(got[:, :3], Eref) <= FIELD_TOL
    assert potential_err(got[:, 3], Vref, Vabs) <= FIELD_TOL


def test_map_interpolation_matches_oracle_trilinear():
    mesh, sigma = _plates()
    nodes = oracle.grid_nodes(LO, HI, DIMS).astype(np.float32)
    rng = np.random.default_rng(4)
    pts = np.concatenate([rng.uniform(LO, HI, (2000, 3)),
                          np.array([[-1e-3, 5e-3, 5e-4], [2e-2, 2e-2, 2e-3]])]).astype(np.float32)
    ctx = _ctx(mesh, sigma)
    try:
        vals = _eval(ctx, nodes)
        got = _eval(ctx, pts)
    finally:
        obem.obem_destroy(ctx)
    ref = oracle.trilinear(vals, LO, HI, DIMS, pts.astype(np.float64))
    # binary32 weights and an 8-term weighted sum: a few tens of ulps (2^-24)
    # of the largest node value, i.e. <= 4e-6 of it
    emax = np.abs(vals[:, :3]).max()
    assert np.abs(got[:, :3] - ref[:, :3]).max() <= 4e-6 * emax
    assert np.abs(got[:, 3] - ref[:, 3]).max() <= 4e-6 * np.abs(vals[:, 3]).max()


def test_step_map_mode_equals_step_with_interpolated_field():
    """OBEM_STEP_FIELD_MAP: the step takes E = map(x) + e_ext; the same step
    given that field through E_in gives the same bits."""
    mesh, sigma = _plates()
    _, gas, ch, trk = inputs.config_small_plates(seed=5, n=800)
    e_ext = (1e3, -2e3, 5e3)
    ctx = _ctx(mesh, sigma, capacity=1024, seed=trk.seed, z_lo=trk.z_lo, z_hi=trk.z_hi,
               flags=obem.OBEM_STEP_FIELD_MAP, e_ext=e_ext)
    try:
        obem.obem_gas_load(ctx, gas)
        a, b = obem.DeviceState(1024), obem.DeviceState(1024)
        a.upload(ch)
        b.upload(ch)
        sa, sb = obem.new_stats(), obem.new_stats()
        for s in range(3):
            obem.obem_step(ctx, a, s, sa)
            n = int(b.download()[0].pos_q.shape[0])
            E = torch.zeros((1024, 4), device="cuda")
            obem.obem_fieldmap_eval(ctx, b.pos_q[:n], E[:n])
            E[:n, 0] += e_ext[0]
            E[:n, 1] += e_ext[1]
            E[:n, 2] += e_ext[2]
            obem.obem_step(ctx, b, s, sb, E_in=E)
        torch.cuda.synchronize()
        ga, _ = a.download()
        gb, _ = b.download()
    finally:
        obem.obem_destroy(ctx)
    for k in ("pos_q", "vel"):
        assert np.array_equal(getattr(ga, k).view(np.uint32), getattr(gb, k).view(np.uint32)), k
    assert np.array_equal(ga.id, gb.id)


def test_fieldmap_errors():
    mesh, sigma = _plates()
    ctx = obem.obem_create(capacity=16, dt=1e-12)
    try:
        out = torch.empty((4, 4), device="cuda")
        with pytest.raises(obem.ObemError) as e:
            obem.obem_fieldmap_eval(ctx, torch.zeros((4, 4), device="cuda"), out)
        assert e.value.code == obem.OBEM_ERR_STATE
        with pytest.raises(obem.ObemError) as e:
            obem.obem_fieldmap_build(ctx, LO, HI, DIMS, to_dev(sigma))
        assert e.value.code == obem.OBEM_ERR_STATE                  # no mesh
        obem.obem_mesh_load(ctx, mesh)
        with pytest.raises(obem.ObemError) as e:
            obem.obem_fieldmap_build(ctx, LO, HI, (1, 4, 4), to_dev(sigma))
        assert e.value.code == obem.OBEM_ERR_ARG
        with pytest.raises(obem.ObemError) as e:
            obem.obem_fieldmap_build(ctx, HI, LO, DIMS, to_dev(sigma))
        assert e.value.code == obem.OBEM_ERR_ARG
    finally:
        obem.obem_destroy(ctx)
