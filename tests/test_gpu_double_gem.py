"""The differentiable field at full size on the double-GEM stack (119,872
cells, 1e5 charges, a 4096-point probe line through the central hole): the
gradient of L = mean |E|^2 on the probe with respect to the cell densities,
the charges and the six electrode voltages.

The oracle cannot factorise this system, so: dL/dsigma at sampled cells and
dL/d(charges) at sampled charges against the oracle's FP64 backward with the
same upstream gradient (each entry depends only on its own cell or charge);
dL/dV_k (adjoint solve) against central differences of the GPU's own loss,
which is quadratic in the voltages, so that the difference quotient is exact
up to rounding for any step."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem
from gpu_util import FIELD_TOL, grad_abs_scales, grad_err

pytestmark = pytest.mark.gpu


def test_double_gem_probe_loss_gradient_at_full_size():
    mesh, gas, ch, trk, d, probe = inputs.config_double_gem(seed=1, n=100_000, n_probe=4096)
    assert mesh.n >= 118_000
    ng = len(mesh.group_voltage)
    ctx = obem.obem_create(capacity=16, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        obem.obem_bem_assemble(ctx, obem.OBEM_LU_BF16)
        sig = torch.empty(mesh.n, dtype=torch.float32, device="cuda")
        rep = obem.obem_bem_solve(ctx, mesh.group_voltage, sig)
        assert rep["status"] == 0 and rep["backward_error"] < 1e-9
        tgt = torch.zeros((len(probe), 4), dtype=torch.float32, device="cuda")
        tgt[:, :3] = torch.from_numpy(probe.astype(np.float32)).cuda()
        src = torch.from_numpy(ch.pos_q).cuda()

        def loss(s):
            E = torch.empty((len(probe), 4), dtype=torch.float32, device="cuda")
            obem.obem_field_eval(ctx, tgt, E, sources=src, sigma=s)
            return E, float((E[:, :3].double() ** 2).sum(dim=1).mean())

        E, L0 = loss(sig)
        g = torch.zeros_like(E)
        g[:, :3] = 2.0 * E[:, :3] / len(probe)
        dsig = torch.empty(mesh.n, dtype=torch.float32, device="cuda")
        dsrc = torch.empty((ch.n, 4), dtype=torch.float32, device="cuda")
        obem.obem_field_eval_backward(ctx, tgt, g, sources=src, sigma=sig, dL_dsigma=dsig, dL_dsources=dsrc)
        dV, arep = obem.obem_bem_solve_adjoint(ctx, dsig, ng)
        assert arep.status == 0
        # central differences of the loss in each voltage (quadratic: exact)
        fd = []
        sk = torch.empty_like(sig)
        for k in range(ng):
            h = 0.05 * max(abs(float(mesh.group_voltage[k])), 10.0)
            vals = []
            for sgn in (1.0, -1.0):
                v = np.array(mesh.group_voltage, np.float64)
                v[k] += sgn * h
                obem.obem_bem_solve(ctx, v, sk)
                vals.append(loss(sk)[1])
            fd.append((vals[0] - vals[1]) / (2 * h))
        g_np = g.cpu().numpy().astype(np.float64)
        dsig_np = dsig.cpu().numpy().astype(np.float64)
        dsrc_np = dsrc.cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)
    fd = np.array(fd)
    dV = np.asarray(dV, np.float64)
    assert np.abs(dV - fd).max() <= 1e-3 * np.abs(fd).max(), (dV, fd)
    rng = np.random.default_rng(0)
    pts = probe.astype(np.float32).astype(np.float64)
    # dL/dsigma at 256 sampled cells
    cells = np.sort(rng.choice(mesh.n, 256, replace=False))
    tri = mesh.tri[cells]
    ds_ref, _, _ = oracle.field_backward(tri, np.zeros(len(cells)), pts, None, False, g_np)
    A_sig, _, _, _ = grad_abs_scales(pts, g_np, tri=tri)
    assert grad_err(dsig_np[cells], ds_ref, A_sig) <= FIELD_TOL
    # dL/d(position, charge) at 256 sampled charges
    qi = np.sort(rng.choice(ch.n, 256, replace=False))
    sub = ch.pos_q[qi].astype(np.float64)
    _, _, dq_ref = oracle.field_backward(None, None, pts, sub, False, g_np)
    _, _, A_sp, A_sq = grad_abs_scales(pts, g_np, src=sub)
    assert grad_err(dsrc_np[qi, :3], dq_ref[:, :3], A_sp) <= FIELD_TOL
    assert grad_err(dsrc_np[qi, 3], dq_ref[:, 3], A_sq) <= FIELD_TOL
    assert np.isfinite(L0) and L0 > 0
