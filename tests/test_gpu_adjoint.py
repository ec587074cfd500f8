"""obem_bem_solve_adjoint and gradients through solve + field (CUDA, through
the C ABI) against the oracle.  As for the forward solve, the GPU matrix
carries the FP32 quadrature error of far cells (~4e-7 per element), so the
adjoint mu is checked by its backward error in the oracle's FP64 transposed
system and by a cond-aware forward margin (2e-4 of max|mu|); gradients that
pass through a solve get the same margin."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem

pytestmark = pytest.mark.gpu


def _sphere_mesh(level=2, n_plate=8):
    return inputs.dielectric_sphere_in_plates(radius=1e-3, level=level, eps_r=4.0, side=2e-2, gap=1e-2,
                                              n_plate=n_plate)


def _probe_line(n=256):
    c = np.array([1e-2, 1e-2, 5e-3])
    t = np.linspace(-1.0, 1.0, n)
    return c + np.column_stack([4e-3 * t, 1.5e-3 + 0 * t, 4e-3 * t])


def test_adjoint_solve_matches_oracle():
    mesh = _sphere_mesh()
    rng = np.random.default_rng(9)
    g = rng.normal(0, 1.0, mesh.n).astype(np.float32)
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        obem.obem_bem_assemble(ctx, obem.OBEM_LU_FP32)
        db = torch.full((mesh.n,), float("nan"), device="cuda")
        dv, rep = obem.obem_bem_solve_adjoint(ctx, torch.from_numpy(g).cuda(), len(mesh.group_voltage), dL_db=db)
        mu = db.cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)
    assert rep.status == 0 and rep.iterations <= 10
    A = oracle.assemble(mesh)
    mu_ref, dv_ref = oracle.bem_solve_adjoint(mesh, g.astype(np.float64))
    r = A.T @ mu - g
    be = np.abs(r).max() / (np.abs(A.T).sum(axis=1).max() * np.abs(mu).max() + np.abs(g).max())
    assert be <= 2e-6
    assert np.abs(mu - mu_ref).max() <= 2e-4 * np.abs(mu_ref).max()
    assert np.abs(dv - dv_ref).max() <= 2e-4 * np.abs(dv_ref).max()


def test_voltage_gradient_of_probe_loss_through_autograd():
    """L = mean |E|^2 on a 256-point probe line, E = field of sigma =
    solve(V) (the differentiable-field workload at small size): dL/dV from
    torch.autograd through BemSolve and FieldEval against the oracle's chain
    and against FP64 central differences of the oracle's forward pipeline."""
    mesh = _sphere_mesh()
    pts = _probe_line()
    V0 = np.array([-300.0, 1000.0])
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        obem.obem_bem_assemble(ctx, obem.OBEM_LU_FP32)
        V = torch.tensor(V0, dtype=torch.float64, requires_grad=True)
        sigma = obem.bem_solve(ctx, V, mesh.n)
        tgt = torch.zeros((len(pts), 4), dtype=torch.float32, device="cuda")
        tgt[:, :3] = torch.from_numpy(pts.astype(np.float32)).cuda()
        E = obem.field_eval(ctx, tgt, None, sigma)
        loss = (E[:, :3].double() ** 2).sum(dim=1).mean()
        loss.backward()
        dV = V.grad.numpy().copy()
    finally:
        obem.obem_destroy(ctx)
    p32 = pts.astype(np.float32).astype(np.float64)
    sig = oracle.bem_solve(mesh, group_voltage=V0)
    Er, _ = oracle.panel_field(mesh.tri, sig, p32)
    g = np.column_stack([2.0 * Er / len(pts), np.zeros(len(pts))])
    dsig, _, _ = oracle.field_backward(mesh.tri, sig, p32, None, False, g)
    _, dV_ref = oracle.bem_solve_adjoint(mesh, dsig)
    assert np.abs(dV - dV_ref).max() <= 2e-4 * np.abs(dV_ref).max()

    def loss_of(Vv):
        s = oracle.bem_solve(mesh, group_voltage=Vv)
        e, _ = oracle.panel_field(mesh.tri, s, p32)
        return float((e ** 2).sum(axis=1).mean())
    for k in range(2):
        h = 1e-4 * abs(V0[k])
        Vp, Vm = V0.copy(), V0.copy()
        Vp[k] += h
        Vm[k] -= h
        fd = (loss_of(Vp) - loss_of(Vm)) / (2 * h)
        assert abs(dV[k] - fd) <= 2e-4 * np.abs(dV_ref).max()


def test_adjoint_before_assemble_is_a_state_error():
    mesh = _sphere_mesh(level=1, n_plate=4)
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        with pytest.raises(obem.ObemError) as e:
            obem.obem_bem_solve_adjoint(ctx, torch.zeros(mesh.n, device="cuda"), 2)
        assert e.value.code == obem.OBEM_ERR_STATE
    finally:
        obem.obem_destroy(ctx)
