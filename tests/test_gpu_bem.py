"""obem_bem_assemble / obem_bem_solve (CUDA, through the C ABI) against the
oracle's FP64 assembly and Gaussian elimination.

The GPU matrix is assembled with FP32 quadrature for far cells (per-element
relative error <= ~4e-7) and stored in FP32, so sigma can differ from the
FP64 solution by up to cond(A) x that; the tests bound the *backward* error of
sigma_gpu in the oracle's FP64 system (a property independent of cond(A))
and the forward difference with a cond-aware margin."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem
from gpu_util import FIELD_TOL, guarded_rel_err

pytestmark = pytest.mark.gpu
EPS0 = 8.8541878128e-12


def _gpu_solve(mesh, precision=obem.OBEM_LU_FP32, drhs=None, sigma_free=None, gv=None):
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        obem.obem_bem_assemble(ctx, precision)
        out = torch.empty(mesh.n, dtype=torch.float32, device="cuda")
        d = torch.from_numpy(np.asarray(drhs, np.float32)).cuda() if drhs is not None else None
        f = torch.from_numpy(np.asarray(sigma_free, np.float32)).cuda() if sigma_free is not None else None
        rep = obem.obem_bem_solve(ctx, mesh.group_voltage if gv is None else gv, out, sigma_free=f, drhs=d)
        return out.cpu().numpy().astype(np.float64), rep
    finally:
        obem.obem_destroy(ctx)


def _backward_error(A, x, b):
    r = A @ x - b
    return np.abs(r).max() / (np.abs(A).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max())


def _check(mesh, sig, A, b, ref, be_tol=2e-6, fwd_tol=2e-4):
    assert np.all(np.isfinite(sig))
    assert _backward_error(A, sig, b) <= be_tol
    assert np.abs(sig - ref).max() <= fwd_tol * np.abs(ref).max()


@pytest.mark.parametrize("precision", [obem.OBEM_LU_FP32, obem.OBEM_LU_TF32, obem.OBEM_LU_BF16,
                                       obem.OBEM_LU_BF16X9])
def test_parallel_plates_all_precisions(precision):
    mesh = inputs.parallel_plates(1e-2, 1e-3, 16, 0.0, 100.0)
    A = oracle.assemble(mesh)
    b = oracle.bem_rhs(mesh)
    ref = oracle.solve(A, b)
    sig, rep = _gpu_solve(mesh, precision)
    assert rep["status"] == 0 and rep["backward_error"] < 1e-9
    _check(mesh, sig, A, b, ref)


def test_conducting_sphere():
    mesh = inputs.conducting_sphere(1e-3, 3, 1.0)
    A = oracle.assemble(mesh)
    b = oracle.bem_rhs(mesh)
    ref = oracle.solve(A, b)
    sig, rep = _gpu_solve(mesh)
    _check(mesh, sig, A, b, ref)
    area = 0.5 * np.linalg.norm(np.cross(mesh.tri[:, 1] - mesh.tri[:, 0], mesh.tri[:, 2] - mesh.tri[:, 0]), axis=1)
    assert abs((sig * area).sum() / (ref * area).sum() - 1) < 1e-5


def test_dielectric_sphere_with_rhs_correction():
    tri = inputs.icosphere(1e-3, 3)
    n = len(tri)
    mesh = inputs.Mesh(tri, np.ones(n, np.int32), -np.ones(n, np.int32), np.full(n, 4.0), np.ones(n),
                       np.zeros(0))
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    drhs = -(1.0 - 4.0) * EPS0 * (nrm @ np.array([0, 0, 1e5]))
    A = oracle.assemble(mesh)
    ref = oracle.solve(A, drhs)
    sig, rep = _gpu_solve(mesh, drhs=drhs, gv=np.zeros(0))
    _check(mesh, sig, A, drhs.astype(np.float32).astype(np.float64), ref)


@pytest.mark.parametrize("precision", [obem.OBEM_LU_FP32, obem.OBEM_LU_BF16])
def test_gem_patch_mixed_electrode_dielectric(precision):
    """Mixed electrode / dielectric rows; with BF16 panels the refinement
    (FP64 residuals) must recover the FP32 solution's accuracy."""
    g = inputs.GemGeometry(rings=1)
    mesh = inputs.gem_mesh(g, n_theta=24, n_r=3, n_zc=1, n_zk=6, n_plane=10)
    A = oracle.assemble(mesh)
    b = oracle.bem_rhs(mesh)
    ref = oracle.solve(A, b)
    sig, rep = _gpu_solve(mesh, precision)
    assert rep["status"] == 0
    _check(mesh, sig, A, b, ref, fwd_tol=1e-3)
    # field from the GPU solution vs the oracle's, in the holes
    rng = np.random.default_rng(1)
    hc = g.hole_centres()
    p = np.column_stack([hc[rng.integers(0, len(hc), 400)], np.zeros(400)]) + rng.normal(0, 15e-6, (400, 3))
    p = p[~inputs.gem_inside_solid(g, p)]
    E1, _ = oracle.panel_field(mesh.tri, sig, p)
    E2, _ = oracle.panel_field(mesh.tri, ref, p)
    assert guarded_rel_err(E1, E2) < 2e-4


def test_free_charge_and_voltage_resolve():
    """Sec. 2.2: the stored factorisation is reused for new voltages and free
    charges (Eq. (charge-up) right-hand side)."""
    g = inputs.GemGeometry(rings=1)
    mesh = inputs.gem_mesh(g, n_theta=24, n_r=2, n_zc=1, n_zk=4, n_plane=8)
    A = oracle.assemble(mesh)
    rng = np.random.default_rng(2)
    sf = np.where(mesh.kind == 1, rng.uniform(-1e-6, 1e-6, mesh.n), 0.0).astype(np.float32)
    gv = mesh.group_voltage * 1.1
    b = oracle.bem_rhs(mesh, sigma_free=sf.astype(np.float64), group_voltage=gv)
    ref = oracle.solve(A, b)
    sig, rep = _gpu_solve(mesh, sigma_free=sf, gv=gv)
    _check(mesh, sig, A, b, ref, fwd_tol=1e-3)


def test_solve_before_assemble_is_a_state_error():
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        mesh = inputs.parallel_plates(1e-2, 1e-3, 4)
        obem.obem_mesh_load(ctx, mesh)
        out = torch.empty(mesh.n, device="cuda")
        with pytest.raises(obem.ObemError) as e:
            obem.obem_bem_solve(ctx, mesh.group_voltage, out)
        assert e.value.code == obem.OBEM_ERR_STATE
    finally:
        obem.obem_destroy(ctx)


def test_bounded_wait_reports_timeout_and_leaves_the_context_usable():
    """Failure detection without a fault: the wait that the LU panel
    factorisation uses between its CTAs (for every CTA's pivot candidate of a
    column) is made to wait for candidates that no block publishes.  Every
    wait gives up after its time limit, the kernel
    records OBEM_ERR_TIMEOUT in its status word and returns (the call reports
    OBEM_OK when it reads that status back); the same context then assembles,
    factorises and solves a small system correctly."""
    mesh = inputs.parallel_plates(1e-2, 1e-3, 8, 0.0, 100.0)
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_selftest_wait_timeout(ctx)
        obem.obem_mesh_load(ctx, mesh)
        obem.obem_bem_assemble(ctx, obem.OBEM_LU_FP32)
        out = torch.empty(mesh.n, dtype=torch.float32, device="cuda")
        rep = obem.obem_bem_solve(ctx, mesh.group_voltage, out)
        assert rep["status"] == 0
        sig = out.cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)
    A = oracle.assemble(mesh)
    b = oracle.bem_rhs(mesh)
    _check(mesh, sig, A, b, oracle.solve(A, b))


def test_solve_and_influence_waits_report_timeout_and_leave_the_context_usable():
    """Failure detection of the two other bounded device waits: the flag wait
    of the one-launch substitutions (a block row that no block solves) and the
    bulk-copy wait of the influence pass (barriers expecting more bytes than
    arrive).  Each runs out, is reported as OBEM_ERR_TIMEOUT and read back;
    the same context then solves the system and evaluates the influence of a
    distant charge correctly."""
    mesh = inputs.parallel_plates(1e-2, 1e-3, 8, 0.0, 100.0)
    assert mesh.n >= 256
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        obem.obem_bem_assemble(ctx, obem.OBEM_LU_FP32)
        obem.obem_selftest_waits(ctx, 1)
        obem.obem_selftest_waits(ctx, 2)
        out = torch.empty(mesh.n, dtype=torch.float32, device="cuda")
        rep = obem.obem_bem_solve(ctx, mesh.group_voltage, out)
        assert rep["status"] == 0
        sig = out.cpu().numpy().astype(np.float64)
        src = torch.tensor([[5e-3, 5e-3, 0.5, 1.602176634e-19]], dtype=torch.float32, device="cuda")
        drhs = torch.empty(mesh.n, dtype=torch.float32, device="cuda")
        obem.obem_influence_rhs(ctx, src, drhs)
        d = drhs.cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)
    A = oracle.assemble(mesh)
    b = oracle.bem_rhs(mesh)
    _check(mesh, sig, A, b, oracle.solve(A, b))
    ref = oracle.influence_rhs(mesh, np.array([[5e-3, 5e-3, 0.5, 1.602176634e-19]]))
    assert np.abs(d - ref).max() <= 1e-5 * np.abs(ref).max()
