"""Charging-up (OBEM_STEP_SURFACE_HITS, obem_surface_charge; CUDA through the
C ABI) against the oracle: the step with cells absorbing the charges that
cross them is bit-identical to the oracle's (states and per-cell deposit
counts), the free density e * count / area is the oracle's, and the re-solve
with it (Eq. (charge-up) fed to Eq. (matrixBEM)) passes the solve's checks."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem
from gpu_util import to_dev

pytestmark = pytest.mark.gpu
ME = 9.1093837015e-31


def _setup(seed=3):
    mesh = inputs.dielectric_sphere_in_plates(radius=1e-3, level=2, eps_r=4.0, side=2e-2, gap=1e-2, n_plate=8)
    rng = np.random.default_rng(seed)
    c = np.array([1e-2, 1e-2, 5e-3])
    n_s, n_p = 1500, 500
    d = rng.normal(size=(n_s, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = rng.uniform(1.0005e-3, 1.003e-3, n_s)
    ps = c + d * r[:, None]
    vs = -d * rng.uniform(3e5, 2e6, n_s)[:, None] + rng.normal(0, 1e5, (n_s, 3))
    pp = np.column_stack([rng.uniform(2e-3, 1.8e-2, (n_p, 2)), rng.uniform(2e-7, 3e-6, n_p)])
    vp = np.column_stack([rng.normal(0, 1e5, (n_p, 2)), -rng.uniform(3e5, 2e6, n_p)])
    pos, vel = np.concatenate([ps, pp]), np.concatenate([vs, vp])
    sp = (rng.random(n_s + n_p) < 0.3).astype(np.uint8)          # 30 % cations
    ch = inputs.make_charges(pos, vel, sp)
    gas = inputs.argon_like_gas()
    trk = inputs.Tracking(dt=1e-12, seed=seed, z_lo=0.0, z_hi=1e-2, beta=-1.0, surface_hits=True)
    return mesh, gas, ch, trk


def test_surface_hits_step_bit_exact_with_deposits():
    mesh, gas, ch, trk = _setup()
    cap = 4096
    ctx = obem.obem_create(capacity=cap, dt=trk.dt, seed=trk.seed, z_lo=trk.z_lo, z_hi=trk.z_hi, beta=trk.beta,
                           flags=obem.OBEM_STEP_SURFACE_HITS)
    dep_o = np.zeros(mesh.n, np.int64)
    try:
        obem.obem_gas_load(ctx, gas)
        obem.obem_mesh_load(ctx, mesh)
        st = obem.DeviceState(cap)
        st.upload(ch)
        stats = obem.new_stats()
        cur, nid = ch, ch.n
        rng = np.random.default_rng(1)
        for s in range(6):
            E = (np.array([0.0, 0.0, -2e5]) + rng.normal(0, 5e4, (cur.pos_q.shape[0], 3))).astype(np.float32)
            buf = np.zeros((cap, 4), np.float32)
            buf[:len(E), :3] = E
            obem.obem_step(ctx, st, s, stats, E_in=to_dev(buf))
            torch.cuda.synchronize()
            gs = obem.read_stats(stats)
            rc, cur, nid, os_ = oracle.step(cur, E, s, nid, gas, trk, cap, mesh=mesh, deposits=dep_o)
            assert rc == 0 and gs["status"] == 0
            gst, gnid = st.download()
            for k in ("pos_q", "vel"):
                assert np.array_equal(getattr(gst, k).view(np.uint32), getattr(cur, k).view(np.uint32)), (s, k)
            assert np.array_equal(gst.id, cur.id) and gnid == nid
            assert gs["absorbed"] == os_["absorbed"]
        dep_g = obem.obem_surface_charge(ctx, mesh.n)
        sig_f = torch.full((mesh.n,), float("nan"), device="cuda")
        dep_g2 = obem.obem_surface_charge(ctx, mesh.n, sigma_free=sig_f, reset=True)
        dep_g3 = obem.obem_surface_charge(ctx, mesh.n)
        sig_f = sig_f.cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)
    assert np.array_equal(dep_g, dep_o) and np.array_equal(dep_g2, dep_o)
    assert np.all(dep_g3 == 0)                                         # reset
    dd = mesh.kind == 1
    assert np.abs(dep_o[dd]).sum() > 20 and np.abs(dep_o[~dd]).sum() > 20
    area = np.array([oracle.tri_geometry(t)[2] for t in mesh.tri])
    ref = np.where(dd, 1.602176634e-19 * dep_o / area, 0.0)
    assert np.abs(sig_f - ref).max() <= 1e-6 * np.abs(ref).max()


def test_resolve_with_collected_charge():
    """The collected free density on the dielectric sphere, fed back through
    Eq. (charge-up) into the solve: backward error of sigma in the oracle's
    FP64 system (the GPU matrix carries FP32 quadrature error)."""
    mesh, gas, ch, trk = _setup(5)
    rng = np.random.default_rng(2)
    dd = np.flatnonzero(mesh.kind == 1)
    counts = np.zeros(mesh.n, np.int64)
    counts[dd] = rng.integers(-40, 41, len(dd))
    area = np.array([oracle.tri_geometry(t)[2] for t in mesh.tri])
    sig_free = np.where(mesh.kind == 1, 1.602176634e-19 * counts / area, 0.0)
    ctx = obem.obem_create(capacity=16, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        obem.obem_bem_assemble(ctx, obem.OBEM_LU_FP32)
        out = torch.empty(mesh.n, dtype=torch.float32, device="cuda")
        rep = obem.obem_bem_solve(ctx, mesh.group_voltage, out, sigma_free=to_dev(sig_free.astype(np.float32)))
        sig = out.cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)
    A = oracle.assemble(mesh)
    b = oracle.bem_rhs(mesh, sigma_free=sig_free.astype(np.float32).astype(np.float64))
    r = A @ sig - b
    be = np.abs(r).max() / (np.abs(A).sum(axis=1).max() * np.abs(sig).max() + np.abs(b).max())
    assert rep["status"] == 0 and be <= 2e-6
