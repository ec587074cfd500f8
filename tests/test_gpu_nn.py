"""Approximate N-body field (obem_nbody_nn_eval, OBEM_STEP_NBODY_NN; CUDA
through the C ABI) against the oracle's implementation of the same
approximation (same cells, FP64 sums): 1e-5 of max(|E|, 1e-2 rms|E|), the
field tolerance.  The NN field is repeatable to binary32 rounding (the order
of the charges inside a cell comes from the counting sort's atomics)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem
from gpu_util import FIELD_TOL, guarded_rel_err, to_dev

pytestmark = pytest.mark.gpu
E = 1.602176634e-19


def _clouds(n, seed):
    rng = np.random.default_rng(seed)
    k = n // 3
    p = np.concatenate([rng.normal([0, 0, 0], 2e-5, (k, 3)), rng.normal([8e-5, 1e-5, 2e-4], 3e-5, (k, 3)),
                        rng.uniform([-1e-4, -1e-4, -1e-4], [3e-4, 2e-4, 4e-4], (n - 2 * k, 3))])
    q = rng.choice([-E, E], n)
    return np.column_stack([p, q]).astype(np.float32)


def _gpu_nn(src, grid, soft):
    ctx = obem.obem_create(capacity=max(len(src), 16), dt=1e-12)
    try:
        out = torch.full((len(src), 4), float("nan"), device="cuda")
        obem.obem_nbody_nn_eval(ctx, to_dev(src), out, grid, soft)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)
    finally:
        obem.obem_destroy(ctx)


@pytest.mark.parametrize("n,grid", [(1, 4), (37, 1), (3000, 2), (3000, 4), (3000, 8), (5000, 16), (4000, 64)])
def test_nn_matches_oracle(n, grid):
    src = _clouds(n, n + grid)
    got = _gpu_nn(src, grid, 1e-9)
    ref = oracle.nbody_nn(src.astype(np.float64), grid, 1e-9)
    assert np.all(got[:, 3] == 0.0)
    if n == 1:
        assert np.all(got[:, :3] == 0.0)
        return
    assert guarded_rel_err(got[:, :3], ref) <= FIELD_TOL


def test_nn_lattice_equals_exact_sum():
    """No two charges in neighbouring cells: every charge centre is exact, so
    the approximation is the exact sum."""
    K, h = 5, 1e-5
    rng = np.random.default_rng(4)
    g = np.arange(K) * 2 * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    p = np.column_stack([X.ravel(), Y.ravel(), Z.ravel()])
    src = np.column_stack([p, rng.choice([-E, E], len(p))]).astype(np.float32)
    got = _gpu_nn(src, 2 * K - 1, 0.0)
    ref = oracle.nbody_field(src[:, :3].astype(np.float64), src.astype(np.float64), True, 0.0)[0]
    assert guarded_rel_err(got[:, :3], ref) <= FIELD_TOL


def test_nn_repeatable_to_rounding_and_step_mode_uses_it():
    """The charges of a cell are summed in the order the counting sort's
    atomics left them, so two evaluations agree to binary32 rounding (not bit
    for bit); the step's NN mode takes that field: a step fed the separately
    evaluated NN field takes the same decisions for (almost) every charge."""
    src = _clouds(3000, 9)
    e1, e2 = _gpu_nn(src, 8, 1e-9), _gpu_nn(src, 8, 1e-9)
    assert guarded_rel_err(e1[:, :3], e2[:, :3]) <= FIELD_TOL     # 32-term binary32 chunks, any order
    gas = inputs.argon_like_gas()
    trk = inputs.Tracking(dt=1e-12, seed=3, z_lo=-1.0, z_hi=1.0, beta=1e-13)
    rng = np.random.default_rng(1)
    sp = (src[:, 3] > 0).astype(np.uint8)                  # electrons (q < 0), cations (q > 0)
    ch = inputs.make_charges(src[:, :3].astype(np.float64), inputs.maxwellian(rng, 3000, 1.0, 9.1093837015e-31), sp)
    cap = 4096
    flags = obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_NBODY_NN
    ctx = obem.obem_create(capacity=cap, dt=trk.dt, seed=trk.seed, softening=1e-9, z_lo=trk.z_lo, z_hi=trk.z_hi,
                           beta=trk.beta, flags=flags, nn_grid=8)
    try:
        obem.obem_gas_load(ctx, gas)
        a, b = obem.DeviceState(cap), obem.DeviceState(cap)
        a.upload(ch)
        b.upload(ch)
        sa, sb = obem.new_stats(), obem.new_stats()
        obem.obem_step(ctx, a, 0, sa)
        Eb = torch.zeros((cap, 4), device="cuda")
        obem.obem_nbody_nn_eval(ctx, b.pos_q[:3000], Eb[:3000], 8, 1e-9)
        obem.obem_step(ctx, b, 0, sb, E_in=Eb)
        torch.cuda.synchronize()
        ga, _ = a.download()
        gb, _ = b.download()
    finally:
        obem.obem_destroy(ctx)
    common, ia, ib = np.intersect1d(ga.id, gb.id, return_indices=True)
    assert len(common) >= 0.99 * max(len(ga.id), len(gb.id))
    va, vb = ga.vel[ia, :3].astype(float), gb.vel[ib, :3].astype(float)
    rel = np.linalg.norm(va - vb, axis=1) / np.maximum(np.linalg.norm(vb, axis=1), 1.0)
    assert (rel < 1e-4).mean() > 0.99


def test_nn_bad_arguments():
    ctx = obem.obem_create(capacity=16, dt=1e-12)
    try:
        t = torch.zeros((4, 4), device="cuda")
        for grid in (0, 65):
            with pytest.raises(obem.ObemError) as e:
                obem.obem_nbody_nn_eval(ctx, t, torch.empty_like(t), grid)
            assert e.value.code == obem.OBEM_ERR_ARG
        big = torch.zeros((17, 4), device="cuda")
        with pytest.raises(obem.ObemError) as e:
            obem.obem_nbody_nn_eval(ctx, big, torch.empty_like(big), 4)
        assert e.value.code == obem.OBEM_ERR_ARG
    finally:
        obem.obem_destroy(ctx)
