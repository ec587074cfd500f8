"""The LU factorisation and refinement of the dense BEM solve (Sec. 2.2,
Eq. (matrixBEM)) on caller-given matrices through obem_dense_factor /
obem_dense_solve, in every arithmetic.

The assembled BEM matrices (rows equilibrated, diagonal large) seldom need a
row swap, so the pivoting is exercised here on rows permuted at random: the
matrix P (c I + G / sqrt(n)) (G standard normal, c = 2) has every eigenvalue of
the unpermuted part within distance 1 of c, so it is well conditioned, and
partial pivoting must undo P column by column.  The solution is compared
with LAPACK's FP64 solve (numpy) by backward and forward error; sizes include
ragged ones (not a multiple of the 64-column panels) and sizes where the BF16
factorisation recurses several levels."""
import numpy as np
import pytest
import torch

from paper_2110_09214_gb300 import obem

pytestmark = pytest.mark.gpu


def _system(n, seed):
    rng = np.random.default_rng(seed)
    M = 2.0 * np.eye(n) + rng.normal(size=(n, n)) / np.sqrt(n)
    A = M[rng.permutation(n)].astype(np.float32)
    b = rng.normal(size=n)
    return A, b


def _solve(A, b, precision):
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_dense_factor(ctx, torch.from_numpy(A).cuda(), precision)
        x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        rep = obem.obem_dense_solve(ctx, torch.from_numpy(b).cuda(), x)
        return x.cpu().numpy(), rep
    finally:
        obem.obem_destroy(ctx)


PRECISIONS = [obem.OBEM_LU_FP32, obem.OBEM_LU_TF32, obem.OBEM_LU_BF16, obem.OBEM_LU_BF16X9]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n", [1, 63, 64, 65, 200, 1000, 3001])
def test_permuted_system_against_lapack(n, precision):
    A, b = _system(n, n + 17 * precision)
    x, rep = _solve(A, b, precision)
    A64 = A.astype(np.float64)
    ref = np.linalg.solve(A64, b)
    assert rep["status"] == 0
    be = np.abs(A64 @ x - b).max() / (np.abs(A64).sum(1).max() * np.abs(x).max() + np.abs(b).max())
    assert be < 2e-12, be
    assert np.abs(x - ref).max() <= 1e-11 * np.abs(ref).max()


def test_bf16_recursive_factorisation_at_8193():
    """Several recursion levels, a ragged last panel, pivoting everywhere."""
    A, b = _system(8193, 5)
    x, rep = _solve(A, b, obem.OBEM_LU_BF16)
    A64 = A.astype(np.float64)
    assert rep["status"] == 0 and rep["backward_error"] < 1e-12
    ref = np.linalg.solve(A64, b)
    assert np.abs(x - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("precision", [obem.OBEM_LU_FP32, obem.OBEM_LU_BF16])
def test_zero_column_is_reported_singular(precision):
    A, _ = _system(300, 3)
    A[:, 170] = 0.0
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        with pytest.raises(obem.ObemError) as e:
            obem.obem_dense_factor(ctx, torch.from_numpy(A).cuda(), precision)
        assert e.value.code == obem.OBEM_ERR_SINGULAR
        # the context stays usable
        A2, b2 = _system(300, 4)
        obem.obem_dense_factor(ctx, torch.from_numpy(A2).cuda(), precision)
        x = torch.zeros(300, dtype=torch.float64, device="cuda")
        rep = obem.obem_dense_solve(ctx, torch.from_numpy(b2).cuda(), x)
        assert rep["status"] == 0
        assert np.allclose(x.cpu().numpy(), np.linalg.solve(A2.astype(np.float64), b2), rtol=0, atol=1e-10)
    finally:
        obem.obem_destroy(ctx)


def test_dense_calls_need_a_context_without_mesh():
    from paper_2110_09214_gb300 import inputs
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        x = torch.zeros(4, dtype=torch.float64, device="cuda")
        with pytest.raises(obem.ObemError) as e:
            obem.obem_dense_solve(ctx, x, x)
        assert e.value.code == obem.OBEM_ERR_STATE
        obem.obem_mesh_load(ctx, inputs.parallel_plates(1e-2, 1e-3, 4))
        with pytest.raises(obem.ObemError) as e:
            obem.obem_dense_factor(ctx, torch.eye(4, device="cuda"))
        assert e.value.code == obem.OBEM_ERR_STATE
    finally:
        obem.obem_destroy(ctx)


def test_bf16_factorisation_at_20480_against_a_known_solution():
    """A system of order 20,480 (made on the GPU: P (2 I + G / sqrt(n)),
    pivoting at every column) with a known solution x: b = A x in FP64.  At
    this order the recursion's TRSM leaves meet right-hand sides wider than
    8192 columns (the thread-per-column leaf) as well as narrow ones (the
    warp-per-columns leaf), and the panels span up to 135 rows per CTA.  The
    refined solution must reproduce x: its error is at most the condition
    number (about 3) times the backward error."""
    n = 20480
    g = torch.Generator(device="cuda").manual_seed(7)
    M = torch.randn((n, n), device="cuda", generator=g) / n ** 0.5
    M.diagonal().add_(2.0)
    A = M[torch.randperm(n, device="cuda", generator=g)].contiguous()
    del M
    x_true = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    b = A.double() @ x_true
    ctx = obem.obem_create(capacity=8, dt=1e-12)
    try:
        obem.obem_dense_factor(ctx, A, obem.OBEM_LU_BF16)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        rep = obem.obem_dense_solve(ctx, b, x)
    finally:
        obem.obem_destroy(ctx)
    assert rep["status"] == 0 and rep["backward_error"] < 1e-12
    err = (x - x_true).abs().max().item() / x_true.abs().max().item()
    assert err < 1e-11, err
