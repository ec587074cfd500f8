"""The tensor-core BF16 path of the dense BEM solve (Sec. 2.2, Eq. (matrixBEM)).

1. obem_tc_gemm, the trailing update C -= A B with BF16 operands and FP32
   accumulation on tcgen05, against an FP64 product of the same BF16-rounded
   operands: ragged sizes (partial 128 x 256 tiles, K not a multiple of the
   64-wide slices), sub-blocks of larger arrays (leading dimensions), and
   nothing written outside the block.
2. The recursive BF16 LU with FP64-residual refinement against the oracle's
   FP64 solve at ~8.5k and ~9k cells (parallel plates; a GEM patch with
   dielectric rows): the backward error of sigma in the oracle's system and
   the forward difference, as in the FP32 tests."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09214_gb300 import inputs, obem
from test_gpu_bem import _check, _gpu_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = obem.obem_create(capacity=8, dt=1e-12)
    yield c
    obem.obem_destroy(c)


def _bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (128, 256, 64), (130, 300, 70), (257, 1000, 333),
                                   (1000, 513, 4100), (3000, 64, 64), (64, 3000, 1536)])
def test_tc_gemm_matches_fp64_product_of_bf16_operands(ctx, M, N, K):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    pad = 5
    big_c = torch.randn(M + 2 * pad, N + 2 * pad + 3, generator=g, dtype=torch.float32)
    big_a = torch.randn(M + pad, K + 9, generator=g, dtype=torch.float32)
    big_b = torch.randn(K + pad, N + 11, generator=g, dtype=torch.float32)
    Cd = big_c.cuda()
    Ad, Bd = big_a.cuda(), big_b.cuda()
    Cv = Cd[pad:pad + M, pad:pad + N]
    Av = Ad[pad:pad + M, 2:2 + K]
    Bv = Bd[1:1 + K, 3:3 + N]
    obem.obem_tc_gemm(ctx, Cv, Av, Bv)
    torch.cuda.synchronize()
    got = Cd.cpu()
    a = _bf16(big_a[pad:pad + M, 2:2 + K])
    b = _bf16(big_b[1:1 + K, 3:3 + N])
    c0 = big_c[pad:pad + M, pad:pad + N].double()
    ref = c0 - a @ b
    scale = c0.abs() + a.abs() @ b.abs()
    err = ((got[pad:pad + M, pad:pad + N].double() - ref).abs() / scale).max().item()
    assert err <= 3e-5, err
    # nothing outside the block changed
    mask = torch.ones_like(big_c, dtype=torch.bool)
    mask[pad:pad + M, pad:pad + N] = False
    assert torch.equal(got[mask], big_c[mask])


def test_tc_gemm_rejects_bad_sizes(ctx):
    """A leading dimension smaller than the row length is rejected before
    any launch."""
    import ctypes as Cc
    C = torch.zeros(4, 4, device="cuda")
    p = Cc.c_void_p(C.data_ptr())
    assert obem.load().obem_tc_gemm(ctx, p, 2, p, 4, p, 4, 4, 4, 4, None) == obem.OBEM_ERR_ARG
    assert obem.load().obem_tc_gemm(ctx, p, 4, p, 4, p, 4, -1, 4, 4, None) == obem.OBEM_ERR_ARG


@pytest.mark.parametrize("case", ["plates", "gem"])
def test_bf16_recursive_lu_against_oracle_at_8k_cells(case):
    if case == "plates":
        mesh = inputs.parallel_plates(1e-2, 1e-3, 46, 0.0, 100.0)              # 8,464 cells
    else:
        mesh = inputs.gem_mesh_target(9000, inputs.GemGeometry(rings=1))
    assert mesh.n >= 8192
    A = oracle.assemble(mesh)
    b = oracle.bem_rhs(mesh)
    ref = oracle.solve(A, b)
    sig, rep = _gpu_solve(mesh, obem.OBEM_LU_BF16)
    assert rep["status"] == 0 and rep["backward_error"] < 1e-9
    _check(mesh, sig, A, b, ref, fwd_tol=1e-3)
