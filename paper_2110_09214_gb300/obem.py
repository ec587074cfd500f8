"""Python binding of the libobem C ABI (include/obem.h).

Argument marshalling only: every function below calls the entry point of the
same name in libobem.so with raw pointers taken from torch CUDA tensors (PyTorch
is used for device memory and streams).  There is no fallback: if the CUDA
library cannot be built or loaded, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

OBEM_OK = 0
OBEM_ERR_ARG, OBEM_ERR_CUDA, OBEM_ERR_STATE, OBEM_ERR_SINGULAR = -1, -2, -3, -4
OBEM_ERR_NOT_CONVERGED, OBEM_ERR_CAPACITY, OBEM_ERR_TIMEOUT, OBEM_ERR_TRIALS = -5, -6, -7, -8
OBEM_LU_FP32, OBEM_LU_TF32, OBEM_LU_BF16, OBEM_LU_BF16X9 = 0, 1, 2, 3
OBEM_STEP_SPACE_CHARGE, OBEM_STEP_CELL_FIELD, OBEM_STEP_FIELD_MAP, OBEM_STEP_PROB_COLLISION = 1, 2, 4, 8
OBEM_STEP_NBODY_NN, OBEM_NN_GMAX, OBEM_STEP_SURFACE_HITS = 16, 64, 32
OBEM_STEP_CELL_GROUPS = 64


class ObemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("obem error %d: %s" % (code, msg))
        self.code = code


class obem_config(C.Structure):
    _fields_ = [("capacity", C.c_int32), ("trial_cap", C.c_int32), ("flags", C.c_int32),
                ("nn_grid", C.c_int32), ("dt", C.c_double), ("seed", C.c_uint64),
                ("softening", C.c_double), ("z_lo", C.c_double), ("z_hi", C.c_double),
                ("beta", C.c_double), ("e_ext", C.c_double * 3)]


class obem_gas(C.Structure):
    _fields_ = [("n_proc", C.c_int32), ("n_energy", C.c_int32), ("energy_eV", C.c_void_p),
                ("sigma_m2", C.c_void_p), ("kind", C.c_void_p), ("mode", C.c_void_p),
                ("threshold_eV", C.c_void_p), ("nu_const", C.c_void_p), ("T", C.c_double),
                ("N", C.c_double), ("M_amu", C.c_double), ("nu_ion", C.c_double)]


class obem_state(C.Structure):
    _fields_ = [("pos_q", C.c_void_p), ("vel", C.c_void_p), ("id", C.c_void_p),
                ("birth", C.c_void_p), ("species", C.c_void_p), ("n", C.c_void_p),
                ("next_id", C.c_void_p), ("capacity", C.c_int32)]


class obem_step_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_before", C.c_int32), ("n_after", C.c_int32),
                ("required_capacity", C.c_int32), ("n_electron", C.c_int32),
                ("n_cation", C.c_int32), ("n_anion", C.c_int32), ("spawned_pairs", C.c_int32),
                ("absorbed", C.c_int32), ("attached", C.c_int32), ("recombined_pairs", C.c_int32),
                ("collisions", C.c_int32), ("trials", C.c_int64), ("sum_e", C.c_double * 3),
                ("sum2_e", C.c_double * 3), ("sum_i", C.c_double * 3), ("sum2_i", C.c_double * 3),
                ("sum_energy_e", C.c_double)]


class obem_solve_report(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("backward_error", C.c_double),
                ("factor_ms", C.c_double), ("solve_ms", C.c_double)]


STATS_BYTES = C.sizeof(obem_step_stats)

_lib = None


def library_path():
    return _build.LIB


def load():
    """Load libobem.so, building it with nvcc first if the sources changed."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = C.CDLL(path)
    P, I, U = C.c_void_p, C.c_int32, C.c_uint32
    lib.obem_create.argtypes = [C.POINTER(P), C.POINTER(obem_config)]
    lib.obem_destroy.argtypes = [P]
    lib.obem_destroy.restype = None
    lib.obem_last_error.argtypes = [P]
    lib.obem_last_error.restype = C.c_char_p
    lib.obem_gas_load.argtypes = [P, C.POINTER(obem_gas)]
    lib.obem_mesh_load.argtypes = [P, I, P, P, P, P, P, I]
    lib.obem_bem_assemble.argtypes = [P, I, P]
    lib.obem_bem_solve.argtypes = [P, P, P, P, P, C.POINTER(obem_solve_report), P]
    lib.obem_bem_solve_adjoint.argtypes = [P, P, P, P, C.POINTER(obem_solve_report), P]
    lib.obem_field_eval.argtypes = [P, P, I, P, I, I, P, P, P]
    lib.obem_field_eval_backward.argtypes = [P, P, I, P, I, I, P, P, P, P, P, P]
    lib.obem_step.argtypes = [P, C.POINTER(obem_state), P, U, P, P]
    lib.obem_field_eval_noalloc.argtypes = [P, I, P, I, I, P, P, I, P, C.c_char_p, I, P]
    lib.obem_field_eval_noalloc.restype = C.c_int
    lib.obem_profile.argtypes = [P, I]
    lib.obem_alu_rates.argtypes = [P, P, P]
    lib.obem_selftest_wait_timeout.argtypes = [P, P]
    lib.obem_selftest_waits.argtypes = [P, C.c_int32, P]
    L64 = C.c_int64
    lib.obem_tc_gemm.argtypes = [P, P, L64, P, L64, P, L64, I, I, I, P]
    lib.obem_tc_gemm.restype = C.c_int
    lib.obem_shard_field.argtypes = [P, C.POINTER(obem_state), P, I, I, P, P]
    lib.obem_shard_propose.argtypes = [P, C.POINTER(obem_state), C.POINTER(obem_state), U, P, P]
    lib.obem_shard_count.argtypes = [P, C.POINTER(obem_state), P, U, P, I, P, P]
    lib.obem_shard_commit.argtypes = [P, C.POINTER(obem_state), P, U, U, I, P, P]
    for f in ("obem_shard_field", "obem_shard_propose", "obem_shard_count", "obem_shard_commit"):
        getattr(lib, f).restype = C.c_int
    lib.obem_influence_rhs.argtypes = [P, P, I, P, P]
    lib.obem_influence_rhs.restype = C.c_int
    lib.obem_dense_factor.argtypes = [P, P, I, I, P]
    lib.obem_dense_factor.restype = C.c_int
    lib.obem_dense_solve.argtypes = [P, P, P, C.POINTER(obem_solve_report), P]
    lib.obem_dense_solve.restype = C.c_int
    lib.obem_fieldmap_build.argtypes = [P, P, P, P, P, P]
    lib.obem_nbody_nn_eval.argtypes = [P, P, I, I, C.c_double, P, P]
    lib.obem_surface_charge.argtypes = [P, P, P, I, P]
    lib.obem_fieldmap_eval.argtypes = [P, P, I, P, P]
    lib.obem_stage_times.argtypes = [P, P, P]
    lib.obem_batch_create.argtypes = [C.POINTER(P), P, I, P, P, P, P]
    lib.obem_batch_destroy.argtypes = [P]
    lib.obem_batch_destroy.restype = None
    lib.obem_batch_layout.argtypes = [P, P]
    lib.obem_batch_cells.argtypes = [P, I, I, P, P]
    lib.obem_batch_field_eval.argtypes = [P, C.POINTER(obem_state), P, P]
    lib.obem_batch_step.argtypes = [P, C.POINTER(obem_state), P, P, P, P]
    lib.obem_batch_step_graph.argtypes = [P, C.POINTER(obem_state), P, P, P]
    lib.obem_batch_autotune.argtypes = [P, C.POINTER(obem_state), I, P, P]
    lib.obem_batch_set_block.argtypes = [P, I]
    for f in ("obem_batch_create", "obem_batch_layout", "obem_batch_cells", "obem_batch_field_eval",
              "obem_batch_step", "obem_batch_step_graph", "obem_batch_autotune", "obem_batch_set_block"):
        getattr(lib, f).restype = C.c_int
    for f in ("obem_create", "obem_gas_load", "obem_mesh_load", "obem_bem_assemble",
              "obem_bem_solve", "obem_bem_solve_adjoint", "obem_field_eval", "obem_field_eval_backward", "obem_step", "obem_profile",
              "obem_stage_times", "obem_alu_rates", "obem_fieldmap_build", "obem_fieldmap_eval",
              "obem_nbody_nn_eval", "obem_surface_charge"):
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _check(ctx, rc):
    if rc != OBEM_OK:
        msg = load().obem_last_error(ctx).decode() if ctx else "invalid argument"
        raise ObemError(rc, msg)


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- entry points
def obem_create(capacity, dt, seed=1, softening=0.0, z_lo=-1.0, z_hi=1.0, beta=-1.0,
                trial_cap=256, flags=OBEM_STEP_SPACE_CHARGE | OBEM_STEP_CELL_FIELD,
                e_ext=(0.0, 0.0, 0.0), nn_grid=0):
    cfg = obem_config(capacity=int(capacity), trial_cap=int(trial_cap), flags=int(flags),
                      nn_grid=int(nn_grid), dt=float(dt), seed=int(seed), softening=float(softening),
                      z_lo=float(z_lo), z_hi=float(z_hi), beta=float(beta),
                      e_ext=(C.c_double * 3)(*[float(x) for x in e_ext]))
    ctx = C.c_void_p()
    rc = load().obem_create(C.byref(ctx), C.byref(cfg))
    if rc != OBEM_OK:
        raise ObemError(rc, "obem_create rejected the configuration")
    return ctx


def obem_destroy(ctx):
    if ctx:
        load().obem_destroy(ctx)


def obem_last_error(ctx):
    return load().obem_last_error(ctx).decode()


def obem_gas_load(ctx, gas):
    eg = _host(gas.egrid, np.float32)
    xs = _host(gas.xs, np.float32)
    kind = _host(gas.kind, np.int32)
    mode = _host(gas.mode, np.int32)
    thr = _host(gas.thr, np.float32)
    nuc = _host(gas.nuc, np.float32)
    g = obem_gas(n_proc=len(kind), n_energy=len(eg), energy_eV=eg.ctypes.data,
                 sigma_m2=xs.ctypes.data, kind=kind.ctypes.data, mode=mode.ctypes.data,
                 threshold_eV=thr.ctypes.data, nu_const=nuc.ctypes.data, T=float(gas.T),
                 N=float(gas.N), M_amu=float(gas.M_amu), nu_ion=float(gas.nu_ion))
    _check(ctx, load().obem_gas_load(ctx, C.byref(g)))


def obem_mesh_load(ctx, mesh):
    tri = _host(mesh.tri, np.float64)
    kind = _host(mesh.kind, np.int32)
    group = _host(mesh.group, np.int32)
    em = _host(mesh.eps_minus, np.float64)
    ep = _host(mesh.eps_plus, np.float64)
    _check(ctx, load().obem_mesh_load(ctx, mesh.n, tri.ctypes.data, kind.ctypes.data,
                                      group.ctypes.data, em.ctypes.data, ep.ctypes.data,
                                      mesh.n_groups))


def obem_bem_assemble(ctx, precision=OBEM_LU_FP32, stream=None):
    _check(ctx, load().obem_bem_assemble(ctx, int(precision), _stream(stream)))


def obem_bem_solve(ctx, group_voltage, sigma_out, sigma_free=None, drhs=None, stream=None,
                   check=True):
    gv = _host(group_voltage, np.float64)
    rep = obem_solve_report()
    rc = load().obem_bem_solve(ctx, gv.ctypes.data if len(gv) else None, _ptr(sigma_free),
                               _ptr(drhs), _ptr(sigma_out), C.byref(rep), _stream(stream))
    if check:
        _check(ctx, rc)
    return {"iterations": rep.iterations, "status": rep.status,
            "backward_error": rep.backward_error, "factor_ms": rep.factor_ms,
            "solve_ms": rep.solve_ms, "rc": rc}


def obem_bem_solve_adjoint(ctx, dL_dsigma, n_groups, dL_db=None, stream=None):
    """Adjoint of obem_bem_solve: returns (dL/dV [n_groups] float64 numpy,
    report) and writes dL/db into dL_db (device [n_panels]) if given."""
    dv = np.zeros(max(int(n_groups), 1), np.float64)
    rep = obem_solve_report()
    _check(ctx, load().obem_bem_solve_adjoint(ctx, _ptr(dL_dsigma), dv.ctypes.data_as(C.c_void_p),
                                              _ptr(dL_db), C.byref(rep), _stream(stream)))
    return dv[:int(n_groups)], rep


class BemSolve(torch.autograd.Function):
    """sigma = bem_solve(V, sigma_free, drhs) as a differentiable op (the
    context must hold the factors of the loaded mesh).  group_voltage is a
    float64 CPU tensor [n_groups]; sigma_free and drhs are device tensors
    [n_panels] or None.  The backward is obem_bem_solve_adjoint."""

    @staticmethod
    def forward(fctx, ctx, group_voltage, sigma_free, drhs, n_panels):
        dev = torch.device("cuda", torch.cuda.current_device())
        sigma = torch.empty(int(n_panels), dtype=torch.float32, device=dev)
        gv = group_voltage.detach().to("cpu", torch.float64).contiguous().numpy()
        obem_bem_solve(ctx, gv, sigma, sigma_free=sigma_free, drhs=drhs)
        fctx.ctx = ctx
        fctx.n_groups = int(group_voltage.numel())
        return sigma

    @staticmethod
    def backward(fctx, grad):
        grad = grad.contiguous().float()
        need_v, need_f, need_d = fctx.needs_input_grad[1:4]
        db = torch.empty_like(grad) if (need_f or need_d) else None
        dv, _ = obem_bem_solve_adjoint(fctx.ctx, grad, fctx.n_groups, dL_db=db)
        gv = torch.from_numpy(dv.copy()) if need_v else None
        return None, gv, db if need_f else None, db if need_d else None, None


def bem_solve(ctx, group_voltage, n_panels, sigma_free=None, drhs=None):
    """Differentiable BEM solve (see BemSolve)."""
    return BemSolve.apply(ctx, group_voltage, sigma_free, drhs, n_panels)


def obem_field_eval(ctx, targets, E_out, sources=None, self_exclude=False, sigma=None,
                    stream=None):
    nt = targets.shape[0]
    ns = sources.shape[0] if sources is not None else 0
    _check(ctx, load().obem_field_eval(ctx, _ptr(targets), nt, _ptr(sources), ns,
                                       int(bool(self_exclude)), _ptr(sigma), _ptr(E_out),
                                       _stream(stream)))


def obem_field_eval_backward(ctx, targets, dL_dE, sources=None, self_exclude=False, sigma=None,
                             dL_dsigma=None, dL_dtargets=None, dL_dsources=None, stream=None):
    """Vector-Jacobian product of obem_field_eval: writes dL/dsigma [n_panels],
    dL/dtargets [nt, 4] (x, y, z, 0) and dL/dsources [ns, 4] (x, y, z, q)
    into whichever output tensors are given."""
    nt = targets.shape[0]
    ns = sources.shape[0] if sources is not None else 0
    _check(ctx, load().obem_field_eval_backward(ctx, _ptr(targets), nt, _ptr(sources), ns,
                                                int(bool(self_exclude)), _ptr(sigma), _ptr(dL_dE),
                                                _ptr(dL_dsigma), _ptr(dL_dtargets), _ptr(dL_dsources),
                                                _stream(stream)))


class FieldEval(torch.autograd.Function):
    """E = field_eval(targets, sources, sigma) as a differentiable op: the
    forward is obem_field_eval, the backward obem_field_eval_backward.
    Gradients flow to targets[:, :3], sources[:, :4] (position and charge)
    and sigma."""

    @staticmethod
    def forward(fctx, ctx, targets, sources, sigma, self_exclude):
        out = torch.empty((targets.shape[0], 4), dtype=torch.float32, device=targets.device)
        obem_field_eval(ctx, targets, out, sources=sources, self_exclude=self_exclude, sigma=sigma,
                        stream=torch.cuda.current_stream(targets.device))
        fctx.ctx = ctx
        fctx.self_exclude = self_exclude
        fctx.save_for_backward(targets, sources, sigma)
        return out

    @staticmethod
    def backward(fctx, grad):
        targets, sources, sigma = fctx.saved_tensors
        need_t, need_s, need_sg = fctx.needs_input_grad[1:4]
        dev = targets.device
        grad = grad.contiguous().float()
        dt = torch.empty((targets.shape[0], 4), dtype=torch.float32, device=dev) if need_t else None
        ds = torch.empty((sources.shape[0], 4), dtype=torch.float32, device=dev) \
            if (need_s and sources is not None) else None
        dsg = torch.empty_like(sigma) if (need_sg and sigma is not None) else None
        obem_field_eval_backward(fctx.ctx, targets, grad, sources=sources, self_exclude=fctx.self_exclude,
                                 sigma=sigma, dL_dsigma=dsg, dL_dtargets=dt, dL_dsources=ds,
                                 stream=torch.cuda.current_stream(dev))
        return None, dt, ds, dsg, None


def field_eval(ctx, targets, sources=None, sigma=None, self_exclude=False):
    """Differentiable field and potential [nt, 4] at targets (see FieldEval)."""
    return FieldEval.apply(ctx, targets, sources, sigma, bool(self_exclude))


def obem_step(ctx, state, step, stats, E_in=None, stream=None):
    _check(ctx, load().obem_step(ctx, C.byref(state.c_struct()), _ptr(E_in), int(step),
                                 _ptr(stats), _stream(stream)))


NOALLOC_MAX_TARGETS, NOALLOC_MAX_CELLS = 262144, 16384


def obem_field_eval_noalloc(targets, E_out, sources=None, self_exclude=False, cell_xyz=None,
                            sigma=None, stream=None):
    """Field at targets without a context or any allocation (fixed scratch
    inside the library); same arguments as obem_field_eval, with the cells
    given directly as FP64 vertices [np, 3, 3] on the device."""
    nt = targets.shape[0]
    ns = sources.shape[0] if sources is not None else 0
    np_ = cell_xyz.shape[0] if cell_xyz is not None else 0
    err = C.create_string_buffer(256)
    rc = load().obem_field_eval_noalloc(_ptr(targets), nt, _ptr(sources), ns, int(bool(self_exclude)),
                                        _ptr(cell_xyz), _ptr(sigma), np_, _ptr(E_out), err, 256,
                                        _stream(stream))
    if rc != OBEM_OK:
        raise ObemError(rc, err.value.decode())


def obem_selftest_wait_timeout(ctx, stream=None):
    """Failure-detection self-test of the bounded device wait (see
    include/obem.h): raises ObemError unless the wait ran out and reported
    OBEM_ERR_TIMEOUT."""
    _check(ctx, load().obem_selftest_wait_timeout(ctx, _stream(stream)))


def obem_selftest_waits(ctx, which, stream=None):
    """Failure-detection self-test of bounded device wait `which` (0: LU panel
    candidate exchange, 1: substitution flags, 2: influence bulk copies); raises unless
    the wait reported OBEM_ERR_TIMEOUT (see include/obem.h)."""
    _check(ctx, load().obem_selftest_waits(ctx, int(which), _stream(stream)))


def obem_shard_field(ctx, state, sources, ns, self_off, E_out, stream=None):
    """Field at a shard's charges from the gathered charges (see obem.h)."""
    _check(ctx, load().obem_shard_field(ctx, C.byref(state.c_struct()), _ptr(sources), int(ns), int(self_off),
                                        _ptr(E_out), _stream(stream)))


def obem_shard_propose(ctx, state, gathered, step, ionkey, stream=None):
    """Recombination proposals of a shard's electrons into ionkey (int64 CUDA
    tensor over the gathered charges; reduce with MIN over the shards)."""
    _check(ctx, load().obem_shard_propose(ctx, C.byref(state.c_struct()), C.byref(gathered.c_struct()), int(step),
                                          _ptr(ionkey), _stream(stream)))


def obem_shard_count(ctx, state, E, step, ionkey, self_off, stats, stream=None):
    _check(ctx, load().obem_shard_count(ctx, C.byref(state.c_struct()), _ptr(E), int(step), _ptr(ionkey),
                                        int(self_off), _ptr(stats), _stream(stream)))


def obem_shard_commit(ctx, state, E, step, id_base, commit, stats, stream=None):
    _check(ctx, load().obem_shard_commit(ctx, C.byref(state.c_struct()), _ptr(E), int(step), int(id_base),
                                         int(bool(commit)), _ptr(stats), _stream(stream)))


def obem_influence_rhs(ctx, sources, drhs, stream=None):
    """drhs (CUDA float [n_panels]) = the right-hand-side correction of the
    charges sources (CUDA float [ns, 4]: x, y, z, q) on the cells, for
    obem_bem_solve(..., drhs=drhs) (Eqs. (BEMpotpart), (BEMfldpart))."""
    ns = sources.shape[0] if sources is not None else 0
    _check(ctx, load().obem_influence_rhs(ctx, _ptr(sources), ns, _ptr(drhs), _stream(stream)))


def obem_dense_factor(ctx, A, precision=OBEM_LU_FP32, stream=None):
    """Factorise a dense FP32 CUDA matrix [n, n] (row-major, contiguous) in
    place of an assembled BEM system (context without a mesh)."""
    n = A.shape[0]
    assert A.shape == (n, n) and A.is_contiguous() and A.element_size() == 4
    _check(ctx, load().obem_dense_factor(ctx, _ptr(A), n, int(precision), _stream(stream)))


def obem_dense_solve(ctx, b, x, stream=None):
    """x = A^-1 b (FP64 CUDA vectors) with the factors of obem_dense_factor
    and FP64-residual refinement; returns the solve report."""
    rep = obem_solve_report()
    _check(ctx, load().obem_dense_solve(ctx, _ptr(b), _ptr(x), C.byref(rep), _stream(stream)))
    return {"iterations": rep.iterations, "status": rep.status, "backward_error": rep.backward_error,
            "factor_ms": rep.factor_ms, "solve_ms": rep.solve_ms}


def obem_tc_gemm(ctx, C_, A, B, stream=None):
    """C_ -= A @ B on the tensor cores with BF16 operands and FP32
    accumulation (the BF16 LU's trailing update); C_, A, B: 2-D FP32 CUDA
    tensors with unit column stride (row-major, any row stride)."""
    M, K = A.shape
    N = B.shape[1]
    assert C_.shape == (M, N) and B.shape[0] == K
    for t in (C_, A, B):
        assert t.dtype.is_floating_point and t.element_size() == 4 and (t.shape[1] <= 1 or t.stride(1) == 1)
    _check(ctx, load().obem_tc_gemm(ctx, _ptr(C_), C_.stride(0), _ptr(A), A.stride(0), _ptr(B), B.stride(0),
                                    M, N, K, _stream(stream)))


def obem_alu_rates(ctx, stream=None):
    """Measured FP32 / rsqrt rates of the GPU (see include/obem.h)."""
    out = np.zeros(7, np.float64)
    _check(ctx, load().obem_alu_rates(ctx, out.ctypes.data_as(C.c_void_p), _stream(stream)))
    return {"fp32_tflops": out[0], "fp32_lane_ops_per_sm_clk": out[1], "rsqrt_per_sm_clk": out[2],
            "mix12_lane_ops_per_sm_clk": out[3], "sm_mhz": out[4], "mix16_lane_ops_per_sm_clk": out[5],
            "mix14_lane_ops_per_sm_clk": out[6]}


def obem_fieldmap_build(ctx, lo, hi, dims, sigma, stream=None):
    """Static field map of the cell field on a regular grid (see include/obem.h)."""
    lo = np.ascontiguousarray(lo, np.float64)
    hi = np.ascontiguousarray(hi, np.float64)
    dims = np.ascontiguousarray(dims, np.int32)
    _check(ctx, load().obem_fieldmap_build(ctx, lo.ctypes.data_as(C.c_void_p), hi.ctypes.data_as(C.c_void_p),
                                           dims.ctypes.data_as(C.c_void_p), _ptr(sigma), _stream(stream)))


def obem_fieldmap_eval(ctx, points, E_out, stream=None):
    _check(ctx, load().obem_fieldmap_eval(ctx, _ptr(points), points.shape[0], _ptr(E_out), _stream(stream)))


def obem_nbody_nn_eval(ctx, pos_q, E_out, grid, softening=0.0, stream=None):
    """Approximate N-body field at the charges (see include/obem.h)."""
    _check(ctx, load().obem_nbody_nn_eval(ctx, _ptr(pos_q), pos_q.shape[0], int(grid), float(softening),
                                          _ptr(E_out), _stream(stream)))


def obem_surface_charge(ctx, n_panels, sigma_free=None, reset=False, stream=None):
    """Charges collected by the cells (units of e, int64 numpy [n_panels]);
    writes e * count / area of the dielectric cells into sigma_free if given."""
    counts = np.zeros(int(n_panels), np.int64)
    _check(ctx, load().obem_surface_charge(ctx, _ptr(sigma_free), counts.ctypes.data_as(C.c_void_p),
                                           int(bool(reset)), _stream(stream)))
    return counts


OBEM_PROFILE_TIMES = 2


def obem_profile(ctx, enable=True):
    """True: stage events and evaluation counters; OBEM_PROFILE_TIMES: stage
    events only (the uncounted kernels run); False: off."""
    mode = OBEM_PROFILE_TIMES if (enable is not True and enable == OBEM_PROFILE_TIMES) else int(bool(enable))
    _check(ctx, load().obem_profile(ctx, mode))


def obem_stage_times(ctx):
    """Stage times (ms, summed over the recorded steps) and counters."""
    ms = np.zeros(5, np.float64)
    cnt = np.zeros(9, np.int64)
    _check(ctx, load().obem_stage_times(ctx, ms.ctypes.data, cnt.ctypes.data))
    return {"cell_ms": ms[0], "pairs_ms": ms[1], "step_ms": ms[2], "total_ms": ms[3], "near_ms": ms[4],
            "steps": int(cnt[0]), "launches": int(cnt[1]), "charge_pairs": int(cnt[2]),
            "cells_1pt": int(cnt[3]), "cells_3pt": int(cnt[4]), "cells_7pt": int(cnt[5]),
            "cells_closed": int(cnt[6]), "cell_points": int(cnt[7]), "cell_pairs_quad": int(cnt[8])}


# ---------------------------------------------------------------- device state
class DeviceState:
    """Charge arrays in device memory (torch tensors) in the layout of
    obem_state, plus the device scalars n and next_id."""

    def __init__(self, capacity, device="cuda"):
        import torch
        self.capacity = int(capacity)
        self.pos_q = torch.zeros((capacity, 4), dtype=torch.float32, device=device)
        self.vel = torch.zeros((capacity, 4), dtype=torch.float32, device=device)
        self.id = torch.zeros(capacity, dtype=torch.int32, device=device)
        self.birth = torch.zeros(capacity, dtype=torch.int32, device=device)
        self.species = torch.zeros(capacity, dtype=torch.uint8, device=device)
        self.scalars = torch.zeros(2, dtype=torch.int32, device=device)   # n, next_id

    def c_struct(self):
        return obem_state(pos_q=self.pos_q.data_ptr(), vel=self.vel.data_ptr(),
                          id=self.id.data_ptr(), birth=self.birth.data_ptr(),
                          species=self.species.data_ptr(), n=self.scalars.data_ptr(),
                          next_id=self.scalars.data_ptr() + 4, capacity=self.capacity)

    def upload(self, ch, next_id=None):
        import torch
        n = ch.pos_q.shape[0]
        if n > self.capacity:
            raise ValueError("state of %d charges exceeds capacity %d" % (n, self.capacity))
        self.pos_q[:n].copy_(torch.from_numpy(np.ascontiguousarray(ch.pos_q, np.float32)))
        self.vel[:n].copy_(torch.from_numpy(np.ascontiguousarray(ch.vel, np.float32)))
        self.id[:n].copy_(torch.from_numpy(np.ascontiguousarray(ch.id).view(np.int32)))
        self.birth[:n].copy_(torch.from_numpy(np.ascontiguousarray(ch.birth).view(np.int32)))
        self.species[:n].copy_(torch.from_numpy(np.ascontiguousarray(ch.species, np.uint8)))
        nid = n if next_id is None else int(next_id)
        self.scalars.copy_(torch.tensor([n, np.uint32(nid).view(np.int32)], dtype=torch.int32))

    def download(self):
        from types import SimpleNamespace
        sc = self.scalars.cpu().numpy()
        n = int(sc[0])
        return SimpleNamespace(
            pos_q=self.pos_q[:n].cpu().numpy(), vel=self.vel[:n].cpu().numpy(),
            id=self.id[:n].cpu().numpy().view(np.uint32), birth=self.birth[:n].cpu().numpy().view(np.uint32),
            species=self.species[:n].cpu().numpy(), n=n), int(sc[1].view(np.uint32))


def new_stats(device="cuda"):
    import torch
    return torch.zeros(STATS_BYTES, dtype=torch.uint8, device=device)


def read_stats(stats):
    raw = stats.cpu().numpy().tobytes()
    s = obem_step_stats.from_buffer_copy(raw)
    out = {f: getattr(s, f) for f, _ in obem_step_stats._fields_}
    for k in ("sum_e", "sum2_e", "sum_i", "sum2_i"):
        out[k] = list(out[k])
    return out


# ---------------------------------------------------------------- batch of chambers
class BatchState:
    """Concatenated charge arrays of a batch of chambers (torch CUDA tensors in
    the layout of obem_state): chamber c owns slots [seg_off[c], seg_off[c+1]);
    n and next_id are per-chamber device arrays."""

    def __init__(self, seg_off, device="cuda"):
        import torch
        self.seg_off = np.asarray(seg_off, np.int64)
        self.nb = len(self.seg_off) - 1
        S = int(self.seg_off[-1])
        self.capacity = S
        self.pos_q = torch.zeros((S, 4), dtype=torch.float32, device=device)
        self.vel = torch.zeros((S, 4), dtype=torch.float32, device=device)
        self.id = torch.zeros(S, dtype=torch.int32, device=device)
        self.birth = torch.zeros(S, dtype=torch.int32, device=device)
        self.species = torch.zeros(S, dtype=torch.uint8, device=device)
        self.n = torch.zeros(self.nb, dtype=torch.int32, device=device)
        self.next_id = torch.zeros(self.nb, dtype=torch.int32, device=device)

    def c_struct(self):
        return obem_state(pos_q=self.pos_q.data_ptr(), vel=self.vel.data_ptr(), id=self.id.data_ptr(),
                          birth=self.birth.data_ptr(), species=self.species.data_ptr(), n=self.n.data_ptr(),
                          next_id=self.next_id.data_ptr(), capacity=self.capacity)

    def host_arrays(self, chambers, next_ids=None):
        """Host copies of the arrays for a list of charge sets (one per chamber)."""
        S = self.capacity
        pos = np.zeros((S, 4), np.float32)
        vel = np.zeros((S, 4), np.float32)
        ids = np.zeros(S, np.uint32)
        birth = np.zeros(S, np.uint32)
        sp = np.zeros(S, np.uint8)
        n = np.zeros(self.nb, np.int32)
        nid = np.zeros(self.nb, np.uint32)
        for c, ch in enumerate(chambers):
            m = ch.pos_q.shape[0]
            o = int(self.seg_off[c])
            if m > self.seg_off[c + 1] - o:
                raise ValueError("chamber %d: %d charges exceed its segment" % (c, m))
            pos[o:o + m] = ch.pos_q
            vel[o:o + m] = ch.vel
            ids[o:o + m] = ch.id
            birth[o:o + m] = ch.birth
            sp[o:o + m] = ch.species
            n[c] = m
            nid[c] = m if next_ids is None else next_ids[c]
        return pos, vel, ids, birth, sp, n, nid

    def upload(self, chambers, next_ids=None):
        import torch
        pos, vel, ids, birth, sp, n, nid = self.host_arrays(chambers, next_ids)
        self.pos_q.copy_(torch.from_numpy(pos))
        self.vel.copy_(torch.from_numpy(vel))
        self.id.copy_(torch.from_numpy(ids.view(np.int32)))
        self.birth.copy_(torch.from_numpy(birth.view(np.int32)))
        self.species.copy_(torch.from_numpy(sp))
        self.n.copy_(torch.from_numpy(n))
        self.next_id.copy_(torch.from_numpy(nid.view(np.int32)))

    def download(self):
        """Per chamber: (charges, next_id)."""
        from types import SimpleNamespace
        n = self.n.cpu().numpy()
        nid = self.next_id.cpu().numpy().view(np.uint32)
        pos, vel = self.pos_q.cpu().numpy(), self.vel.cpu().numpy()
        ids, birth = self.id.cpu().numpy().view(np.uint32), self.birth.cpu().numpy().view(np.uint32)
        sp = self.species.cpu().numpy()
        out = []
        for c in range(self.nb):
            o, m = int(self.seg_off[c]), int(n[c])
            out.append((SimpleNamespace(pos_q=pos[o:o + m].copy(), vel=vel[o:o + m].copy(), id=ids[o:o + m].copy(),
                                        birth=birth[o:o + m].copy(), species=sp[o:o + m].copy(), n=m),
                        int(nid[c])))
        return out


def new_batch_stats(nb, device="cuda"):
    import torch
    return torch.zeros(nb * STATS_BYTES, dtype=torch.uint8, device=device)


def read_batch_stats(stats, nb):
    raw = stats.cpu().numpy().tobytes()
    out = []
    for c in range(nb):
        s = obem_step_stats.from_buffer_copy(raw[c * STATS_BYTES:(c + 1) * STATS_BYTES])
        d = {f: getattr(s, f) for f, _ in obem_step_stats._fields_}
        for k in ("sum_e", "sum2_e", "sum_i", "sum2_i"):
            d[k] = list(d[k])
        out.append(d)
    return out


class Batch:
    """obem_batch_* (include/obem.h): chambers stepped together, borrowing ctx
    (gas and step settings); per chamber capacity, planes and seed."""

    def __init__(self, ctx, capacity, z_lo, z_hi, seed):
        capacity = _host(capacity, np.int32)
        self.nb = len(capacity)
        self.ctx = ctx
        z_lo, z_hi = _host(z_lo, np.float64), _host(z_hi, np.float64)
        seed = _host(seed, np.uint64)
        h = C.c_void_p()
        _check(ctx, load().obem_batch_create(C.byref(h), ctx, self.nb, capacity.ctypes.data_as(C.c_void_p),
                                             z_lo.ctypes.data_as(C.c_void_p), z_hi.ctypes.data_as(C.c_void_p),
                                             seed.ctypes.data_as(C.c_void_p)))
        self.h = h
        off = np.zeros(self.nb + 1, np.int64)
        _check(ctx, load().obem_batch_layout(h, off.ctypes.data_as(C.c_void_p)))
        self.seg_off = off

    def destroy(self):
        if self.h:
            load().obem_batch_destroy(self.h)
            self.h = None

    def state(self, device="cuda"):
        return BatchState(self.seg_off, device)

    def cells(self, chamber, tri, sigma):
        tri = _host(tri, np.float64)
        sigma = _host(sigma, np.float32)
        _check(self.ctx, load().obem_batch_cells(self.h, int(chamber), int(tri.shape[0]),
                                                 tri.ctypes.data_as(C.c_void_p), sigma.ctypes.data_as(C.c_void_p)))

    def field_eval(self, st, E_out, stream=None):
        _check(self.ctx, load().obem_batch_field_eval(self.h, C.byref(st.c_struct()), _ptr(E_out), _stream(stream)))

    def step(self, st, step, stats, E_in=None, stream=None):
        """step: device uint32/int32 scalar tensor (advanced on commit)."""
        _check(self.ctx, load().obem_batch_step(self.h, C.byref(st.c_struct()), _ptr(E_in), _ptr(step), _ptr(stats),
                                                _stream(stream)))

    def step_graph(self, st, step, stats, stream=None):
        _check(self.ctx, load().obem_batch_step_graph(self.h, C.byref(st.c_struct()), _ptr(step), _ptr(stats),
                                                      _stream(stream)))

    def autotune(self, st, reps=3, stream=None):
        out = np.zeros(4, np.float64)
        _check(self.ctx, load().obem_batch_autotune(self.h, C.byref(st.c_struct()), int(reps),
                                                    out.ctypes.data_as(C.c_void_p), _stream(stream)))
        return {"cells_per_block": int(out[0]), "ms": float(out[1]), "ms_512": float(out[2])}

    def set_block(self, cells_per_block):
        _check(self.ctx, load().obem_batch_set_block(self.h, int(cells_per_block)))
