#!/usr/bin/env python
"""Throughput of the fused field + tracking step on the headline workload.

Workload: single-GEM patch meshed into 60,000 triangles (electrode and
dielectric cells), 1e6 charges (half electrons, half cations) in Gaussian
clouds on the hole axes, synthetic argon-like gas, dt = 1 ps, space charge and
recombination on.  One "step" = one obem_step: cell field + all-pairs Coulomb
field at every charge, recombination, flight with null-collision trials,
ionisation spawn, compaction, moments.

Prints one JSON line.  value: electron-steps/s with the state resident in HBM;
e2e: the same metric through the C ABI with the state copied from pinned host
buffers and back every step.  --impl reference times the CPU oracle instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "electron-steps/s & field pair-evals/s (1e6 charges, 60k panels), % FP32 peak"
UNIT = "electron-steps/s"
FLOPS_PER_PAIR = 18          # 3 sub, 3 fma (r^2), 3 mul, 3 fma (E): FFMA counted as 2
LANE_OPS_PER_PAIR = 7        # FP32-pipe lane operations per ordered pair in the symmetric
                             # kernel: 14 + 1 rsqrt per pair evaluated once for both charges
                             # when both tiles hold one charge value (every tile pair here but
                             # those with the sign-boundary or the padded last tile: 16 + 1)
FP32_LANES_PER_SM = 128
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "nbsym_kernel_dram_traffic.json")


def _file_sha256(path):
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def sym_items(n_charges, tile=1024):
    """Off-diagonal tile pairs of the symmetric all-pairs kernel (each
    writes one source-side partial of 12 B per charge of its tile)."""
    n = (n_charges + tile - 1) // tile
    h = n // 2
    return n * h - (n // 2 if n % 2 == 0 else 0)


def nbody_traffic_per_launch(n_charges):
    """DRAM bytes per launch of the all-pairs kernel from the committed ncu
    record, or None when the kernel source has changed since the counters were
    taken.  The record gives bytes per tile pair (the partial sums written,
    which dominate) and bytes per charge (positions, sources re-read from L2);
    a launch is scaled by both."""
    try:
        with open(TRAFFIC_RECORD) as f:
            rec = json.load(f)
        if kernel_source_sha256(rec["source"], rec["section_begin"], rec["section_end"]) != rec["source_sha256"]:
            return None
        return rec["dram_bytes_per_item"] * sym_items(n_charges) + rec["dram_bytes_per_charge"] * n_charges
    except (OSError, KeyError, ValueError):
        return None


def kernel_source_sha256(source, begin, end):
    """sha256 of the kernel's own source text: from the line holding `begin`
    up to (not including) the line holding `end`."""
    import hashlib
    with open(os.path.join(ROOT, source)) as f:
        text = f.read()
    i = text.index(begin)
    j = text.index(end, i)
    return hashlib.sha256(text[i:j].encode()).hexdigest()


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--charges", type=int, default=1_000_000)
    p.add_argument("--cells", type=int, default=60000)
    p.add_argument("--precision", default="bf16", choices=["fp32", "tf32", "bf16", "bf16x9"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-fieldmap", action="store_true")
    p.add_argument("--no-nn", action="store_true")
    p.add_argument("--no-dynamic", action="store_true")
    p.add_argument("--no-gradient", action="store_true")
    p.add_argument("--sharded", action="store_true",
                   help="split the headline charges among the ranks (target sharding with NCCL exchanges, "
                        "strong scaling) instead of one independent workload per rank")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-bem-precisions", action="store_true")
    p.add_argument("--no-avalanche", action="store_true")
    p.add_argument("--avalanche-only", action="store_true")
    p.add_argument("--double-gem", action="store_true",
                   help="also time the double-GEM gradient and charging-up workload (~120k cells)")
    p.add_argument("--double-gem-only", action="store_true")
    p.add_argument("--lu-dense", type=int, default=0,
                   help="only factorise and solve a synthetic dense system of this order (BF16 LU + refinement)")
    p.add_argument("--no-cell-groups", dest="cell_groups", action="store_false",
                   help="far cells by the per-cell tiers only (default: distant groups of 32 cells as "
                        "fitted equivalent charges, OBEM_STEP_CELL_GROUPS)")
    p.add_argument("--batch-chambers", type=int, default=256)
    p.add_argument("--batch-only", action="store_true")
    p.add_argument("--batch-skip-single", action="store_true",
                   help="batched sweep without the single-instance comparison (for profiling)")
    return p.parse_args()


def reduce_over_ranks(ms, counts, device):
    """Whole-job figures of N replicas: the slowest rank's timed region (max)
    and the work of all ranks (sum), over the initialised process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot = torch.tensor([float(c) for c in counts], dtype=torch.float64, device=device)
    dist.all_reduce(tot)
    return float(t.item()), [float(x) for x in tot.tolist()]


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(", ") for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (IndexError, ValueError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _workload(seed, n, cells):
    from paper_2110_09214_gb300 import inputs
    return inputs.config_gem(seed=seed, n=n, target_panels=cells)


def workload_name(mesh, ch):
    return ("single-GEM patch: %d cells (electrode + dielectric), %d charges (e-/cation), argon-like gas, "
            "dt 1 ps, space charge + recombination" % (mesh.n, ch.n))


def _synthetic_sigma(mesh):
    """A smooth density on the cells, used only by the CPU baseline's timing
    (its cost does not depend on the values)."""
    cen = mesh.tri.mean(axis=1)
    return 1e-6 * (1.0 + 0.3 * np.sin(cen[:, 0] / 1e-4)) * np.where(mesh.kind == 0, 1.0, 0.3)


def cpu_baseline(mesh, ch, gas, trk, seconds, rng_seed=0):
    """The oracle on the host cores, on a bounded sample of the workload:
    the FP64 field (all cells + all charges) at S sampled electrons and the
    binary32 step of those S electrons; electron-steps/s = S / time."""
    import oracle
    sig = _synthetic_sigma(mesh)
    rng = np.random.default_rng(rng_seed)
    el = np.flatnonzero(ch.species == 0)
    src = ch.pos_q.astype(np.float64)

    def run(S):
        idx = np.sort(rng.choice(el, S, replace=False))
        pts = ch.pos_q[idx, :3].astype(np.float64)
        t0 = time.perf_counter()
        E1, _ = oracle.panel_field(mesh.tri, sig, pts)
        E2, _ = oracle.nbody_field(pts, src, False, trk.softening)
        from types import SimpleNamespace
        sub = SimpleNamespace(pos_q=ch.pos_q[idx], vel=ch.vel[idx], id=ch.id[idx], birth=ch.birth[idx],
                              species=ch.species[idx])
        oracle.step(sub, (E1 + E2).astype(np.float32), 0, int(ch.id.max()) + 1, gas, trk, 4 * S + 64)
        return time.perf_counter() - t0

    # calibrate on growing samples: a few targets leave most host cores idle,
    # so the cost per electron is only linear once every core has work
    S, t = 8, run(8)
    for frac in (0.05, 1.0, 1.0):
        if frac == 1.0 and t >= 0.66 * seconds:
            break
        S = int(max(8, min(len(el), S * frac * seconds / max(t, 1e-3))))
        t = run(S)
    return {"value": S / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d sampled electrons: FP64 field from all %d cells and all %d charges, "
                      "plus their binary32 step (%.1f s)" % (S, mesh.n, ch.n, t)}


def run_reference(a, ws, rank):
    """--impl reference: the CPU oracle as it stands, same workload and metric."""
    if rank != 0:
        return
    from paper_2110_09214_gb300 import inputs  # noqa: F401
    mesh, gas, ch, trk, geo = _workload(1, a.charges, a.cells)
    trk.softening = 1e-9
    per = max(2.0, min(a.cpu_seconds, 150.0 / max(1, a.steps + a.warmup)))
    vals = []
    for i in range(a.warmup + a.steps):
        r = cpu_baseline(mesh, ch, gas, trk, per, rng_seed=i)
        if i >= a.warmup:
            vals.append(r["value"])
    v = float(np.mean(vals))
    n_e = int((ch.species == 0).sum())
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup,
            # one full step of the workload at the sampled rate (each timed step is a bounded sample)
            "ms_per_step": 1e3 * n_e / v if v > 0 else None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 field / f32 step",
            "data": "synthetic (seeded GEM mesh, charge clouds, argon-like cross sections)",
            "config": {"workload": workload_name(mesh, ch), "cells": mesh.n, "charges": ch.n},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(a, ws, rank, local):
    import torch
    from paper_2110_09214_gb300 import obem
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    prec = {"fp32": obem.OBEM_LU_FP32, "tf32": obem.OBEM_LU_TF32, "bf16": obem.OBEM_LU_BF16,
            "bf16x9": obem.OBEM_LU_BF16X9}[a.precision]
    mesh, gas, ch, trk, geo = _workload(1 + rank, a.charges, a.cells)
    trk.softening = 1e-9
    cap = int(ch.n * 1.6) + 1024
    ctx = obem.obem_create(capacity=cap, dt=trk.dt, seed=trk.seed, softening=trk.softening,
                           z_lo=trk.z_lo, z_hi=trk.z_hi, beta=trk.beta, trial_cap=256,
                           flags=obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD
                           | (obem.OBEM_STEP_CELL_GROUPS if a.cell_groups else 0))
    obem.obem_gas_load(ctx, gas)
    obem.obem_mesh_load(ctx, mesh)
    t0 = time.perf_counter()
    obem.obem_bem_assemble(ctx, prec)
    t_asm = time.perf_counter() - t0
    sigma = torch.empty(mesh.n, dtype=torch.float32, device=dev)
    rep = obem.obem_bem_solve(ctx, mesh.group_voltage, sigma)
    st = obem.DeviceState(cap)
    st.upload(ch)
    # The timed snapshot is the uploaded workload itself: every warm-up and
    # every timed step starts from it (restored by a device copy) with the
    # same step index, so each step does the same work and the workload does
    # not depend on --warmup.
    step_index = 0
    n_start = int((ch.species == 0).sum())
    snap = {k: getattr(st, k).clone() for k in ("pos_q", "vel", "id", "birth", "species", "scalars")}

    def restore():
        for key, v in snap.items():
            getattr(st, key).copy_(v, non_blocking=True)

    stats = [obem.new_stats() for _ in range(max(a.steps, a.warmup) + 1)]
    stats_c = obem.new_stats()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for k in range(a.warmup):
        restore()
        obem.obem_step(ctx, st, step_index, stats[k])
    torch.cuda.synchronize()
    for k in range(a.warmup):
        w = obem.read_stats(stats[k])
        assert w["status"] == 0, "warm-up step failed: %s" % w
    clocks = Clocks(local)
    obem.obem_profile(ctx, obem.OBEM_PROFILE_TIMES)      # stage events; uncounted kernels
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()          # a profiler started with --profile-from-start off sees these steps only
    ev0.record()
    for k in range(a.steps):
        flush.zero_()
        restore()
        obem.obem_step(ctx, st, step_index, stats[k])
    ev1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = obem.obem_stage_times(ctx)
    # evaluation counts: one more pass over the same snapshot (untimed), in
    # the counting kernels; every timed step did the same evaluations
    restore()
    obem.obem_profile(ctx, True)
    obem.obem_step(ctx, st, step_index, stats_c)
    cnt = obem.obem_stage_times(ctx)
    obem.obem_profile(ctx, False)
    for key in ("charge_pairs", "cells_1pt", "cells_3pt", "cells_7pt", "cells_closed", "cell_points",
                "cell_pairs_quad"):
        prof[key] = cnt[key] * a.steps
    sts = [obem.read_stats(stats[k]) for k in range(a.steps)]
    for s_ in sts:
        assert s_["status"] == 0, "timed step failed: %s" % s_
    e_counts = [n_start] * a.steps
    c_counts = [s_["n_before"] for s_ in sts]
    print("bench: steps %s" % [(s_["n_before"], s_["n_after"], s_["spawned_pairs"], s_["absorbed"],
                                s_["recombined_pairs"], s_["trials"]) for s_ in sts], file=sys.stderr)
    print("bench: profile %s" % prof, file=sys.stderr)
    electron_steps = float(sum(e_counts))
    pairs = prof["charge_pairs"]
    # field pair evaluations: ordered charge pairs + (target, cell) pairs, the
    # latter by quadrature or in the closed form
    cell_pairs = prof["cell_pairs_quad"] + prof["cells_closed"]
    charge_steps, pair_evals = float(sum(c_counts)), float(pairs + cell_pairs)
    if ws > 1:
        ms, (electron_steps, charge_steps, pair_evals) = reduce_over_ranks(
            ms, [electron_steps, charge_steps, pair_evals], dev)
    sec = ms / 1e3
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12          # TFLOP/s at max clock
    kern_s = prof["pairs_ms"] / 1e3
    achieved = FLOPS_PER_PAIR * pairs / kern_s / 1e12 if kern_s > 0 else 0.0
    peak_load = sms * FP32_LANES_PER_SM * 2 * (clk.get("sm_mhz") or sm_max) * 1e6 / 1e12
    # measured FP32 rate of this GPU right after the timed region (FFMA2 chains)
    alu = obem.obem_alu_rates(ctx)
    peak_meas = alu["fp32_tflops"]
    # the kernel's FP32-pipe rate against the measured ceiling of its own mix
    # (14 lane-ops per rsqrt), both per SM per clock at the clock under load
    mhz_load = clk.get("sm_mhz") or alu["sm_mhz"]
    lane_rate = LANE_OPS_PER_PAIR * pairs / kern_s / sms / (mhz_load * 1e6) if kern_s > 0 else 0.0
    traffic = nbody_traffic_per_launch(ch.n)
    # whole-step and cell-stage FP32 rates: 18 flops per ordered charge pair
    # and per (target, quadrature point) evaluation of the cell kernels (the
    # same pair formula); the FP64 closed form of targets within one cell size
    # is not counted in FP32 flops
    cell_s = prof["cell_ms"] / 1e3
    step_flops = FLOPS_PER_PAIR * (pairs + prof["cell_points"])
    step_rate = step_flops / sec / 1e12 if sec > 0 else 0.0
    cell_rate = FLOPS_PER_PAIR * prof["cell_points"] / cell_s / 1e12 if cell_s > 0 else 0.0
    # ---- end to end: state from pinned host memory and back, every step
    e2e = None
    if not a.no_e2e:
        for key, v in snap.items():
            getattr(st, key).copy_(v)
        e2e = run_e2e(ctx, st, a.steps, step_index, dev)
    dyn = None
    if ws == 1 and not a.no_dynamic:
        restore()
        n_now = int(st.download()[0].pos_q.shape[0])
        dyn = dynamic_resolve_timing(ctx, mesh, st.pos_q[:n_now], dev)
        obem.obem_bem_solve(ctx, mesh.group_voltage, sigma)         # back to the static sigma
    grad = None
    if ws == 1 and not a.no_gradient:
        restore()
        n_now = int(st.download()[0].pos_q.shape[0])
        grad = gradient_timing(ctx, mesh, geo, st.pos_q[:n_now], sigma, dev)
    nnres = None
    if ws == 1 and not a.no_nn:
        for key, v in snap.items():
            getattr(st, key).copy_(v)
        n_now = int(st.download()[0].pos_q.shape[0])
        nnres = nn_timing(ctx, st.pos_q[:n_now], dev, trk.softening)
    obem.obem_destroy(ctx)
    if rank != 0:
        return
    fmap = None
    if ws == 1 and not a.no_fieldmap:
        fmap = fieldmap_timing(dev)
    bres = None
    if ws == 1 and not a.no_batch:
        bres = batch_timing(dev, a.batch_chambers)
    bemp = None
    lu_gemm = None
    if ws == 1 and not a.no_bem_precisions:
        bemp = bem_precision_timing(mesh, dev)
        lu_gemm = lu_gemm_roofline(dev, mesh.n)
    aval = None
    if ws == 1 and not a.no_avalanche:
        aval = avalanche_timing(dev)
    dgem = None
    if ws == 1 and a.double_gem:
        dgem = double_gem_timing(dev, precision=a.precision)
    cpu = None
    if ws == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(mesh, ch, gas, trk, a.cpu_seconds)
    line = {
        "metric": METRIC, "value": electron_steps / sec, "unit": UNIT, "n_gpus": ws,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded GEM mesh, charge clouds, argon-like cross sections)",
        "config": {"workload": workload_name(mesh, ch),
                   "cells": mesh.n, "charges": ch.n, "l2": "flushed (256 MiB write) before every timed step",
                   "snapshot": "every warm-up and timed step starts from the generated workload (restored "
                               "by a device copy) with step index %d: identical work per step" % step_index,
                   "bem_precision": a.precision, "bem_assemble_factor_s": round(t_asm, 3),
                   "cell_groups": bool(a.cell_groups),
                   "bem_factor_ms": rep["factor_ms"], "bem_solve_ms": rep["solve_ms"],
                   "bem_ir_iterations": rep["iterations"], "bem_backward_error": rep["backward_error"]},
        "charge_steps_per_s": charge_steps / sec,
        "field_pair_evals_per_s": pair_evals / sec,
        "fp32_peak_frac": achieved / peak if peak else None,
        "fp32_peak_frac_at_load_clock": achieved / peak_load if peak_load else None,
        "stage_ms_per_step": {"cells": prof["cell_ms"] / a.steps, "cells_near": prof["near_ms"] / a.steps,
                              "pairs": prof["pairs_ms"] / a.steps,
                              "step": prof["step_ms"] / a.steps},
        "cell_evals_per_step": {"target_cell_pairs_quadrature": prof["cell_pairs_quad"] / a.steps,
                                "target_cell_pairs_closed_form": prof["cells_closed"] / a.steps,
                                "target_point_evals": prof["cell_points"] / a.steps,
                                "block_cell_pairs_by_tier": {"centroid": prof["cells_1pt"] / a.steps,
                                                             "3_to_6pt": prof["cells_3pt"] / a.steps,
                                                             "7pt_or_more": prof["cells_7pt"] / a.steps}},
        "roofline": {"bound": "alu", "kernel": "nbsym_kernel (symmetric all-pairs field)", "achieved": achieved,
                     "peak": peak_meas, "unit": "TFLOP/s", "frac": achieved / peak_meas if peak_meas else None,
                     "peak_source": "measured: packed f32x2 FMA chains on all %d SMs at %.0f MHz "
                                    "(obem_alu_rates, run after the timed region)" % (sms, alu["sm_mhz"]),
                     "peak_nominal": peak,
                     "frac_of_nominal": achieved / peak if peak else None,
                     "nominal_source": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (max SM clock)" % (sms, sm_max),
                     "flops_note": "achieved counts 18 flops per ordered pair (the method's N(N-1) pair "
                                   "evaluations); the symmetric kernel executes 7 FP32 lane-ops and half an "
                                   "rsqrt per ordered pair (k_C q factored out of tile pairs of one "
                                   "charge value)",
                     "mix_ceiling": {"kernel_lane_ops_per_sm_clk": lane_rate,
                                     "measured_mix14_lane_ops_per_sm_clk": alu["mix14_lane_ops_per_sm_clk"],
                                     "frac": lane_rate / alu["mix14_lane_ops_per_sm_clk"]
                                     if alu["mix14_lane_ops_per_sm_clk"] else None,
                                     "rsqrt_per_sm_clk": alu["rsqrt_per_sm_clk"]},
                     "step": {"achieved": step_rate, "frac": step_rate / peak_meas if peak_meas else None,
                              "unit": "TFLOP/s",
                              "note": "whole fused step (ms_per_step): 18 flops per ordered charge pair and per "
                                      "(target, quadrature point) of the cell kernels; FP64 closed form not "
                                      "counted"},
                     "cells": {"achieved": cell_rate, "frac": cell_rate / peak_meas if peak_meas else None,
                               "unit": "TFLOP/s", "note": "cell stage (binning, near and far kernels): 18 flops "
                                                          "per (target, quadrature point)"},
                     "traffic": traffic,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per target, "
                                       "scaled to %d targets (%s)" % (ch.n, os.path.relpath(TRAFFIC_RECORD, ROOT))
                                       if traffic is not None else "no ncu record for the current kernel source"},
        "clocks": clk,
        "gpu_launches": prof["launches"],
        "e2e": e2e,
        "cpu_baseline": cpu,
        "fieldmap": fmap,
        "batched_sweep": bres,
        "bem_precisions": bemp,
        "roofline_lu_gemm": lu_gemm,
        "nbody_nn": nnres,
        "dynamic_resolve": dyn,
        "gradient": grad,
        "avalanche_snapshots": aval,
        "double_gem": dgem,
    }
    print(json.dumps(line), flush=True)


def run_sharded(a, ws, rank, local):
    """--sharded: the headline workload split among the ranks in contiguous
    id ranges (target sharding: every step an all-gather of the charges, an
    all-reduce(MIN) of the recombination keys, the spawn-id scan and the
    rebalancing, over torch.distributed).  Every timed step starts from the
    same shards (restored by device copies), step index 0.  value: electron
    steps of the whole job per second (strong scaling: the total work is
    fixed)."""
    import torch
    import torch.distributed as dist
    from paper_2110_09214_gb300 import obem, shard
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not dist.is_initialized():
        dist.init_process_group("nccl", device_id=dev)
    prec = {"fp32": obem.OBEM_LU_FP32, "tf32": obem.OBEM_LU_TF32, "bf16": obem.OBEM_LU_BF16,
            "bf16x9": obem.OBEM_LU_BF16X9}[a.precision]
    mesh, gas, ch, trk, geo = _workload(1, a.charges, a.cells)
    trk.softening = 1e-9
    part = shard.split_charges(ch, ws)[rank]
    cap_g = int(ch.n * 1.6) + 1024                 # the gathered charges (spatial-hash scratch)
    cap = int(len(part.id) * 1.6) + 1024
    ctx = obem.obem_create(capacity=cap_g, dt=trk.dt, seed=trk.seed, softening=trk.softening, z_lo=trk.z_lo,
                           z_hi=trk.z_hi, beta=trk.beta, trial_cap=256,
                           flags=obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD)
    obem.obem_gas_load(ctx, gas)
    obem.obem_mesh_load(ctx, mesh)
    obem.obem_bem_assemble(ctx, prec)
    sigma = torch.empty(mesh.n, dtype=torch.float32, device=dev)
    obem.obem_bem_solve(ctx, mesh.group_voltage, sigma)
    st = obem.DeviceState(cap)
    st.upload(part, ch.n)
    sh = shard.Shard(ctx, st, obem.new_stats(), torch.zeros((cap, 4), dtype=torch.float32, device=dev))
    ex = shard.DistExchange()
    snap = {k: getattr(st, k).clone() for k in ("pos_q", "vel", "id", "birth", "species", "scalars")}

    def restore():
        for key, v in snap.items():
            getattr(st, key).copy_(v, non_blocking=True)

    n_e = int((ch.species == 0).sum())
    for _ in range(a.warmup):
        restore()
        status, _, _ = shard.sharded_step([sh], ex, 0, ch.n)
        assert status == obem.OBEM_OK, "warm-up step failed: %d" % status
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    clocks = Clocks(local)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(a.steps):
        flush.zero_()
        restore()
        status, _, _ = shard.sharded_step([sh], ex, 0, ch.n)
        assert status == obem.OBEM_OK
    ev1.record()
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    wall = (time.perf_counter() - t0) * 1e3
    ms, (tot,) = reduce_over_ranks(ms, [float(n_e) * a.steps / ws], dev)
    obem.obem_destroy(ctx)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": tot / (ms / 1e3), "unit": UNIT, "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded GEM mesh, charge clouds, argon-like "
                                                          "cross sections)",
            "config": {"workload": workload_name(mesh, ch), "cells": mesh.n, "charges": ch.n,
                       "parallelism": "target sharding over %d ranks (contiguous id ranges)" % ws,
                       "l2": "flushed (256 MiB write) before every timed step",
                       "snapshot": "every step restores the initial shards, step index 0",
                       "host_wall_ms_per_step_rank0": wall / a.steps},
            "clocks": clk}), flush=True)
    dist.destroy_process_group()


def nn_timing(ctx, pos_q, dev, soft, grids=(16, 32)):
    """The approximate N-body field (Sec. 3.2.4 "NN" option) on the headline
    charges: time per evaluation and accuracy against the exact all-pairs
    sum -- the share of charges whose field is within 5 % (the paper's
    criterion: 96.8 % of ~1e6 charges in its worst case)."""
    import torch
    from paper_2110_09214_gb300 import obem
    n = pos_q.shape[0]
    exact = torch.empty((n, 4), dtype=torch.float32, device=dev)
    obem.obem_field_eval(ctx, pos_q, exact, sources=pos_q, self_exclude=True)
    out = {}
    for G in grids:
        E = torch.empty((n, 4), dtype=torch.float32, device=dev)
        obem.obem_nbody_nn_eval(ctx, pos_q, E, G, 0.0)           # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        obem.obem_nbody_nn_eval(ctx, pos_q, E, G, 0.0)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rel = (torch.linalg.norm(E[:, :3] - exact[:, :3], dim=1) /
               torch.linalg.norm(exact[:, :3], dim=1).clamp_min(1e-30))
        bad_nn = int((~torch.isfinite(E[:, :3])).any(dim=1).sum())
        bad_ex = int((~torch.isfinite(exact[:, :3])).any(dim=1).sum())
        out["grid_%d" % G] = {"ms": ms, "within_5pct": float((rel < 0.05).float().mean()),
                              "median_rel_err": float(rel.nanmedian()),
                              "non_finite": {"nn": bad_nn, "exact": bad_ex}}
    out["charges"] = n
    out["exact_reference"] = "symmetric all-pairs field, no softening"
    return out


def batch_timing(dev, n_chambers=256, steps=3, swarm_steps=12, single=True):
    """The batched sweep: n_chambers independent parallel-plate chambers
    (gaps 0.5-3 mm, fields 0.1-30 kV/cm, 1e2-1e5 charges log-uniform, 1024-4096
    cells each, argon-like gas), every chamber's cell densities from its own
    GPU solve.  Times one step of every chamber (field + tracking) as the
    captured CUDA graph of the batched step, after the autotuner picked the
    cell block size, and the same work as the plain single-instance form (one
    context per chamber, obem_step one after the other) from the same states;
    both start every timed step from the same snapshot.  Swarm parameters per
    chamber (Eqs. (vd), (diffusion), (townsend)) from a short batched run."""
    import torch
    from paper_2110_09214_gb300 import inputs, obem, swarm
    chambers = inputs.config_batch(seed=1, n_chambers=n_chambers)
    gas = inputs.argon_like_gas()
    flags = obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD
    # Plummer length 0.1 um: with 1 nm the pairs that ionisations place ~1 nm
    # apart (Eq. (distIoni)) drive their electrons to keV energies in one 1 ps
    # step of step-start field, and the avalanches run away
    soft = 1e-7
    t0 = time.perf_counter()
    caps = [max(2 * c.charges.n, 1024) for c in chambers]
    ctxs, sts, sig = [], [], []
    for c, cap in zip(chambers, caps):
        ctx = obem.obem_create(capacity=cap, dt=c.trk.dt, seed=c.trk.seed, softening=soft, z_lo=c.trk.z_lo,
                               z_hi=c.trk.z_hi, beta=c.trk.beta, flags=flags)
        obem.obem_gas_load(ctx, gas)
        obem.obem_mesh_load(ctx, c.mesh)
        obem.obem_bem_assemble(ctx, obem.OBEM_LU_FP32)
        sg = torch.empty(c.mesh.n, dtype=torch.float32, device=dev)
        obem.obem_bem_solve(ctx, c.mesh.group_voltage, sg)
        st = obem.DeviceState(cap)
        st.upload(c.charges)
        ctxs.append(ctx)
        sts.append(st)
        sig.append(sg.cpu().numpy())
    t_setup = time.perf_counter() - t0
    bctx = obem.obem_create(capacity=16, dt=1e-12, softening=soft, beta=1e-13, flags=flags)
    obem.obem_gas_load(bctx, gas)
    b = obem.Batch(bctx, caps, [c.trk.z_lo for c in chambers], [c.trk.z_hi for c in chambers],
                   [c.trk.seed for c in chambers])
    out = {}
    try:
        for k, c in enumerate(chambers):
            b.cells(k, c.mesh.tri, sig[k])
        bst = b.state()
        bst.upload([c.charges for c in chambers])
        snap_b = {k: getattr(bst, k).clone() for k in ("pos_q", "vel", "id", "birth", "species", "n", "next_id")}
        snap_s = [{k: getattr(st, k).clone() for k in ("pos_q", "vel", "id", "birth", "species", "scalars")}
                  for st in sts]
        tune = b.autotune(bst, reps=2)
        step = torch.zeros(1, dtype=torch.int32, device=dev)
        stats = obem.new_batch_stats(n_chambers)
        sstats = [obem.new_stats() for _ in chambers]

        def restore_b():
            for k, v in snap_b.items():
                getattr(bst, k).copy_(v)
            step.zero_()

        def restore_s():
            for st, sn in zip(sts, snap_s):
                for k, v in sn.items():
                    getattr(st, k).copy_(v)

        def timed(fn, restore):
            tot = 0.0
            for r in range(steps + 1):                 # first round warms up (and captures)
                restore()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                if r:
                    tot += e0.elapsed_time(e1)
            return tot / steps

        ms_b = timed(lambda: b.step_graph(bst, step, stats), restore_b)
        gsb = obem.read_batch_stats(stats, n_chambers)
        assert all(g["status"] == 0 for g in gsb), "batched step failed"

        def one_by_one():
            for ctx, st, ss in zip(ctxs, sts, sstats):
                obem.obem_step(ctx, st, 0, ss)
        ms_s = None
        if single:
            ms_s = timed(one_by_one, restore_s)
            for ss in sstats:
                assert obem.read_stats(ss)["status"] == 0, "single-instance step failed"
        n = np.array([c.charges.n for c in chambers], np.float64)
        npan = np.array([c.mesh.n for c in chambers], np.float64)
        ne = np.array([int((c.charges.species == 0).sum()) for c in chambers], np.float64)
        pairs = float((n * (n - 1)).sum() + (n * npan).sum())
        # per-chamber swarm parameters from a short batched run
        restore_b()
        hist = [[] for _ in chambers]
        for _ in range(swarm_steps):
            b.step_graph(bst, step, stats)
            for k, g in enumerate(obem.read_batch_stats(stats, n_chambers)):
                hist[k].append(g)
        sw = [swarm.swarm_params(h, 1e-12) for h in hist]
        vd = np.array([x[0] for x in sw])
        out = {
            "chambers": n_chambers, "charges": int(n.sum()), "electrons": int(ne.sum()), "cells": int(npan.sum()),
            "charges_min_max": [int(n.min()), int(n.max())],
            "pair_evals_per_step": pairs,
            "batched_graph_ms_per_step": ms_b,
            "single_instance_ms_per_step": ms_s,
            "speedup_vs_single_instance": ms_s / ms_b if ms_b > 0 and ms_s else None,
            "electron_steps_per_s": float(ne.sum()) / (ms_b * 1e-3),
            "field_pair_evals_per_s": pairs / (ms_b * 1e-3),
            "autotune": tune,
            "setup_s": t_setup,
            "swarm": {"steps": swarm_steps, "drift_velocity_m_s_median": float(np.median(vd)),
                      "per_chamber_first4": [{"e_kv_cm": round(chambers[k].e_kv_cm, 3),
                                              "vd_m_s": sw[k][0], "dl_m2_s": sw[k][1], "alpha_1_m": sw[k][2]}
                                             for k in range(min(4, n_chambers))]},
            "note": "same chambers, same charges, same GPU; both forms compute the fused field (cells + "
                    "all-pairs, FP32) and the tracking step; the single-instance form runs one context per "
                    "chamber in sequence",
        }
    finally:
        b.destroy()
        obem.obem_destroy(bctx)
        for ctx in ctxs:
            obem.obem_destroy(ctx)
    return out


def measured_peaks():
    """Denominators of the rooflines: the machine's measured copy bandwidth and
    BF16 GEMM rate (MEASURED_PEAKS.json beside this file), else the profiling
    fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured (MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def lu_gemm_roofline(dev, n_cells):
    """The tensor-core kernel of the BF16 LU alone: the top-level trailing
    update of the recursive factorisation of the headline system (M = N = K =
    n/2), C -= A B through obem_tc_gemm (BF16 operands rounded from FP32,
    FP32 accumulation), best of 3 launches timed with CUDA events on the
    launching stream; 2 M N K flops against the measured BF16 burst rate."""
    import torch
    from paper_2110_09214_gb300 import obem
    h = n_cells // 2
    ctx = obem.obem_create(capacity=16, dt=1e-12)
    try:
        A = torch.randn(h, h, device=dev)
        B = torch.randn(h, h, device=dev)
        C = torch.randn(h, h, device=dev)
        obem.obem_tc_gemm(ctx, C, A, B)
        best = None
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            obem.obem_tc_gemm(ctx, C, A, B)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        del A, B, C
        torch.cuda.empty_cache()
    finally:
        obem.obem_destroy(ctx)
    pk = measured_peaks()
    tf = 2.0 * h ** 3 / (best * 1e-3) / 1e12
    return {"bound": "tensor", "kernel": "tc_gemm_kernel (tcgen05 BF16 GEMM, FP32 accumulation)",
            "shape": [h, h, h], "ms": best, "achieved": tf, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
            "frac": tf / pk["bf16_tflops"], "peak_source": pk["source"] + ", BF16 burst",
            "note": "time includes the BF16 rounding of both operands (two conversion kernels)"}


def gradient_timing(ctx, mesh, geo, pos_q, sigma, dev, n_probe=4096, reps=2):
    """The differentiable field on the headline workload: L = mean |E|^2 on a
    4096-point probe line along the central hole's axis (drift plane to
    anode); forward (cells + all charges at the probe) and backward (dL/dsigma
    for every cell, dL/d(position, charge) for every charge) through
    obem_field_eval / obem_field_eval_backward.  Best of reps, CUDA events."""
    import torch
    from paper_2110_09214_gb300 import obem
    c = geo.hole_centres()[0]
    z = np.linspace(geo.z_anode, geo.z_drift, n_probe + 2)[1:-1]
    tgt = torch.zeros((n_probe, 4), dtype=torch.float32, device=dev)
    tgt[:, 0], tgt[:, 1] = float(c[0]), float(c[1])
    tgt[:, 2] = torch.from_numpy(z.astype(np.float32)).to(dev)
    E = torch.empty((n_probe, 4), dtype=torch.float32, device=dev)
    dsig = torch.empty(mesh.n, dtype=torch.float32, device=dev)
    dsrc = torch.empty((pos_q.shape[0], 4), dtype=torch.float32, device=dev)

    def timed(fn):
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    fwd = timed(lambda: obem.obem_field_eval(ctx, tgt, E, sources=pos_q, sigma=sigma))
    g = torch.zeros_like(E)
    g[:, :3] = 2.0 * E[:, :3] / n_probe
    bwd = timed(lambda: obem.obem_field_eval_backward(ctx, tgt, g, sources=pos_q, sigma=sigma, dL_dsigma=dsig,
                                                      dL_dsources=dsrc))
    pairs = float(n_probe) * (mesh.n + pos_q.shape[0])
    return {"probe_points": n_probe, "forward_ms": fwd, "backward_ms": bwd,
            "backward_pairs_per_s": pairs / (bwd * 1e-3),
            "note": "backward: dL/dsigma of every cell and dL/d(position, charge) of every charge (the probe "
                    "points' own gradient not requested)",
            "finite": bool(torch.isfinite(dsig).all() and torch.isfinite(dsrc).all())}


def dynamic_resolve_timing(ctx, mesh, pos_q, dev, reps=2):
    """The paper's dynamic option (Sec. 3.2.2) at the headline size: the
    influence of every charge on every cell (obem_influence_rhs, Eqs.
    (potpart), (fldpart); the same cell-charge pairs as the field
    evaluation) and the re-solve of the cell charges with it (obem_bem_solve
    with drhs, refinement on the stored factors).  Best of reps, CUDA events."""
    import torch
    from paper_2110_09214_gb300 import obem
    drhs = torch.empty(mesh.n, dtype=torch.float32, device=dev)
    sig = torch.empty(mesh.n, dtype=torch.float32, device=dev)
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        obem.obem_influence_rhs(ctx, pos_q, drhs)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    rep = obem.obem_bem_solve(ctx, mesh.group_voltage, sig, drhs=drhs)
    pairs = float(mesh.n) * float(pos_q.shape[0])
    return {"influence_ms": best, "cell_charge_pairs": pairs, "pairs_per_s": pairs / (best * 1e-3),
            "resolve_ms": rep["solve_ms"], "resolve_ir_iterations": rep["iterations"],
            "resolve_backward_error": rep["backward_error"]}


def dense_lu_timing(n, dev, precision="bf16"):
    """The factorisation and refined solve alone (obem_dense_factor /
    obem_dense_solve) on a synthetic dense system of order n: uniform
    entries in [-1/2, 1/2] plus sqrt(n) on the diagonal, rows permuted at
    random so that partial pivoting swaps at almost every column (the BEM
    matrix's size without its assembly)."""
    import torch
    from paper_2110_09214_gb300 import obem
    prec = {"fp32": obem.OBEM_LU_FP32, "tf32": obem.OBEM_LU_TF32, "bf16": obem.OBEM_LU_BF16,
            "bf16x9": obem.OBEM_LU_BF16X9}[precision]
    g = torch.Generator(device=dev).manual_seed(1)
    A = torch.rand((n, n), device=dev, generator=g) - 0.5
    A += torch.diag(torch.full((n,), float(n) ** 0.5, device=dev))
    A = A[torch.randperm(n, device=dev, generator=g)].contiguous()
    ctx = obem.obem_create(capacity=16, dt=1e-12)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        obem.obem_dense_factor(ctx, A, prec)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        b = torch.rand(n, device=dev, dtype=torch.float64, generator=g)
        x = torch.empty_like(b)
        rep = obem.obem_dense_solve(ctx, b, x)
    finally:
        obem.obem_destroy(ctx)
    pk = measured_peaks()
    tf = 2.0 / 3.0 * float(n) ** 3 / (rep["factor_ms"] * 1e-3) / 1e12
    return {"n": n, "precision": precision, "factor_wall_s": wall, **rep,
            "factor_roofline": {"bound": "tensor", "achieved": tf, "peak": pk["bf16_tflops_sustained"],
                                "unit": "TFLOP/s", "frac": tf / pk["bf16_tflops_sustained"],
                                "peak_source": pk["source"] + ", BF16 sustained"}}


def bem_precision_timing(mesh, dev):
    """The dense BEM solve of the headline mesh (Eq. (matrixBEM), 59,968
    cells) with the LU's trailing updates in each arithmetic -- FP32 SIMT,
    TF32, BF16 and BF16x9 on the tensor cores -- each followed by iterative
    refinement with FP64 residuals: factorisation time, solve time,
    refinement iterations, backward error, and the largest difference of sigma
    from the FP32 solution (relative to max |sigma|)."""
    import torch
    from paper_2110_09214_gb300 import obem
    out, ref = {}, None
    for name, prec in (("fp32", obem.OBEM_LU_FP32), ("tf32", obem.OBEM_LU_TF32), ("bf16", obem.OBEM_LU_BF16),
                       ("bf16x9", obem.OBEM_LU_BF16X9)):
        ctx = obem.obem_create(capacity=16, dt=1e-12)
        try:
            obem.obem_mesh_load(ctx, mesh)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            obem.obem_bem_assemble(ctx, prec)
            torch.cuda.synchronize()
            t_af = time.perf_counter() - t0
            sig = torch.empty(mesh.n, dtype=torch.float32, device=dev)
            r = obem.obem_bem_solve(ctx, mesh.group_voltage, sig, check=False)
            sg = sig.double()
            if ref is None:
                ref = sg
            out[name] = {"assemble_factor_s": round(t_af, 3), "factor_ms": r["factor_ms"], "solve_ms": r["solve_ms"],
                         "ir_iterations": r["iterations"], "backward_error": r["backward_error"],
                         "status": r["status"], "rc": r["rc"],
                         "sigma_vs_fp32": float((sg - ref).abs().max() / ref.abs().max())}
        finally:
            obem.obem_destroy(ctx)
    out["cells"] = int(mesh.n)
    n = float(mesh.n)
    pk = measured_peaks()
    bf = out["bf16"]
    tf = 2.0 / 3.0 * n ** 3 / (bf["factor_ms"] * 1e-3) / 1e12
    out["bf16_factor_roofline"] = {"bound": "tensor", "flops": 2.0 / 3.0 * n ** 3, "achieved": tf,
                                   "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                                   "frac": tf / pk["bf16_tflops_sustained"],
                                   "peak_source": pk["source"] + ", BF16 sustained"}
    out["bf16_vs_fp32_total_speedup"] = ((out["fp32"]["factor_ms"] + out["fp32"]["solve_ms"]) /
                                         (bf["factor_ms"] + bf["solve_ms"]))
    out["note"] = ("bf16: recursive LU, every trailing update and off-diagonal TRSM block on this library's "
                   "tcgen05 GEMM (BF16 operands, FP32 accumulation); fp32 / tf32 / bf16x9: right-looking blocked "
                   "LU with the trailing updates through cuBLAS in the named arithmetic; pivoting panels, "
                   "triangular solves and the FP64 residuals of the refinement are this library's kernels in "
                   "every case")
    return out


def avalanche_timing(dev, sizes=(10_000, 100_000, 1_000_000), steps=5, warmup=3, e_kv_cm=10.0):
    """Fused-step throughput on the parallel-plate avalanche counter (2 mm gap,
    1 cm plates of 32 x 32 x 2 triangles: 4096 cells, argon-like gas, beta =
    1e-7 cm^3/s, 10 kV/cm) at fixed snapshot sizes: an avalanche-shaped cloud
    of n charges (half electrons, half cations).  After the warm-up steps every
    timed step restarts from the same state (device copy) after a 256 MiB L2
    flush, both inside the timed region."""
    import torch
    from paper_2110_09214_gb300 import inputs, obem
    mesh, gas, _, trk = inputs.config_avalanche(seed=1, e_kv_cm=e_kv_cm)
    trk.softening = 1e-9
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = {"cells": int(mesh.n), "field_kv_cm": e_kv_cm, "steps": steps, "warmup": warmup,
           "l2": "flushed (256 MiB write) before every timed step"}
    for n in sizes:
        ch = inputs.avalanche_snapshot(np.random.default_rng(100 + n), n, gap=trk.z_hi)
        cap = int(n * 1.6) + 1024
        ctx = obem.obem_create(capacity=cap, dt=trk.dt, seed=trk.seed, softening=trk.softening,
                               z_lo=trk.z_lo, z_hi=trk.z_hi, beta=trk.beta, trial_cap=256,
                               flags=obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD)
        try:
            obem.obem_gas_load(ctx, gas)
            obem.obem_mesh_load(ctx, mesh)
            obem.obem_bem_assemble(ctx, obem.OBEM_LU_FP32)
            sigma = torch.empty(mesh.n, dtype=torch.float32, device=dev)
            obem.obem_bem_solve(ctx, mesh.group_voltage, sigma)
            st = obem.DeviceState(cap)
            st.upload(ch)
            stats = [obem.new_stats() for _ in range(steps + 1)]
            for k in range(warmup):
                obem.obem_step(ctx, st, k, stats[steps])
            torch.cuda.synchronize()
            w = obem.read_stats(stats[steps])
            assert w["status"] == 0, "avalanche warm-up step failed: %s" % w
            snap = {k: getattr(st, k).clone() for k in ("pos_q", "vel", "id", "birth", "species", "scalars")}
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            obem.obem_profile(ctx, obem.OBEM_PROFILE_TIMES)      # stage events; uncounted kernels
            torch.cuda.synchronize()
            ev0.record()
            for k in range(steps):
                flush.zero_()
                for key, v in snap.items():
                    getattr(st, key).copy_(v, non_blocking=True)
                obem.obem_step(ctx, st, warmup + k, stats[k])
            ev1.record()
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / steps
            prof = obem.obem_stage_times(ctx)
            sts = [obem.read_stats(stats[k]) for k in range(steps)]
            for s_ in sts:
                assert s_["status"] == 0, "avalanche timed step failed: %s" % s_
        finally:
            obem.obem_destroy(ctx)
        nc = sts[0]["n_before"]
        ne = w["n_electron"]
        out["n_%d" % n] = {"charges": nc, "electrons": ne, "ms_per_step": ms,
                           "electron_steps_per_s": ne / (ms / 1e3),
                           "charge_steps_per_s": nc / (ms / 1e3),
                           "pair_evals_per_step": float(nc) * (nc - 1) + float(nc) * mesh.n,
                           "spawned_pairs_per_step": sts[0]["spawned_pairs"],
                           "stage_ms_per_step": {"cells": prof["cell_ms"] / steps,
                                                 "cells_near": prof["near_ms"] / steps,
                                                 "pairs": prof["pairs_ms"] / steps,
                                                 "step": prof["step_ms"] / steps},
                           "launches_per_step": prof["launches"] / steps}
    return out


def double_gem_timing(dev, steps=100, precision="bf16", n_charges=100_000, n_probe=4096):
    """The differentiable field and charging-up on the double-GEM stack (two
    single-GEM foils 2 mm apart, ~120k cells, 1e5 charges, a 4096-point probe
    line through the central hole's axis): BEM set-up in the given LU
    arithmetic; the gradient of L = mean |E|^2 on the probe line with respect
    to the cell densities, the charges (positions and q) and the six electrode
    voltages (adjoint solve); `steps` fused steps with surface hits, then the
    collected charge turned into free density and the system re-solved."""
    import torch
    from paper_2110_09214_gb300 import inputs, obem
    prec = {"fp32": obem.OBEM_LU_FP32, "tf32": obem.OBEM_LU_TF32, "bf16": obem.OBEM_LU_BF16,
            "bf16x9": obem.OBEM_LU_BF16X9}[precision]
    mesh, gas, ch, trk, d, probe = inputs.config_double_gem(seed=1, n=n_charges, n_probe=n_probe)
    # a 0.1 um Plummer length, as the swarm runs: with 1 nm, freshly ionised
    # pairs held in their mutual field for 1 ps run away and the avalanche in
    # the holes grows several-fold per step
    trk.softening = 1e-7
    cap = 40 * ch.n + 1024       # room for the avalanche in the holes' field over `steps` steps
    ng = len(mesh.group_voltage)
    ctx = obem.obem_create(capacity=cap, dt=trk.dt, seed=trk.seed, softening=trk.softening,
                           z_lo=trk.z_lo, z_hi=trk.z_hi, beta=trk.beta, trial_cap=256,
                           flags=obem.OBEM_STEP_SPACE_CHARGE | obem.OBEM_STEP_CELL_FIELD
                           | obem.OBEM_STEP_SURFACE_HITS)
    out = {"cells": int(mesh.n), "charges": int(ch.n), "probe_points": int(n_probe), "lu": precision,
           "softening_m": trk.softening,
           "geometry": "two single-GEM foils (19 holes each) 2 mm apart, drift 2 / transfer 3 / "
                       "induction 3 kV/cm, 400 V per foil"}

    def ev_ms(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    try:
        obem.obem_gas_load(ctx, gas)
        obem.obem_mesh_load(ctx, mesh)
        t0 = time.perf_counter()
        obem.obem_bem_assemble(ctx, prec)
        out["assemble_factor_s"] = time.perf_counter() - t0
        sigma = torch.empty(mesh.n, dtype=torch.float32, device=dev)
        rep = obem.obem_bem_solve(ctx, mesh.group_voltage, sigma)
        out["solve"] = {k: rep[k] for k in ("iterations", "backward_error", "factor_ms", "solve_ms")}
        # ---- gradient of the probe loss
        tgt = torch.zeros((n_probe, 4), dtype=torch.float32, device=dev)
        tgt[:, :3] = torch.from_numpy(probe.astype(np.float32)).to(dev)
        src = torch.from_numpy(ch.pos_q).to(dev)
        E = torch.empty((n_probe, 4), dtype=torch.float32, device=dev)
        obem.obem_field_eval(ctx, tgt, E, sources=src, sigma=sigma)          # warm-up
        fwd_ms, _ = ev_ms(lambda: obem.obem_field_eval(ctx, tgt, E, sources=src, sigma=sigma))
        gE = torch.zeros_like(E)
        gE[:, :3] = 2.0 * E[:, :3] / n_probe
        dsig = torch.empty(mesh.n, dtype=torch.float32, device=dev)
        dsrc = torch.empty((ch.n, 4), dtype=torch.float32, device=dev)
        obem.obem_field_eval_backward(ctx, tgt, gE, sources=src, sigma=sigma, dL_dsigma=dsig, dL_dsources=dsrc)
        bwd_ms, _ = ev_ms(lambda: obem.obem_field_eval_backward(ctx, tgt, gE, sources=src, sigma=sigma,
                                                                 dL_dsigma=dsig, dL_dsources=dsrc))
        adj_ms, (dV, arep) = ev_ms(lambda: obem.obem_bem_solve_adjoint(ctx, dsig, ng))
        loss = float((E[:, :3].double() ** 2).sum(dim=1).mean())
        out["gradient"] = {"loss_V2_per_m2": loss, "forward_ms": fwd_ms, "backward_ms": bwd_ms,
                           "adjoint_solve_ms": adj_ms, "adjoint_iterations": arep.iterations,
                           "dL_dV": [float(x) for x in dV],
                           "finite": bool(torch.isfinite(dsig).all() and torch.isfinite(dsrc).all()
                                          and np.all(np.isfinite(dV)))}
        # ---- charging-up: steps with surface hits, the collected charge as
        # free density on the dielectric cells, re-solve
        st = obem.DeviceState(cap)
        st.upload(ch)
        stats = [obem.new_stats(dev) for _ in range(steps)]
        obem.obem_surface_charge(ctx, mesh.n, reset=True)

        def run_steps():
            for k in range(steps):
                obem.obem_step(ctx, st, k, stats[k])

        step_ms, _ = ev_ms(run_steps)
        sts = [obem.read_stats(s) for s in stats]
        bad = [k for k, s_ in enumerate(sts) if s_["status"] != 0]
        sf = torch.zeros(mesh.n, dtype=torch.float32, device=dev)
        counts = obem.obem_surface_charge(ctx, mesh.n, sigma_free=sf)
        sig2 = torch.empty_like(sigma)
        res_ms, rep2 = ev_ms(lambda: obem.obem_bem_solve(ctx, mesh.group_voltage, sig2, sigma_free=sf))
        dd = mesh.kind == inputs.KIND_DIELECTRIC
        out["charging_up"] = {"steps": steps, "ms_per_step": step_ms / steps,
                              "first_failed_step": bad[0] if bad else None,
                              "status": sts[bad[0]]["status"] if bad else 0,
                              "charges_first_last": [sts[0]["n_before"], sts[-1]["n_after"]],
                              "collected_e": int(np.abs(counts).sum()),
                              "dielectric_cells_charged": int(((counts != 0) & dd).sum()),
                              "resolve_ms": res_ms, "resolve_iterations": rep2["iterations"],
                              "resolve_backward_error": rep2["backward_error"],
                              "sigma_change_rel": float((sig2 - sigma).abs().max() / sigma.abs().max())}
    finally:
        obem.obem_destroy(ctx)
    return out


def fieldmap_timing(dev, n_grid=256):
    """The static field map at the size of the paper's grid timings (Sec. 2.4:
    a 256^3 grid, two parallel plates of 8,192 cells in total): build time of
    obem_fieldmap_build.  Plates 1 cm x 1 cm, 1 cm apart, 64 x 32 x 2
    triangles each, sigma from the GPU solve; grid over the gap, 0.2 mm clear
    of the plates."""
    import torch
    from paper_2110_09214_gb300 import inputs, obem
    mesh = inputs.parallel_plates(1e-2, 1e-2, 64, 0.0, 1000.0, ny=32)
    ctx = obem.obem_create(capacity=16, dt=1e-12)
    try:
        obem.obem_mesh_load(ctx, mesh)
        obem.obem_bem_assemble(ctx, obem.OBEM_LU_FP32)
        sigma = torch.empty(mesh.n, dtype=torch.float32, device=dev)
        obem.obem_bem_solve(ctx, mesh.group_voltage, sigma)
        lo, hi, dims = [0.0, 0.0, 2e-4], [1e-2, 1e-2, 1e-2 - 2e-4], [n_grid] * 3
        obem.obem_fieldmap_build(ctx, lo, hi, [16, 16, 16], sigma)      # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        obem.obem_fieldmap_build(ctx, lo, hi, dims, sigma)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    finally:
        obem.obem_destroy(ctx)
    nodes = n_grid ** 3
    return {"grid": dims, "cells": int(mesh.n), "nodes": nodes, "seconds": t,
            "cell_pair_evals_per_s": nodes * mesh.n / t,
            "geometry": "two 1 cm plates 1 cm apart, 64x32x2 triangles each; grid over the gap",
            "paper_context": "Sec. 2.4 table: 256^3 grid, 8,192 cells, 37 s on one V100-era GPU "
                             "(their geometry and precision are not stated; context only)"}


def run_e2e(ctx, st, steps, step0, dev):
    """Same metric through obem_step with the state in pinned host buffers:
    H2D of the whole state before, D2H of the new state and the stats after.
    Every step starts from the same host state with the same step index, as
    the device-resident timing does."""
    import torch
    from paper_2110_09214_gb300 import obem
    cap = st.capacity
    n = int(st.scalars[0].item())
    host = {k: torch.empty_like(getattr(st, k), device="cpu").pin_memory()
            for k in ("pos_q", "vel", "id", "birth", "species")}
    hs = torch.empty(2, dtype=torch.int32).pin_memory()
    out = {k: torch.empty_like(getattr(st, k), device="cpu").pin_memory()
           for k in ("pos_q", "vel", "id", "birth", "species")}
    hstat = torch.empty(obem.STATS_BYTES, dtype=torch.uint8).pin_memory()
    for k in host:
        host[k][:n].copy_(getattr(st, k)[:n])
    hs.copy_(st.scalars)
    stats = obem.new_stats()
    torch.cuda.synchronize()
    h2d = d2h = 0
    e_steps = 0.0
    n_e = int((host["species"][:n] == 0).sum())
    t0 = time.perf_counter()
    step = step0
    for _ in range(steps):
        n = int(hs[0].item())
        for k in host:
            getattr(st, k)[:n].copy_(host[k][:n], non_blocking=True)
            h2d += host[k][:n].numel() * host[k].element_size()
        st.scalars.copy_(hs, non_blocking=True)
        h2d += 8
        obem.obem_step(ctx, st, step, stats)
        m_dev = st.scalars.to("cpu", non_blocking=False)
        m = int(m_dev[0])
        for k in out:
            out[k][:m].copy_(getattr(st, k)[:m], non_blocking=True)
            d2h += out[k][:m].numel() * out[k].element_size()
        hstat.copy_(stats, non_blocking=False)
        d2h += 8 + obem.STATS_BYTES
        torch.cuda.synchronize()
        s_ = obem.obem_step_stats.from_buffer_copy(hstat.numpy().tobytes())
        if s_.status != 0:
            raise RuntimeError("e2e step failed with status %d" % s_.status)
        e_steps += float(n_e)
    sec = time.perf_counter() - t0
    return {"value": e_steps / sec, "unit": UNIT, "h2d_bytes_per_step": h2d // steps,
            "d2h_bytes_per_step": d2h // steps}


def main():
    a = _args()
    ws, rank, local = _dist()
    if a.impl == "reference":
        run_reference(a, ws, rank)
    elif a.lu_dense > 0:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"dense_lu": dense_lu_timing(a.lu_dense, "cuda:%d" % local, a.precision)}))
    elif a.double_gem_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"double_gem": double_gem_timing("cuda:%d" % local, precision=a.precision)}))
    elif a.avalanche_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"avalanche_snapshots": avalanche_timing("cuda:%d" % local)}))
    elif a.batch_only:
        # the batched sweep alone (for profiling it): one JSON object
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"batched_sweep": batch_timing("cuda:%d" % local, a.batch_chambers,
                                                        single=not a.batch_skip_single)}))
    elif a.sharded:
        run_sharded(a, ws, rank, local)
    else:
        run_ours(a, ws, rank, local)


if __name__ == "__main__":
    main()
