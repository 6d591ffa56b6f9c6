#!/usr/bin/env python
"""Benchmark of the GB300 B-spline cloth hot path.

One timed step = one projected-Newton iteration (``bsc_newton_step``) of the
largest single-GPU workload, the 1024 x 1024 wrinkle field (1,048,576 control
points, 1,044,484 spans) in FP32 bulk precision: span evaluation (E, g, 27x27
H), FP64 SPD projection, gather assembly, PCG solve to 1e-8 and the
backtracking line search.  Reported:

  value         spans/s of the E + grad + Hessian (+ SPD projection) + assembly
                phase, from CUDA events recorded on the launching stream at the
                phase boundaries inside every timed step
  ms_per_step   Newton-step ms (whole iteration)
  e2e           the full step through the C ABI with host buffers (pinned H2D
                of C and Chat, D2H of C) in spans/s
  fp64          the same step with the plain FP64 GPU path (speedup context)
  roofline      the dominant kernel (the FP64 projection) against the FP64 pipe
  cpu_baseline  the FP64 CPU oracle on a bounded crop of the same state

``--workload batch64`` times the batched-garment workload instead: 64
independent patches (sides uniform in 16..192, per-patch materials and rest
rotations) stepped together - one launch per phase, the persistent PCG split
into per-patch block groups, the Newton iteration replayed from a CUDA graph,
tile shapes from the autotuner; ``--workload drape256`` the 256 x 256 drape.
The default line also carries short measurements of the drape under
``drape256``, of the batch under ``batched``, and under ``learned`` the
learned preconditioner on held-out 512 x 512 Newton systems (block-Jacobi
PCG vs flexible CG with the trained network: iterations and ms to 1e-8 per
solve, and ms per Newton step with each solver).

``--impl reference`` times the oracle itself (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2506_18867_gb300 import inputs  # noqa: E402

METRIC = "spans/s (E+grad+Hessian+assembly) and Newton-step ms"
# FP64 peak of a GB300 (no FP64 entry in the measured peaks): 152 SMs x 2 DFMA
# per clock x 2 flops x 2.07 GHz = 1.26 TFLOP/s, NVIDIA's nominal 1.25; a
# throughput microbenchmark of independent DFMA chains measured 1.0 TFLOP/s
FP64_PEAK_TFLOPS = 1.25
FP64_DFMA_MEASURED_TFLOPS = 1.0

WORKLOADS = {
    # name: (builder of the list of patches, description)
    "drape256": (lambda seed: [inputs.config_drape(seed, 256, 1e-5)],
                 "drape, 256x256 control points (65,536 cp, 64,516 spans), 2 m x 2 m, mu_bd = 1e-5 N m, "
                 "sigma = 1 mm noise, u = 0 edge pinned, dt = 0.01 s"),
    "square32": (lambda seed: [inputs.config_square(seed, 32)],
                 "square, 32x32 control points (900 spans), 1 m x 1 m, two top corners pinned"),
    "wrinkle512": (lambda seed: [inputs.config_wrinkle(seed, 512, 2.0)],
                   "the wrinkle field on 512x512 control points (261,121 spans), 2 m x 2 m, same span length "
                   "and material as wrinkle1024: the size the profiles are captured at"),
    "wrinkle1024": (lambda seed: [inputs.config_wrinkle(seed, 1024)],
                    "precision-sweep patch, 1024x1024 control points (1,048,576 cp, 1,044,484 spans), 4 m x 4 m, "
                    "seeded multi-frequency wrinkle field (8 sinusoids, wavelengths 4-64 spans, amplitudes 1-5 mm), "
                    "E = 1e5 Pa, nu = 0.3, h = 1 mm, 200 kg/m^2, two top corners pinned, gravity -z, "
                    "dt = 0.01 s"),
    "batch64": (lambda seed: inputs.config_batch(seed, 64),
                "batched garments: 64 independent patches, nu and nv uniform in [16, 192], E log-uniform in "
                "[1e4, 1e6] Pa, Poisson ratio uniform in [0.2, 0.45], random rest rotations, 1 cm spans, "
                "sigma = 1 mm noise, two top corners pinned, dt = 0.01 s; one graph-replayed Newton iteration "
                "over all patches"),
}

def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="bsc", choices=["bsc", "reference"])
    p.add_argument("--workload", default="wrinkle1024", choices=sorted(WORKLOADS))
    p.add_argument("--tuning-out", default=None,
                   help="write the autotuner's choices for the main workload to this JSON file")
    p.add_argument("--tuning-in", default=None,
                   help="apply these autotuner choices (from --tuning-out) instead of autotuning the main workload: "
                        "a run under a profiler, whose timings differ, then launches the same kernels")
    p.add_argument("--k-layout", default="symmetric", choices=("symmetric", "full"),
                   help="layout of the Newton step's matrix (bsc_set_k_storage; symmetric is the library default)")
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-batch", action="store_true", help="skip the batched-garment sub-measurement")
    p.add_argument("--no-drape", action="store_true", help="skip the 256x256 drape sub-measurement")
    p.add_argument("--no-contact", action="store_true", help="skip the drape-on-a-sphere contact sub-measurement")
    p.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner sub-measurement")
    p.add_argument("--no-point", action="store_true", help="skip the per-point projection sub-measurement")
    p.add_argument("--no-sweep", action="store_true", help="skip the 1024x1024 precision sweep sub-measurement")
    p.add_argument("--no-trajectory", action="store_true",
                   help="skip the 20-time-step drape trajectories (mu_bd sweep, FP32 vs FP64)")
    return p.parse_args()


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.lines, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- flop model

def ldlt_flops(n):
    """The FP64 PSD test of a reduced Hessian of size n: the infinity norm
    (n^2 absolute values summed), the shift, and the right-looking LDL^T with
    one reciprocal, n - k - 1 multipliers and (n - k - 1)(n - k) / 2 FMAs
    (2 flops each) per pivot k."""
    f = n * n + n
    for k in range(n):
        m = n - k - 1
        f += 1 + m + m * (m + 1)
    return f


def projection_flops(nred, nneg, nm, nb, psd=False, open_frac=1.0, border_psd=False, border_open_frac=1.0):
    """Algorithmic FP64 flops of the SPD projection of one span per Newton
    iteration as implemented: reduced Hessian formation from the reduced
    derivative vectors (the span's orthonormal basis and the vectors in it
    depend on the rest geometry only and are computed once per context, so
    they are not counted), Householder tridiagonalisation (4/3 n^3), the
    inertia count, and per negative eigenvalue: the FP64 check of its FP32
    bracket and the regula-falsi refinement (5 characteristic-polynomial
    evaluations of 4 n flops on average), the pivoted LU and two solves of
    the shifted tridiagonal, the Rayleigh quotient, the back-transformation
    (2 n^2), the mapping to span DOFs and the rank-one update of the 378
    packed entries (FP32 bracketing and FP32 updates are not counted).
    With the PSD test (interior spans, psd=True) a span pays the formation
    and the LDL^T test in FP64 with probability open_frac (the share of the
    interior spans the FP32 certificate leaves open; 1 without it - the
    certificate's own work is FP32 and not counted), and only the spans with
    a projected eigenvalue go on to the formation again and the
    eigendecomposition.  Border spans (n = 24) pay the FP64 test when it
    is on (border_psd: every border path tests first) with probability
    border_open_frac (the share the warp paths' FP32 certificate leaves
    open; 1 without it)."""
    n = nred
    D = n // 3
    form = nm * 2 * (36 * D + 9 * D * (D + 1)) + nb * (2 * D * (D + 1))  # T_k and blocks per point
    f = 0.0
    if psd and n == 15:
        f += open_frac * (form + ldlt_flops(n))
        if not nneg:
            return f
    if border_psd and n == 24:
        f += border_open_frac * (form + ldlt_flops(n))
        if not nneg:
            return f
    f += form
    f += 4.0 * n ** 3 / 3.0 + 4 * n                    # tridiagonalisation, scaling
    f += 4 * n                                         # inertia count at -tau
    if nneg:
        f += nneg * (5 * 4 * n + 10 * n + 2 * 8 * n + 6 * n + 2 * n * n + 54 * D)
    return f


# --------------------------------------------------------------------------- GPU arm

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(dist, times_ms, spans, device):
    """Across ranks (replicas, or the patches of one batch split over them):
    every rank steps its own patches, so the job's time is the slowest rank's
    (max of every time) and its work the sum of the ranks' spans.  No
    data-path collective: only these scalars."""
    import torch
    out = dict(times_ms)
    out["spans"] = spans
    if dist is None:
        return out
    keys = sorted(times_ms)
    t = torch.tensor([float(times_ms[k]) for k in keys], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(spans)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    for k, v in zip(keys, t.tolist()):
        out[k] = v
    out["spans"] = int(n.item())
    return out


def make_context(bsc, pats, prec):
    if len(pats) == 1:
        return bsc.context_for_patch(pats[0], precision=prec, pcg_rel_tol=1e-8)
    return bsc.batch_for_patches(pats, precision=prec, pcg_rel_tol=1e-8)


def stacked(ctx, arrays, torch, np):
    """Per-patch (N_p, 3) arrays -> the context's (3, N) layout (host, float64)."""
    out = np.zeros((3, ctx.N))
    for p, a in enumerate(arrays):
        out[:, ctx.cp_offset[p]:ctx.cp_offset[p + 1]] = np.asarray(a).T
    return torch.from_numpy(out)


def apply_tuning(ctx, t):
    """The autotuner's choices (bsc_tuning as a dict) set through the C ABI."""
    ctx.set_tiles([max(int(v), 0) for v in t["tile_tu"]])
    ctx.set_border_path(int(t["border_path"]))
    ctx.set_p2_variant(int(t["p2_variant"]))
    ctx.set_psd_test(int(t["psd_test"]))
    ctx.set_pcg_grid(int(t["pcg_grid"]))
    ctx.set_pcg_form(int(t["pcg_form"]))


def time_newton(ctx, C, C0, Chat, steps, warmup, flush, stream, torch):
    """Newton steps from the same state; per step the L2 flush and the reset
    of C run outside the CUDA events.  Returns (step ms list, summed phase
    ms, reports, launches)."""
    from paper_2506_18867_gb300 import bsc
    for _ in range(warmup):
        C.copy_(C0)
        ctx.newton_step(C, Chat)
    torch.cuda.synchronize()
    phases = {k: 0.0 for k in bsc.Context.PHASES}
    step_ms, reports = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launch_count()
    for _ in range(steps):
        flush.zero_()
        C.copy_(C0)
        ev0.record(stream)
        rep = ctx.newton_step(C, Chat)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        for k, v in ctx.phase_times().items():
            phases[k] += v
        reports.append(rep.as_dict())
    return step_ms, phases, reports, ctx.launch_count() - launches0


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2506_18867_gb300 import bsc
    from paper_2506_18867_gb300 import build as _build

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    bsc.load()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    builder, desc = WORKLOADS[args.workload]
    partitioned = args.workload == "batch64" and world > 1
    if partitioned:
        # one batch of garments split over the ranks (no exchange): strong scaling
        from paper_2506_18867_gb300 import partition
        _, pats = partition.rank_patches(builder(1), rank, world)
    else:
        pats = builder(1 + rank)
    prec = bsc.FP32 if args.precision == "fp32" else bsc.FP64
    ctx = make_context(bsc, pats, prec)
    ctx.set_profiling(True)
    ctx.set_k_storage(args.k_layout == "symmetric")
    Nsp, Ncp = ctx.n_spans, ctx.N
    C0 = stacked(ctx, [p.C for p in pats], torch, np).to(device="cuda", dtype=ctx.dtype)
    Chat = stacked(ctx, [p.Chat for p in pats], torch, np).to(device="cuda", dtype=ctx.dtype)
    C = C0.clone()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    if args.tuning_in:
        with open(args.tuning_in) as fh:
            tuning = json.load(fh)
        apply_tuning(ctx, tuning)
    else:
        tuning = ctx.autotune(C0, Chat)
    if args.tuning_out and rank == 0:
        with open(args.tuning_out, "w") as fh:
            json.dump(tuning, fh)

    barrier()
    clocks = ClockSampler(local).start()
    barrier()
    t_wall = time.perf_counter()
    step_ms, phases, reports, launches = time_newton(ctx, C, C0, Chat, args.steps, args.warmup, flush, stream,
                                                     torch)
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()

    K = args.steps
    ms_step = sum(step_ms) / K
    eval_ms = (phases["span_eval"] + phases["project"] + phases["assemble"]) / K
    proj_ms = phases["project"] / K
    # the projection flops of the last step (the workload is identical every step)
    nneg, nred = ctx.projection_stats()
    nm = np.bincount(ctx.quadrature_tables(0)[:, 24].astype(np.int64), minlength=Nsp)
    nb = np.bincount(ctx.quadrature_tables(1)[:, 24].astype(np.int64), minlength=Nsp)
    flops = 0.0
    psd = bool(tuning.get("psd_test"))
    psd_counts = ctx.psd_counts()   # interior spans, FP64-tested, eigendecomposed
    open_frac = psd_counts[1] / max(psd_counts[0], 1)
    border_open_frac = psd_counts[5] / max(psd_counts[3], 1)
    for s_ in range(Nsp):
        flops += projection_flops(int(nred[s_]), int(nneg[s_]), int(nm[s_]), int(nb[s_]), psd, open_frac,
                                  psd, border_open_frac)
    achieved_tflops = flops / (proj_ms * 1e-3) / 1e12

    # e2e: the same Newton step through the C ABI from pinned host buffers
    host_C = C0.cpu().pin_memory()
    host_Chat = Chat.cpu().pin_memory()
    host_out = torch.empty_like(host_C).pin_memory()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = []
    for i in range(args.warmup + K):
        flush.zero_()
        ev0.record(stream)
        C.copy_(host_C, non_blocking=True)
        Chat.copy_(host_Chat, non_blocking=True)
        ctx.newton_step(C, Chat)
        host_out.copy_(C, non_blocking=True)
        ev1.record(stream)
        ev1.synchronize()
        if i >= args.warmup:
            e2e_ms.append(ev0.elapsed_time(ev1))
    e2e_step = sum(e2e_ms) / len(e2e_ms)
    tsz = 4 if prec == bsc.FP32 else 8

    agg = reduce_over_ranks(dist, {"eval": eval_ms, "step": ms_step, "e2e": e2e_step}, Nsp, "cuda")
    eval_ms_max, ms_step_max, e2e_max = agg["eval"], agg["step"], agg["e2e"]
    total_spans = agg["spans"]
    value = total_spans / (eval_ms_max * 1e-3)

    # The sub-measurements below run in single-GPU runs only: a multi-GPU run
    # times the replicated step and holds its GPUs no longer than that.
    fp64 = None
    if not args.no_fp64 and prec == bsc.FP32 and world == 1:
        ctx64 = make_context(bsc, pats, bsc.FP64)
        ctx64.set_profiling(True)
        C64_0 = C0.double()
        Chat64 = Chat.double()
        C64 = C64_0.clone()
        K64 = max(2, K // 3)
        ms64, ph64, reps64, _ = time_newton(ctx64, C64, C64_0, Chat64, K64, 2, flush, stream, torch)
        e64 = (ph64["span_eval"] + ph64["project"] + ph64["assemble"]) / K64
        fp64 = {"newton_step_ms": sum(ms64) / K64, "eval_assembly_ms": e64,
                "spans_per_s": Nsp / (e64 * 1e-3), "steps": K64,
                "newton_step_speedup_fp32_vs_fp64": (sum(ms64) / K64) / ms_step,
                "phases_ms": {k: v / K64 for k, v in ph64.items()}, "pcg_iters": reps64[-1]["pcg_iters"]}
        ctx64.close()
        del C64, C64_0, Chat64

    drape = None
    if args.workload != "drape256" and not args.no_drape and prec == bsc.FP32 and world == 1:
        drape = measure_drape(bsc, flush, stream, torch, np, K, args.warmup)
    contact = None
    if args.workload != "batch64" and not args.no_contact and prec == bsc.FP32 and world == 1:
        contact = measure_contact(bsc, flush, stream, torch, np)
    batched = None
    if args.workload != "batch64" and not args.no_batch and prec == bsc.FP32 and world == 1:
        batched = measure_batch(bsc, flush, stream, torch, np, seed=1 + rank)
    learned = None
    if args.workload != "batch64" and not args.no_learned and prec == bsc.FP32 and world == 1:
        learned = measure_learned(bsc, np, torch, flush)
    sweep = None
    if args.workload != "batch64" and not args.no_sweep and world == 1:
        sweep = measure_sweep(bsc, torch)
    trajectory = None
    if args.workload != "batch64" and not args.no_trajectory and world == 1:
        trajectory = measure_trajectories(bsc, torch)
    point = None
    if len(pats) == 1 and not args.no_point and world == 1:
        point = measure_point_projection(bsc, pats[0], prec, ctx, C0, Chat, K, args.warmup, ms_step, flush, stream,
                                         torch)

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline(args, pats)

    if rank == 0:
        rep = reports[-1]
        cfg = {"workload": f"{args.workload}_{args.precision}", "description": desc,
               "patches": len(pats), "spans": Nsp, "control_points": Ncp,
               "precision": ("FP32 span evaluation, assembly, SpMV and PCG vectors; FP64 SPD projection, "
                             "energy sums and norms") if prec == bsc.FP32 else "FP64 throughout",
               "pcg_rel_tol": 1e-8, "l2": "flushed (256 MB write) before every timed step",
               "step": "one projected-Newton iteration (bsc_newton_step, CUDA-graph replay) from the same "
                       "seeded state",
               "ranks": ("the 64 patches of one batch split over the ranks by the longest-processing-time "
                         "rule on span counts, no exchange" if partitioned else
                         "one independent workload per GPU (seed 1 + rank)")}
        if len(pats) == 1:
            cfg.update(nu=pats[0].nu, nv=pats[0].nv)
        # the linear solve: the persistent PCG streams K once per iteration
        # (HBM-bound at this size); algorithmic bytes per iteration and
        # control point: the stencil K as the Newton step stores it (13
        # blocks of the symmetric layout = 117 entries, the default; 225 in
        # the full one) plus the SpMV's x and y and five vector passes (11
        # vectors of 3 components), in T
        pcg_ms = phases["solve"] / K
        iters = sum(r["pcg_iters"] for r in reports) / len(reports)
        k_sym = args.k_layout == "symmetric"
        k_entries = 117 if k_sym else 225
        pcg_bytes = iters * Ncp * tsz * (k_entries + 6 + 15)
        hbm, hbm_src = hbm_peak_gbs()
        pcg_gbs = pcg_bytes / (pcg_ms * 1e-3) / 1e9
        roof_pcg = {"kernel": "persistent block-Jacobi PCG (k_pcg or k_pcg_pipe)", "bound": "hbm",
                    "achieved": pcg_gbs, "peak": hbm, "unit": "GB/s", "frac": pcg_gbs / hbm,
                    "traffic": pcg_traffic(args.workload, prec == bsc.FP32, tuning, iters, k_sym),
                    "algorithmic_bytes_per_launch": pcg_bytes, "iterations": iters,
                    "bytes_per_cp_per_iteration": tsz * (k_entries + 6 + 15),
                    "k_layout": "symmetric (13 blocks)" if k_sym else "full (25 blocks)", "launch_ms": pcg_ms,
                    "launch_ms_source": "solve phase of bsc_phase_times (rhs, block-Jacobi inverses and the PCG "
                                        "launch, CUDA events on the launching stream)",
                    "peak_source": hbm_src,
                    "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of one k_pcg launch (three-pass "
                                      "form, symmetric layout) of the 512x512 wrinkle field "
                                      "(profiles/k_pcg_wrinkle512_fp32.md), scaled by control points x iterations "
                                      "to this launch (a lower bound above 512x512: the vectors leave L2); null "
                                      "for another form or layout, or once the kernel changed"}
        roof_proj = {"kernel": "SPD projection (k_proj_pf: FP32 certificate; k_proj_p0, k_proj_p1, k_proj_p2, "
                               "k_proj_corr, k_project_ring: FP64)",
                     "psd_counts": {"interior_spans": psd_counts[0], "fp64_tested": psd_counts[1],
                                    "eigendecomposed": psd_counts[2], "border_spans": psd_counts[3],
                                    "border_eigendecomposed": psd_counts[4], "border_fp64_tested": psd_counts[5],
                                    "mode": tuning.get("psd_test")},
                     "bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved_tflops / FP64_PEAK_TFLOPS,
                     "traffic": projection_traffic(args.workload, prec == bsc.FP32, tuning),
                     "algorithmic_flops_per_step": flops, "launch_ms": proj_ms,
                     "peak_source": "GB300 FP64 from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flops x "
                                    "2.07 GHz = 1.26 TFLOP/s (nominal 1.25); no FP64 entry in the measured peaks",
                     "frac_of_dfma_microbenchmark": achieved_tflops / FP64_DFMA_MEASURED_TFLOPS,
                     "arithmetic": ("PSD test and phase 1 of the thread-per-span kernels in double-float (pairs of "
                                    "FP32) on the FP32 pipe, the eigenpair phase and the border warps' test in "
                                    "FP64; the algorithmic FP64 flops of all of it are counted against the FP64 "
                                    "peak") if prec == bsc.FP32 else "FP64 throughout",
                     "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of the projection launches "
                                       "of one step (ncu capture summarised in profiles/), null when no capture "
                                       "of the current kernels exists for this workload",
                     "executed": projection_executed(args.workload, prec == bsc.FP32, tuning, proj_ms,
                                             clk.get("sm_mhz") or 2070.0,
                                             torch.cuda.get_device_properties(local).multi_processor_count)}
        roof_main = roof_pcg if pcg_ms >= proj_ms else roof_proj
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "spans/s",
            "n_gpus": world,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": ms_step_max,
            "higher_is_better": True,
            "scaling": "strong" if partitioned else "weak",
            "vs_baseline": None,
            "dtype": "f32" if prec == bsc.FP32 else "f64",
            "data": "synthetic",
            "config": cfg,
            "newton_step_ms": ms_step_max,
            "newton_spans_per_s": total_spans / (ms_step_max * 1e-3),
            "eval_assembly_ms": eval_ms_max,
            "phases_ms": {k: v / K for k, v in phases.items()},
            "wall_ms_per_step": wall * 1e3 / (K + args.warmup),
            "newton": {"pcg_iters": rep["pcg_iters"], "pcg_rel_res": rep["pcg_rel_res"], "alpha": rep["alpha"],
                       "ls_halvings": rep["ls_halvings"], "spans_projected": rep["spans_projected"],
                       "dir_inf_over_dt": rep["dir_inf"] / pats[0].dt, "E0": rep["E0"], "E1": rep["E1"]},
            "autotune": tuning,
            "e2e": {"value": total_spans / (e2e_max * 1e-3), "unit": "spans/s",
                    "scope": "bsc_newton_step with host buffers: pinned H2D of C and Chat, D2H of C, per step",
                    "ms_per_step": e2e_max, "h2d_bytes_per_step": 2 * 3 * Ncp * tsz,
                    "d2h_bytes_per_step": 3 * Ncp * tsz},
            "gpu_launches": int(launches),
            "gpu_launches_per_step": launches / K,
            "roofline": roof_main,
            "rooflines": {"pcg": roof_pcg, "projection": roof_proj},
            "fp64": fp64,
            "drape256": drape,
            "contact": contact,
            "batched": batched,
            "learned": learned,
            "point_projection": point,
            "precision_sweep": sweep,
            "trajectories": trajectory,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def hbm_peak_gbs():
    """The measured copy bandwidth of the GB300s, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measure_sweep(bsc, torch, n=1024, spmvs=50):
    """The 1024 x 1024 wrinkle field (1,044,484 spans) in FP32 and FP64: energy,
    gradient and the projected Hessian (span evaluation + FP64 projection +
    assembly), one call each after a warm-up call, then 50 SpMVs with that K.
    K (225 entries per control point) is far larger than L2, so every product
    streams it from HBM; the algorithmic bytes of one product are K + x + y."""
    pat = inputs.config_wrinkle(1, n)
    peak, src = hbm_peak_gbs()
    out = {"workload": f"wrinkle{n}", "spans": (n - 2) * (n - 2), "control_points": n * n, "spmvs": spmvs}
    for prec, name in ((bsc.FP32, "fp32"), (bsc.FP64, "fp64")):
        ctx = bsc.context_for_patch(pat, precision=prec, pcg_rel_tol=1e-8)
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        ctx.energy(C, Ch)
        ctx.gradient(C, Ch)
        K = ctx.assemble_hessian(C, project=True)
        x = torch.randn((3, ctx.N), dtype=ctx.dtype, device="cuda", generator=torch.Generator("cuda").manual_seed(9))
        y = ctx.new_vec()
        ctx.spmv(x, K=K, out=y)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record()
        ctx.energy(C, Ch)
        ev[1].record()
        ctx.gradient(C, Ch, out=y)
        ev[2].record()
        ctx.assemble_hessian(C, project=True, out=K)
        ev[3].record()
        for _ in range(spmvs):
            ctx.spmv(x, K=K, out=y)
        ev[4].record()
        ev[4].synchronize()
        spmv_ms = ev[3].elapsed_time(ev[4]) / spmvs
        tsz = 4 if prec == bsc.FP32 else 8
        nbytes = ctx.N * tsz * (225 + 3 + 3)
        gbs = nbytes / (spmv_ms * 1e-3) / 1e9
        hess_ms = ev[2].elapsed_time(ev[3])
        out[name] = {"energy_ms": ev[0].elapsed_time(ev[1]), "gradient_ms": ev[1].elapsed_time(ev[2]),
                     "hessian_ms": hess_ms, "hessian_spans_per_s": out["spans"] / (hess_ms * 1e-3),
                     "spmv_ms": spmv_ms, "spmv_bytes": nbytes, "spmv_gbs": gbs, "spmv_frac_of_hbm": gbs / peak}
        ctx.close()
        del K, x, y, C, Ch
    out["hbm_peak_gbs"] = peak
    out["hbm_peak_source"] = src
    return out


def drape_trajectory(bsc, torch, pat, prec, steps, tol=1e-2, max_newton=30):
    """`steps` implicit-Euler time steps of the drape from rest velocity:
    Chat = C + dt v, Newton iterations until ||d||_inf / dt < tol, then
    v = (C - C_prev) / dt.  Device time of the whole trajectory (CUDA
    events), Newton and PCG iteration counts, and the final positions."""
    ctx = bsc.context_for_patch(pat, precision=prec, pcg_rel_tol=1e-8)
    C = ctx.to_device(pat.C)
    ctx.autotune(C, C)
    v = torch.zeros_like(C)
    C_prev, Chat = torch.empty_like(C), torch.empty_like(C)  # fixed buffers: the captured graph stays valid
    newton, pcg, worst = 0, 0, 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # warm-up outside the timed region: the vector operations' first launches and the
    # capture of the Newton graph on these buffers; then back to the initial state
    C_prev.copy_(C)
    torch.add(C, v, alpha=pat.dt, out=Chat)
    ctx.newton_step(C, Chat)
    torch.sub(C, C_prev, out=v)
    v.div_(pat.dt)
    C.copy_(C_prev)
    v.zero_()
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(steps):
        C_prev.copy_(C)
        torch.add(C, v, alpha=pat.dt, out=Chat)
        for _ in range(max_newton):
            rep = ctx.newton_step(C, Chat)
            newton += 1
            pcg += rep.pcg_iters
            if rep.status != 0 or rep.dir_inf / pat.dt < tol:
                break
        worst = max(worst, rep.dir_inf / pat.dt)
        torch.sub(C, C_prev, out=v)
        v.div_(pat.dt)
    ev1.record()
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    final = C.double().cpu()
    ctx.close()
    return {"time_steps": steps, "newton_iterations": newton, "pcg_iterations": pcg, "ms": ms,
            "ms_per_time_step": ms / steps, "ms_per_newton_iteration": ms / newton,
            "last_dir_inf_over_dt_max": worst}, final


def measure_trajectories(bsc, torch, steps=20):
    """The drape over 20 time steps (dt = 0.01 s) for mu_bd = 1e-6, 1e-5 and
    1e-4 N m in FP32 bulk, and for 1e-5 also in FP64; the FP32 trajectory's
    final positions against the FP64 one's (the FP64 path holds the oracle's
    1e-12 parity), relative to the cloth width."""
    out = {"workload": "drape256", "stop_rule": "||d||_inf / dt < 1e-2 m/s per time step", "runs": {}}
    finals = {}
    for mu_bd in (1e-6, 1e-5, 1e-4):
        pat = inputs.config_drape(1, 256, mu_bd)
        for prec, name in ((bsc.FP32, "fp32"), (bsc.FP64, "fp64")):
            if prec == bsc.FP64 and mu_bd != 1e-5:
                continue
            rec, final = drape_trajectory(bsc, torch, pat, prec, steps)
            out["runs"][f"mu_bd={mu_bd:g} {name}"] = rec
            finals[(mu_bd, name)] = final
        if mu_bd == 1e-5:
            width = float((pat.rest.max(axis=0) - pat.rest.min(axis=0)).max())
            d = (finals[(mu_bd, "fp32")] - finals[(mu_bd, "fp64")]).abs().max().item()
            out["fp32_vs_fp64_final_max_abs_over_width"] = d / width
    return out


def newton_to_convergence(ctx, C, C0, Chat, dt, stream, torch, tol=1e-2, max_iter=30):
    """Newton iterations of one time step from C0 until ||d||_inf / dt < tol
    (the paper's stopping rule, Sec. 6): iterations and device ms."""
    C.copy_(C0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    it = 0
    for it in range(1, max_iter + 1):
        rep = ctx.newton_step(C, Chat)
        if rep.status != 0 or rep.dir_inf / dt < tol:
            break
    ev1.record(stream)
    ev1.synchronize()
    return {"iterations": it, "ms": ev0.elapsed_time(ev1), "status": rep.status,
            "dir_inf_over_dt": rep.dir_inf / dt}


def measure_point_projection(bsc, pat, prec, ctx_span, C0, Chat, steps, warmup, span_ms, flush, stream, torch):
    """The same workload with the per-point closed-form projection of the FBW
    terms (BSC_PROJECT_POINT) instead of the FP64 span projection: Newton-step
    time, and Newton iterations to convergence for both projections."""
    ctx = bsc.context_for_patch(pat, precision=prec, project=bsc.PROJECT_POINT, pcg_rel_tol=1e-8)
    ctx.set_profiling(True)
    ctx.autotune(C0, Chat)
    C = C0.clone()
    ms, ph, reps, launches = time_newton(ctx, C, C0, Chat, steps, warmup, flush, stream, torch)
    step_ms = sum(ms) / steps
    eval_ms = (ph["span_eval"] + ph["project"] + ph["assemble"]) / steps
    conv = {"point": newton_to_convergence(ctx, C, C0, Chat, pat.dt, stream, torch),
            "span": newton_to_convergence(ctx_span, C, C0, Chat, pat.dt, stream, torch)}
    ctx.close()
    # the paper's ablation baseline (Sec. 6.5, case A): 2x2 Gauss on the
    # interior spans, same projection, same state
    ctx = bsc.context_for_patch(pat, precision=prec, project=bsc.PROJECT_POINT, pcg_rel_tol=1e-8,
                                quadrature=(bsc.QUAD_STANDARD, bsc.QUAD_STANDARD))
    ctx.set_profiling(True)
    ctx.autotune(C0, Chat)
    ms_a, ph_a, reps_a, _ = time_newton(ctx, C, C0, Chat, steps, warmup, flush, stream, torch)
    pts = lambda c: (len(c.quadrature_tables(0)), len(c.quadrature_tables(1)))  # noqa: E731
    ablation = {"quadrature": "2x2 Gauss on interior spans, reduced placements on boundary spans",
                "newton_step_ms": sum(ms_a) / steps, "phases_ms": {k: v / steps for k, v in ph_a.items()},
                "pcg_iters": reps_a[-1]["pcg_iters"], "points_membrane_bending": pts(ctx),
                "to_convergence": newton_to_convergence(ctx, C, C0, Chat, pat.dt, stream, torch)}
    ctx.close()
    return {"newton_step_ms": step_ms, "eval_assembly_ms": eval_ms, "spans_per_s": ctx_span.n_spans / (eval_ms * 1e-3),
            "phases_ms": {k: v / steps for k, v in ph.items()}, "pcg_iters": reps[-1]["pcg_iters"],
            "newton_step_speedup_vs_span_projection": span_ms / step_ms, "gpu_launches_per_step": launches / steps,
            "points_membrane_bending": pts(ctx_span), "to_convergence": conv,
            "stop_rule": "||d||_inf / dt < 1e-2 m/s", "ablation_standard_2x2": ablation}


def measure_drape(bsc, flush, stream, torch, np, steps, warmup):
    """The 256 x 256 drape (65,536 cp, 64,516 spans) in FP32 bulk and in FP64:
    Newton-step ms, phases, spans/s of the evaluation + assembly phase."""
    pat = WORKLOADS["drape256"][0](1)[0]
    out = {"workload": "drape256", "spans": pat.n_spans, "control_points": pat.n_cp}
    for prec, name, k in ((bsc.FP32, "fp32", steps), (bsc.FP64, "fp64", max(2, steps // 3))):
        ctx = bsc.context_for_patch(pat, precision=prec, pcg_rel_tol=1e-8)
        ctx.set_profiling(True)
        C0, Chat = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        C = C0.clone()
        tuning = ctx.autotune(C0, Chat)
        ms, ph, reps, launches = time_newton(ctx, C, C0, Chat, k, warmup, flush, stream, torch)
        ev = (ph["span_eval"] + ph["project"] + ph["assemble"]) / k
        out[name] = {"newton_step_ms": sum(ms) / k, "eval_assembly_ms": ev, "spans_per_s": pat.n_spans / (ev * 1e-3),
                     "phases_ms": {kk: v / k for kk, v in ph.items()}, "pcg_iters": reps[-1]["pcg_iters"],
                     "launches_per_step": launches / k, "steps": k, "autotune": tuning}
        if prec == bsc.FP32:
            nneg, nred = ctx.projection_stats()
            nm = np.bincount(ctx.quadrature_tables(0)[:, 24].astype(np.int64), minlength=pat.n_spans)
            nb = np.bincount(ctx.quadrature_tables(1)[:, 24].astype(np.int64), minlength=pat.n_spans)
            psd = bool(tuning.get("psd_test"))
            pc = ctx.psd_counts()
            fl = sum(projection_flops(int(nred[i]), int(nneg[i]), int(nm[i]), int(nb[i]), psd,
                                      pc[1] / max(pc[0], 1), psd, pc[5] / max(pc[3], 1))
                     for i in range(pat.n_spans))
            pms = ph["project"] / k
            out[name]["projection"] = {"ms": pms, "algorithmic_flops": fl,
                                       "tflops": fl / (pms * 1e-3) / 1e12,
                                       "frac_of_nominal_fp64": fl / (pms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                                       "traffic": projection_traffic("drape256", True, tuning)}
        ctx.close()
    out["newton_step_speedup_fp32_vs_fp64"] = out["fp64"]["newton_step_ms"] / out["fp32"]["newton_step_ms"]
    return out


def measure_contact(bsc, flush, stream, torch, np, steps=5, warmup=2):
    """The drape (256x256, FP32) resting on a sphere (radius 0.4 m, 9,216
    triangles) 4 mm below its centre, IPC barrier with dhat = 1 cm, kappa =
    1e3 Pa, contact mesh of about twice the control points: Newton-step ms
    with and without the contact term, from the same state."""
    pat = inputs.config_drape(1, 256, 1e-5)
    V, T = inputs.sphere_obstacle((1.0, 1.0, -0.404), 0.4, 48, 96)
    out = {"workload": "drape256 on a sphere", "obstacle_triangles": int(len(T)), "dhat_m": 0.01,
           "kappa_pa": 1e3}
    for name, with_contact in (("without", False), ("with", True)):
        ctx = bsc.context_for_patch(pat, precision=bsc.FP32, pcg_rel_tol=1e-8)
        ctx.set_profiling(True)
        if with_contact:
            ctx.contact_attach(V, T, 0.01, 1e3)
        C0, Chat = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        C = C0.clone()
        ctx.autotune(C0, Chat)
        ms, ph, reps, launches = time_newton(ctx, C, C0, Chat, steps, warmup, flush, stream, torch)
        rec = {"newton_step_ms": sum(ms) / steps, "phases_ms": {k: v / steps for k, v in ph.items()},
               "alpha": reps[-1]["alpha"], "pcg_iters": reps[-1]["pcg_iters"], "launches_per_step": launches / steps}
        if with_contact:
            rec.update(ctx.contact_stats())
        out[name] = rec
        ctx.close()
    out["contact_overhead_ms"] = out["with"]["newton_step_ms"] - out["without"]["newton_step_ms"]
    return out


def measure_batch(bsc, flush, stream, torch, np, seed=1, steps=3, warmup=2):
    """Short measurement of the batched-garment workload (FP32, autotuned, graph)."""
    pats = WORKLOADS["batch64"][0](seed)
    ctx = make_context(bsc, pats, bsc.FP32)
    ctx.set_profiling(True)
    C0 = stacked(ctx, [p.C for p in pats], torch, np).to(device="cuda", dtype=ctx.dtype)
    Chat = stacked(ctx, [p.Chat for p in pats], torch, np).to(device="cuda", dtype=ctx.dtype)
    C = C0.clone()
    tuning = ctx.autotune(C0, Chat)
    step_ms, phases, reports, launches = time_newton(ctx, C, C0, Chat, steps, warmup, flush, stream, torch)
    eval_ms = (phases["span_eval"] + phases["project"] + phases["assemble"]) / steps
    out = {"workload": "batch64_fp32", "patches": len(pats), "spans": ctx.n_spans, "control_points": ctx.N,
           "spans_per_s": ctx.n_spans / (eval_ms * 1e-3), "newton_step_ms": sum(step_ms) / steps,
           "eval_assembly_ms": eval_ms, "phases_ms": {k: v / steps for k, v in phases.items()},
           "launches_per_step": launches / steps, "max_pcg_iters": reports[-1]["pcg_iters"],
           "max_ls_halvings": reports[-1]["ls_halvings"], "tile_tu": tuning["tile_tu"],
           "autotune": tuning, "graph": ctx.graph_state(), "steps": steps}
    ctx.close()
    # the same batch with the per-point projection of the FBW terms
    ctx = bsc.batch_for_patches(pats, precision=bsc.FP32, pcg_rel_tol=1e-8, project=bsc.PROJECT_POINT)
    ctx.set_profiling(True)
    ctx.autotune(C0, Chat)
    C = C0.clone()
    step_ms, phases, reports, _ = time_newton(ctx, C, C0, Chat, steps, warmup, flush, stream, torch)
    out["point_projection"] = {"newton_step_ms": sum(step_ms) / steps,
                               "phases_ms": {k: v / steps for k, v in phases.items()},
                               "max_pcg_iters": reports[-1]["pcg_iters"]}
    ctx.close()
    return out


WEIGHTS = os.path.join(ROOT, "paper_2506_18867_gb300", "weights", "cnn_learned512.npz")


def measure_learned(bsc, np, torch, flush, seeds=(1_000_000, 1_000_001, 1_000_002, 1_000_003), n=512, steps=3):
    """The learned preconditioner on held-out Newton systems of the 512 x 512
    workload: block-Jacobi PCG vs flexible CG with the trained network, both
    to 1e-8 (CUDA events around each solve; one warm-up solve each first);
    then whole Newton steps of the same held-out states with each solver
    (graph replay, the step from the same state every time, L2 flushed)."""
    from paper_2506_18867_gb300 import train_cnn
    if not os.path.exists(WEIGHTS):
        return {"unavailable": "no trained weights file"}
    sy = train_cnn.Systems(n)
    net = bsc.Cnn(sy.ctx)
    net.set_params(np.load(WEIGHTS)["params"])
    train_cnn.evaluate(sy, net, seeds[:1])            # warm-up (graph capture, first launches)
    rows = train_cnn.evaluate(sy, net, seeds)
    summ = train_cnn.summarize(rows)
    ctx = sy.ctx
    ctx.set_profiling(True)
    stream = torch.cuda.current_stream()
    newton = {"pcg": [], "learned": []}
    for s in seeds:
        pat = inputs.config_learned(s, n)
        ctx.set_material(pat.material)
        C0, Chat = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        C = C0.clone()
        for name, solver in (("pcg", None), ("learned", net)):
            ctx.set_learned_solver(solver)
            ms, ph, reps, _ = time_newton(ctx, C, C0, Chat, steps, 1, flush, stream, torch)
            newton[name].append({"seed": int(s), "newton_step_ms": sum(ms) / steps, "solve_ms": ph["solve"] / steps,
                                 "iters": reps[-1]["pcg_iters"], "fcg_iters": reps[-1]["fcg_iters"],
                                 "fell_back": reps[-1]["fell_back"], "alpha": reps[-1]["alpha"]})
    ctx.set_learned_solver(None)
    mean = lambda rows, k: float(np.mean([r[k] for r in rows]))  # noqa: E731
    summ["newton_step"] = {
        "pcg_ms_mean": mean(newton["pcg"], "newton_step_ms"), "learned_ms_mean": mean(newton["learned"], "newton_step_ms"),
        "pcg_solve_ms_mean": mean(newton["pcg"], "solve_ms"),
        "learned_solve_ms_mean": mean(newton["learned"], "solve_ms"),
        "pcg_iters_mean": mean(newton["pcg"], "iters"), "learned_iters_mean": mean(newton["learned"], "iters"),
        "step_time_ratio_pcg_over_learned": mean(newton["pcg"], "newton_step_ms") / mean(newton["learned"],
                                                                                        "newton_step_ms"),
        "rows": newton}
    net.close()
    sy.ctx.close()
    summ.update({"workload": f"learned{n}", "grid": f"{n}x{n}", "rel_tol": 1e-8,
                 "heldout_seeds": list(seeds), "weights": "paper_2506_18867_gb300/weights/cnn_learned512.npz"})
    return summ


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the projection
# phase per Newton step, from a metrics-only ncu capture of the 512x512 wrinkle
# field (every projection launch of four steps, tuning applied from a plain
# run; profiles/k_proj_psd_wrinkle512_fp32.md), keyed by the autotuner's border
# path and phase-2 variant and by a hash of the projection sources it was taken
# with.  Border path 3, variant 0, per step: border certificate and test 7.2 +
# failing border spans 5.8 + FP32 certificate 101.2 + double-float test 93.0 +
# p1 43.8 + p2 66.2 + corrections 386.1 MB = 703.2 MB.  (Hash renewed after a
# comment and a guard for vanishing matrices, which change no launch here.)
PROJECTION_TRAFFIC_HASH = "a080953cd404bc6f"
PROJECTION_TRAFFIC = {("wrinkle512", True, 3, 0): 703.2e6,
                      # the 512x512 capture scaled by the span count (1,044,484 / 260,100): every
                      # projection kernel's traffic is per span (classes and failing shares alike)
                      ("wrinkle1024", True, 3, 0): 703.2e6 * 1044484 / 260100}
PROJECTION_SOURCES = ("k_project.cu", "proj_core.cuh", "k_project_ring.cu")
# Executed FP64 work of the projection kernels of one drape step (border path 2,
# phase-2 variant 0), from the same kind of capture with the metrics
# sm__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on.sum and
# sm__pipe_fp64_cycles_active.sum: FLOPs (DADD + DMUL + 2 DFMA) and FP64-pipe
# cycles summed over the SMs.
PROJECTION_EXECUTED = {("drape256", True, 2, 0): (938.5e6, 367.4e6)}


def projection_executed(workload, fp32, tuning, launch_ms, sm_mhz, num_sms):
    """Executed FP64 FLOP/s of the projection and the busy fraction of the SMs'
    FP64 pipes over its live time, from the captured counts, or None."""
    rec = PROJECTION_EXECUTED.get((workload, bool(fp32), tuning.get("border_path"), tuning.get("p2_variant")))
    if rec is None or projection_traffic(workload, fp32, tuning) is None:
        return None
    flops, cycles = rec
    return {"executed_flops_per_step": flops, "executed_tflops": flops / (launch_ms * 1e-3) / 1e12,
            "fp64_pipe_busy": cycles / (num_sms * launch_ms * 1e-3 * sm_mhz * 1e6)}


# DRAM bytes (read + write) of one k_pcg launch (three-pass form, symmetric
# matrix layout, FP32) on the 512x512 wrinkle field, 32 iterations: 3.689 GB
# read + 0.448 GB written (metrics-only capture, profiles/k_pcg_wrinkle512_fp32.md),
# i.e. 493 B per control point and iteration.  K (0.47 KB per control point)
# is about the L2's size there and the vectors mostly stay in L2, so the figure
# scaled by control points x iterations to 1024x1024 is a lower bound.  Keyed
# by a hash of the solver sources, the form and the layout (the hash was
# renewed after a change to the two-pass form only, which this instance does
# not compile).
PCG_TRAFFIC_PER_CP_ITER = 4.137e9 / (32 * 262144)
PCG_TRAFFIC_HASH = "0a6ced550a009569"
PCG_TRAFFIC_FORM = 0
PCG_TRAFFIC_WORKLOADS = ("wrinkle512", "wrinkle1024")
# the solver kernels and the product rows they inline
PCG_SOURCES = ("k_solve.cu", "bsc_internal.cuh")


def pcg_traffic(workload, fp32, tuning, iters, k_sym=True):
    import hashlib
    if workload not in PCG_TRAFFIC_WORKLOADS or not fp32 or tuning.get("pcg_form") != PCG_TRAFFIC_FORM or not k_sym:
        return None
    hs = hashlib.sha256()
    for f in PCG_SOURCES:
        with open(os.path.join(ROOT, "paper_2506_18867_gb300", "csrc", f), "rb") as fh:
            hs.update(fh.read())
    if hs.hexdigest()[:16] != PCG_TRAFFIC_HASH:
        return None
    n = {"wrinkle512": 512 * 512, "wrinkle1024": 1024 * 1024}[workload]
    return PCG_TRAFFIC_PER_CP_ITER * n * iters


def projection_traffic(workload, fp32, tuning):
    """The captured DRAM traffic of the projection phase for the autotuner's
    choices, or None when no capture exists for them or the kernels changed
    since it."""
    import hashlib
    rec = PROJECTION_TRAFFIC.get((workload, bool(fp32), tuning.get("border_path"), tuning.get("p2_variant")))
    if rec is None:
        return None
    h = hashlib.sha256()
    for f in PROJECTION_SOURCES:
        with open(os.path.join(ROOT, "paper_2506_18867_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec if h.hexdigest()[:16] == PROJECTION_TRAFFIC_HASH else None


# --------------------------------------------------------------------------- CPU oracle

def _oracle_eval_sample(orc, pat_crop):
    prob = orc.Problem.from_patch(pat_crop)
    sc = orc.Scene.from_patch(pat_crop, project=True)
    t0 = time.perf_counter()
    orc.evaluate(prob, sc, pat_crop.C, pat_crop.Chat)
    return time.perf_counter() - t0


def cpu_baseline(args, pats, m=160, budget_spans=25000):
    """The oracle on a bounded sample: a leading crop of a single patch, or the
    first patches of a batch up to about budget_spans spans."""
    import oracle as orc
    orc.build()
    if len(pats) == 1:
        sample = [inputs.crop(pats[0], min(m, pats[0].nu), min(m, pats[0].nv))]
        what = f"the leading {sample[0].nu}x{sample[0].nv} control points ({sample[0].n_spans} spans) of the state"
    else:
        sample, tot = [], 0
        for p in pats:
            sample.append(p)
            tot += p.n_spans
            if tot >= budget_spans:
                break
        what = f"the first {len(sample)} patches ({tot} spans) of the batch"
    secs = sum(_oracle_eval_sample(orc, p) for p in sample)
    spans = sum(p.n_spans for p in sample)
    return {"value": spans / secs, "unit": "spans/s", "cores": 1, "kind": "oracle",
            "sample": f"E+grad+projected Hessian+stencil assembly of {what}, FP64, one thread",
            "seconds": secs, "all_cores": _oracle_all_cores(orc, pats[0])}


def _oracle_all_cores(orc, pat, m=96):
    """The same oracle evaluation on every host core at once: one thread per
    core, each evaluating its own copy of a leading m x m crop (the ctypes
    calls release the GIL, and the oracle keeps no global state)."""
    from concurrent.futures import ThreadPoolExecutor
    n = os.cpu_count() or 1
    crop = inputs.crop(pat, min(m, pat.nu), min(m, pat.nv))

    def work(_):
        prob = orc.Problem.from_patch(crop)
        sc = orc.Scene.from_patch(crop, project=True)
        orc.evaluate(prob, sc, crop.C.copy(), crop.Chat.copy())

    t0 = time.perf_counter()
    with ThreadPoolExecutor(n) as ex:
        list(ex.map(work, range(n)))
    wall = time.perf_counter() - t0
    return {"value": n * crop.n_spans / wall, "unit": "spans/s", "cores": n, "seconds": wall,
            "sample": f"{n} concurrent evaluations of the leading {crop.nu}x{crop.nv} control points "
                      f"({crop.n_spans} spans each), one per thread"}


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle as orc
    orc.build()
    builder, desc = WORKLOADS[args.workload]
    pats = builder(1)
    if len(pats) == 1:
        sample = [inputs.crop(pats[0], min(96, pats[0].nu), min(96, pats[0].nv))]
        what = f"leading {sample[0].nu}x{sample[0].nv} control points ({sample[0].n_spans} spans)"
    else:
        sample, tot = [], 0
        for p in pats:
            sample.append(p)
            tot += p.n_spans
            if tot >= 8000:
                break
        what = f"first {len(sample)} patches ({tot} spans)"
    spans = sum(p.n_spans for p in sample)

    def one():
        return sum(_oracle_eval_sample(orc, p) for p in sample)

    for _ in range(args.warmup):
        one()
    t = [one() for _ in range(args.steps)]
    sec = sum(t) / len(t)
    value = spans / sec
    line = {"metric": METRIC, "value": value, "unit": "spans/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{args.workload}_{args.precision}", "description": desc, "sample": what},
            "cpu_baseline": {"value": value, "unit": "spans/s", "cores": 1, "kind": "oracle",
                             "sample": f"E+grad+projected Hessian+assembly of the {what} of the same state per "
                                       "step, FP64, one thread"},
            "e2e": {"value": value, "unit": "spans/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
