#!/usr/bin/env python
"""Throughput of the GB300 FMM self-gravity solve (one JSON line on rank 0).

A step is one full solve -- leaf moments, M2M, every cell-to-cell
interaction of every level in one persistent launch, L2L and evaluation of
phi and g -- on one density field resident in HBM.  The default workload is
the largest single-GPU configuration: the AMR octree refined to level 8
around a mass-ratio-0.7 binary of polytropes (43,240 leaves of 8^3 cells,
22.1M cells), plain FP64.

value      = directed cell interactions (far multipole + exact near + mixed
             near pairs) per second, summed over all ranks; the median and
             the mean of the per-step device times are both reported
e2e        = the same through ot_solve_gravity_host: densities copied in from
             pinned host memory and phi, g copied back, every step
roofline   = the interaction launch (the dominant kernel): algorithmic flops
             of the executed pair formulas / its CUDA-event time, against the
             CUDA-core peaks measured in the same run by ot_alu_peaks (FP64
             FMA and FP32 FMA throughput kernels); the peaks derived from the
             unit counts and the maximum SM clock are reported beside them
companions (rank 0, one GPU): the FP32-bulk form and the wide FP32 form
             (time, speed-up, error against the FP64 form, momentum and torque
             residuals, mixed roofline), the adjoint, six resident solves on
             densities updated in place (the two solves per stage of an RK3
             step), the uniform level-3 binary in every form, and the CPU
             oracle on a bounded sample.
--impl reference times the CPU oracle (the plain FP64 statement of the same
solve) on the host cores, on a bounded sample of the same workload.
Multi-GPU runs are independent replicas (weak scaling); the solve has no
exchange step on one tree.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM cell-interactions/s and leaf subgrids/s on 1 GB300; % of FP64/FP32 peak"
UNIT = "cell-interactions/s"
NUM_SMS = 152
SM_MAX_MHZ = 2070.0
# CUDA-core peaks from unit counts and the maximum SM clock (context beside
# the measured ones): 2 FP64 FMA and 128 FP32 FMA per SM per clock
PEAK_FP64_DERIVED = NUM_SMS * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12
PEAK_FP32_DERIVED = NUM_SMS * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (read + write) of one interaction phase, per form, from ncu
# captures of the interaction kernels summarised in profiles/ (per launch;
# binary_amr8 from its full-size one-pass capture).  A workload or form
# without a capture of the current kernels reports null.
TRAFFIC_BYTES = {("binary_l3", "fp64"): 14.44e6 + 10.64e6,
                 ("binary_l3", "fp32_bulk"): 17.39e6 + 10.64e6,
                 ("binary_l3", "fp32_wide"): 12.54e6 + 10.66e6 + 9.56e6,
                 ("binary_amr8", "fp64"): 5.360e9 + 1.536e9 + 0.911e9 + 0.653e9,
                 ("binary_amr8", "fp32_bulk"): 6.558e9 + 1.513e9 + 0.912e9 + 0.653e9}

WORKLOAD_TEXT = {
    "sphere_l1": "uniform level-1 octree, 8 leaves of 8^3 (4,096 cells), one polytrope",
    "binary_l3": "uniform level-3 octree, 512 leaves of 8^3 (262,144 cells), binary "
                 "polytropes rho_c 1.0/0.6, R 0.18/0.12, 1e-10 atmosphere, 1e-3 noise",
    "binary_amr6": "AMR octree to level 6 refined on the binary (4,852 leaves, 2.48M cells)",
    "binary_amr8": "AMR octree to level 8 refined on a mass-ratio-0.7 binary (43,240 leaves of "
                   "8^3, 22.1M cells), 1e-10 atmosphere, 1e-3 noise",
}

FORMS = {"fp64": 0, "fp32_bulk": 1, "fp32_wide": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="binary_amr8", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--precision", default="fp64", choices=sorted(FORMS))
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the companions (other forms, adjoint, resident solves, level-3 "
                         "binary) and the CPU baseline")
    ap.add_argument("--table", action="store_true",
                    help="time every workload in every precision form (no oracle) and print a "
                         "markdown table and one JSON object per row")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (default: tune the persistent launch before timing)")
    ap.add_argument("--hydro-only", type=int, default=None, metavar="LEVEL",
                    help="time only the hydro companions (PPM values and the right-hand side) on a "
                         "uniform tree of this level and print them as one JSON object")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi takes a while to print its first row: start timing only
        # once it samples, so the samples fall inside the timed region
        t0 = time.time()
        while not self.rows and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.rows.clear()  # samples from here on belong to the timed region

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        # a timed region shorter than the sampling period: take the first
        # sample that arrives after it (the clocks at its end)
        t0 = time.time()
        while not self.rows and time.time() - t0 < 2.0 and self.proc.poll() is None:
            time.sleep(0.005)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_setup(n_gpus: int):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not torch.distributed.is_initialized():
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    import torch
    if world > 1:
        torch.distributed.barrier()


def _reduce(world, x: float, op) -> float:
    import torch
    if world == 1:
        return x
    # NCCL reduces device tensors, gloo host tensors
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(world, x: float) -> float:
    import torch
    return _reduce(world, x, torch.distributed.ReduceOp.MAX if world > 1 else None)


def sum_over_ranks(world, x: float) -> float:
    import torch
    return _reduce(world, x, torch.distributed.ReduceOp.SUM if world > 1 else None)


def aggregate(world, per_rank_ms: float, per_rank_units: float):
    """Whole-job throughput of weak-scaled replicas: the slowest rank's time
    and the units every rank processed."""
    total_ms = max_over_ranks(world, per_rank_ms)
    return total_ms, sum_over_ranks(world, per_rank_units) / (total_ms / 1e3)


def time_steps(tree, rho, phi, g, opts, steps, flush, per_step_times=True):
    """Device time (ms) of each solve, L2 flushed before each step."""
    import torch
    stream = torch.cuda.current_stream()
    solve_ms, inter_ms = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tree.solve(rho, phi, g, **opts)
        e1.record(stream)
        e1.synchronize()
        solve_ms.append(e0.elapsed_time(e1))
        if per_step_times:
            inter_ms.append(tree.last_times()[0])
    return solve_ms, inter_ms


def residuals(leaves, rho, g):
    """(momentum, torque) residuals |sum F| / sum |F| and |sum x x F| /
    sum |x x F| of F = m g over every leaf cell (x about the domain centre)."""
    import torch
    from paper_2412_15518_gb300 import inputs
    h = torch.from_numpy(1.0 / (8.0 * 2.0 ** leaves[:, 0])).to(rho.device)
    f = (rho * (h ** 3)[:, None])[:, None, :] * g
    x = torch.from_numpy(inputs.cell_centres(leaves) - 0.5).to(rho.device)
    mom = (f.sum((0, 2)).abs().max() / f.abs().sum()).item()
    tq = torch.cross(x, f.permute(0, 2, 1), dim=2)
    return mom, (tq.sum((0, 1)).abs().max() / tq.abs().sum()).item()


def rel_err(a, ref):
    return float((a - ref).abs().max() / ref.abs().max())


def roofline(info, form, inter_ms, peaks):
    """Roofline of the interaction launch for one form.  FP64: FP64 flops
    against the FP64 peak.  FP32 forms: the launch is bound by whichever pipe
    takes longer for its share of the flops (the mixed bound); frac is the
    bound's time over the measured time."""
    p64, p32 = peaks["fp64_tflops"], peaks["fp32_tflops"]
    t = inter_ms / 1e3
    if form == "fp64":
        f64, f32 = info["flops_am"], 0.0
    elif form == "fp32_bulk":
        f64, f32 = info["flops_bulk64"], info["flops_bulk32"]
    else:
        f64, f32 = info["flops_near"], info["flops_am"] - info["flops_near"]
    bound = max(f64 / (p64 * 1e12), f32 / (p32 * 1e12))
    bound_derived = max(f64 / (PEAK_FP64_DERIVED * 1e12), f32 / (PEAK_FP32_DERIVED * 1e12))
    r = {"launch_ms": inter_ms, "fp64_flops_per_launch": f64, "fp32_flops_per_launch": f32,
         "fp64_tflops": f64 / t / 1e12, "fp32_tflops": f32 / t / 1e12,
         "bound_ms": 1e3 * bound, "frac_of_bound": 1e3 * bound / inter_ms,
         "frac_of_bound_derived_peaks": 1e3 * bound_derived / inter_ms}
    return r


def run_form(tree, rho, form, steps, flush, autotune, warm=3):
    """Autotunes (optionally) and times `steps` solves of one form; returns
    (phi, g, solve_ms list, interaction ms list, tuned shape)."""
    import torch
    prec = FORMS[form]
    if autotune:
        tree.autotune(rho, precision=prec)
    phi, g = tree.empty_outputs()
    opts = dict(precision=prec)
    time_steps(tree, rho, phi, g, opts, warm, flush)
    torch.cuda.synchronize()
    ms, im = time_steps(tree, rho, phi, g, opts, steps, flush)
    i = tree.info()
    shape = {"chunk": i["tuned_chunk"], "ctas_per_sm": i["tuned_ctas_per_sm"],
             "lattice_ctas_per_sm": i["tuned_lattice_ctas_per_sm"], "work_items": i["n_work_items"]}
    return phi, g, ms, im, shape


def companion_form(tree, leaves, rho, form, steps, flush, autotune, ref, ref_ms, info, peaks):
    """One FP32 form beside the FP64 line: time, speed-up, error against the
    FP64 GPU solve, conservation residuals and the mixed roofline."""
    phi, g, ms, im, shape = run_form(tree, rho, form, steps, flush, autotune)
    n_int = info["n_m2l"] + info["n_p2p"] + info["n_seam"]
    mom, ang = residuals(leaves, rho, g)
    out = {"ms_per_step": statistics.mean(ms), "ms_per_step_median": statistics.median(ms),
           "value": n_int / (statistics.median(ms) / 1e3),
           "speedup_vs_fp64": statistics.median(ref_ms) / statistics.median(ms),
           "max_rel_err_vs_fp64": {"phi": rel_err(phi, ref[0]), "g": rel_err(g, ref[1])},
           "residuals": {"momentum": mom, "torque": ang},
           "roofline": roofline(info, form, statistics.median(im), peaks), "tuned": shape}
    del phi, g
    return out


def resident_six(tree, rho, form, flush):
    """Six solves per step on a resident tree, the density updated in place on
    the device before each (as the two solves per stage of an RK3 step would
    see it): device time per six solves, host time per solve call (the graph
    replay), and the device time between the solves."""
    import torch
    prec = FORMS[form]
    phi, g = tree.empty_outputs()
    r = rho.clone()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        tree.solve(r, phi, g, precision=prec)
    torch.cuda.synchronize()
    step_ms, host_us, gap_ms = [], [], []
    for step in range(3):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(12)]
        for k in range(6):
            r.mul_(1.0 + 1e-6 * (1 if (step + k) % 2 else -1))  # the hydro update stands in
            ev[2 * k].record(stream)
            t0 = time.perf_counter()
            tree.solve(r, phi, g, precision=prec)
            host_us.append(1e6 * (time.perf_counter() - t0))
            ev[2 * k + 1].record(stream)
        ev[11].synchronize()
        solves = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(6))
        total = ev[0].elapsed_time(ev[11])
        step_ms.append(total)
        gap_ms.append((total - solves) / 5)
    return {"ms_per_six_solves": statistics.median(step_ms),
            "host_us_per_solve_call": statistics.median(host_us),
            "device_gap_ms_between_solves": statistics.median(gap_ms),
            "includes": "per solve: an in-place density update (one elementwise kernel) and the "
                        "graph replay of the solve; L2 flushed once per six"}


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_2412_15518_gb300 import fmm, inputs
    peaks = fmm.ot_alu_peaks(local, 5)
    leaves, rho_np = inputs.workload(args.workload)
    form = args.precision
    prec = FORMS[form]
    opts = dict(precision=prec)
    tree = fmm.Tree(leaves, device=local)
    rho = torch.from_numpy(rho_np).cuda()
    phi, g = tree.empty_outputs()
    if not args.no_autotune:
        tree.autotune(rho, precision=prec)
    info = tree.info()
    n_int = info["n_m2l"] + info["n_p2p"] + info["n_seam"]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    time_steps(tree, rho, phi, g, opts, max(3, args.warmup), flush)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    solve_ms, inter_ms = time_steps(tree, rho, phi, g, opts, args.steps, flush)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    total_ms, value = aggregate(world, sum(solve_ms), n_int * args.steps)
    ms_per_step = total_ms / args.steps
    subgrids = sum_over_ranks(world, leaves.shape[0] * args.steps) / (total_ms / 1e3)

    # roofline of the interaction launch, against the measured peaks
    inter_med = statistics.median(inter_ms)
    rf = roofline(info, form, inter_med, peaks)
    if form == "fp64":
        achieved, peak, peak_d = rf["fp64_tflops"], peaks["fp64_tflops"], PEAK_FP64_DERIVED
        kernel = "k_interact<double> + k_lattice<0> (concurrent graph branches)"
    elif form == "fp32_bulk":
        achieved, peak, peak_d = rf["fp64_tflops"], peaks["fp64_tflops"], PEAK_FP64_DERIVED
        kernel = "k_interact_split + k_lattice<0> (concurrent graph branches; FP64-bound)"
    else:
        achieved, peak, peak_d = rf["fp32_tflops"], peaks["fp32_tflops"], PEAK_FP32_DERIVED
        kernel = "k_interact<float> + k_lattice<1> + k_lattice<2> (concurrent graph branches)"
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": TRAFFIC_BYTES.get((args.workload, form)),
            "kernel": kernel,
            "peak_source": "measured in this run by ot_alu_peaks (FMA throughput kernels on "
                           "every SM, best of 5)",
            "peak_derived": peak_d, "frac_derived": achieved / peak_d,
            "flops_per_launch": rf["fp64_flops_per_launch"] + rf["fp32_flops_per_launch"],
            "launch_ms": inter_med, "launch_ms_mean": statistics.mean(inter_ms)}
    if form != "fp64":
        roof.update({k: rf[k] for k in ("fp64_flops_per_launch", "fp32_flops_per_launch",
                                        "bound_ms", "frac_of_bound")})
    mom, ang = residuals(leaves, rho, g)

    # end to end through the host-buffer entry point
    hr = torch.from_numpy(rho_np).pin_memory()
    hp = torch.empty((leaves.shape[0], 512), dtype=torch.float64).pin_memory()
    hg = torch.empty((leaves.shape[0], 3, 512), dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        tree.solve_host(hr, hp, hg, **opts)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tree.solve_host(hr, hp, hg, **opts)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    _, e2e_value = aggregate(world, sum(e2e_ms), n_int * args.steps)
    del hr, hp, hg
    n_cells = leaves.shape[0] * 512
    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        ref = (phi.clone(), g.clone())
        csteps = max(3, min(args.steps, 10))
        for other in ("fp32_bulk", "fp32_wide"):
            if other != form:
                extra[other] = companion_form(tree, leaves, rho, other, csteps, flush,
                                              not args.no_autotune, ref, solve_ms, info, peaks)
        del ref
        # the adjoint (FP64): dJ/drho for J = sum(w1 phi + w2 . g)
        tree.set_launch_shape(info["tuned_chunk"], info["tuned_ctas_per_sm"],
                              info["tuned_lattice_ctas_per_sm"])
        w1n, w2n = inputs.weights(leaves.shape[0])
        w1, w2 = torch.from_numpy(w1n).cuda(), torch.from_numpy(w2n).cuda()
        del w1n, w2n
        drho = torch.empty_like(rho)
        for _ in range(2):
            tree.backward(rho, w1, w2, drho)
        torch.cuda.synchronize()
        bms = []
        for _ in range(min(args.steps, 5)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tree.backward(rho, w1, w2, drho)
            e1.record(stream)
            e1.synchronize()
            bms.append(e0.elapsed_time(e1))
        adj = {"ms_per_step": statistics.median(bms), "includes": "forward solve + reverse sweep",
               "ratio_to_forward": statistics.median(bms) / statistics.median(solve_ms)}
        if info.get("flops_adjoint"):
            rev_ms = statistics.median(bms) - statistics.median(solve_ms)
            adj["reverse_interaction_fp64_flops"] = info["flops_adjoint"]
            adj["reverse_sweep_ms_est"] = rev_ms
            adj["fp64_tflops_est"] = info["flops_adjoint"] / (rev_ms / 1e3) / 1e12
            adj["frac_of_fp64_peak_est"] = adj["fp64_tflops_est"] / peaks["fp64_tflops"]
        extra["adjoint_fp64"] = adj
        del w1, w2, drho
        # the tangent (time derivative of phi and g for densities changing at
        # rho_dot = rho u, u uniform in [-1, 1]), FP64 dual numbers
        rd = rho * torch.from_numpy(np.random.default_rng(7).uniform(-1.0, 1.0, rho_np.shape)).cuda()
        pd, gd = tree.empty_outputs()
        for _ in range(2):
            fmm.ot_solve_gravity_tangent(tree.handle, rho, rd, None, None, pd, gd)
        torch.cuda.synchronize()
        tms = []
        for _ in range(min(args.steps, 5)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fmm.ot_solve_gravity_tangent(tree.handle, rho, rd, None, None, pd, gd)
            e1.record(stream)
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
        tmed = statistics.median(tms)
        extra["tangent_fp64"] = {
            "ms_per_step": tmed, "ratio_to_forward": tmed / statistics.median(solve_ms),
            "includes": "values and tangents of every step (dual numbers)",
            "interaction_fp64_flops": info["flops_tangent"],
            "fp64_tflops_whole_solve": info["flops_tangent"] / (tmed / 1e3) / 1e12,
            "frac_of_fp64_peak_whole_solve": info["flops_tangent"] / (tmed / 1e3) / 1e12 /
                                             peaks["fp64_tflops"]}
        del rd, pd, gd
        extra["resident_6"] = {f: resident_six(tree, rho, f, flush) for f in ("fp64", "fp32_bulk")}
        extra["resident_6"]["ms_per_six_solves_if_separate"] = 6 * statistics.median(solve_ms)
        if args.workload != "binary_l3":
            extra["binary_l3"] = companion_workload("binary_l3", flush, not args.no_autotune, peaks)
        extra["ppm_reconstruction"] = ppm_companion(flush, peaks)
        extra["hydro_rhs"] = hydro_companion(flush, peaks)
        extra["hydro_rhs_workload_tree"] = hydro_tree_companion(tree, leaves, args.workload, flush, peaks)
        extra["rk3_step_workload_tree"] = step_companion(tree, leaves, args.workload, flush)
        extra["cpu_baseline"] = cpu_baseline(leaves, rho_np)
    # library kernels of one solve: leaf moments; per parent level the M2M
    # kernel for cells with interior children and/or the one for cells with
    # leaf children; the general interaction kernel; the lattice kernels (1 in
    # the FP64 and FP32-bulk forms, near + far in the wide FP32 form; none
    # without leaf nodes below the root); per level the L2L kernel for its
    # interior cells below the root (or a leaf root) and/or the one
    # evaluating its leaf children
    nl = info["n_levels"]
    leaf_at = lambda L: info["n_leaf_nodes"][L] if 0 <= L < nl else 0
    inner_at = lambda L: info["n_nodes"][L] - info["n_leaf_nodes"][L] if 0 <= L < nl else 0
    m2m = sum((inner_at(L + 1) > 0) + (leaf_at(L + 1) > 0) for L in range(nl - 1))
    l2l = sum((leaf_at(0) > 0 if L == 0 else inner_at(L) > 0) + (leaf_at(L + 1) > 0)
              for L in range(nl))
    lattice = sum(info["n_leaf_nodes"][1:nl]) > 0
    n_lat = (2 if form == "fp32_wide" else 1) if lattice else 0
    launches = (1 + m2m + 1 + n_lat + l2l) * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step,
        "ms_per_step_median": statistics.median(solve_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if form == "fp64" else "f32+f64",
        "data": "synthetic (seeded polytrope binary)",
        "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                   "precision": form, "theta": 0.5, "am_correction": True,
                   "cells": n_cells, "leaf_subgrids": int(leaves.shape[0]),
                   "interactions_per_step": n_int,
                   "l2": "flushed before every step (256 MiB write, untimed)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "work_items": info["n_work_items"], "chunk": info["tuned_chunk"],
                   "ctas_per_sm": info["tuned_ctas_per_sm"]},
        "leaf_subgrids_per_s": subgrids,
        "roofline": roof,
        "peaks_measured": peaks,
        "residuals": {"momentum": mom, "torque": ang},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n_cells * 8,
                "d2h_bytes_per_step": n_cells * 4 * 8},
        "gpu_launches": launches,
        "clocks": clk,
    }
    line.update(extra)
    if "cpu_baseline" not in line:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    tree.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def hbm_peak():
    """The measured copy bandwidth (GB/s) the driver writes beside the repo,
    else the machine's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def ppm_companion(flush, peaks, level=4, steps=20):
    """The hydro solver's PPM reconstruction of the 26 directional values on
    a uniform tree (8^level leaf sub-grids) with the five conserved fields:
    median time and rooflines.  The kernel is FP64-bound on this GPU: per
    cell, field and line 25 FP64 operations (one boundary value: 2 adds, 2
    multiplies, 1 subtract, 4 min/max; the limiter: 10 adds and multiplies, 3
    comparisons, 3 for one update) against the measured FP64 instruction rate
    (the FMA peak / 2); the HBM share is the algorithmic bytes (each average
    read once, its 26 values written once) over the measured copy rate."""
    import numpy as np
    import torch
    from paper_2412_15518_gb300 import fmm, inputs
    leaves = inputs.uniform_leaves(level)
    u = torch.from_numpy(inputs.hydro_fields(leaves)).cuda()
    tree = fmm.Tree(leaves)
    out = torch.empty((u.shape[0], u.shape[1], 26, 512), dtype=torch.float64, device="cuda")
    for _ in range(3):
        fmm.ot_ppm_reconstruct(tree.handle, u, out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fmm.ot_ppm_reconstruct(tree.handle, u, out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    med = statistics.median(ms)
    cells = leaves.shape[0] * 512
    nf = u.shape[1]
    nbytes = cells * nf * 8 * (1 + 26)
    ops = cells * nf * 13 * 25
    hbm, src = hbm_peak()
    gops = ops / (med / 1e3) / 1e12
    peak_ops = peaks["fp64_tflops"] / 2.0
    tree.close()
    del u, out
    return {"workload": f"uniform level-{level} octree ({leaves.shape[0]} leaf sub-grids, {cells} cells), "
                        "5 conserved fields of the rotating binary",
            "ms_per_launch": med, "cells_per_s": cells / (med / 1e3),
            "roofline": {"bound": "alu", "achieved": gops, "peak": peak_ops, "unit": "T FP64 ops/s",
                         "frac": gops / peak_ops,
                         "peak_source": "measured FP64 FMA rate (ot_alu_peaks) / 2, one FP64 operation "
                                        "per lane per issue slot",
                         "fp64_ops_per_launch": ops, "fp64_ops_per_cell_field_line": 25},
            "hbm": {"achieved_gbs": nbytes / (med / 1e3) / 1e9, "peak_gbs": hbm, "peak_source": src,
                    "frac": nbytes / (med / 1e3) / 1e9 / hbm, "bytes_per_launch": nbytes}}


# FP64 operations of the hydro right-hand side (hydro.cu), counted from its
# code: per face point 83 (two states' Euler fluxes and wave speeds, 23 each
# with the reciprocal and the square root as one operation; the Rusanov flux,
# 27; the weighted sum, 10), per cell 44 (divergence 30, scale 5, source 9);
# a leaf computes 3 x 9 x 8 x 8 faces of 9 points.
# FP64 operations of the hydro right-hand side, the correctly rounded
# reciprocal and square root counted as one each: per face point the two
# states' fluxes from their primitives (7 each), the Rusanov flux (27) and the
# weighted sum (10); per own cell and direction the state's primitives (16,
# formed once); per cell the divergence, scale and source (44).  The ghost
# states' primitives at refinement jumps are not counted.
HYDRO_OPS_PER_POINT = 51
HYDRO_OPS_PER_STATE = 16
HYDRO_OPS_PER_CELL = 44


def hydro_companion(flush, peaks, level=4, steps=20):
    """The hydro solver's right-hand side dU/dt on a uniform tree
    (8^level leaf sub-grids) with the rotating binary's five conserved fields
    and the gravity solve's acceleration: PPM values, face fluxes and the
    gravity source in one call.  Median time and the FP64 roofline of the
    whole call (the PPM kernel's and the flux kernel's operations against the
    measured FP64 instruction rate, the FMA peak / 2)."""
    import torch
    from paper_2412_15518_gb300 import fmm, inputs
    leaves = inputs.uniform_leaves(level)
    u = torch.from_numpy(inputs.hydro_fields(leaves)).cuda()
    tree = fmm.Tree(leaves)
    phi, g = tree.solve(u[:, 0].contiguous())
    out = torch.empty_like(u)
    for _ in range(3):
        fmm.ot_hydro_rhs(tree.handle, u, g, 5.0 / 3.0, out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fmm.ot_hydro_rhs(tree.handle, u, g, 5.0 / 3.0, out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    med = statistics.median(ms)
    n_leaf = leaves.shape[0]
    cells = n_leaf * 512
    ops_ppm = cells * 5 * 13 * 25
    ops_flux = (n_leaf * 3 * 576 * 9 * HYDRO_OPS_PER_POINT + cells * 26 * HYDRO_OPS_PER_STATE
                + cells * HYDRO_OPS_PER_CELL)
    gops = (ops_ppm + ops_flux) / (med / 1e3) / 1e12
    peak_ops = peaks["fp64_tflops"] / 2.0
    tree.close()
    del u, out, phi, g
    return {"workload": f"uniform level-{level} octree ({n_leaf} leaf sub-grids, {cells} cells), "
                        "5 conserved fields of the rotating binary, g from the gravity solve",
            "ms_per_launch": med, "cells_per_s": cells / (med / 1e3),
            "roofline": {"bound": "alu", "achieved": gops, "peak": peak_ops, "unit": "T FP64 ops/s",
                         "frac": gops / peak_ops,
                         "peak_source": "measured FP64 FMA rate (ot_alu_peaks) / 2, one FP64 operation "
                                        "per lane per issue slot",
                         "fp64_ops_per_launch": ops_ppm + ops_flux, "ppm_ops": ops_ppm,
                         "flux_ops": ops_flux}}


def hydro_tree_companion(tree, leaves, name, flush, peaks, steps=5):
    """The hydro right-hand side on the workload's own tree (adaptive for the
    AMR workloads: halos across refinement jumps, flux matching), with the
    workload's density plus the rotating binary's momentum and energy, and g
    from an FP64 gravity solve of that density: median time, the same
    operation count as hydro_companion (the leaves' own cells), and the
    volume-weighted totals of the rates against their magnitudes (what the
    fluxes move between cells cancels; the rest is the gravity source and
    the domain boundary)."""
    import torch
    from paper_2412_15518_gb300 import fmm, inputs
    u = torch.from_numpy(inputs.hydro_fields(leaves, inputs.WORKLOAD_STARS[name])).cuda()
    phi, g = tree.solve(u[:, 0].contiguous())
    out = torch.empty_like(u)
    for _ in range(2):
        fmm.ot_hydro_rhs(tree.handle, u, g, 5.0 / 3.0, out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fmm.ot_hydro_rhs(tree.handle, u, g, 5.0 / 3.0, out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    med = statistics.median(ms)
    n_leaf = leaves.shape[0]
    cells = n_leaf * 512
    ops = (cells * 5 * 13 * 25 + n_leaf * 3 * 576 * 9 * HYDRO_OPS_PER_POINT + cells * 26 * HYDRO_OPS_PER_STATE
           + cells * HYDRO_OPS_PER_CELL)
    gops = ops / (med / 1e3) / 1e12
    peak_ops = peaks["fp64_tflops"] / 2.0
    # mass rate without gravity: fluxes only, so its total is the domain
    # boundary's (the bench's trees span the unit cube)
    fmm.ot_hydro_rhs(tree.handle, u, None, 5.0 / 3.0, out)
    try:
        status = tree.info()["device_status"]
    except fmm.OTError as e:
        status = e.info["device_status"]
    h = 1.0 / (8.0 * 2.0 ** torch.from_numpy(leaves[:, 0].astype("float64")).cuda())
    w = (h ** 3)[:, None]
    mass_rate = out[:, 0]
    res = {"workload": f"{name}'s tree ({n_leaf} leaf sub-grids, {cells} cells, levels "
                       f"{int(leaves[:, 0].min())}-{int(leaves[:, 0].max())}), the workload's density, "
                       "5 conserved fields, g from the FP64 gravity solve",
           "ms_per_launch": med, "cells_per_s": cells / (med / 1e3),
           "roofline": {"bound": "alu", "achieved": gops, "peak": peak_ops, "unit": "T FP64 ops/s",
                        "frac": gops / peak_ops, "fp64_ops_per_launch": ops},
           "mass_rate_total_over_magnitude": float((mass_rate * w).sum() / (mass_rate.abs() * w).sum()),
           "device_status": status}
    del u, out, phi, g
    return res


def step_companion(tree, leaves, name, flush, steps=2):
    """One coupled time step on the workload's own tree, on the device: the
    third-order Runge-Kutta scheme, each of its 3 stages a gravity solve of
    the stage's density (FP64) and the hydro right-hand side, with the
    combinations between them (ot_hydro_rk3_step).  Median time per step."""
    import torch
    from paper_2412_15518_gb300 import fmm, inputs
    u0 = torch.from_numpy(inputs.hydro_fields(leaves, inputs.WORKLOAD_STARS[name])).cuda()
    u = u0.clone()
    fmm.ot_hydro_rk3_step(tree.handle, u, 1e-5, 5.0 / 3.0, 1)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        u.copy_(u0)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fmm.ot_hydro_rk3_step(tree.handle, u, 1e-5, 5.0 / 3.0, 1)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    med = statistics.median(ms)
    cells = leaves.shape[0] * 512
    try:
        status = tree.info()["device_status"]
    except fmm.OTError as e:  # the latched bits (the density bit: a stage state below zero)
        status = e.info["device_status"]
    del u, u0
    return {"workload": f"{name}'s tree ({cells} cells), the workload's density plus the rotating "
                        "binary's momentum and energy, dt = 1e-5",
            "ms_per_step": med, "cell_updates_per_s": cells / (med / 1e3),
            "includes": "3 stages x (FP64 gravity solve of the stage density + hydro right-hand side "
                        "+ Runge-Kutta combination)",
            "device_status": status,
            "device_status_note": "bit 4: some stage state had a density <= 0 (the 1e-10 atmosphere at "
                                  "the stars' surfaces; the scheme has no positivity fix)"}


def companion_workload(name, flush, autotune, peaks):
    """Every form on another workload (its own tree): ms per solve, the
    interaction rooflines, the FP32 forms' errors and residuals."""
    import torch
    from paper_2412_15518_gb300 import fmm, inputs
    leaves, rho_np = inputs.workload(name)
    tree = fmm.Tree(leaves)
    rho = torch.from_numpy(rho_np).cuda()
    info = tree.info()
    n_int = info["n_m2l"] + info["n_p2p"] + info["n_seam"]
    out = {"workload": f"{name}: {WORKLOAD_TEXT[name]}"}
    ref = None
    for form in ("fp64", "fp32_bulk", "fp32_wide"):
        phi, g, ms, im, shape = run_form(tree, rho, form, 20, flush, autotune)
        mom, ang = residuals(leaves, rho, g)
        r = {"ms_per_step_median": statistics.median(ms), "ms_per_step": statistics.mean(ms),
             "value": n_int / (statistics.median(ms) / 1e3),
             "residuals": {"momentum": mom, "torque": ang},
             "roofline": roofline(info, form, statistics.median(im), peaks), "tuned": shape}
        if ref is None:
            ref = (phi.clone(), g.clone(), ms)
        else:
            r["max_rel_err_vs_fp64"] = {"phi": rel_err(phi, ref[0]), "g": rel_err(g, ref[1])}
            r["speedup_vs_fp64"] = statistics.median(ref[2]) / statistics.median(ms)
        out[form] = r
    tree.close()
    return out


def cpu_baseline(leaves, rho, budget_s: float = 20.0):
    """The oracle (plain FP64 C++ on the host cores), timed once on a bounded
    sample: the full solve when it fits the budget, else a seeded sample of
    leaf cells with their ancestors' expansions."""
    import numpy as np
    import oracle
    cores = oracle.set_threads(0)
    n_cells = leaves.shape[0] * 512
    probe_cells = np.arange(0, n_cells, max(1, n_cells // 512))
    t0 = time.perf_counter()
    _, _, c = oracle.solve_sample(leaves, rho, probe_cells, return_counts=True)
    probe = time.perf_counter() - t0
    rate = (c["m2l"] + c["p2p"] + c["seam"]) / max(probe, 1e-6)
    per_cell = (c["m2l"] + c["p2p"] + c["seam"]) / probe_cells.size
    full = None
    try:
        import paper_2412_15518_gb300.fmm as F
        info = F.host_only_counts(leaves)
        full = info["n_m2l"] + info["n_p2p"] + info["n_seam"]
    except Exception:
        pass
    if full is not None and full / rate <= budget_s:
        t0 = time.perf_counter()
        _, _, c = oracle.solve(leaves, rho, return_counts=True)
        dt = time.perf_counter() - t0
        sample = f"one full oracle solve of the workload ({n_cells:,} cells)"
    else:
        k = int(min(n_cells, max(512, budget_s * rate / max(per_cell, 1.0))))
        rng = np.random.default_rng(0)
        s = np.sort(rng.choice(n_cells, size=k, replace=False))
        t0 = time.perf_counter()
        _, _, c = oracle.solve_sample(leaves, rho, s, return_counts=True)
        dt = time.perf_counter() - t0
        sample = f"oracle solve of {k:,} seeded leaf cells and their ancestors' expansions"
    n = c["m2l"] + c["p2p"] + c["seam"]
    out = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
           "seconds": dt, "interactions": n}
    # brute force beside it: direct O(N^2) summation on the 4,096-cell sphere
    # (16.8M pairs) against the oracle's FMM solve of the same field
    from paper_2412_15518_gb300 import inputs
    lv1, r1 = inputs.workload("sphere_l1")
    t0 = time.perf_counter()
    oracle.direct(lv1, r1)
    t_direct = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.solve(lv1, r1)
    t_fmm = time.perf_counter() - t0
    out["sphere_l1_direct_s"] = t_direct
    out["sphere_l1_fmm_oracle_s"] = t_fmm
    # the same oracle on one core, on a smaller seeded sample (about 5 s)
    if cores > 1:
        oracle.set_threads(1)
        k1 = int(min(n_cells, max(64, 5.0 * (rate / cores) / max(per_cell, 1.0))))
        s1 = np.sort(np.random.default_rng(1).choice(n_cells, size=k1, replace=False))
        t0 = time.perf_counter()
        _, _, c1 = oracle.solve_sample(leaves, rho, s1, return_counts=True)
        dt1 = time.perf_counter() - t0
        oracle.set_threads(0)
        out["value_1core"] = (c1["m2l"] + c1["p2p"] + c1["seam"]) / dt1
        out["sample_1core"] = f"oracle solve of {k1:,} seeded leaf cells on 1 core"
    return out


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2412_15518_gb300 import inputs
    leaves, rho = inputs.workload(args.workload)
    cores = oracle.set_threads(0)
    n_cells = leaves.shape[0] * 512
    budget = max(1.0, 150.0 / (args.steps + args.warmup))
    rng = np.random.default_rng(0)
    k = 2048
    for _ in range(args.warmup):      # calibrate the sample so a step takes ~budget
        s = np.sort(rng.choice(n_cells, size=min(k, n_cells), replace=False))
        t0 = time.perf_counter()
        oracle.solve_sample(leaves, rho, s)
        dt = time.perf_counter() - t0
        k = int(min(n_cells, max(256, k * budget / max(dt, 1e-3))))
    total_n, total_t = 0, 0.0
    for _ in range(args.steps):
        s = np.sort(rng.choice(n_cells, size=min(k, n_cells), replace=False))
        t0 = time.perf_counter()
        _, _, c = oracle.solve_sample(leaves, rho, s, return_counts=True)
        total_t += time.perf_counter() - t0
        total_n += c["m2l"] + c["p2p"] + c["seam"]
    value = total_n / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded polytrope binary)",
        "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                   "precision": "fp64", "theta": 0.5, "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"per step: oracle solve of {k:,} seeded leaf cells of "
                                   f"{n_cells:,} and their ancestors' expansions"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_table(args):
    """Every workload x every form on this GPU: median solve time, throughput,
    interaction roofline against the measured peaks, conservation residuals,
    speed-up and difference against the FP64 form."""
    import torch
    from paper_2412_15518_gb300 import fmm, inputs
    torch.cuda.set_device(0)
    peaks = fmm.ot_alu_peaks(0, 5)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = []
    for name in ("sphere_l1", "binary_l3", "binary_amr6", "binary_amr8"):
        leaves, rho_np = inputs.workload(name)
        tree = fmm.Tree(leaves)
        rho = torch.from_numpy(rho_np).cuda()
        info = tree.info()
        n_int = info["n_m2l"] + info["n_p2p"] + info["n_seam"]
        ref = None
        for form in ("fp64", "fp32_bulk", "fp32_wide"):
            phi, g, ms, im, shape = run_form(tree, rho, form, args.steps, flush, not args.no_autotune)
            med = statistics.median(ms)
            mom, ang = residuals(leaves, rho, g)
            rf = roofline(info, form, statistics.median(im), peaks)
            row = {"workload": name, "form": form, "cells": int(leaves.shape[0]) * 512,
                   "leaf_subgrids": int(leaves.shape[0]), "interactions": n_int,
                   "ms_median": med, "ms_mean": statistics.mean(ms),
                   "interact_ms_median": statistics.median(im),
                   "cell_interactions_per_s": n_int / (med / 1e3),
                   "leaf_subgrids_per_s": leaves.shape[0] / (med / 1e3),
                   "frac_of_bound": rf["frac_of_bound"], "roofline": rf,
                   "momentum": mom, "torque": ang, "tuned": shape}
            if ref is None:
                ref = (phi.clone(), g.clone(), med)
            else:
                row["speedup_vs_fp64"] = ref[2] / med
                row["max_rel_diff_vs_fp64"] = max(rel_err(phi, ref[0]), rel_err(g, ref[1]))
            rows.append(row)
            print(json.dumps(row), flush=True)
            del phi, g
        del ref
        tree.close()
        del rho
        torch.cuda.empty_cache()
    print(f"peaks measured: {json.dumps(peaks)}")
    print("| workload | form | ms (median) | cell-int/s | leaf subgrids/s | frac of bound | "
          "momentum | torque | speed-up vs FP64 |")
    print("|---|---|---:|---:|---:|---:|---:|---:|---:|")
    for r in rows:
        print(f"| {r['workload']} | {r['form']} | {r['ms_median']:.3f} | {r['cell_interactions_per_s']:.3g} | "
              f"{r['leaf_subgrids_per_s']:.3g} | {r['frac_of_bound']:.3f} | {r['momentum']:.1e} | "
              f"{r['torque']:.1e} | {r.get('speedup_vs_fp64', 1.0):.2f} |")


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.table:
        run_table(args)
    elif args.hydro_only is not None:
        import torch
        from paper_2412_15518_gb300 import fmm
        peaks = fmm.ot_alu_peaks(0, 3)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        print(json.dumps({"ppm_reconstruction": ppm_companion(flush, peaks, args.hydro_only, args.steps),
                          "hydro_rhs": hydro_companion(flush, peaks, args.hydro_only, args.steps)}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
