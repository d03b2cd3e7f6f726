#!/usr/bin/env python
"""Throughput of the GB300 FMM self-gravity solve (one JSON line on rank 0).

A step is one full solve -- leaf moments, M2M, every cell-to-cell
interaction of every level in one persistent launch, L2L and evaluation of
phi and g -- on one density field resident in HBM.  The default workload is
the uniform level-3 octree (512 leaves of 8^3 cells, 262,144 cells) with a
seeded binary of two polytropes, plain FP64.

value      = directed cell interactions (far multipole + exact near + mixed
             near pairs) per second, summed over all ranks
e2e        = the same through ot_solve_gravity_host: densities copied in from
             pinned host memory and phi, g copied back, every step
roofline   = the interaction launch (the dominant kernel): algorithmic flops
             of the executed pair formulas / its CUDA-event time, against the
             FP64 (or FP32) CUDA-core peak derived from the unit counts and
             the maximum SM clock
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
# CUDA-core peaks from unit counts and the maximum SM clock: 2 FP64 FMA and
# 128 FP32 FMA per SM per clock, 2 flops per FMA
PEAK_FP64_TFLOPS = NUM_SMS * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12
PEAK_FP32_TFLOPS = NUM_SMS * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (read + write) of one interaction phase, from the ncu capture of
# the interaction kernels summarised in profiles/ (k_interact + the lattice
# kernels of the form, per launch).  Valid for these kernels as captured; a
# workload or form without a capture reports null.
TRAFFIC_BYTES = {("binary_l3", "fp64"): 15.327e6 + 10.637e6,
                 ("binary_l3", "fp32_bulk"): 13.473e6 + 10.664e6 + 9.564e6}

WORKLOAD_TEXT = {
    "sphere_l1": "uniform level-1 octree, 8 leaves of 8^3 (4,096 cells), one polytrope",
    "binary_l3": "uniform level-3 octree, 512 leaves of 8^3 (262,144 cells), binary "
                 "polytropes rho_c 1.0/0.6, R 0.18/0.12, 1e-10 atmosphere, 1e-3 noise",
    "binary_amr6": "AMR octree to level 6 refined on the binary (4,852 leaves, 2.48M cells)",
    "binary_amr8": "AMR octree to level 8, mass-ratio-0.7 binary (43,240 leaves, 22.1M cells)",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="binary_l3", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_bulk"])
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the companion FP32-bulk run and the CPU baseline")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (default: tune the persistent launch before timing)")
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


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_2412_15518_gb300 import fmm, inputs
    leaves, rho_np = inputs.workload(args.workload)
    prec = fmm.OT_PRECISION_FP64 if args.precision == "fp64" else fmm.OT_PRECISION_FP32_BULK
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

    # roofline of the interaction launch
    inter_avg = statistics.mean(inter_ms)
    flops = info["flops_am"]
    if prec == fmm.OT_PRECISION_FP64:
        achieved = flops / (inter_avg / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": PEAK_FP64_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / PEAK_FP64_TFLOPS,
                "traffic": TRAFFIC_BYTES.get((args.workload, "fp64")),
                "kernel": "k_interact<double> + k_lattice<0> (concurrent graph branches)",
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz",
                "flops_per_launch": flops, "launch_ms": inter_avg}
    else:
        f32 = flops - info["flops_near"]
        achieved = f32 / (inter_avg / 1e3) / 1e12
        # the FP64 near pairs bound the launch too: the mixed roofline is the
        # larger of the two pipes' times
        mixed_ms = 1e3 * max(f32 / (PEAK_FP32_TFLOPS * 1e12),
                             info["flops_near"] / (PEAK_FP64_TFLOPS * 1e12))
        roof = {"bound": "alu", "achieved": achieved, "peak": PEAK_FP32_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / PEAK_FP32_TFLOPS,
                "traffic": TRAFFIC_BYTES.get((args.workload, "fp32_bulk")),
                "kernel": "k_interact<float> + k_lattice<1> + k_lattice<2> (concurrent graph branches)",
                "peak_source": "derived: 152 SMs x 128 FP32 FMA/clk x 2 flops x 2070 MHz",
                "flops_per_launch": f32, "fp64_flops_per_launch": info["flops_near"],
                "launch_ms": inter_avg, "mixed_bound_ms": mixed_ms,
                "frac_of_mixed_bound": mixed_ms / inter_avg}

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
    n_cells = leaves.shape[0] * 512
    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        if prec == fmm.OT_PRECISION_FP64:
            # the FP32-bulk form on the same workload, and its error against FP64
            ref_phi, ref_g = phi.clone(), g.clone()
            o32 = dict(precision=fmm.OT_PRECISION_FP32_BULK)
            if not args.no_autotune:
                tree.autotune(rho, precision=fmm.OT_PRECISION_FP32_BULK)
            time_steps(tree, rho, phi, g, o32, 3, flush)
            ms32, int32 = time_steps(tree, rho, phi, g, o32, args.steps, flush)
            torch.cuda.synchronize()
            ep = float((phi - ref_phi).abs().max() / ref_phi.abs().max())
            eg = float((g - ref_g).abs().max() / ref_g.abs().max())
            f32 = info["flops_am"] - info["flops_near"]
            a32 = f32 / (statistics.mean(int32) / 1e3) / 1e12
            mixed_ms = 1e3 * max(f32 / (PEAK_FP32_TFLOPS * 1e12),
                                 info["flops_near"] / (PEAK_FP64_TFLOPS * 1e12))
            extra["fp32_bulk"] = {
                "ms_per_step": sum(ms32) / args.steps,
                "value": n_int * args.steps / (sum(ms32) / 1e3),
                "speedup_vs_fp64": sum(solve_ms) / sum(ms32),
                "max_rel_err_vs_fp64": {"phi": ep, "g": eg},
                "interact_ms": statistics.mean(int32),
                "interact_fp32_tflops": a32, "frac_of_fp32_peak": a32 / PEAK_FP32_TFLOPS,
                "mixed_bound_ms": mixed_ms,
                "frac_of_mixed_bound": mixed_ms / statistics.mean(int32)}
            i32 = tree.info()
            extra["fp32_bulk"]["tuned"] = {"chunk": i32["tuned_chunk"],
                                           "ctas_per_sm": i32["tuned_ctas_per_sm"],
                                           "lattice_ctas_per_sm": i32["tuned_lattice_ctas_per_sm"],
                                           "work_items": i32["n_work_items"]}
            # the adjoint (FP64): dJ/drho for J = sum(w1 phi + w2 . g)
            w1n, w2n = inputs.weights(leaves.shape[0])
            w1, w2 = torch.from_numpy(w1n).cuda(), torch.from_numpy(w2n).cuda()
            drho = torch.empty_like(rho)
            for _ in range(2):
                tree.backward(rho, w1, w2, drho)
            torch.cuda.synchronize()
            bms = []
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                tree.backward(rho, w1, w2, drho)
                e1.record(stream)
                e1.synchronize()
                bms.append(e0.elapsed_time(e1))
            extra["adjoint_fp64"] = {"ms_per_step": sum(bms) / args.steps,
                                     "includes": "forward solve + reverse sweep",
                                     "ratio_to_forward": sum(bms) / sum(solve_ms)}
        extra["cpu_baseline"] = cpu_baseline(leaves, rho_np)
    # library kernels of one solve: leaf moments; per parent level the M2M
    # kernel for cells with interior children and/or the one for cells with
    # leaf children; the general interaction kernel; the lattice kernels (1 in
    # the FP64 form, near + far in the FP32-bulk form; none without leaf nodes
    # below the root); per level the L2L kernel for its interior cells below
    # the root (or a leaf root) and/or the one evaluating its leaf children
    nl = info["n_levels"]
    leaf_at = lambda L: info["n_leaf_nodes"][L] if 0 <= L < nl else 0
    inner_at = lambda L: info["n_nodes"][L] - info["n_leaf_nodes"][L] if 0 <= L < nl else 0
    m2m = sum((inner_at(L + 1) > 0) + (leaf_at(L + 1) > 0) for L in range(nl - 1))
    l2l = sum((leaf_at(0) > 0 if L == 0 else inner_at(L) > 0) + (leaf_at(L + 1) > 0)
              for L in range(nl))
    lattice = sum(info["n_leaf_nodes"][1:nl]) > 0
    n_lat = (2 if prec == fmm.OT_PRECISION_FP32_BULK else 1) if lattice else 0
    launches = (1 + m2m + 1 + n_lat + l2l) * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == fmm.OT_PRECISION_FP64 else "f32+f64",
        "data": "synthetic (seeded polytrope binary)",
        "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                   "precision": args.precision, "theta": 0.5, "am_correction": True,
                   "cells": n_cells, "leaf_subgrids": int(leaves.shape[0]),
                   "interactions_per_step": n_int,
                   "l2": "flushed before every step (256 MiB write, untimed)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "work_items": info["n_work_items"], "chunk": info["tuned_chunk"],
                   "ctas_per_sm": info["tuned_ctas_per_sm"]},
        "leaf_subgrids_per_s": subgrids,
        "roofline": roof,
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


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
