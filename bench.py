#!/usr/bin/env python
"""Benchmark of the temporally blocked 3D 7-point Jacobi library on GB300.

Default workload (what the headline metric is quoted on): FP64 512^3
interior, interior U[0,1), halo 0 except the k=0 plane = 1, T = 100 sweeps
per step (one step = one jacobi_sweep call = the whole hot path: halo copy,
pass planning, all passes).  Metric: GLUP/s = nx*ny*nz*T / time (the
paper's LUP/s, Sect. 1.2), and the fraction of the HBM roofline of Eq. (2),
P0 = M_s / (2 s) per pass (16 B/LUP for FP64), effective d * P0 after
temporal blocking.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   (the CPU oracle on the host cores)

Under torchrun (N > 1) every rank sweeps its own replica of the workload
(weak scaling; the method needs no exchange on one grid per GPU) and rank 0
prints one JSON line with the max-over-ranks time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GLUP/s (3D 7-pt Jacobi) and % of HBM roofline, blocked vs plain, 1×GB300"
POISSON_METRIC = "time to relative residual 1e-10 (Poisson 96^3, refinement vs plain FP64 Jacobi)"
M_S_FALLBACK = 6800.0  # GB/s, used only if MEASURED_PEAKS.json is absent
# FP64 pipe of GB300: 1.25 TFLOP/s nominal counting an FMA as 2 flops, i.e.
# 2 FP64 lanes per SM per clock (1.25e12 / (2 * 152 * 2.07e9)).
FP64_LANES_PER_SM_CLK = 2
# Of the five additions of a cell update, the library's FP64 kernels run the
# first and the last on the integer pipe; three issue on the FP64 pipe.
FP64_PIPE_ADDS = 3
# Integer ALU pipe: 16 lanes per SM sub-partition and clock, 64 per SM
# (ncu: 536.6 M ALU warp instructions in 952.8 us at 90.15 % of peak on the
# 512^3 launch = 2.0 warp instructions per SM and clock).
ALU_LANES_PER_SM_CLK = 64
# ALU-pipe lane instructions per cell update (smsp__inst_executed_pipe_alu.sum
# x 32 / LUPs of the launch, ncu): kernel, dtype -> (count, capture tag).
MEASURED_ALU = {
    ("plain_pass_kernel", "f64"): (128.0, "ncu: plain_pass_kernel<double> 512^3, 32x16 threads, 32 planes"),
}
SMS = 152
# Temporally blocked pass used for the comparison line (one CTA applying d
# levels): kernel, depth, tile bx x by, z chunk, ring (unused), threads.
BLOCKED_REF = {"f64": (4, 4, 64, 32, 64, 0, 512), "f32": (4, 4, 32, 32, 128, 0, 256)}  # kernel TB_CTA
# DRAM bytes per LUP of one launch (dram__bytes_read.sum + dram__bytes_write.sum
# over the LUPs of the launch), from ncu captures of the same kernel build:
# (kernel, dtype, depth) -> (bytes per LUP, capture tag).
BATCH_SWEEP_TRAFFIC = (12.62, "ncu: batch_sweep_kernel, 256-grid workload, one sweep")
MEASURED_TRAFFIC = {
    ("plain_pass_kernel", "f64", 1): (15.92, "ncu: plain_pass_kernel<double>, 512^3"),
    ("tbc4_pass_kernel", "f32", 2): (3.97, "ncu: tbc4_pass_kernel depth 2, FP32 512^3"),
    ("tbc4_pass_kernel", "f32", 4): (2.04, "ncu: tbc4_pass_kernel depth 4, FP32 512^3"),
    ("tbr_pass_kernel", "f32", 3): (2.82, "ncu: tbr_pass_kernel depth 3, region 64x32, FP32 512^3, one pass"),
    ("cg_f32_kernel", "f32", 3): (3.05, "ncu: cg_f32_kernel depth 3, 128-plane chunks, FP32 512^3, one pass"),
}
SM_MAX_MHZ = 2070.0

WORKLOADS = {
    "fp64_512": dict(n=(512, 512, 512), dtype="f64", T=100, gen="dirichlet_z0", seed=2,
                     name="jacobi3d_fp64_512cubed_T100_z0face1"),
    "fp64_64": dict(n=(64, 64, 64), dtype="f64", T=10, gen="uniform", seed=1,
                    name="jacobi3d_fp64_64cubed_T10"),
    # the paper's grid shape (Sect. 2.3: a 600^3 domain; its values are not
    # given), as a context configuration
    "fp64_600": dict(n=(600, 600, 600), dtype="f64", T=100, gen="uniform", seed=6,
                     name="jacobi3d_fp64_600cubed_T100_paper_shape"),
    "fp32_1024": dict(n=(1024, 1024, 1024), dtype="f32", T=200, gen="mode", seed=3,
                      name="jacobi3d_fp32_1024cubed_T200_mode16"),
    "compressed1024": dict(n=(1024, 1024, 1024), dtype="f32", T=200, gen="mode", seed=3,
                           name="jacobi3d_fp32_1024cubed_T200_mode16_compressed_grid"),
    "batch256": dict(n=None, dtype="mixed", T=50, gen="batch", seed=4,
                     name="jacobi3d_batch_256grids_32to192_half_fp64_T50"),
    "poisson96": dict(n=(96, 96, 96), dtype="f64", T=500, gen="poisson", seed=5,
                      name="poisson_96cubed_h1over97_refine_to_1e-10"),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": M_S_FALLBACK}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1, 0
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    return dist, rank, ws, local


def reduce_max(dist, x: float, device) -> float:
    """Max of a per-rank float over all ranks (identity without a process
    group); `device` is where the collective's tensor lives (the GPU for
    NCCL, the CPU for gloo)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_glups(ws: int, lups_per_step: float, steps: int, max_ms: float) -> float:
    """Whole-job GLUP/s: every rank sweeps its own replica (weak scaling)."""
    return ws * lups_per_step * steps / (max_ms * 1e-3) / 1e9


def _make_grid(w, device):
    import torch
    from paper_1006_3148_gb300 import inputs
    nx, ny, nz = w["n"]
    dt = torch.float64 if w["dtype"] == "f64" else torch.float32
    if w["gen"] == "dirichlet_z0":
        return inputs.dirichlet_z0_grid(nx, ny, nz, w["seed"], dtype=dt, device=device)
    if w["gen"] == "uniform":
        return inputs.uniform_grid(nx, ny, nz, w["seed"], dtype=dt, device=device)
    return inputs.mode_grid(nx, ny, nz, w["seed"], dtype=dt, device=device)


def cpu_oracle_sample(w, budget_s: float):
    """Times the CPU oracle (as it stands) on the host cores: the workload's
    grid, sweeps in pairs until budget_s of CPU work.  Returns dict."""
    import numpy as np
    import oracle

    nx, ny, nz = w["n"]
    if w["dtype"] == "f32" and nx * ny * nz > 256 ** 3:
        nx = ny = nz = 256  # bounded sample of the FP32 workload (same recipe)
    ww = dict(w, n=(nx, ny, nz))
    A = _make_grid(ww, "cpu").numpy()
    B = np.empty_like(A)
    oracle.jacobi(A, B, 2)  # first touch / warm
    sweeps, t0 = 0, time.perf_counter()
    while True:
        oracle.jacobi(A, B, 2)
        sweeps += 2
        dt = time.perf_counter() - t0
        if dt >= budget_s or sweeps >= w["T"]:
            break
    g = nx * ny * nz * sweeps / dt / 1e9
    cores = oracle.threads()
    # the same oracle on one core: two sweeps of the same grid
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.jacobi(A, B, 2)
    g1 = nx * ny * nz * 2 / (time.perf_counter() - t1) / 1e9
    oracle.set_threads(cores)
    return {"value": g, "unit": "GLUP/s", "cores": cores, "kind": "oracle",
            "sample": "%dx%dx%d %s grid of the workload recipe, %d sweeps in %.1f s" % (
                nx, ny, nz, w["dtype"], sweeps, dt),
            "single_thread": {"value": g1, "unit": "GLUP/s", "sample": "2 sweeps of the same grid on 1 core"}}


# ------------------------------------------------------------------ context
class Ctx:
    """Process placement: rank, world size, local GPU, and the process group
    (None for a single process)."""

    def __init__(self, gpu: bool):
        self.dist, self.rank, self.ws, self.local = _dist()
        self.dev = None
        if gpu:
            import torch
            if self.dist is not None:
                torch.cuda.set_device(self.local)
                self.dist.init_process_group("nccl")
            self.dev = torch.device("cuda", torch.cuda.current_device())

    def barrier(self):
        import torch
        torch.cuda.synchronize()
        if self.dist is not None:
            self.dist.barrier()
        torch.cuda.synchronize()

    def close(self):
        if self.dist is not None and self.dev is not None:
            self.dist.barrier()
            self.dist.destroy_process_group()


def _parallelism(ws: int) -> str:
    return "replicas" if ws > 1 else "single"


def grid_config(w, ws: int) -> dict:
    """The workload's config keys, identical in both arms."""
    nx, ny, nz = w["n"]
    es = 8 if w["dtype"] == "f64" else 4
    gb = (nx + 2) * (ny + 2) * (nz + 2) * es / 1e9
    held = "one %.2f GB grid in one buffer" % gb if "compressed_grid" in w["name"] else "two %.2f GB grids" % gb
    return {"workload": w["name"], "nx": nx, "ny": ny, "nz": nz, "T": w["T"], "parallelism": _parallelism(ws),
            "l2": "inputs larger than L2 (%s)" % held}


def batch_config(w, ws: int) -> dict:
    from paper_1006_3148_gb300 import inputs
    dims, f32 = inputs.batch_dims(256, seed=w["seed"])
    nbytes = sum((nx + 2) * (ny + 2) * (nz + 2) * (4 if f else 8) for (nx, ny, nz), f in zip(dims, f32))
    return {"workload": w["name"], "grids": len(dims), "T": w["T"], "fp32_grids": int(sum(f32)),
            "cells": int(sum(nx * ny * nz for nx, ny, nz in dims)), "parallelism": _parallelism(ws),
            "l2": "inputs larger than L2 (%.2f GB of grids)" % (2 * nbytes / 1e9)}


def poisson_config(w, ws: int) -> dict:
    return {"workload": w["name"], "nx": w["n"][0], "ny": w["n"][1], "nz": w["n"][2], "inner_sweeps": w["T"],
            "tol": 1e-10, "parallelism": _parallelism(ws)}


def _ref_line(args, w, value, unit, hib, ms_per_step, dtype, config, cores, sample):
    return {
        "impl": "reference", "metric": METRIC if unit == "GLUP/s" else POISSON_METRIC, "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": hib, "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference(args, w):
    """The CPU oracle as it stands, timed on the host cores on a bounded
    sample of the workload per step; rank 0 only."""
    ctx = Ctx(gpu=False)
    if ctx.rank != 0:
        return None
    import numpy as np
    import oracle
    from paper_1006_3148_gb300 import inputs

    cores = oracle.threads()
    if w["gen"] == "batch":
        # per step: the next 4 grids of the batch, T sweeps each
        dims, f32 = inputs.batch_dims(256, seed=w["seed"])
        grids = [(g, inputs.uniform_grid(*d, seed=1000 + g).to(
            __import__("torch").float32 if f32[g] else __import__("torch").float64).numpy())
            for g, d in enumerate(dims)]
        per_step = 4

        def step(i):
            lups = 0
            for g, a in grids[(per_step * i) % 256:(per_step * i) % 256 + per_step]:
                oracle.jacobi(a.copy(), np.empty_like(a), w["T"])
                lups += a[1:-1, 1:-1, 1:-1].size * w["T"]
            return lups
        for i in range(args.warmup):
            step(i)
        t0, lups = time.perf_counter(), 0
        for i in range(args.steps):
            lups += step(args.warmup + i)
        dt = time.perf_counter() - t0
        g = lups / dt / 1e9
        line = _ref_line(args, w, g, "GLUP/s", True, dt * 1e3 / args.steps, "f64+f32", batch_config(w, ctx.ws),
                         cores, "%d grids of the batch per step (next in order), %d sweeps each" % (per_step, w["T"]))
    elif w["gen"] == "poisson":
        # one full refinement solve gives the outer-step count; each timed
        # step is one outer step (residual + inner sweeps + update); the
        # value is the time per outer step x the outer steps of the solve
        n = w["n"][0]
        hg = 1.0 / (n + 1)
        f = inputs.normal_rhs(n, n, n, seed=w["seed"]).numpy()
        u = np.zeros_like(f)
        st, outer_full, rel = oracle.refine(u, f, hg, 1e-10, w["T"], 400)
        u = np.zeros_like(f)
        for _ in range(args.warmup):
            oracle.refine(u, f, hg, 0.0, w["T"], 1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.refine(u, f, hg, 0.0, w["T"], 1)
        per_outer = (time.perf_counter() - t0) / args.steps
        value = per_outer * outer_full
        line = _ref_line(args, w, value, "s", False, per_outer * 1e3, "f64+f32", poisson_config(w, ctx.ws), cores,
                         "one outer refinement step per step (%d inner FP32 sweeps + FP64 residual and update); "
                         "value = time per outer step x %d outer steps of a full oracle solve" % (w["T"], outer_full))
    else:
        nx, ny, nz = w["n"]
        A = _make_grid(w, "cpu").numpy()
        B = np.empty_like(A)
        per_step = 2  # bounded sample per step: 2 sweeps of the full grid
        for _ in range(args.warmup):
            oracle.jacobi(A, B, per_step)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.jacobi(A, B, per_step)
        dt = time.perf_counter() - t0
        g = nx * ny * nz * per_step * args.steps / dt / 1e9
        line = _ref_line(args, w, g, "GLUP/s", True, dt * 1e3 / args.steps, w["dtype"], grid_config(w, ctx.ws), cores,
                         "%d sweeps per step of the %dx%dx%d grid" % (per_step, nx, ny, nz))
    return line


def _kernel_name(J, kernel: int, dtype: str) -> str:
    return {J.KERNEL_TB: "tb_pass_kernel", J.KERNEL_PLAIN: "plain_pass_kernel", J.KERNEL_PLAIN_X2: "plain_x2_kernel",
            J.KERNEL_TB_CTA: "tbc4_pass_kernel" if dtype == "f32" else "tbc_pass_kernel",
            J.KERNEL_TB_REG: "tbr_pass_kernel", J.KERNEL_TB_CHAIN: "tbx_pass_kernel"}[kernel]


def run_ours(args, w, ctx, sub=False):
    """One step = one jacobi_sweep call of T sweeps on the workload's grid.
    sub: a secondary line inside the default run (no end-to-end, blocked
    comparison or CPU baseline)."""
    import torch
    from paper_1006_3148_gb300 import jacobi as J

    dist, rank, ws, dev = ctx.dist, ctx.rank, ctx.ws, ctx.dev
    nx, ny, nz = w["n"]
    T = w["T"]
    es = 8 if w["dtype"] == "f64" else 4
    lups_step = nx * ny * nz * T
    dt = torch.float64 if w["dtype"] == "f64" else torch.float32

    h = J.Handle(nx, ny, nz, dt)
    A = _make_grid(w, dev)
    B = torch.empty_like(A)
    tune_glups = None
    if args.plan and not sub:
        f = args.plan.split(":")
        ring = int(f[5]) if len(f) > 5 else 0
        threads = int(f[6]) if len(f) > 6 else 0
        J.jacobi_set_plan(h, {"tb": J.KERNEL_TB, "plain": J.KERNEL_PLAIN, "x2": J.KERNEL_PLAIN_X2,
                              "cta": J.KERNEL_TB_CTA, "reg": J.KERNEL_TB_REG, "chain": J.KERNEL_TB_CHAIN}[f[0]], int(f[1]), int(f[2]), int(f[3]), int(f[4]), ring, threads)
    elif not args.no_tune:
        sa, sb = torch.empty_like(A), torch.empty_like(A)
        tune_glups = J.jacobi_tune(h, sa, sb)
        del sa, sb
        torch.cuda.empty_cache()
    plan = J.jacobi_get_plan(h)
    stream = torch.cuda.current_stream()

    J.jacobi_profile_enable(h, True)
    for _ in range(args.warmup):
        J.jacobi_sweep(h, A, B, T, stream)
    ctx.barrier()
    J.jacobi_profile_read(h)
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    ctx.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        J.jacobi_sweep(h, A, B, T, stream)
    e1.record(stream)
    ctx.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    prof = J.jacobi_profile_read(h)
    assert J.jacobi_get_status(h) == 0, "device status word set during the timed region"
    ms = reduce_max(dist, ms, dev)
    value = aggregate_glups(ws, lups_step, args.steps, ms)

    # ---- roofline of the dominant kernel (the pass kernel), live events
    peaks, peak_src = _peaks()
    m_s = float(peaks.get("hbm_gbs", M_S_FALLBACK))
    n_pass = prof["pass_launches"]
    pass_ms = prof["pass_ms"] / max(1, n_pass)
    passes_per_step = n_pass / args.steps
    lup_launch = nx * ny * nz * (T / passes_per_step)
    bytes_launch = 2.0 * es * nx * ny * nz  # read src once, write dst once
    hbm_ach = bytes_launch / (pass_ms * 1e-3) / 1e9
    clk = (clocks or {}).get("sm_mhz") or SM_MAX_MHZ
    roof = None
    if w["dtype"] == "f64":
        # FP64 sweeps are bound on chip: three FP64-pipe additions per LUP
        # (the other two and the division by 6 run on the integer pipe),
        # whose ALU instructions are the binding unit
        kname = _kernel_name(J, plan["kernel"], w["dtype"])
        fp64_ach = FP64_PIPE_ADDS * lup_launch / (pass_ms * 1e-3) / 1e12
        fp64_peak = FP64_LANES_PER_SM_CLK * SMS * SM_MAX_MHZ * 1e6 / 1e12
        fp64 = {"achieved": fp64_ach, "peak": fp64_peak, "unit": "T adds/s", "frac": fp64_ach / fp64_peak,
                "note": "FP64 pipe: 2 lanes/SM/clk x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s FMA-counted); "
                        "%d FP64-pipe additions per LUP" % FP64_PIPE_ADDS}
        hbm = {"achieved": hbm_ach, "peak": m_s, "unit": "GB/s", "frac": hbm_ach / m_s, "peak_source": peak_src}
        alu = MEASURED_ALU.get((kname, w["dtype"]))
        if alu is not None:
            alu_ach = alu[0] * lup_launch / (pass_ms * 1e-3) / 1e12
            alu_peak = ALU_LANES_PER_SM_CLK * SMS * SM_MAX_MHZ * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "T int-ops/s",
                    "frac": alu_ach / alu_peak, "traffic": None,
                    "note": "integer ALU pipe: 64 lanes/SM/clk x 152 SMs x 2070 MHz; achieved = %.0f ALU lane "
                            "instructions per LUP (%s) x LUP/s" % alu,
                    "fp64_pipe": fp64, "hbm": hbm}
        elif fp64["frac"] > hbm["frac"]:
            roof = dict(fp64, bound="alu", unit="TFLOP/s", traffic=None, hbm=hbm)
    if roof is None:
        roof = {"bound": "hbm", "achieved": hbm_ach, "peak": m_s, "unit": "GB/s", "frac": hbm_ach / m_s,
                "traffic": None, "peak_source": peak_src,
                "note": "algorithmic bytes: read and write the grid once per pass (2 x %d B per cell)" % es}
    roof["kernel"] = _kernel_name(J, plan["kernel"], w["dtype"])
    roof["avg_launch_ms"] = pass_ms
    roof["sm_mhz_during"] = clk
    measured = MEASURED_TRAFFIC.get((roof["kernel"], w["dtype"], plan["depth"]))
    if measured is not None:
        # bytes per LUP of the captured launch x the LUPs of one launch here
        roof["traffic"] = measured[0] * lup_launch
        roof["traffic_source"] = measured[1] + " (bytes per LUP x LUPs of this launch)"

    p0 = m_s / (2.0 * es)  # Eq. (2) for element size es
    line = {
        "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": w["dtype"], "data": "synthetic",
        "config": grid_config(w, ws), "plan": plan,
        "hbm_roofline": {"P0_glups": p0, "per_pass_frac": value / ws / p0,
                         "effective_frac": value / ws / (p0 * plan["depth"]), "M_s_gbs": m_s,
                         "peak_source": peak_src},
        "roofline": roof,
        "gpu_launches": prof["pass_launches"] + prof["other_launches"],
        "clocks": clocks,
    }
    if tune_glups is not None:
        line["tuner_best_glups"] = tune_glups

    # ---- comparison kernels, outside value: the scalar single-pass kernel
    # (code balance of Eq. (2)) and a temporally blocked pass of fixed depth
    if rank == 0 and not args.no_plain:
        def glups_of(kernel, *fields):
            hp = J.Handle(nx, ny, nz, dt)
            J.jacobi_set_plan(hp, kernel, *fields)
            Tp = min(T, 20)
            J.jacobi_sweep(hp, A, B, Tp, stream)
            torch.cuda.synchronize()
            e0.record(stream)
            J.jacobi_sweep(hp, A, B, Tp, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            hp.close()
            return nx * ny * nz * Tp / (e0.elapsed_time(e1) * 1e-3) / 1e9, Tp
        gp, Tp = glups_of(J.KERNEL_PLAIN)
        line["plain"] = {"value": gp, "unit": "GLUP/s", "sweeps": Tp, "per_pass_frac": gp / p0}
        line["tuned_vs_plain"] = (value / ws) / gp
        if not sub:
            bd = BLOCKED_REF[w["dtype"]]
            gb, Tb = glups_of(*bd)
            line["blocked"] = {"value": gb, "unit": "GLUP/s", "sweeps": Tb,
                               "plan": dict(zip(("kernel", "depth", "bx", "by", "bz", "ring", "threads"), bd)),
                               "hbm_bytes_per_lup_ideal": 2.0 * es / bd[1]}

    # ---- end to end through the host-buffer entry point
    if not args.no_e2e and not sub:
        host_in = A.cpu().pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        del A, B
        torch.cuda.empty_cache()
        J.jacobi_profile_enable(h, False)
        for _ in range(max(2, args.warmup)):  # warm-up: device grids of the host entry point, pinned pages
            J.jacobi_sweep_host(h, host_in, host_out, T, stream)
        ctx.barrier()
        ke = max(1, min(args.steps, 3))
        calls = []
        t0 = time.perf_counter()
        for _ in range(ke):
            tc = time.perf_counter()
            J.jacobi_sweep_host(h, host_in, host_out, T, stream)
            calls.append((time.perf_counter() - tc) * 1e3)
        dt_e = time.perf_counter() - t0
        dt_e = reduce_max(dist, dt_e, dev)
        nbytes = host_in.numel() * es
        line["e2e"] = {"value": ws * lups_step * ke / dt_e / 1e9, "unit": "GLUP/s", "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes, "steps": ke, "call_ms": calls}
        del host_in, host_out
    else:
        del A, B

    # ---- CPU oracle baseline on the host cores (rank 0, N = 1 only)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not sub:
        line["cpu_baseline"] = cpu_oracle_sample(w, args.cpu_budget)

    h.close()
    torch.cuda.empty_cache()
    return line


def run_batch(args, w, ctx, sub=False):
    """256 independent grids (sizes U{32..192} per axis, half FP64 / half
    FP32, interior and halo U[0,1), T = 50 each): one step = one
    jacobi_batch_run (a CUDA graph: halo copy, then one launch per sweep over
    all grids, or one persistent launch, as the batch tuner chose)."""
    import torch
    import numpy as np
    from paper_1006_3148_gb300 import inputs
    from paper_1006_3148_gb300 import jacobi as J

    dist, rank, ws, dev = ctx.dist, ctx.rank, ctx.ws, ctx.dev
    dims, f32 = inputs.batch_dims(256, seed=w["seed"])
    T = w["T"]
    dts = [torch.float32 if f else torch.float64 for f in f32]
    b = J.Batch(dims, dts, [T] * len(dims))
    A = [inputs.uniform_grid(*d, seed=1000 + g, dtype=torch.float64, device=dev).to(dts[g])
         for g, d in enumerate(dims)]
    B = [torch.empty_like(x) for x in A]
    tune = None
    if args.batch_fp32_depth:
        J.jacobi_batch_set_fp32_depth(b, args.batch_fp32_depth)
    if not args.no_tune:
        sa = [torch.empty_like(x) for x in A]
        sb = [torch.empty_like(x) for x in A]
        tune = J.jacobi_batch_tune(b, sa, sb)
        del sa, sb
        torch.cuda.empty_cache()
    info = J.jacobi_batch_get_info(b)
    eng = J.jacobi_batch_get_engine(b)
    depth32 = J.jacobi_batch_get_fp32_depth(b)
    sweeps_engine = eng["engine"] == J.BATCH_SWEEPS
    launches_per_run = (1 + T) if sweeps_engine else 2
    passes32 = T
    if depth32 > 1:
        # FP32 grids in blocked passes: one launch per pass and row-pitch parity
        passes32 = len(J.jacobi_plan_passes(T, depth32))
        pitches = {(nx + 2) % 2 for (nx, ny, nz), f in zip(dims, f32) if f}
        launches_per_run += passes32 * len(pitches)
    lups = float(sum(nx * ny * nz for nx, ny, nz in dims)) * T
    lups64 = float(sum(nx * ny * nz for (nx, ny, nz), f in zip(dims, f32) if not f)) * T
    # algorithmic bytes: read and write each cell once per sweep (FP64, and
    # FP32 at depth 1) or once per blocked pass (FP32 at depth > 1)
    bytes_alg = float(sum(2 * 8 * nx * ny * nz for (nx, ny, nz), f in zip(dims, f32) if not f)) * T + \
        float(sum(2 * 4 * nx * ny * nz for (nx, ny, nz), f in zip(dims, f32) if f)) * passes32
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        J.jacobi_batch_run(b, A, B, stream)
    ctx.barrier()
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    ctx.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        J.jacobi_batch_run(b, A, B, stream)
    e1.record(stream)
    ctx.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    assert J.jacobi_batch_get_status(b) == 0
    ms = reduce_max(dist, ms, dev)
    step_s = ms * 1e-3 / args.steps
    value = ws * lups / step_s / 1e9
    peaks, peak_src = _peaks()
    m_s = float(peaks.get("hbm_gbs", M_S_FALLBACK))
    hbm_ach = bytes_alg / step_s / 1e9
    alu_peak = FP64_LANES_PER_SM_CLK * SMS * SM_MAX_MHZ * 1e6 / 1e12
    alu_ach = FP64_PIPE_ADDS * lups64 / step_s / 1e12
    if alu_ach / alu_peak > hbm_ach / m_s:
        roof = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_ach / alu_peak,
                "traffic": None, "note": "FP64 pipe, %d FP64-pipe additions per FP64 LUP (two additions and the "
                "division run on the integer pipe); the launch also sweeps the FP32 grids" % FP64_PIPE_ADDS,
                "hbm": {"achieved": hbm_ach, "peak": m_s, "unit": "GB/s", "frac": hbm_ach / m_s}}
    else:
        roof = {"bound": "hbm", "achieved": hbm_ach, "peak": m_s, "unit": "GB/s", "frac": hbm_ach / m_s,
                "traffic": None, "peak_source": peak_src}
    roof["kernel"] = "batch_sweep_kernel" if sweeps_engine else "batch_kernel"
    if sweeps_engine and depth32 == 1 and BATCH_SWEEP_TRAFFIC is not None:
        # DRAM bytes per LUP of one sweep launch over the batch (ncu capture)
        roof["traffic"] = BATCH_SWEEP_TRAFFIC[0] * lups / T
        roof["traffic_source"] = BATCH_SWEEP_TRAFFIC[1]
    # the halo copy is ~1 % of a step; the rest is the sweep launches
    roof["avg_launch_ms"] = step_s * 1e3 / (T if sweeps_engine else 1)
    line = {
        "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": batch_config(w, ws),
        "plan": {"engine": "sweeps" if sweeps_engine else "persistent", "fp32_depth": depth32,
                 **({"planes_per_thread": eng["kz"]} if sweeps_engine else
                    {"tile": [info["bx"], info["by"], info["bz"]], "items": info["items"],
                     "persistent_ctas": info["blocks"]})},
        "roofline": roof, "gpu_launches": launches_per_run * args.steps, "clocks": clocks,
    }
    if tune is not None:
        line["tuner_best_glups"] = tune
    if not args.no_e2e and not sub:
        hosts = [x.cpu().pin_memory() for x in A]
        outs_h = [torch.empty_like(x).pin_memory() for x in hosts]
        ctx.barrier()
        ke = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(ke):
            for g in range(len(A)):
                A[g].copy_(hosts[g], non_blocking=True)
            outs = J.jacobi_batch_run(b, A, B, stream)
            for g in range(len(A)):
                outs_h[g].copy_(outs[g], non_blocking=True)
            torch.cuda.synchronize()
        dt_e = time.perf_counter() - t0
        nbytes = sum(x.numel() * x.element_size() for x in hosts)
        line["e2e"] = {"value": ws * lups * ke / dt_e / 1e9, "unit": "GLUP/s", "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes, "steps": ke}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not sub:
        import oracle
        t0 = time.perf_counter()
        done = 0.0
        ng = 0
        for g, (nx, ny, nz) in enumerate(dims):
            a = inputs.uniform_grid(nx, ny, nz, seed=1000 + g).to(dts[g]).numpy()
            oracle.jacobi(a, np.empty_like(a), T)
            done += nx * ny * nz * T
            ng += 1
            if time.perf_counter() - t0 > args.cpu_budget:
                break
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / dt / 1e9, "unit": "GLUP/s", "cores": oracle.threads(),
                                "kind": "oracle", "sample": "first %d of the 256 grids, %d sweeps each" % (ng, T)}
    b.close()
    del A, B
    torch.cuda.empty_cache()
    return line


def run_compressed(args, w, ctx, sub=False):
    """The FP32 1024^3 workload swept in ONE buffer (compressed grid,
    jacobi_sweep_compressed): one step = T sweeps, the grid moving between
    its two positions in the buffer pass by pass."""
    import torch
    from paper_1006_3148_gb300 import jacobi as J

    dist, ws, dev = ctx.dist, ctx.ws, ctx.dev
    nx, ny, nz = w["n"]
    T = w["T"]
    es = 8 if w["dtype"] == "f64" else 4
    dt = torch.float64 if w["dtype"] == "f64" else torch.float32
    h = J.Handle(nx, ny, nz, dt)
    if args.cg_plan:
        J.jacobi_compressed_set_plan(h, *(int(v) for v in args.cg_plan.split(":")))
    cg = J.jacobi_compressed_get_plan(h)
    U = J.compressed_buffer(h, device=dev)
    J.compressed_view(h, U, 1).copy_(_make_grid(w, dev))
    stream = torch.cuda.current_stream()
    pos = 1
    for _ in range(args.warmup):
        pos = J.jacobi_sweep_compressed(h, U, T, pos, stream)
    ctx.barrier()
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    ctx.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        pos = J.jacobi_sweep_compressed(h, U, T, pos, stream)
    e1.record(stream)
    ctx.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    assert J.jacobi_get_status(h) == 0, "device status word set during the timed region"
    ms = reduce_max(dist, ms, dev)
    value = aggregate_glups(ws, nx * ny * nz * T, args.steps, ms)
    passes = (T + cg["depth"] - 1) // cg["depth"]
    # one pass kernel per pass (plus a counter reset); its algorithmic bytes:
    # the grid read and written once
    pass_ms = ms / args.steps / passes
    peaks, peak_src = _peaks()
    m_s = float(peaks.get("hbm_gbs", M_S_FALLBACK))
    hbm_ach = 2.0 * es * nx * ny * nz / (pass_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": hbm_ach, "peak": m_s, "unit": "GB/s", "frac": hbm_ach / m_s,
            "traffic": None, "peak_source": peak_src, "kernel": "cg_f32_kernel" if es == 4 else "cg_f64_kernel",
            "avg_launch_ms": pass_ms,
            "note": "algorithmic bytes: read and write the grid once per pass (2 x %d B per cell); pass time = "
                    "step time / passes (one launch per pass and a counter reset)" % es}
    measured = MEASURED_TRAFFIC.get((roof["kernel"], w["dtype"], cg["depth"]))
    if measured is not None and cg["bz"] == 128:
        # bytes per LUP of the captured launch x the LUPs of one pass here
        roof["traffic"] = measured[0] * nx * ny * nz * cg["depth"]
        roof["traffic_source"] = measured[1] + " (bytes per LUP x LUPs of this pass)"
    grid_bytes = (nx + 2) * (ny + 2) * (nz + 2) * es
    line = {
        "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": w["dtype"], "data": "synthetic", "config": grid_config(w, ws),
        "plan": dict(cg, memory_vs_one_grid=U.numel() * es / grid_bytes, memory_vs_two_grids=U.numel() * es / (2 * grid_bytes)),
        "roofline": roof, "gpu_launches": passes * args.steps, "clocks": clocks,
    }
    h.close()
    del U
    torch.cuda.empty_cache()
    return line


def run_poisson(args, w, ctx):
    """-Lap u = f, 96^3, h = 1/97, f ~ N(0,1), zero halo: time to a relative
    residual of 1e-10 by mixed-precision refinement (FP64 residual/update,
    500 FP32 inner sweeps per outer step) and by plain FP64 Jacobi.  One
    step = one refinement solve from u = 0."""
    import torch
    from paper_1006_3148_gb300 import inputs
    from paper_1006_3148_gb300 import jacobi as J

    n = w["n"][0]
    hg = 1.0 / (n + 1)
    f = inputs.normal_rhs(n, n, n, seed=w["seed"]).to(ctx.dev)
    H = J.Handle(n, n, n, torch.float64)
    u = torch.zeros_like(f)
    for _ in range(args.warmup):
        u.zero_()
        J.jacobi_refine(H, u, f, hg, 1e-10, w["T"], 400)
    torch.cuda.synchronize()
    times, outers = [], []
    J.jacobi_profile_enable(H, True)
    J.jacobi_profile_read(H)
    for _ in range(args.steps):
        u.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, outer, rel = J.jacobi_refine(H, u, f, hg, 1e-10, w["T"], 400)
        times.append(time.perf_counter() - t0)
        outers.append(outer)
        assert st == 0
    t_ref = statistics.median(times)
    launches = J.jacobi_profile_read(H)["other_launches"]
    inner_lups = float(n ** 3) * w["T"] * outers[-1]
    # plain FP64 Jacobi to the same residual: chunks of 2000 sweeps
    u.zero_()
    tmp = torch.empty_like(u)
    sweeps, t0 = 0, time.perf_counter()
    rel_p = 1.0
    while rel_p > 1e-10 and sweeps < 200000:
        out = J.jacobi_poisson_jacobi(H, u, tmp, f, hg, 2000)
        sweeps += 2000
        if out is not u:
            u, tmp = tmp, u
        rel_p = J.jacobi_poisson_residual(H, u, f, hg)
    t_plain = time.perf_counter() - t0
    return {
        "metric": POISSON_METRIC, "value": t_ref, "unit": "s", "n_gpus": ctx.ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ref * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": poisson_config(w, ctx.ws), "outer_steps": outers[-1], "final_rel": rel,
        "refine_inner_glups": inner_lups / t_ref / 1e9,
        "plain_fp64_jacobi": {"seconds": t_plain, "sweeps": sweeps, "final_rel": rel_p,
                              "glups": float(n ** 3) * sweeps / t_plain / 1e9},
        "speedup_refine_vs_plain_fp64": t_plain / t_ref,
        "gpu_launches": launches,
    }


SUB_KEYS = ("value", "unit", "steps", "warmup", "ms_per_step", "dtype", "config", "plan", "hbm_roofline", "roofline",
            "clocks", "gpu_launches", "tuner_best_glups", "plain", "tuned_vs_plain")


def sub_line(line: dict) -> dict:
    """The keys of a secondary workload's line kept inside the default line."""
    return {k: line[k] for k in SUB_KEYS if k in line}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fp64_512", choices=sorted(WORKLOADS))
    ap.add_argument("--plan", default=None, help="force a plan kernel:depth:bx:by:bz[:ring[:threads]], kernel tb, cta, "
                    "reg, chain (ring = CTAs), plain or x2, e.g. tb:4:64:16:64:8, cta:4:64:32:64:0:512 or x2:1:32:8:16")
    ap.add_argument("--cg-plan", default=None, help="compressed grid plan depth:bz:waves")
    ap.add_argument("--batch-fp32-depth", type=int, default=0, help="FP32 depth of the batch (with --no-tune)")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="default workload only: skip the FP32 1024^3 and "
                    "256-grid batch lines measured beside it")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--n", type=int, default=None, help="override the cubic interior size (profiling cases)")
    ap.add_argument("--T", type=int, default=None, help="override the sweeps per step (profiling cases)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    w = dict(WORKLOADS[args.workload])
    resized = args.n is not None or args.T is not None
    if args.n is not None:
        w["n"] = (args.n, args.n, args.n)
        w["name"] += "_resized_%d" % args.n
    if args.T is not None:
        w["T"] = args.T
        w["name"] += "_T%d" % args.T
    if args.impl == "reference":
        line = run_reference(args, w)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0
    ctx = Ctx(gpu=True)
    try:
        if w["gen"] == "batch":
            line = run_batch(args, w, ctx)
        elif w["gen"] == "poisson":
            line = run_poisson(args, w, ctx)
        elif args.workload == "compressed1024":
            line = run_compressed(args, w, ctx)
        else:
            line = run_ours(args, w, ctx)
            if args.workload == "fp64_512" and not resized and not args.no_sub and not args.plan:
                # the FP32 and batched workloads, measured in the same run
                line["fp32_1024"] = sub_line(run_ours(args, dict(WORKLOADS["fp32_1024"]), ctx, sub=True))
                line["batch256"] = sub_line(run_batch(args, dict(WORKLOADS["batch256"]), ctx, sub=True))
                line["compressed_fp32_1024"] = sub_line(
                    run_compressed(args, dict(WORKLOADS["compressed1024"]), ctx, sub=True))
        if ctx.rank == 0:
            print(json.dumps(line), flush=True)
    finally:
        ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
