"""Benchmark: MSP-preconditioned FGMRES solves of the SPE10-shaped synthetic Jacobian.

One step = one Newton-like linear solve through the C ABI: the step's Jacobian values
(same pattern, off-diagonal couplings perturbed by U[0.95, 1.05], diagonal blocks
rebalanced, see synthetic.perturb_values) are loaded with msp_update_values (the first
step uses the values the solver was set up with), then msp_solve runs the adaptive setup decision of Section 3.2
(SETUP again iff the previous solve took more than mu iterations) and FGMRES(30) with
the multi-stage preconditioner to relative residual 1e-6.

Workload (default): 60x220x85 cells (1,122,000) + 4 wells, 4 unknowns per cell, FP64,
seed 2209 -- the plain FP64 GPU path.  The matrix (about 1 GB of values) and every
step's values and right-hand side are resident in HBM before the timed region (inputs
larger than L2, no flush needed).  `e2e` repeats the measurement through the host-buffer
entry points (values and right-hand side copied in from pinned host memory, the solution
copied out, every step).

`--impl reference` times the CPU oracle (single thread) on the same workload; each of
its steps is one FGMRES iteration of the oracle on the full matrix, and its solves/s are
extrapolated as 1 / (setup share + It * seconds per iteration) with the GPU solve's
iteration count and setup frequency (stated in `cpu_baseline.sample`).

Multi-GPU: the solve does not shard, so `--gpus N` (under torchrun) runs N independent
replicas, one per GPU, and reports the total solves/s (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s to 1e-6 rel. residual (1.1M cells x4)"
# timing call sites of the library (msp_stats_*) -> the kernel each one launches
SITE_KERNELS = {
    "krylov_spmv": "bsr_spmv_kernel", "api_spmv": "bsr_spmv_kernel",
    "krylov_multi_dot": "multi_dot1_kernel", "krylov_basis_dot": "multi_dot1_kernel",
    "krylov_finalize_dot": "multi_dot1_kernel",
    "krylov_multi_axpy": "multi_axpy_norm_kernel",
    "stageN_bgs_sweep": "bgs_colour_kernel", "stageN_scale": "nscale_kernel",
    "stageP_residual_restrict": "bsr_restrict_p_kernel",
    "stageP_correct_residual": "bsr_col0_update_kernel",
    "stageP_prolong": "prolong_p_kernel",
    "stageR_bilu_fwd": "bilu_fwd_kernel", "stageR_bilu_bwd": "bilu_bwd_kernel",
    "amg_prolong": "prolong_add_kernel", "coarse_gemv": "dense_gemv_kernel",
    "batch_spmv": "bsr_spmv_kernel",
    "batch_multi_dot": "seg_multi_dot2_kernel", "batch_finalize_dot": "seg_multi_dot_kernel",
    "batch_multi_axpy": "seg_multi_axpy_norm_kernel",
}
SITE_PREFIX_KERNELS = {"amg_gs_pre_l": "ell_gs_colour_kernel",
                       "amg_gs_post_l": "ell_gs_colour_kernel",
                       "amg_gs_csr_pre_l": "csr_gs_colour_kernel",
                       "amg_gs_csr_post_l": "csr_gs_colour_kernel",
                       "amg_residual_restrict_l": "ell_residual_restrict_kernel",
                       "amg_pjac_l": "jacobi_sweep_kernel",
                       "amg_pgs_no_l": "pgs_no_sweep_kernel",
                       "amg_residual_restrict_csr_l": "csr_residual_restrict_kernel"}
TOL = 1e-6


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=6)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    p.add_argument("--smoother", default="pgs_mc", choices=["pgs_mc", "pjac", "pgs_no"],
                   help="AMG smoother: PGS-MC (the paper's), PJAC-NO or PGS-NO "
                        "(Section 5.1.1, Table 2)")
    p.add_argument("--colouring", default="alg41", choices=["alg41", "jp"],
                   help="Algorithms 4.1/4.2 (the paper's) or greedy in Jones-Plassmann "
                        "priority order (parallel rounds)")
    p.add_argument("--wells", default="rows", choices=["rows", "eliminate"],
                   help="wells as ordinary block rows of the solved system (default), or "
                        "eliminated by the Schur complement of A_WW before the solve")
    p.add_argument("--mu", type=int, default=180)
    p.add_argument("--autotune", action="store_true",
                   help="time the lanes per row of the AMG levels' ELL kernels at SETUP and "
                        "keep the fastest (msp_config.autotune)")
    p.add_argument("--nx", type=int, default=60)
    p.add_argument("--ny", type=int, default=220)
    p.add_argument("--nz", type=int, default=85)
    p.add_argument("--value-sets", type=int, default=4)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--mu0-steps", type=int, default=4,
                   help="solves timed with mu = 0 (plain MSP: SETUP before every solve)")
    p.add_argument("--profile-steps", type=int, default=0)
    p.add_argument("--mu-sweep", action="store_true",
                   help="SetupCalls / SetupRatio / Iter / Time against mu on a drifting "
                        "Newton-like sequence (Tables 3, 5, 7) instead of the benchmark")
    p.add_argument("--serve", action="store_true",
                   help="request-loop benchmark: Newton sequences of systems of many sizes "
                        "arriving over time, solved through the server (p50/p99 latency)")
    p.add_argument("--serve-reservoirs", type=int, default=8)
    p.add_argument("--serve-cells", type=float, nargs=2, default=[1e4, 2e6])
    p.add_argument("--serve-blocks", type=int, nargs=2, default=[4, 8])
    p.add_argument("--serve-rate", type=float, default=200.0,
                   help="offered requests per second (reservoir arrivals are Poisson at this "
                        "rate divided by the mean Newton steps per reservoir)")
    p.add_argument("--serve-slots", type=int, nargs="+", default=[1, 4])
    p.add_argument("--serve-budget-gb", type=float, default=150.0)
    p.add_argument("--latency", action="store_true",
                   help="latency of single solves of the small 16x16x8, b = 3 system (C1: "
                        "launch- and latency-bound; p50/p99 over --steps solves)")
    p.add_argument("--batch", action="store_true",
                   help="batched instances: many uneven systems stacked block-diagonally and "
                        "solved together, against the same systems one at a time")
    p.add_argument("--batch-instances", type=int, default=64)
    p.add_argument("--batch-cells", type=float, nargs=2, default=[2e4, 5e5])
    p.add_argument("--batch-steps", type=int, default=2)
    p.add_argument("--batch-profile", action="store_true",
                   help="time every call site of one more batched step (stats mode 3)")
    p.add_argument("--time-steps", type=int, default=6)
    p.add_argument("--newton-steps", type=int, default=3)
    p.add_argument("--rel-step", type=float, default=0.15)
    p.add_argument("--rel-newton", type=float, default=0.02)
    return p.parse_args()


def workload_name(args):
    return ("spe10-shaped %dx%dx%d + 4 wells, 4x4 BSR, coupling blocks -T_ij (R_ij + 3 I) "
            "(R_ij ~ U[0.1,1]), Newton steps: couplings x U[0.95,1.05] with rebalanced "
            "diagonal blocks, %s%s") % (
        args.nx, args.ny, args.nz, "FP64" if args.precision == "fp64" else
        "FP32 preconditioner / FP64 Krylov",
        ", Jones-Plassmann-order colouring" if args.colouring == "jp" else "") + (
        ", AMG smoother %s" % {"pjac": "PJAC-NO", "pgs_no": "PGS-NO"}[args.smoother]
        if args.smoother != "pgs_mc" else "") + (
        ", wells eliminated (Schur complement)" if args.wells == "eliminate" else "")


def colouring_of(args, msp):
    return msp.MSP_COLOURING_JP if args.colouring == "jp" else msp.MSP_COLOURING_ALG41


def smoother_of(args, msp):
    return {"pgs_mc": msp.MSP_SMOOTHER_PGS_MC, "pjac": msp.MSP_SMOOTHER_PJAC,
            "pgs_no": msp.MSP_SMOOTHER_PGS_NO}[args.smoother]


# call sites that run on a branch of the preconditioner's graph, beside the coarse AMG
# levels: their device time overlaps other kernels' and is not part of the step's critical
# path, so they are reported apart and left out of the per-kernel table and the roofline
OVERLAPPED_SITES = {"krylov_basis_dot"}


def kernels_from_sites(sites):
    """{kernel: [launches, ms, bytes, flops]} summed over the call sites that launch it
    (containers such as the whole graph replay, and the overlapped sites, are left out)."""
    out = {}
    for site, rec in sites.items():
        if site in OVERLAPPED_SITES:
            continue
        n, ms, by = rec[:3]
        fl = rec[3] if len(rec) > 3 else 0.0
        k = SITE_KERNELS.get(site)
        if k is None:
            k = next((v for p, v in SITE_PREFIX_KERNELS.items() if site.startswith(p)), None)
        if k is None:
            continue
        acc = out.setdefault(k, [0, 0.0, 0.0, 0.0])
        acc[0] += n
        acc[1] += ms
        acc[2] += by
        acc[3] += fl
    return out


# FP64 FMA units: 152 SMs x 2 FMA per clock (the nominal 1.25 TFLOP/s FP64 of this part at
# 2070 MHz); the peak of a kernel bound by FP64 arithmetic, at the SM clock measured under load
FP64_FMA_PER_CLOCK_PER_SM = 2


def roofline_of(name, rec, peak_gbs, peak_kind, sms, sm_mhz, fma64_measured, live_ms, steps):
    """The binding roof of one kernel: HBM (algorithmic bytes / time against the measured
    copy bandwidth) or, where its algorithmic FP64 flops need longer at the FP64 FMA rate
    than its bytes need at the HBM rate, the FP64 ALU (flops / time against the derived FP64
    peak)."""
    n_l, tot_ms, tot_b, tot_f = rec
    t = (tot_ms / n_l) / 1000.0
    by, fl = tot_b / n_l, tot_f / n_l
    fp64_peak = sms * FP64_FMA_PER_CLOCK_PER_SM * 2 * sm_mhz * 1e6
    out = {"kernel": name, "algorithmic_bytes_per_launch": round(by, 1),
           "algorithmic_flops_per_launch": round(fl, 1), "avg_launch_ms": round(t * 1000, 5),
           "launches": n_l, "share_of_step": round(tot_ms / live_ms, 4),
           "hbm_GBps": round(by / t / 1e9, 1), "hbm_frac": round(by / t / 1e9 / peak_gbs, 4)}
    if fl > 0 and fl / fp64_peak > by / (peak_gbs * 1e9):
        out.update({"bound": "alu", "achieved": round(fl / t / 1e12, 4),
                    "peak": round(fp64_peak / 1e12, 4), "unit": "TFLOP/s",
                    "frac": round(fl / t / fp64_peak, 4),
                    "peak_kind": "derived: %d SMs x %d FP64 FMA/clock x 2 flops x %.0f MHz "
                                 "(measured FMA-chain kernel: %.4f TFLOP/s)" % (
                                     sms, FP64_FMA_PER_CLOCK_PER_SM, sm_mhz,
                                     fma64_measured / 1e12)})
    else:
        out.update({"bound": "hbm", "achieved": round(by / t / 1e9, 1), "peak": peak_gbs,
                    "unit": "GB/s", "frac": round(by / t / 1e9 / peak_gbs, 4),
                    "peak_kind": peak_kind})
    return out


def static_config(args, a):
    """The workload's configuration, the same in the native and the reference line."""
    return {"workload": workload_name(args), "cells": args.nx * args.ny * args.nz,
            "block_rows": a.nb, "nnzb": a.nnzb, "mu": args.mu, "restart": 30, "tol": TOL,
            "l2": "inputs larger than L2 (1 GB of values), no flush",
            "parallelism": "single GPU or independent replicas (one per GPU)"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.samples = []
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 6:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if not self.samples:
            return None
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if s[2 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def kernel_source_sha(kernel):
    """Hash of the source a kernel is compiled from: the whole .cu file in csrc/ that
    defines it (its helpers live there too) and the shared headers, so a committed ncu
    figure can be matched to the code it measured."""
    import glob
    import re
    csrc = os.path.join(ROOT, "paper_2208_08594_gb300", "csrc")
    for path in sorted(glob.glob(os.path.join(csrc, "*.cu"))):
        src = open(path).read()
        if re.search(r"__global__ void[^;{]*?\b%s\(" % re.escape(kernel), src):
            h = hashlib.sha256(src.encode())
            for hdr in ("common.cuh", "kernels.h"):
                with open(os.path.join(csrc, hdr)) as f:
                    h.update(f.read().encode())
            return h.hexdigest()[:16]
    return None


def traffic_for(kernel):
    """DRAM bytes (read + write) per launch of `kernel` at the benchmark size, from the
    committed ncu summary, if it was taken on the current source of that kernel (null
    otherwise)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        e = t.get(kernel)
        if e and e.get("kernel_source_sha") == kernel_source_sha(kernel):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def combine_over_ranks(times_ms):
    """Max over ranks of each local time (the slowest replica bounds the job); a no-op
    without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(times_ms)
    dev = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor(list(times_ms), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def total_throughput(steps, world, ms):
    """Whole-job solves/s: every replica solved `steps` systems within `ms`."""
    return steps * world / (ms / 1000.0)


def make_inputs(args, rank):
    from synthetic import grid_spe10, perturb_values, random_rhs
    a = grid_spe10(seed=2209 + rank, nx=args.nx, ny=args.ny, nz=args.nz)
    sets = [perturb_values(a, 5000 + 17 * rank + k) for k in range(args.value_sets)]
    rhs = [random_rhs(a, 7000 + 13 * rank + k) for k in range(args.value_sets)]
    return a, sets, rhs


def run_native(args):
    import torch
    import torch.distributed as dist

    import paper_2208_08594_gb300 as msp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    a, sets, rhs = make_inputs(args, rank)
    d_rp = torch.from_numpy(a.row_ptr).to(dev)
    d_ci = torch.from_numpy(a.col_idx).to(dev)
    d_sets = [torch.from_numpy(v.reshape(-1)).to(dev) for v in sets]
    d_v0 = d_sets[0]
    d_rhs = [torch.from_numpy(r).to(dev) for r in rhs]
    x = torch.zeros(a.n, dtype=torch.float64, device=dev)
    prec = msp.MSP_PRECISION_FP32 if args.precision == "fp32" else msp.MSP_PRECISION_FP64

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    opts = dict(mu=args.mu, precision=prec, colouring=colouring_of(args, msp),
                smoother=smoother_of(args, msp), autotune=int(args.autotune))
    if args.wells == "eliminate":
        solver = msp.WellEliminatedSolver(a.nb, a.b, a.n_wells, d_rp, d_ci, d_v0, **opts)
        inner = solver.solver
        reduced = {"reduced_block_rows": solver.wells.nr,
                   "reduced_nnzb": int(solver.wells.col_idx.numel())}
    else:
        solver = inner = msp.Solver(a.nb, a.b, d_rp, d_ci, d_v0, **opts)
        reduced = {}
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    nsets = len(d_sets)

    def step(k, infos):
        if k > 0:
            solver.update_values(d_sets[k % nsets])
        info = solver.solve(d_rhs[k % nsets], x, TOL)
        if info["status"] != 0:
            raise RuntimeError("solve failed: %s" % info)
        infos.append(info)

    warm = []
    for k in range(args.warmup):
        step(k, warm)

    # headline: the preconditioner replayed as its CUDA graph; every kernel launch is
    # counted, nothing is timed inside the region but the region itself
    msp.msp_stats_reset()
    msp.msp_stats_enable(1)
    clocks = ClockSampler(torch.cuda.current_device())
    infos = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(args.warmup + k, infos)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = msp.msp_stats_launches()

    # instrumented: the same steps again, the graph re-captured with a pair of CUDA event
    # nodes around every call site inside it and the launches outside it timed with
    # events on the solver stream: per-site device time of every kernel launch
    msp.msp_stats_reset()
    msp.msp_stats_enable(3)
    live_infos = []
    torch.cuda.synchronize()
    i0 = torch.cuda.Event(enable_timing=True)
    i1 = torch.cuda.Event(enable_timing=True)
    i0.record(stream)
    for k in range(args.steps):
        step(args.warmup + k, live_infos)
    i1.record(stream)
    torch.cuda.synchronize()
    live_ms = i0.elapsed_time(i1)
    live = msp.msp_stats_get()

    # plain MSP (mu = 0, the first CUDA rows of Tables 3, 5 and 7): every solve regenerates
    # the preconditioner (SETUP) before FGMRES; the same value sets, one solver per pass
    mu0 = None
    if args.mu0_steps > 0:
        mu0_solver = msp.Solver(a.nb, a.b, d_rp, d_ci, d_v0, mu=0, precision=prec,
                                colouring=colouring_of(args, msp),
                                smoother=smoother_of(args, msp))
        mu0_infos = []

        def mu0_step(k):
            mu0_solver.update_values(d_sets[k % nsets])
            info = mu0_solver.solve(d_rhs[k % nsets], x, TOL)
            if info["status"] != 0:
                raise RuntimeError("solve failed: %s" % info)
            mu0_infos.append(info)

        mu0_step(1)  # the first solve uses msp_setup's preconditioner: not timed
        mu0_infos.clear()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.mu0_steps):
            mu0_step(args.warmup + k)
        torch.cuda.synchronize()
        mu0_s = time.perf_counter() - t0
        # one more plain-MSP solve with every setup phase timed by CUDA events (not part of
        # the timed solves above): where a SETUP's time goes
        msp.msp_stats_reset()
        msp.msp_stats_enable(2)
        mu0_step(args.warmup + args.mu0_steps)
        mu0_infos.pop()
        msp.msp_stats_enable(0)
        setup_sites = {k: round(v[1], 2) for k, v in sorted(msp.msp_stats_get().items(),
                                                            key=lambda kv: -kv[1][1])
                       if k.startswith("setup:")}
        msp.msp_stats_reset()
        mu0_solver.close()
        t_set = sum(i["t_setup_ms"] for i in mu0_infos) / 1000.0
        mu0 = {"mu": 0, "solves": len(mu0_infos),
               "solves_per_s": round(len(mu0_infos) / mu0_s, 4),
               "ms_per_solve": round(1000.0 * mu0_s / len(mu0_infos), 1),
               "setup_calls": int(sum(i["setup_performed"] for i in mu0_infos)),
               "setup_ratio": round(t_set / mu0_s, 4),
               "setup_ms_mean": round(1000.0 * t_set / len(mu0_infos), 1),
               "iterations": [i["iterations"] for i in mu0_infos],
               "setup_phases_ms": setup_sites,
               "timed": "host wall clock around update_values + solve (SETUP inside the "
                        "solve, timed by the library as SetupRatio's numerator)"}

    # FMA ceilings of this GPU, measured now (the FP64 block kernels do one FMA per
    # 8-byte value and can be bound by the FP64 rate, not by HBM)
    fma64 = msp.msp_fma_rate(msp.MSP_PRECISION_FP64)
    fma32 = msp.msp_fma_rate(msp.MSP_PRECISION_FP32)

    # optional: the steps launched eagerly (no graph), every launch timed
    stats, prof_ms = {}, None
    if args.profile_steps > 0:
        msp.msp_stats_reset()
        msp.msp_stats_enable(2)
        prof_infos = []
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for k in range(args.profile_steps):
            step(args.warmup + k, prof_infos)
        p1.record(stream)
        torch.cuda.synchronize()
        prof_ms = p0.elapsed_time(p1) / args.profile_steps
        stats = msp.msp_stats_get()
    msp.msp_stats_enable(0)

    # end to end through the host-buffer entry points
    e2e = None
    if not args.no_e2e:
        pin_sets = [torch.from_numpy(v.reshape(-1)).pin_memory() for v in sets]
        pin_rhs = [torch.from_numpy(r).pin_memory() for r in rhs]
        pin_x = torch.zeros(a.n, dtype=torch.float64).pin_memory()
        e2e_infos = []
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        copy_stream = torch.cuda.Stream()
        if args.wells == "eliminate":
            stage_v = torch.empty_like(d_v0)
            stage_r = torch.empty(a.n, dtype=torch.float64, device=dev)
        for k in range(args.steps):
            kk = (args.warmup + k) % nsets
            if args.wells == "eliminate":
                # the full system's values and right-hand side in, the solution out
                stage_v.copy_(pin_sets[kk], non_blocking=True)
                solver.update_values(stage_v)
                stage_r.copy_(pin_rhs[kk], non_blocking=True)
                info = solver.solve(stage_r, x, TOL)
                pin_x.copy_(x, non_blocking=True)
            else:
                # the next step's values are copied on a second stream while this step
                # solves (pipelined, as a simulator would); each update waits for its copy
                if k == 0:
                    solver.stage_values_host(pin_sets[kk].numpy(), copy_stream)
                solver.update_values_staged(stream)
                if k + 1 < args.steps:
                    solver.stage_values_host(pin_sets[(kk + 1) % nsets].numpy(), copy_stream)
                info = solver.solve_host(pin_rhs[kk].numpy(), pin_x.numpy(), TOL)
            e2e_infos.append(info)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = f0.elapsed_time(f1)
        e2e = {"ms": e2e_ms, "h2d": (a.nnzb * a.b * a.b + a.n) * 8, "d2h": a.n * 8}

    # max over ranks
    ms, e2e_ms = combine_over_ranks([ms, e2e["ms"] if e2e else 0.0])
    if e2e:
        e2e["ms"] = e2e_ms
    solver_levels = inner.num_levels
    level_info = [msp.msp_level_info(inner.h, l) for l in range(solver_levels)]
    level_tiles = [msp.msp_level_tiles(inner.h, l) for l in range(solver_levels)]
    solver.close()
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return None

    total_solves = args.steps * world
    value = total_throughput(args.steps, world, ms)
    its = [i["iterations"] for i in infos]
    setups = sum(i["setup_performed"] for i in infos)
    peak, peak_kind = load_peaks()
    # Per kernel: the instrumented pass's call sites grouped by the kernel they launch;
    # the roofline is reported for the kernel with the most device time (the same
    # ranking as the shares of the ncu launch list under profiles/).
    kern = kernels_from_sites(live)
    roofline = None
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if kern:
        name, rec = max(kern.items(), key=lambda kv: kv[1][1])
        roofline = roofline_of(name, rec, peak, peak_kind, sms, sm_mhz, fma64, live_ms,
                               args.steps)
        roofline.update({"traffic": traffic_for(name),
                    "measured": "CUDA event pairs around every call site (one launch, or "
                                "the consecutive launches of one kernel over the colours of "
                                "a sweep), as event nodes inside the preconditioner's CUDA "
                                "graph and event records on the solver stream outside it, "
                                "over a second timed pass of the same steps"})
    kernels = {k: {"launches_per_step": round(v[0] / args.steps, 1),
                   "ms_per_step": round(v[1] / args.steps, 3),
                   "GBps": round(v[2] / (v[1] / 1000.0) / 1e9, 1) if v[1] > 0 else None,
                   "frac": round(v[2] / (v[1] / 1000.0) / 1e9 / peak, 4) if v[1] > 0 else None,
                   "TFLOPs": round(v[3] / (v[1] / 1000.0) / 1e12, 4)
                   if v[1] > 0 and v[3] > 0 else None}
               for k, v in sorted(kern.items(), key=lambda kv: -kv[1][1])}
    sites = {k: {"launches_per_step": round(v[0] / args.steps, 1),
                 "ms_per_step": round(v[1] / args.steps, 3),
                 "GBps": round(v[2] / (v[1] / 1000.0) / 1e9, 1) if v[1] > 0 else None,
                 **({"overlapped": True} if k in OVERLAPPED_SITES else {})}
             for k, v in sorted(live.items(), key=lambda kv: -kv[1][1])}
    eager = {k: {"launches": v[0], "ms": round(v[1], 3),
                 "GBps": round(v[2] / (v[1] / 1000.0) / 1e9, 1) if v[1] > 0 else None}
             for k, v in sorted(stats.items(), key=lambda kv: -kv[1][1])}
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32-precond/f64-krylov",
        "data": "synthetic (seeded SPE10-shaped Jacobian; SPE10 data not available)",
        "config": static_config(args, a),
        "run": {**reduced, "levels": solver_levels,
                   "level_sizes": [li[0] for li in level_info],
                   "level_nnz": [li[1] for li in level_info],
                   "level_colours": [li[2] for li in level_info],
                   "level_tiles": [list(t) for t in level_tiles],
                   "autotune": bool(args.autotune),
                   "amg_operator_complexity": round(sum(li[1] for li in level_info)
                                                    / max(1, level_info[0][1]), 3),
                   "amg_grid_complexity": round(sum(li[0] for li in level_info)
                                                / max(1, level_info[0][0]), 3),
                   "iterations": its, "setups_in_timed_steps": setups,
                   "setup_s_first": round(setup_s, 3)},
        "gpu_launches": launches,
        "roofline": roofline,
        "fma_rates": {"fp64_tflops": round(fma64 / 1e12, 4), "fp32_tflops": round(fma32 / 1e12, 3),
                      "fp64_fma_ceiling_GBps": round(fma64 / 2 * 8 / 1e9, 1),
                      "how": "msp_fma_rate: 8 blocks of 256 threads per SM, 8 independent FMA "
                             "chains of 2048 steps per thread, best of 5 launches, CUDA events; "
                             "ceiling = the bytes/s of kernels doing one FP64 FMA per 8-byte "
                             "value"},
        "plain_msp_mu0": mu0,
        "kernels": kernels,
        "sites": sites,
        "instrumented_ms_per_step": round(live_ms / args.steps, 3),
        "clocks": clk,
    }
    if eager:
        out["eager_sites"] = eager
        out["eager_ms_per_step"] = round(prof_ms, 3)
    if e2e:
        out["e2e"] = {"value": round(total_solves / (e2e["ms"] / 1000.0), 4), "unit": "solves/s",
                      "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                      "copies": "from pinned host memory inside the timed region; each step's "
                                "matrix values are copied on a second stream while the "
                                "previous step solves" if args.wells == "rows" else
                                "from pinned host memory inside the timed region"}
    out["_its_mean"] = float(np.mean(its))
    out["_setup_frac"] = setups / max(1, args.steps)
    return out


def oracle_sample(args, its_mean, setup_frac, steps, warmup, full_solve=False):
    """Time the oracle (single thread) on the full workload: SETUP once, then per step one
    Arnoldi iteration, measured as (solve capped at 2 iterations) - (capped at 1);
    returns (solves/s extrapolated to `its_mean` iterations and a `setup_frac` share of
    setups, seconds per iteration, setup seconds, its_mean).  With `full_solve`, the
    oracle first solves the system to the tolerance once and its own iteration count
    replaces `its_mean`."""
    import oracle
    from synthetic import grid_spe10, random_rhs
    from synthetic import BSRMatrix
    a = grid_spe10(seed=2209, nx=args.nx, ny=args.ny, nz=args.nz)
    rhs = random_rhs(a, 7000)
    t0 = time.perf_counter()
    if getattr(args, "wells", "rows") == "eliminate":
        W = oracle.Wells(a, a.n_wells)
        rp, ci, v = W.reduced()
        rhs = W.reduce_rhs(rhs)
        a = BSRMatrix(nb=W.nr, b=a.b, row_ptr=rp, col_idx=ci, values=v.reshape(-1, a.b, a.b),
                      n_cells=W.nr)
    o = oracle.Oracle(a, mu=10 ** 9)
    setup_s = time.perf_counter() - t0
    if full_solve:
        _, info = o.solve(rhs, TOL)
        its_mean = float(info["iterations"])
    per = []
    for k in range(warmup + steps):
        o.set_max_it(1)
        t = time.perf_counter()
        o.solve(rhs, TOL)
        t1 = time.perf_counter() - t
        o.set_max_it(2)
        t = time.perf_counter()
        o.solve(rhs, TOL)
        t2 = time.perf_counter() - t
        if k >= warmup:
            per.append(max(t2 - t1, 1e-9))
    t_it = float(np.median(per))
    value = 1.0 / (setup_frac * setup_s + its_mean * t_it)
    return value, t_it, setup_s, its_mean


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    # the oracle's own iteration count comes from one full solve of the first system; the
    # timed steps are single Arnoldi iterations.  SETUP counts in every solve at mu = 0
    # (plain MSP) and in none when mu is above the iteration count (the GPU arm's timed
    # solves reuse their first SETUP)
    t0 = time.perf_counter()
    value, t_it, setup_s, its_mean = oracle_sample(args, 0.0, 0.0, args.steps, args.warmup,
                                                   full_solve=True)
    setup_frac = 1.0 if args.mu < its_mean else 0.0
    value = 1.0 / (setup_frac * setup_s + its_mean * t_it)
    wall = time.perf_counter() - t0
    sample = ("oracle on the full %dx%dx%d matrix: SETUP once (%.1f s), one full solve to "
              "1e-6 (%d iterations), then %d timed single Arnoldi iterations (each a solve "
              "capped at 2 iterations minus one capped at 1; median %.3f s); solves/s = "
              "1 / (%.2f * setup + %d iterations)" % (args.nx, args.ny, args.nz, setup_s, its_mean, args.steps, t_it,
                               setup_frac, its_mean))
    from synthetic import grid_spe10
    a = grid_spe10(seed=2209, nx=args.nx, ny=args.ny, nz=args.nz)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(t_it * 1000, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": static_config(args, a),
           "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": 1,
                            "host_cores": os.cpu_count(), "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0},
           "wall_s": round(wall, 1)}
    return out


def run_mu_sweep(args):
    """Section 3.2, Tables 3, 5 and 7: SetupCalls, SetupRatio, Iter and Time of a whole
    Newton-like sequence of solves for several thresholds mu.  The sequence
    (synthetic.newton_sequence) drifts: a preconditioner kept across time steps goes stale
    and costs iterations, one regenerated every solve costs SETUPs.  mu is swept at the
    multiples 0, 1.0, 1.1, 1.2, 1.4 and 2.0 of the mean iteration count at mu = 0 (the
    paper's mu = 0, 10, 20, 30, 40 span 0-2.6 times its mean count of about 15.6 in
    Table 3, over a much wider spread of counts than this sequence has).  One JSON line
    per mu; the time of a run covers the solver's construction (the first SETUP), every
    value update and every solve."""
    import torch

    import paper_2208_08594_gb300 as msp
    from synthetic import grid_spe10, newton_sequence, random_rhs

    dev = torch.device("cuda", 0)
    a = grid_spe10(seed=2209, nx=args.nx, ny=args.ny, nz=args.nz)
    seq = newton_sequence(a, args.time_steps, args.newton_steps, seed=4242,
                          rel_newton=args.rel_newton, rel_step=args.rel_step)
    d_rp = torch.from_numpy(a.row_ptr).to(dev)
    d_ci = torch.from_numpy(a.col_idx).to(dev)
    d_vals = [torch.from_numpy(v.reshape(-1)).to(dev) for v in seq]
    d_rhs = [torch.from_numpy(random_rhs(a, 9000 + k)).to(dev) for k in range(len(seq))]
    x = torch.zeros(a.n, dtype=torch.float64, device=dev)
    prec = msp.MSP_PRECISION_FP32 if args.precision == "fp32" else msp.MSP_PRECISION_FP64

    def run(mu):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver = msp.Solver(a.nb, a.b, d_rp, d_ci, d_vals[0], mu=mu, precision=prec,
                            colouring=colouring_of(args, msp), smoother=smoother_of(args, msp))
        torch.cuda.synchronize()
        t_first = time.perf_counter() - t0
        setups, setup_s, iters, its, unconverged = 0, t_first, 0, [], 0
        for k in range(len(seq)):
            if k:
                solver.update_values(d_vals[k])
            info = solver.solve(d_rhs[k], x, TOL)
            # a preconditioner kept too long may not reach the tolerance in MaxIt
            # iterations: that is part of the trade-off being measured (the next solve
            # regenerates it); any other status is an error
            if info["status"] == msp.MSP_NOT_CONVERGED:
                unconverged += 1
            elif info["status"] != 0:
                raise RuntimeError("solve failed: %s" % info)
            setups += info["setup_performed"]
            setup_s += info["t_setup_ms"] / 1000.0
            iters += info["iterations"]
            its.append(info["iterations"])
        torch.cuda.synchronize()
        total = time.perf_counter() - t0
        solver.close()
        return {"mu": mu, "setup_calls": setups, "setup_ratio": round(setup_s / total, 4),
                "iter": iters, "time_s": round(total, 3), "solves": len(seq),
                "unconverged": unconverged, "iterations": its}

    run(0)  # warm-up (module load, allocator)
    base = run(0)
    it0 = base["iter"] / base["solves"]
    rows = [base]
    for f in (1.0, 1.1, 1.2, 1.4, 2.0):
        rows.append(run(int(round(f * it0))))
    for r in rows:
        r["mu_over_mean_it0"] = round(r["mu"] / it0, 2)
        r["speedup_vs_mu0"] = round(base["time_s"] / r["time_s"], 3)
        r["workload"] = "%s, Newton-like sequence: %d time steps x %d Newton steps, drift " \
                        "U[1 +- %.2f] per time step, U[1 +- %.2f] per Newton step" % (
                            workload_name(args), args.time_steps, args.newton_steps,
                            args.rel_step, args.rel_newton)
        print(json.dumps(r))


def serve_workload(args):
    """Seeded reservoirs: cells log-uniform in --serve-cells on a random box (nz 5-40, the
    rest split with aspect U[1, 4]), b uniform in --serve-blocks, 0-4 wells, 3-8 Newton steps
    whose matrices alternate between the base values and a copy perturbed by up to 5 % (the
    values change at every step, the pattern never), one right-hand side per step."""
    from synthetic import box_jacobian, perturb_values, random_rhs
    rng = np.random.default_rng(4242)
    lo, hi = np.log(args.serve_cells[0]), np.log(args.serve_cells[1])
    out = []
    for r in range(args.serve_reservoirs):
        cells = float(np.exp(rng.uniform(lo, hi)))
        nz = int(rng.integers(5, 41))
        b = int(rng.integers(args.serve_blocks[0], args.serve_blocks[1] + 1))
        aspect = float(rng.uniform(1.0, 4.0))
        area = max(cells / nz, 4.0)
        nx = max(2, int(round(np.sqrt(area / aspect))))
        ny = max(2, int(round(area / nx)))
        wells = int(rng.integers(0, 5))
        steps = int(rng.integers(3, 9))
        a = box_jacobian(nx, ny, nz, b, 9000 + r, layered=True, kz_ratio=0.1, n_wells=wells)
        v0 = np.ascontiguousarray(a.values.reshape(-1))
        v1 = np.ascontiguousarray(perturb_values(a, 9100 + r).reshape(-1))
        rhs = [np.ascontiguousarray(random_rhs(a, 9200 + 10 * r + k)) for k in range(steps)]
        out.append({"a": a, "vals": (v0, v1), "rhs": rhs, "steps": steps,
                    "dims": (nx, ny, nz), "b": b})
    return out


def run_serve_once(args, res, slots, precision):
    """Reservoirs arrive as a Poisson process; each runs its Newton sequence closed-loop (the
    next step is submitted when the previous solve returns).  Returns per-request results
    and the wall time from the first arrival to the last completion."""
    import paper_2208_08594_gb300 as msp
    mean_steps = float(np.mean([r["steps"] for r in res]))
    rate_res = args.serve_rate / mean_steps
    arr = np.cumsum(np.random.default_rng(77).exponential(1.0 / rate_res, size=len(res)))
    arr -= arr[0]
    server = msp.Server(slots=slots, hbm_budget=int(args.serve_budget_gb * 1e9), mu=args.mu,
                        precision=precision, colouring=colouring_of(args, msp),
                        smoother=smoother_of(args, msp))
    xs = [np.zeros(r["a"].nb * r["a"].b) for r in res]
    pending = {}  # ticket -> (reservoir, step)
    next_step = [0] * len(res)
    results = []
    t0 = time.perf_counter()

    def submit(i):
        r, k = res[i], next_step[i]
        a = r["a"]
        last = k == r["steps"] - 1
        t = server.submit(i, a.nb, a.b, r["rhs"][k], xs[i], values=r["vals"][k % 2],
                          row_ptr=a.row_ptr, col_idx=a.col_idx, rel_tol=TOL, release=last)
        pending[t] = (i, k)
        next_step[i] += 1

    arrived = 0
    while arrived < len(res) or pending:
        now = time.perf_counter() - t0
        while arrived < len(res) and arr[arrived] <= now:
            submit(arrived)
            arrived += 1
        done = []
        for t in list(pending):
            out = server.wait(t, 0.0)
            if out is not None:
                done.append((t, out))
        for t, out in done:
            i, k = pending.pop(t)
            out["reservoir"], out["step"] = i, k
            out["cells"] = res[i]["a"].nb
            out["n"] = res[i]["a"].nb * res[i]["a"].b
            results.append(out)
            if next_step[i] < res[i]["steps"]:
                submit(i)
        if not done:
            time.sleep(0.0005)
    wall = time.perf_counter() - t0
    stats = server.stats()
    server.close()
    return results, wall, stats


def run_serve(args):
    import paper_2208_08594_gb300 as msp
    prec_of = {"fp64": msp.MSP_PRECISION_FP64, "fp32": msp.MSP_PRECISION_FP32}
    t_gen = time.perf_counter()
    res = serve_workload(args)
    t_gen = time.perf_counter() - t_gen
    cfg = msp.msp_config_default(mu=args.mu, precision=prec_of[args.precision])
    est = [msp.msp_estimate_device_bytes(r["a"].nb, r["a"].b, r["a"].nnzb, cfg) for r in res]
    runs = []
    for slots in args.serve_slots:
        results, wall, stats = run_serve_once(args, res, slots, prec_of[args.precision])
        bad = [r for r in results if r["status"] != 0]
        lat = np.array([r["latency_ms"] for r in results])
        runs.append({
            "slots": slots, "solves": len(results), "failed": len(bad), "wall_s": round(wall, 3),
            "solves_per_s": round(len(results) / wall, 3),
            "cell_solves_per_s": round(sum(r["cells"] for r in results) / wall, 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 1),
            "p99_ms": round(float(np.percentile(lat, 99)), 1),
            "mean_queue_ms": round(float(np.mean([r["queue_ms"] for r in results])), 1),
            "setups": int(sum(r["setup"] for r in results)),
            "asmsp_setups": int(sum(r["info"]["setup_performed"] for r in results)),
            "iterations": int(sum(r["info"]["iterations"] for r in results)),
            "max_rel_residual": float(max(r["info"]["rel_residual"] for r in results)),
            "peak_charged_gb": round(stats["peak_charged_bytes"] / 1e9, 2),
            "footprint_over_estimate": [
                round(max(r["device_bytes"] for r in results if r["reservoir"] == i) / est[i], 3)
                for i in range(len(res))],
            "evictions": stats["evictions"]})
    out = {"metric": "request loop: solves/s and p50/p99 latency", "unit": "solves/s",
           "value": runs[-1]["solves_per_s"], "higher_is_better": True, "n_gpus": 1,
           "dtype": "f64" if args.precision == "fp64" else "f32-precond/f64-krylov",
           "data": "synthetic", "vs_baseline": None,
           "config": {"workload": "%d reservoirs, cells log-uniform %.0f-%.0f, b %d-%d, "
                                  "3-8 Newton steps each, +-5%% values" % (
                                      args.serve_reservoirs, args.serve_cells[0],
                                      args.serve_cells[1], args.serve_blocks[0],
                                      args.serve_blocks[1]),
                      "offered_requests_per_s": args.serve_rate, "mu": args.mu,
                      "hbm_budget_gb": args.serve_budget_gb, "tol": TOL,
                      "reservoirs": [{"dims": r["dims"], "b": r["b"], "block_rows": r["a"].nb,
                                      "nnzb": r["a"].nnzb, "steps": r["steps"]} for r in res],
                      "generation_s": round(t_gen, 1)},
           "runs": runs}
    print(json.dumps(out))


def batch_workload(args):
    """Seeded instances: cells log-uniform in --batch-cells on random boxes (nz 5-40, the
    rest split with aspect U[1, 4]), b 4 or 6, 0-2 wells; one right-hand side each."""
    from synthetic import box_jacobian, random_rhs
    rng = np.random.default_rng(6464)
    lo, hi = np.log(args.batch_cells[0]), np.log(args.batch_cells[1])
    out = []
    for k in range(args.batch_instances):
        cells = float(np.exp(rng.uniform(lo, hi)))
        nz = int(rng.integers(5, 41))
        b = int(rng.choice([4, 6]))
        aspect = float(rng.uniform(1.0, 4.0))
        area = max(cells / nz, 4.0)
        nx = max(2, int(round(np.sqrt(area / aspect))))
        ny = max(2, int(round(area / nx)))
        a = box_jacobian(nx, ny, nz, b, 7000 + k, layered=True, kz_ratio=0.1,
                         n_wells=int(rng.integers(0, 3)))
        out.append((a, random_rhs(a, 7100 + k)))
    return out


def run_batch(args):
    """Every instance solved `--batch-steps` times (values fixed, preconditioner reused):
    (a) batched: one stack per block size, msp_solve_batch; (b) one at a time: a handle
    per instance, msp_solve.  Both timed with CUDA events on the same stream."""
    import torch

    import paper_2208_08594_gb300 as msp
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    prec = msp.MSP_PRECISION_FP32 if args.precision == "fp32" else msp.MSP_PRECISION_FP64
    opts = dict(mu=args.mu, precision=prec, colouring=colouring_of(args, msp),
                smoother=smoother_of(args, msp), autotune=int(args.autotune))
    t_gen = time.perf_counter()
    inst = batch_workload(args)
    t_gen = time.perf_counter() - t_gen
    cells = sum(a.nb for a, _ in inst)

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # (a) batched, one stack per block size
    groups = {}
    for k, (a, r) in enumerate(inst):
        groups.setdefault(a.b, []).append(k)
    stacks, t_setup_b = [], time.perf_counter()
    for b, ks in sorted(groups.items()):
        nb, bb, rp, ci, v, off = msp.stack_block_diagonal([inst[k][0] for k in ks])
        rhs = np.concatenate([inst[k][1] for k in ks])
        solver = msp.BatchSolver(nb, bb, torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev),
                                 torch.from_numpy(v).to(dev), off, **opts)
        stacks.append({"b": b, "ks": ks, "solver": solver, "rhs": torch.from_numpy(rhs).to(dev),
                       "x": torch.zeros(nb * bb, dtype=torch.float64, device=dev),
                       "nb": nb, "nnzb": int(ci.size), "levels": solver.num_levels,
                       "colours": msp.msp_level_info(solver.h, 0)[2],
                       "tiles": [msp.msp_level_tiles(solver.h, l)
                                 for l in range(solver.num_levels)]})
    torch.cuda.synchronize()
    t_setup_b = time.perf_counter() - t_setup_b
    its_b = {}

    st_b = {}

    def batched():
        for st in stacks:
            infos = st["solver"].solve_batch(st["rhs"], st["x"], TOL)
            for k, i in zip(st["ks"], infos):
                if i["status"] < 0:
                    raise RuntimeError("instance %d: %s" % (k, i))
                its_b[k] = i["iterations"]
                st_b[k] = i["status"]

    batched()  # warm-up
    msp.msp_stats_reset()
    msp.msp_stats_enable(1)
    ms_b = timed(batched, args.batch_steps)
    launches_b = msp.msp_stats_launches()
    msp.msp_stats_enable(0)
    profile_b = None
    if args.batch_profile:  # one more step with every call site timed: where the time goes
        msp.msp_stats_reset()
        msp.msp_stats_enable(3)
        batched()
        msp.msp_stats_enable(0)
        profile_b = {k: {"launches": v[0], "ms": round(v[1], 2)}
                     for k, v in sorted(msp.msp_stats_get().items(), key=lambda kv: -kv[1][1])[:25]}
        msp.msp_stats_reset()
    stack_info = [dict({k: st[k] for k in ("b", "nb", "nnzb", "levels", "colours", "tiles")},
                       instances=len(st["ks"])) for st in stacks]
    for st in stacks:
        st["solver"].close()
    del stacks

    # (b) one at a time
    t_setup_1 = time.perf_counter()
    singles = []
    for a, r in inst:
        solver = msp.Solver(a.nb, a.b, torch.from_numpy(a.row_ptr).to(dev),
                            torch.from_numpy(a.col_idx).to(dev),
                            torch.from_numpy(a.values.reshape(-1)).to(dev), **opts)
        singles.append((solver, torch.from_numpy(r).to(dev),
                        torch.zeros(a.nb * a.b, dtype=torch.float64, device=dev)))
    torch.cuda.synchronize()
    t_setup_1 = time.perf_counter() - t_setup_1
    its_1 = {}

    st_1 = {}

    def one_by_one():
        for k, (solver, r, x) in enumerate(singles):
            i = solver.solve(r, x, TOL)
            if i["status"] < 0:
                raise RuntimeError("instance %d: %s" % (k, i))
            its_1[k] = i["iterations"]
            st_1[k] = i["status"]

    one_by_one()
    msp.msp_stats_reset()
    msp.msp_stats_enable(1)
    ms_1 = timed(one_by_one, args.batch_steps)
    launches_1 = msp.msp_stats_launches()
    msp.msp_stats_enable(0)
    for solver, _, _ in singles:
        solver.close()

    n_solves = args.batch_steps * len(inst)
    out = {"metric": "batched instances: solves/s", "unit": "solves/s",
           "value": round(n_solves / (ms_b / 1000.0), 3), "higher_is_better": True, "n_gpus": 1,
           "dtype": "f64" if args.precision == "fp64" else "f32-precond/f64-krylov",
           "data": "synthetic", "vs_baseline": None,
           "config": {"workload": "%d instances, cells log-uniform %.0f-%.0f, b 4 or 6" % (
                          len(inst), args.batch_cells[0], args.batch_cells[1]),
                      "cells": cells, "steps": args.batch_steps, "mu": args.mu, "tol": TOL,
                      "generation_s": round(t_gen, 1)},
           "batched": {"ms_per_step": round(ms_b / args.batch_steps, 1),
                       "solves_per_s": round(n_solves / (ms_b / 1000.0), 3),
                       "cell_solves_per_s": round(cells * args.batch_steps / (ms_b / 1000.0), 1),
                       "launches_per_step": round(launches_b / args.batch_steps, 1),
                       "setup_s": round(t_setup_b, 2),
                       "iterations_total": int(sum(its_b.values())),
                       "iterations_max": int(max(its_b.values())),
                       "not_converged": sorted(k for k, v in st_b.items() if v != 0)},
           "one_at_a_time": {"ms_per_step": round(ms_1 / args.batch_steps, 1),
                             "solves_per_s": round(n_solves / (ms_1 / 1000.0), 3),
                             "cell_solves_per_s": round(cells * args.batch_steps / (ms_1 / 1000.0), 1),
                             "launches_per_step": round(launches_1 / args.batch_steps, 1),
                             "setup_s": round(t_setup_1, 2),
                             "iterations_total": int(sum(its_1.values())),
                             "iterations_max": int(max(its_1.values())),
                             "not_converged": sorted(k for k, v in st_1.items() if v != 0)},
           "stacks": stack_info}
    if profile_b:
        out["batched_sites_one_step"] = profile_b
    print(json.dumps(out))


def run_latency(args):
    """Latency of one solve of the small system (16x16x8 cells, b = 3, no wells, RHS N(0,1)):
    SETUP once, then `steps` solves of the same system timed one by one with CUDA events on
    the solver stream (device-resident inputs) and, through the host-buffer entry points,
    with the host clock (rhs in, x out)."""
    import torch

    import paper_2208_08594_gb300 as msp
    from synthetic import grid_small
    a = grid_small()
    rng = np.random.default_rng(2208)
    rhs = rng.normal(size=a.n)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    prec = msp.MSP_PRECISION_FP32 if args.precision == "fp32" else msp.MSP_PRECISION_FP64
    t0 = time.perf_counter()
    s = msp.Solver(a.nb, a.b, torch.from_numpy(a.row_ptr).to(dev),
                   torch.from_numpy(a.col_idx).to(dev),
                   torch.from_numpy(a.values.reshape(-1)).to(dev), mu=args.mu, precision=prec)
    torch.cuda.synchronize()
    setup_ms = 1000.0 * (time.perf_counter() - t0)
    g = torch.from_numpy(rhs).to(dev)
    x = torch.zeros(a.n, dtype=torch.float64, device=dev)
    for _ in range(max(args.warmup, 3)):
        s.solve(g, x, TOL)
    dev_ms, its = [], []
    msp.msp_stats_reset()
    msp.msp_stats_enable(1)
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = s.solve(g, x, TOL)
        e1.record(stream)
        torch.cuda.synchronize()
        dev_ms.append(e0.elapsed_time(e1))
        its.append(info["iterations"])
    launches = msp.msp_stats_launches()
    msp.msp_stats_enable(0)
    host_ms = []
    xh = np.zeros(a.n)
    for _ in range(args.steps):
        t = time.perf_counter()
        s.solve_host(rhs, xh, TOL)
        host_ms.append(1000.0 * (time.perf_counter() - t))
    s.close()
    res = a.to_scipy() @ xh - rhs
    out = {"metric": "solve latency, 16x16x8 cells x3 (C1)", "unit": "ms",
           "value": round(float(np.percentile(dev_ms, 50)), 4), "higher_is_better": False,
           "n_gpus": 1, "steps": args.steps, "dtype": "f64" if prec == msp.MSP_PRECISION_FP64
           else "f32-precond/f64-krylov", "data": "synthetic",
           "config": {"workload": "16x16x8 box, b = 3, ln k ~ N(0,1), no wells, RHS ~ N(0,1)",
                      "block_rows": a.nb, "nnzb": a.nnzb, "tol": TOL, "mu": args.mu},
           "p50_ms": round(float(np.percentile(dev_ms, 50)), 4),
           "p99_ms": round(float(np.percentile(dev_ms, 99)), 4),
           "mean_ms": round(float(np.mean(dev_ms)), 4),
           "iterations": sorted(set(its)), "launches_per_solve": launches / args.steps,
           "host_buffers": {"p50_ms": round(float(np.percentile(host_ms, 50)), 4),
                            "p99_ms": round(float(np.percentile(host_ms, 99)), 4)},
           "true_rel_residual": float(np.linalg.norm(res) / np.linalg.norm(rhs)),
           "setup_ms": round(setup_ms, 1)}
    print(json.dumps(out))


def main():
    args = parse()
    if args.latency:
        run_latency(args)
        return
    if args.batch:
        run_batch(args)
        return
    if args.serve:
        run_serve(args)
        return
    if args.mu_sweep:
        run_mu_sweep(args)
        return
    if args.impl == "reference":
        out = run_reference(args)
        if out is not None:
            print(json.dumps(out))
        return
    out = run_native(args)
    if out is None:
        return
    # CPU baseline: the oracle, bounded sample (rank 0, N = 1 only)
    if out["n_gpus"] == 1 and os.environ.get("MSP_BENCH_NO_CPU") != "1":
        value, t_it, setup_s, _ = oracle_sample(args, out["_its_mean"], out["_setup_frac"], 2, 1)
        out["cpu_baseline"] = {
            "value": round(value, 6), "unit": "solves/s", "cores": 1,
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle on the full matrix: SETUP once (%.1f s) + 2 timed single Arnoldi "
                      "iterations (median %.3f s), extrapolated to %.1f iterations and a setup "
                      "share of %.2f" % (setup_s, t_it, out["_its_mean"], out["_setup_frac"])}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
