#!/usr/bin/env python3
"""Benchmark of the Chebyshev propagation hot path on GB300.

Workload (one line of output): the batched disorder ensemble -- 64 zigzag ribbons of uneven
size (W in U{40..160}, L in U{500..4000}, 15.5 M sites), Anderson disorder W = 0.5/1/2 cycled
over ribbons, 4 wave packets per ribbon (k0 = pi/6, pi/4, pi/3, pi/2), complex64 vectors with
FP64 coefficients and reductions, dt = 1 (M = 19/20/21 per ribbon).  One step = one time step
dt of the whole ensemble: M fused recurrence kernels, all ribbons in each launch.

Metric: Chebyshev matvec-steps/s (one matvec-step = one application of H~ inside the
recurrence to one vector of one ribbon), with the recurrence kernel's achieved algorithmic
HBM bandwidth against the measured copy bandwidth, the complex128 single-vector path on the
same ensemble for comparison, the oracle on the host as the CPU baseline, and an end-to-end
figure through the C ABI with host buffers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank propagates its own 64-ribbon ensemble (disorder streams offset by
rank): weak scaling, no collective on the data path.
"""
from __future__ import annotations

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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = ("Chebyshev matvec-steps/s and achieved HBM GB/s (% of GB300 peak), "
          "complex64-batched vs FP64")
UNIT = "matvec-steps/s"
WORKLOAD = "ensemble of 64 uneven zigzag ribbons x 4 packets, complex64, dt=1"

# Algorithmic bytes per unit (one site or basis row, one Chebyshev order) of the unblocked
# fused recurrence that moves every operand once: T_j, T_{j-1}, T_{j+1}, psi read and written,
# the on-site array, plus the stored matrix for the SELL operator.  "achieved" in the bench
# line is this figure x the units a launch processes / the launch's duration, so a kernel that
# reuses data on chip (temporal blocking, grouped accumulation) can exceed the copy bandwidth;
# its own DRAM bytes are reported as "traffic".
ALG_BYTES_PER_UNIT = {
    ("ensemble", "c64"): 164.0,   # 4 packets share the on-site array: 4 * 40 + 4
    ("ribbon", "c64"): 44.0, ("ribbon", "f64"): 88.0,
    ("doublewell", "f64"): 88.0, ("doublewell", "c64"): 44.0,
    ("holstein", "c64"): 71.0, ("holstein", "f64"): 127.0,          # SELL-32 (~3.9 entries)
    ("holstein-mf", "c64"): 40.0, ("holstein-mf", "f64"): 80.0,     # vectors only
}

# DRAM bytes of one step of the paper's polaron run with the matrix-free operator, by
# (precision, M), same capture method
POLARON_MF_DRAM_BYTES_PER_STEP = {("c64", 24): 497.5e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle timing (profiling runs)")
    ap.add_argument("--lean", action="store_true",
                    help="timed region only: no e2e, FP64 or accuracy legs (profiling runs)")
    ap.add_argument("--workload", default="ensemble",
                    choices=["ensemble", "ribbon", "holstein", "doublewell", "paperwell", "adjoint",
                             "polaron", "armchair", "driven"],
                    help="ensemble (default, the headline line); the others measure the other "
                         "configurations of the hot path")
    ap.add_argument("--prec", default=None, choices=["c64", "c128"],
                    help="vector precision for --workload ribbon/holstein (default c128)")
    ap.add_argument("--matrix-free", action="store_true",
                    help="--workload holstein/polaron: matrix-free Holstein operator instead of "
                         "the stored SELL matrix")
    ap.add_argument("--sweep", action="store_true",
                    help="ensemble only: time whole steps (graph replay, CUDA events) for the "
                         "compiled blocked shapes of both blocked kernels and print one JSON line "
                         "per shape with the work model (profiling runs; no contract line)")
    ap.add_argument("--sell-sigma", type=int, default=0,
                    help="--workload holstein/polaron with the stored matrix: SELL-C-sigma window "
                         "(0: library default, 1: rows unsorted)")
    ap.add_argument("--hol-size", default=None,
                    help="L:NPH -- Holstein chain size for --workload holstein (profiling runs; "
                         "default 12:10)")
    ap.add_argument("--blocking", default=None,
                    help="S:SPT[:THREADS[:KERNEL]] -- force S orders per launch with SPT sites per "
                         "thread (THREADS per CTA, default 256; KERNEL 'runs': the register-run "
                         "kernel, 'runs_tma': the same with boxes staged by TMA) "
                         "and skip the autotuner (profiling runs); 0:0 forces single-order "
                         "launches")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------------------
# reference arm: the oracle on the host
# ----------------------------------------------------------------------------------------
def oracle_ensemble_sample(ens: wl.RibbonEnsemble, ribbons, nsteps: int = 1):
    """Propagate the packets of the given ribbons by nsteps with the oracle; returns
    (seconds, matvec-steps, site-steps)."""
    import oracle

    t = 0.0
    mv = 0
    ss = 0
    for r in ribbons:
        rb = ens.ribbon(r)
        H = oracle.honeycomb(rb.W, rb.L, rb.hop, rb.onsite())
        a, b = oracle.rescale(*rb.bounds(), 0.0)
        C, M = oracle.coeffs(a, b, rb.dt)
        for k0 in ens.k0s:
            psi = rb.packet(k0)
            t0 = time.perf_counter()
            H.evolve(a, b, C, nsteps, psi)
            t += time.perf_counter() - t0
            mv += M * nsteps
            ss += M * nsteps * rb.W * rb.L
    return t, mv, ss


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    ens = wl.RibbonEnsemble()
    # one step = one dt for 4 ribbons of the ensemble (cycling through all 64), 4 packets each
    per_step = 4
    for w in range(args.warmup):
        oracle_ensemble_sample(ens, [(w * per_step + i) % ens.n_ribbons for i in range(per_step)])
    tt, mv, ss = 0.0, 0, 0
    for s in range(args.steps):
        rs = [((args.warmup + s) * per_step + i) % ens.n_ribbons for i in range(per_step)]
        t, m, x = oracle_ensemble_sample(ens, rs)
        tt += t
        mv += m
        ss += x
    value = mv / tt
    sample = (f"{args.steps} steps, each one dt of 4 ribbons x 4 packets of the ensemble "
              f"(cycling through the 64 ribbons), single-threaded FP64 oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "4 ribbons x 4 packets per step"},
        "site_steps_per_s": ss / tt,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
def make_plan(cb, ens, prec, nvec, packets):
    import torch

    W = [w for w, _ in ens.sizes]
    L = [l for _, l in ens.sizes]
    eps = torch.from_numpy(ens.onsite()).to("cuda")
    desc, keep = cb.desc_ribbons(W, L, ens.hop, eps)
    lo, hi = ens.bounds()
    plan = cb.Plan(desc, lo, hi, 0.0, prec, nvec, keep=keep)
    dt = torch.complex64 if prec == cb.CHEB_C64 else torch.complex128
    psi = torch.from_numpy(packets).to(dt).to("cuda").contiguous()
    return plan, psi


def blocked_roofline(cb, plan, kms, kcount, steps, alg_per_unit, unit_definition):
    """Roofline of the recurrence launches of the timed region (their CUDA-event time).

    Temporal blocking (k_rec_tb): the launches reuse every vector element for s orders out of
    shared memory, so their bound is the shared-memory pipe, not HBM.  achieved = the
    shared-memory bytes the launches move (cheb_plan_step_model: per formed site-order the
    own-site, neighbour and T_{k-2} loads and the T_k store, plus region copies and read-back)
    / their event time, against the shared-memory load bandwidth measured in this run by the
    library's probe.  Beside it: DRAM bytes derived from the tile set (every operand once per
    launch) against HBM, and the streaming-equivalent rate (the per-unit bytes an unblocked
    kernel would move for the same useful site-orders) against HBM.
    Single-order launches: bound HBM, achieved = their algorithmic DRAM bytes / time."""
    peak_hbm, hbm_kind = measured_peaks()
    model = plan.step_model()
    lps = model["launches"]
    ms_per_launch = kms / max(kcount, 1)
    sec = ms_per_launch / 1e3
    useful_pl = model["useful_site_orders"] / lps
    stream_equiv = alg_per_unit * useful_pl / sec / 1e9
    dram_pl = model["dram_bytes"] / lps
    blk = tuple(plan.blocking_shape())
    common = {"launches": kcount, "launches_per_step": lps, "kernel_ms_total": kms,
              "ms_per_launch": ms_per_launch, "unit_definition": unit_definition,
              "useful_site_orders_per_launch": useful_pl,
              "streaming_equivalent": {"achieved": stream_equiv, "peak": peak_hbm,
                                       "frac": stream_equiv / peak_hbm, "unit": "GB/s",
                                       "alg_bytes_per_unit": alg_per_unit,
                                       "note": "per-unit bytes of an unblocked kernel x useful "
                                               "site-orders / time; above 1 when data is reused "
                                               "on chip"}}
    if blk[0]:
        smem_peak = cb.cheb_measure_peak(cb.CHEB_PEAK_SMEM_LOAD_GBS)
        smem_pl = model["smem_bytes"] / lps
        achieved = smem_pl / sec / 1e9
        r = {"bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
             "frac": achieved / smem_peak, "traffic": dram_pl,
             "kernel": ("k_rec_tbr<%s,%d,%d> (all launches of the step)"
                        % ("float4" if plan.nvec >= 2 else "float2", blk[1], blk[2])
                        if plan.blocking_kernel() in (cb.CHEB_TB_RUNS, cb.CHEB_TB_RUNS_TMA) else
                        "k_rec_tb<%d,%d,%d> (all launches of the step)" % (plan.nvec, blk[1], blk[2])),
             "peak_kind": "shared-memory load bandwidth measured in this run by the library's "
                          "probe (cheb_measure_peak; MEASURED_PEAKS.json has no shared-memory "
                          "figure)",
             "smem_bytes_per_launch": smem_pl,
             "computed_over_useful": model["computed_site_orders"] / model["useful_site_orders"],
             "traffic_source": "derived from the tile set: every operand crossing DRAM once per "
                               "launch, halo re-reads served by L2 (ncu cross-check in profiles/)",
             "l2_bytes_per_launch": model["l2_bytes"] / lps,
             "dram": {"achieved": dram_pl / sec / 1e9, "peak": peak_hbm,
                      "frac": dram_pl / sec / 1e9 / peak_hbm, "unit": "GB/s",
                      "peak_kind": f"{hbm_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}}
    else:
        achieved = dram_pl / sec / 1e9
        r = {"bound": "hbm", "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
             "frac": achieved / peak_hbm, "traffic": dram_pl,
             "kernel": "k_rec<float,%d,StencilOp> (all launches of the step)" % plan.launch_shape()[3],
             "peak_kind": f"{hbm_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
             "traffic_source": "algorithmic: every operand read or written once per launch"}
    r.update(common)
    return r


SWEEP_SHAPES = [("sites", 6, 512), ("sites", 3, 1024), ("runs", 3, 768), ("runs", 5, 512),
                ("runs", 7, 384), ("runs", 9, 256), ("runs_tma", 5, 512), ("runs_tma", 7, 384),
                ("runs_tma", 9, 256)]
KERNEL_NAMES = {"sites": 0, "runs": 1, "runs_tma": 2}  # cheb_tb_kernel values


def kernel_of(name):
    return KERNEL_NAMES.get(name, 0)


def kernel_name(k):
    return {v: n for n, v in KERNEL_NAMES.items()}.get(k, "sites")


def run_sweep(args, local):
    """Whole-step times of the ensemble for blocked shapes: orders per launch 8, 10, 12 for each
    (kernel, sites per thread, threads), graph-replayed steps between CUDA events."""
    import torch

    import paper_0907_3022_gb300 as cb

    torch.cuda.set_device(local)
    ens = wl.RibbonEnsemble()
    plan, psi = make_plan(cb, ens, cb.CHEB_C64, ens.nvec, ens.packets())
    plan.evolve(psi, ens.dt, 0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nst = max(args.steps, 3)
    for kname, spt, tpb in SWEEP_SHAPES:
        kern = kernel_of(kname)
        for s in (8, 10, 12):
            plan.set_blocking_kernel(s, spt, tpb, kern)
            plan.evolve(psi, ens.dt, max(args.warmup, 3))
            plan.sync()
            e0.record()
            plan.evolve(psi, ens.dt, nst)
            e1.record()
            torch.cuda.synchronize()
            m = plan.step_model()
            print(json.dumps({"kernel": kname, "sites_per_thread": spt, "threads": tpb,
                              "orders_per_launch": s, "ms_per_step": e0.elapsed_time(e1) / nst,
                              "computed_over_useful": m["computed_site_orders"] / m["useful_site_orders"],
                              "smem_gb_per_step": m["smem_bytes"] / 1e9,
                              "dram_gb_per_step": m["dram_bytes"] / 1e9,
                              "launches_per_step": m["launches"]}), flush=True)
    plan.close()
    return 0


def run_ours(args, world, rank, local):
    import torch

    import paper_0907_3022_gb300 as cb

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ens = wl.RibbonEnsemble(stream0=rank * 64)
    packets = ens.packets()
    plan, psi = make_plan(cb, ens, cb.CHEB_C64, ens.nvec, packets)
    psi0 = psi.clone()
    plan.evolve(psi, ens.dt, 0)  # coefficients for dt
    if args.blocking is None:
        plan.autotune()
    else:
        f = args.blocking.split(":")
        kern = kernel_of(f[3]) if len(f) > 3 else cb.CHEB_TB_SITES
        parts = [int(x) for x in f[:3]]
        bs, bspt = parts[0], parts[1]
        btpb = parts[2] if len(parts) > 2 else 256
        plan.set_blocking_kernel(bs, bspt if bs else 4, btpb if bs else 256, kern)
    Ms = [plan.block(q)["M"] for q in range(ens.n_ribbons)]
    sites = [w * l for w, l in ens.sizes]
    mv_per_step = ens.nvec * sum(Ms)
    ss_per_step = ens.nvec * sum(m * s for m, s in zip(Ms, sites))
    stream = torch.cuda.current_stream()

    # warm-up (graph path)
    plan.evolve(psi, ens.dt, args.warmup)
    plan.sync()

    # timed region: K steps; each recurrence launch bracketed by CUDA events on this stream
    plan.set_timing(True)
    plan.kernel_stats(reset=True)
    clocks = Clocks(local)
    launches0 = plan.launches()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.evolve(psi, ens.dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms_local = e0.elapsed_time(e1)
    gpu_launches = plan.launches() - launches0
    kms, kcount, kbytes = plan.kernel_stats(reset=True)
    plan.set_timing(False)
    ms = max_over_ranks(ms_local, world)
    value = sum_over_ranks(mv_per_step * args.steps, world) / (ms / 1e3)
    site_steps = sum_over_ranks(ss_per_step * args.steps, world) / (ms / 1e3)

    roofline = blocked_roofline(cb, plan, kms, kcount, args.steps,
                                ALG_BYTES_PER_UNIT[("ensemble", "c64")],
                                "one site (4 packets) and one Chebyshev order")

    out = {}
    if not args.lean:
        # end to end through the C ABI with host buffers: H2D of the packets, one step, D2H
        # cheb_evolve_host: every step is one job whose packets come from pinned host memory
        # and whose result goes back to it; the copies of the neighbouring jobs overlap the
        # propagation (host wall clock around the call, which synchronises)
        pinned_in = torch.from_numpy(packets.astype(np.complex64)).pin_memory()
        pinned_out = torch.empty_like(pinned_in).pin_memory()
        plan.evolve_host(pinned_in, pinned_out, 2, ens.dt, 1, in_stride=0, out_stride=0)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.evolve_host(pinned_in, pinned_out, args.steps, ens.dt, 1, in_stride=0, out_stride=0)
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, world)
        nbytes = pinned_in.numel() * pinned_in.element_size()
        out["e2e"] = {"value": sum_over_ranks(mv_per_step * args.steps, world) / (e2e_ms / 1e3),
                      "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                      "api": "cheb_evolve_host (pinned host buffers, copies overlapped with "
                             "the propagation of the neighbouring steps)"}

        # accuracy over the configuration's 200 steps: the smallest ribbon against the FP64
        # oracle (4 packets) and the norm drift of every (ribbon, packet)
        import oracle

        nsteps_acc = ens.nsteps
        psi.copy_(torch.from_numpy(packets.astype(np.complex64)))
        n2_0 = torch.zeros((ens.n_ribbons, ens.nvec), dtype=torch.float64, device=dev)
        n2 = torch.zeros_like(n2_0)
        plan.observables(psi, cb.CHEB_OBS_NORM2, 0.0, n2_0)
        plan.evolve(psi, ens.dt, nsteps_acc)
        plan.observables(psi, cb.CHEB_OBS_NORM2, 0.0, n2)
        res = psi.cpu().numpy().astype(np.complex128)
        off = ens.offsets()
        r = int(np.argmin(sites))
        rb = ens.ribbon(r)
        H = oracle.honeycomb(rb.W, rb.L, rb.hop, rb.onsite())
        a, b = oracle.rescale(*rb.bounds(), 0.0)
        C, M = oracle.coeffs(a, b, rb.dt)
        errs = []
        for v, k0 in enumerate(ens.k0s):
            ref = H.evolve(a, b, C, nsteps_acc, rb.packet(k0))
            errs.append(float(np.linalg.norm(res[off[r]:off[r + 1], v] - ref) / np.linalg.norm(ref)))
        out["accuracy"] = {
            "rel_l2_vs_fp64_oracle": max(errs),
            "sample": f"ribbon {r} ({rb.W}x{rb.L}), 4 packets, {nsteps_acc} steps",
            "max_norm_drift": float((n2 - n2_0).abs().max()),
            "norm_drift_steps": nsteps_acc,
        }

        # the plain FP64 single-vector path on the same ensemble (packet k0 = pi/3)
        plan64, psi64 = make_plan(cb, ens, cb.CHEB_C128, 1, packets[:, 2:3].copy())
        plan64.evolve(psi64, ens.dt, 0)
        if args.blocking is None:
            plan64.autotune()
        plan64.evolve(psi64, ens.dt, 2)
        k64 = max(5, args.steps // 5)
        plan64.set_timing(True)
        plan64.kernel_stats(reset=True)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        plan64.evolve(psi64, ens.dt, k64)
        f1.record(stream)
        torch.cuda.synchronize()
        f_ms = f0.elapsed_time(f1)
        k64ms, k64n, k64b = plan64.kernel_stats(reset=True)
        ss64 = sum(m * s for m, s in zip(Ms, sites)) * k64 / (f_ms / 1e3)
        # FP64 roofline of the single-order kernel k_rec<double,1,StencilOp>: per site-order it
        # issues 4 DADD (neighbour sums) + 4 DFMA (2 H~ x - p) on the FP64 pipe, plus 6 DFMA
        # of the psi accumulation every third order: 10 FP64 pipe instructions on average,
        # against the FP64 FMA rate measured in this run by the library's probe
        fp64_peak = cb.cheb_measure_peak(cb.CHEB_PEAK_FP64_GFLOPS)  # GFLOP/s, 2 per DFMA
        ss64_k = sum(m * s for m, s in zip(Ms, sites)) * k64 / (k64ms / 1e3)  # kernel time only
        inst_rate = 10.0 * ss64_k / 1e9  # G FP64 instructions / s
        out["fp64_single_vector"] = {
            "matvec_steps_per_s": sum(Ms) * k64 / (f_ms / 1e3),
            "site_steps_per_s": ss64,
            "complex64_batched_site_vector_steps_per_s": site_steps,
            "speedup_c64_batched_over_fp64": site_steps / ss64,
            "kernel_achieved_gbs": k64b / (k64ms / 1e3) / 1e9,
            "roofline": {"bound": "fp64", "achieved": inst_rate, "peak": fp64_peak / 2.0,
                         "unit": "G FP64 pipe instructions/s", "frac": inst_rate / (fp64_peak / 2.0),
                         "kernel": "k_rec<double,1,StencilOp>",
                         "per_unit": "10 FP64 instructions per site-order (4 DADD + 4 DFMA, "
                                     "6 DFMA every third order)",
                         "peak_kind": "DFMA rate measured in this run by the library's probe "
                                      "(cheb_measure_peak)",
                         "hbm_frac": k64b / (k64ms / 1e3) / 1e9 / measured_peaks()[0]},
            "steps": k64,
            "note": "same ensemble, one packet (k0 = pi/3), complex128",
        }
        plan64.close()

    if not args.no_cpu_baseline and rank == 0 and world == 1:
        # bounded sample: one dt of the first 24 ribbons x 4 packets on one host core
        t, mv, ss = oracle_ensemble_sample(ens, list(range(24)))
        out["cpu_baseline"] = {"value": mv / t, "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(), "kind": "oracle",
                               "sample": "one dt of ribbons 0-23 x 4 packets (FP64 oracle, "
                                         "single thread)",
                               "site_steps_per_s": ss / t, "seconds": t}

    wss = (psi.numel() * psi.element_size() * 4) / 1e9  # psi, T_a, T_b, tail
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {
            "workload": WORKLOAD, "n_ribbons": ens.n_ribbons, "sites": int(sum(sites)),
            "packets_per_ribbon": ens.nvec, "dt": ens.dt, "M_per_ribbon": sorted(set(Ms)),
            "l2": f"inputs larger than L2 (working set {wss:.2f} GB of vectors)",
            "launch_shape": dict(zip(("threads", "sites_per_thread", "grid", "vecs_per_thread"),
                                     plan.launch_shape())),
            "temporal_blocking": dict(zip(("orders_per_launch", "sites_per_thread", "threads"),
                                          plan.blocking_shape()),
                                      kernel=kernel_name(plan.blocking_kernel())),
            "parallelism": f"replicas x{world} (one ensemble per GPU)",
        },
        "site_vector_steps_per_s": site_steps,
        "roofline": roofline,
        "gpu_launches": gpu_launches,
        "clocks": clk,
    }
    line.update(out)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    return 0


# ----------------------------------------------------------------------------------------
# the other configurations (one problem per GPU): --workload ribbon | holstein | doublewell |
# adjoint
# ----------------------------------------------------------------------------------------
def _single_setup(args):
    """(name, build_plan(cb) -> (plan, psi, host_packet), dt, nsteps_config, oracle_operator,
    emin/emax/alpha, sites, description)"""
    wk = args.workload
    if wk == "ribbon":
        rb = wl.Ribbon()
        return dict(name="zigzag ribbon 128x2048, W=1, single vector, dt=1", sites=rb.n_sites,
                    dt=rb.dt, nsteps=rb.nsteps, kind="ribbon", obj=rb, bounds=rb.bounds(),
                    alpha=0.0, packet=rb.packet())
    if wk == "holstein":
        hs = wl.Holstein()
        if args.hol_size:
            L, nph = (int(x) for x in args.hol_size.split(":"))
            hs = wl.Holstein(L=L, nph=nph)
        return dict(name=f"Holstein L={hs.L} periodic, nph<={hs.nph} (D={hs.dim:,}), dt=0.25",
                    sites=hs.dim,
                    dt=hs.dt, nsteps=hs.nsteps, kind="holstein", obj=hs, bounds=hs.bounds(),
                    alpha=hs.alpha, packet=hs.initial_state())
    if wk == "paperwell":
        d = wl.PaperDoubleWell()
        return dict(name="double well of Sec. 3.1, N=2048, dt=0.4 to t=40", sites=d.n, dt=d.dt,
                    nsteps=d.nsteps, kind="doublewell", obj=d, bounds=d.bounds(), alpha=0.01,
                    packet=d.packet(), exact=True)
    if wk == "doublewell":
        d = wl.DoubleWell1D()
        return dict(name="1D double well N=2048, dt=0.5 (M=6353)", sites=d.n, dt=d.dt,
                    nsteps=d.nsteps, kind="doublewell", obj=d, bounds=d.bounds(), alpha=0.01,
                    packet=d.packet())
    rb = wl.Ribbon(W=60, L=1000, disorder=1.0, seed=3022, c0=250, r0=30)
    return dict(name="adjoint gradient of P_R (x_R=500) on a 60x1000 ribbon, T=300, dt=1",
                sites=rb.n_sites, dt=rb.dt, nsteps=300, kind="adjoint", obj=rb,
                bounds=rb.bounds(), alpha=0.0, packet=rb.packet())


def _single_plan(cb, cfg, prec):
    import torch

    o = cfg["obj"]
    if cfg["kind"] in ("ribbon", "adjoint"):
        eps = torch.from_numpy(o.onsite()).to("cuda")
        desc, keep = cb.desc_ribbons([o.W], [o.L], o.hop, eps)
    elif cfg["kind"] == "holstein":
        desc = cb.desc_holstein(o.L, o.nph, o.periodic, o.hop, o.omega0, o.g,
                                matrix_free=cfg.get("matrix_free", False),
                                sell_sigma=cfg.get("sell_sigma", 0))
        keep = ()
    else:
        V = torch.from_numpy(o.potential()).to("cuda")
        desc, keep = cb.desc_lat1d(o.n, o.dx, V), (V,)
    lo, hi = cfg["bounds"]
    plan = cb.Plan(desc, [lo], [hi], cfg["alpha"], prec, 1, keep=keep)
    dt = torch.complex64 if prec == cb.CHEB_C64 else torch.complex128
    psi = torch.from_numpy(cfg["packet"]).to(dt).to("cuda").contiguous()
    return plan, psi


def _oracle_operator(cfg):
    import oracle

    o = cfg["obj"]
    if cfg["kind"] in ("ribbon", "adjoint"):
        return oracle.honeycomb(o.W, o.L, o.hop, o.onsite())
    if cfg["kind"] == "holstein":
        return oracle.holstein(o.L, o.nph, o.periodic, o.hop, o.omega0, o.g)
    return oracle.lattice1d(o.n, o.dx, o.potential())


def run_single(args, world, rank, local):
    import torch

    import oracle
    import paper_0907_3022_gb300 as cb

    torch.cuda.set_device(local)
    cfg = _single_setup(args)
    cfg["matrix_free"] = bool(args.matrix_free)
    cfg["sell_sigma"] = args.sell_sigma
    prec = cb.CHEB_C64 if args.prec == "c64" else cb.CHEB_C128
    plan, psi = _single_plan(cb, cfg, prec)
    stream = torch.cuda.current_stream()
    plan.evolve(psi, cfg["dt"], 0)
    if args.blocking is None:
        plan.autotune()
    else:  # fixed launch shape (profiling runs): blocking as given, else the plan's default
        f = args.blocking.split(":")
        if int(f[0]) > 0:
            kern = kernel_of(f[3]) if len(f) > 3 else cb.CHEB_TB_SITES
            plan.set_blocking_kernel(int(f[0]), int(f[1]), int(f[2]) if len(f) > 2 else 256, kern)
    M = plan.block(0)["M"]
    a, b = oracle.rescale(*cfg["bounds"], cfg["alpha"])
    out = {}
    if cfg["kind"] == "adjoint":
        # one step = one gradient of P_R through T = 300 time steps (forward, checkpointed
        # recompute and reverse sweep); matvec-steps counted: forward T M, checkpoint forward
        # T M, segment recompute <= T M, reverse T (M + 1)
        T = cfg["nsteps"]
        grad = torch.zeros(cfg["sites"], dtype=torch.float64, device="cuda")
        P = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            plan.adjoint_potential(psi, cfg["dt"], T, region_col=500, grad=grad, P=P)
        mv_per_step = T * (4 * M + 1)
        launches0 = plan.launches()
        clocks = Clocks(local)
        torch.cuda.synchronize()
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.adjoint_potential(psi, cfg["dt"], T, region_col=500, grad=grad, P=P)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        gpu_launches = plan.launches() - launches0
        value = mv_per_step * args.steps / (ms / 1e3)
        roofline = adjoint_roofline(cb, M, T, cfg["sites"], ms / args.steps, prec == cb.CHEB_C128)
        if not args.no_cpu_baseline:
            H = _oracle_operator(cfg)
            C, _ = oracle.coeffs(a, b, cfg["dt"])
            mask = (np.arange(cfg["sites"]) % cfg["obj"].L > 500).astype(np.uint8)
            t0 = time.perf_counter()
            Pr, gref, _ = H.adjoint_region(a, b, C, 20, cfg["packet"], mask)
            tcpu = time.perf_counter() - t0
            out["cpu_baseline"] = {"value": 20 * (4 * M + 1) / tcpu, "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(),
                                   "kind": "oracle", "sample": "gradient through 20 of the 300 "
                                   "time steps (FP64 oracle stores every v_k)"}
        line_cfg = {"workload": cfg["name"], "checkpointing": "ceil(sqrt(M+1)) pairs per step"}
        dtype = "f64" if prec == cb.CHEB_C128 else "c64"
        unit_note = {"gradients_per_s": args.steps / (ms / 1e3)}
    else:
        ss_per_step = M * cfg["sites"]
        mv_per_step = M
        plan.evolve(psi, cfg["dt"], args.warmup)
        plan.sync()
        # value: the graph path (small problems are launch-latency bound, so per-launch events
        # would distort it); kernel durations: a second, event-bracketed run of a few steps
        launches0 = plan.launches()
        clocks = Clocks(local)
        torch.cuda.synchronize()
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.evolve(psi, cfg["dt"], args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        gpu_launches = plan.launches() - launches0
        plan.set_timing(True)
        plan.kernel_stats(reset=True)
        plan.evolve(psi, cfg["dt"], min(args.steps, 5))
        kms, kcount, kbytes = plan.kernel_stats(reset=True)
        plan.set_timing(False)
        value = mv_per_step * args.steps / (ms / 1e3)
        peak, peak_kind = measured_peaks()
        dkey = "f64" if prec == cb.CHEB_C128 else "c64"
        ukind = cfg["kind"] + ("-mf" if cfg["matrix_free"] and cfg["kind"] == "holstein" else "")
        per_unit = ALG_BYTES_PER_UNIT[(ukind, dkey)]
        ms_per_launch = kms / max(kcount, 1)
        alg_per_launch = per_unit * cfg["sites"] * M * min(args.steps, 5) / max(kcount, 1)
        achieved = alg_per_launch / (ms_per_launch / 1e3) / 1e9
        bound = "hbm"
        note = None
        if prec == cb.CHEB_C128:
            bound = "alu"
            note = ("complex128: about 10 FP64 instructions per site-order against ~1.19 "
                    "TFLOP/s FP64 (measured FMA probe); the HBM figures are for reference")
        l2_note = ("working set in L2" if cfg["sites"] * 16 * 5 < 100e6 else "inputs larger than L2")
        rtype = "double" if prec == cb.CHEB_C128 else "float"
        if cfg["matrix_free"] and cfg["kind"] == "holstein":
            kname = "k_rec_holmf<%s>" % rtype
        elif cfg["kind"] == "doublewell" and plan.cluster():
            kname = "k_step_cluster<%s> (%d-CTA cluster, one launch per step)" % (rtype, plan.cluster())
        elif cfg["kind"] == "ribbon" and plan.blocking()[0]:
            kname = "k_rec_tb<1,%d,%d> (temporal blocking)" % tuple(plan.blocking_shape()[1:])
        else:
            kname = "k_rec<%s,1,%s>" % (rtype, "SellOp" if cfg["kind"] == "holstein" else "StencilOp")
        roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None, "kernel": kname,
                    "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "launches": kcount, "kernel_ms_total": kms,
                    "alg_bytes_per_launch": alg_per_launch, "alg_bytes_per_unit": per_unit,
                    "unit_definition": "one row (site) and one Chebyshev order",
                    "kernel_bytes_per_launch": kbytes / max(kcount, 1), "note": note}
        if cfg["kind"] == "ribbon" and plan.blocking()[0]:
            roofline = blocked_roofline(cb, plan, kms, kcount, min(args.steps, 5), per_unit,
                                        "one site and one Chebyshev order")
        if cfg["kind"] == "doublewell" and plan.cluster():
            roofline = cluster_roofline(cb, plan, cfg["sites"] * M * min(args.steps, 5), kms,
                                        prec == cb.CHEB_C128, local, roofline)
        # accuracy: against the oracle after min(steps done, config) steps from the packet
        nacc = {"holstein": 2, "ribbon": 50}.get(cfg["kind"], cfg["nsteps"])
        if args.lean:
            nacc = 0
        if nacc:
            x = torch.from_numpy(cfg["packet"]).to(psi.dtype).to("cuda").contiguous()
            plan.evolve(x, cfg["dt"], nacc)
            H = _oracle_operator(cfg)
            C, _ = oracle.coeffs(a, b, cfg["dt"])
            ref = H.evolve(a, b, C, nacc, cfg["packet"])
            res = x.cpu().numpy().astype(np.complex128)
            out["accuracy"] = {"rel_l2_vs_fp64_oracle": float(np.linalg.norm(res - ref) /
                                                              np.linalg.norm(ref)),
                               "sample": f"{nacc} steps from the initial state"}
            if cfg.get("exact"):
                # against full diagonalisation (Sec. 3.1 quotes < 2e-11 for the Chebyshev
                # method), absolute error in the continuum normalisation psi_i / sqrt(dx)
                from scipy.linalg import eigh_tridiagonal

                dd, ee = cfg["obj"].tridiagonal()
                E, U = eigh_tridiagonal(dd, ee)
                ex = U @ (np.exp(-1j * E * nacc * cfg["dt"]) * (U.T @ cfg["packet"]))
                out["accuracy"]["max_abs_err_vs_exact_diagonalisation"] = float(
                    np.max(np.abs(res - ex)) / np.sqrt(cfg["obj"].dx))
        if not args.no_cpu_baseline and not args.lean:
            H = _oracle_operator(cfg)
            C, _ = oracle.coeffs(a, b, cfg["dt"])
            psi0 = cfg["packet"]
            t0 = time.perf_counter()
            H.step(a, b, C, psi0)
            tcpu = time.perf_counter() - t0
            out["cpu_baseline"] = {"value": mv_per_step / tcpu, "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(),
                                   "kind": "oracle", "sample": "one time step (FP64 oracle)",
                                   "site_steps_per_s": ss_per_step / tcpu}
        # e2e: every step one job from pinned host memory through cheb_evolve_host
        pin = torch.from_numpy(cfg["packet"]).to(psi.dtype).pin_memory()
        pout = torch.empty_like(pin).pin_memory()
        plan.evolve_host(pin, pout, 2, cfg["dt"], 1, in_stride=0, out_stride=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.evolve_host(pin, pout, args.steps, cfg["dt"], 1, in_stride=0, out_stride=0)
        e2e_s = time.perf_counter() - t0
        nb = pin.numel() * pin.element_size()
        out["e2e"] = {"value": mv_per_step * args.steps / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
                      "api": "cheb_evolve_host (pinned host buffers)"}
        if cfg["kind"] == "holstein" and not cfg["matrix_free"]:
            st = plan.sell_stats()
            out["sell"] = {"sigma": st["sigma"], "stored_entries": st["stored"],
                           "offdiag_entries": st["offdiag"],
                           "padding": st["stored"] / max(st["offdiag"], 1) - 1.0}
        line_cfg = {"workload": cfg["name"], "sites": cfg["sites"], "M": M, "l2": l2_note,
                    "operator": ("matrix-free" if cfg["matrix_free"] else "SELL-32")
                    if cfg["kind"] == "holstein" else "stencil",
                    "launch_shape": dict(zip(("threads", "sites_per_thread", "grid",
                                              "vecs_per_thread"), plan.launch_shape()))}
        dtype = "f64" if prec == cb.CHEB_C128 else "c64"
        unit_note = {"site_steps_per_s": ss_per_step * args.steps / (ms / 1e3)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": line_cfg, "roofline": roofline, "gpu_launches": gpu_launches,
            "clocks": clk}
    line.update(unit_note)
    line.update(out)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    return 0


def cluster_roofline(cb, plan, site_orders, kms, fp64, local, hbm):
    """The cluster step runs on the cluster's SMs only (8 or 16), a chunk of the chain each, and
    is bound by their arithmetic (complex128: FP64) or by its barriers (complex64).  Counted per
    useful site-order from the kernel: complex128 8 FP64 pipe instructions (2 DADD neighbour
    sums, 4 DFMA for beta and d, 2 for the accumulation), complex64 12 FP32 (2 FADD, 4 FFMA for
    beta as a float pair, 2 for d, 4 for the accumulation as a float pair); the super-steps'
    recomputed edge sites are not counted.  Peak: the library's probe of the whole GPU's FMA
    rate, times the cluster's CTAs over the SMs."""
    import torch

    ctas = plan.cluster()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    per = 8 if fp64 else 12
    probe = cb.cheb_measure_peak(cb.CHEB_PEAK_FP64_GFLOPS if fp64 else cb.CHEB_PEAK_FP32_GFLOPS)
    peak = probe / 2.0 * ctas / sms  # G FMA instructions/s of the cluster's SMs
    achieved = per * site_orders / (kms / 1e3) / 1e9
    return {"bound": "fp64" if fp64 else "latency", "achieved": achieved, "peak": peak,
            "unit": "G %s pipe instructions/s" % ("FP64" if fp64 else "FP32"),
            "frac": achieved / peak, "traffic": None, "kernel": hbm["kernel"],
            "peak_kind": "FMA rate measured in this run by the library's probe, x %d CTAs / %d SMs"
                         % (ctas, sms),
            "per_unit": "%d %s instructions per useful site-order" % (per, "FP64" if fp64 else "FP32"),
            "note": None if fp64 else "complex64: the cluster barriers between super-steps, not "
                                      "FP32, bound the step; the FP32 fraction is for reference",
            "hbm_reference": {"achieved": hbm["achieved"], "peak": hbm["peak"], "unit": "GB/s",
                              "frac": hbm["frac"], "alg_bytes_per_unit": hbm["alg_bytes_per_unit"]}}


def adjoint_roofline(cb, M, T, sites, ms_per_gradient, fp64):
    """FP64 roofline of one gradient (complex128): FP64 pipe instructions per site, counted
    from the kernels' arithmetic -- the fused forward step 10 per order (4 DADD neighbour sums,
    4 DFMA for 2 H~ x - p, 2 for the accumulation on average), the checkpoint and segment
    recompute kernel 12 (the stencil 10, the subtraction 2), the reverse kernel 27 (the
    conjugated coefficient 8, the stencil 10, the update 4, the gradient term 5) and 8 at the
    last order (no matvec) -- times the launches of the sqrt(M) schedule, over the whole
    gradient's time (launch gaps included), against the DFMA rate measured in this run."""
    S = math.ceil(math.sqrt(M + 1))
    nseg = (M + 1 + S - 1) // S
    kc = min(M - 1, (nseg - 1) * S + 1)
    rec = sum(max(0, min(min(j * S + S - 1, M), M - 1) - j * S - 1) for j in range(nseg))
    per_step = M * 10 + kc * 12 + rec * 12 + M * 27 + 8
    inst = per_step * T * sites
    achieved = inst / (ms_per_gradient / 1e3) / 1e9
    out = {"kernel": "k_adj_forward/k_adj_reverse + fused forward steps (whole gradient)",
           "unit": "G FP64 pipe instructions/s", "traffic": None,
           "launches_per_gradient": T * (M + kc + rec + M + 1) + 1,
           "fp64_instructions_per_gradient": inst,
           "per_unit": "per site and time step: 10 M (forward) + 12 (kc + recomputed) + 27 M + 8 "
                       "(reverse) FP64 instructions"}
    if not fp64:
        out.update({"bound": "launch", "achieved": None, "peak": None, "frac": None,
                    "note": "complex64: FP32 arithmetic; the gradient is bound by the launch "
                            "latency of its ~3 M kernels per time step"})
        return out
    peak = cb.cheb_measure_peak(cb.CHEB_PEAK_FP64_GFLOPS) / 2.0
    out.update({"bound": "fp64", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                "peak_kind": "DFMA rate measured in this run by the library's probe"})
    return out


def run_reference_single(args, world, rank):
    """The oracle as the reference arm for --workload != ensemble (one step per step)."""
    if rank != 0:
        return 0
    import oracle

    cfg = _single_setup(args)
    H = _oracle_operator(cfg)
    a, b = oracle.rescale(*cfg["bounds"], cfg["alpha"])
    C, M = oracle.coeffs(a, b, cfg["dt"])
    psi = cfg["packet"]
    for _ in range(args.warmup):
        psi = H.step(a, b, C, psi)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        psi = H.step(a, b, C, psi)
    tt = time.perf_counter() - t0
    value = M * args.steps / tt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} time steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_driven(args, world, rank, local):
    """Time-dependent H(t) (Sec. 2.2), piecewise constant over each step: the 128 x 2048
    zigzag ribbon with an oscillating field F sin(Omega t) (c - L/2)/L along the ribbon added
    to its disorder, sampled at the step midpoints; every step rescales the diagonal on the
    device before its M launches."""
    import torch

    import oracle
    import paper_0907_3022_gb300 as cb

    torch.cuda.set_device(local)
    prec = cb.CHEB_C64 if args.prec == "c64" else cb.CHEB_C128
    cdt = torch.complex64 if prec == cb.CHEB_C64 else torch.complex128
    rb = wl.Ribbon()
    F, Om = 0.5, 0.2
    col = (np.arange(rb.n_sites) % rb.L - rb.L / 2) / rb.L
    base = rb.onsite()

    def field(t):
        return base + F * math.sin(Om * t) * col

    K = args.steps
    seq = torch.from_numpy(np.stack([field((s + 0.5) * rb.dt) for s in range(K)])).to("cuda")
    lo, hi = rb.bounds()
    lo, hi = lo - F / 2, hi + F / 2
    eps = torch.from_numpy(base).to("cuda")
    desc, keep = cb.desc_ribbons([rb.W], [rb.L], rb.hop, eps)
    plan = cb.Plan(desc, [lo], [hi], 0.0, prec, 1, keep=keep)
    psi = torch.from_numpy(rb.packet()).to(cdt).to("cuda").contiguous()
    plan.evolve(psi, rb.dt, 0)
    plan.autotune()
    M = plan.block(0)["M"]
    plan.evolve_td(psi, rb.dt, max(args.warmup, 3), seq)
    stream = torch.cuda.current_stream()
    launches0 = plan.launches()
    clocks = Clocks(local)
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.evolve_td(psi, rb.dt, K, seq)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    gpu_launches = plan.launches() - launches0
    # the same number of steps with H fixed (graph path), for the cost of the per-step update
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    plan.evolve(psi, rb.dt, K)
    s1.record(stream)
    torch.cuda.synchronize()
    out = {}
    if not args.lean:
        nacc = 3
        x = torch.from_numpy(rb.packet()).to(cdt).to("cuda").contiguous()
        plan.evolve_td(x, rb.dt, nacc, seq)
        a, b = oracle.rescale(lo, hi, 0.0)
        C, _ = oracle.coeffs(a, b, rb.dt)
        t0 = time.perf_counter()
        ref = oracle.evolve_piecewise(lambda V: oracle.honeycomb(rb.W, rb.L, rb.hop, V),
                                      [field((s + 0.5) * rb.dt) for s in range(nacc)], a, b, C,
                                      rb.packet())
        tcpu = time.perf_counter() - t0
        res = x.cpu().numpy().astype(np.complex128)
        out["accuracy"] = {"rel_l2_vs_fp64_oracle": float(np.linalg.norm(res - ref)
                                                          / np.linalg.norm(ref)),
                           "sample": f"{nacc} steps from the packet"}
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = {"value": M * nacc / tcpu, "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(),
                                   "kind": "oracle", "sample": f"{nacc} driven steps (operator "
                                   "rebuilt every step, FP64 oracle, single thread)"}
    line = {"metric": METRIC, "value": M * K / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": max(args.warmup, 3), "ms_per_step": ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64" if prec == cb.CHEB_C64 else "f64", "data": "synthetic",
            "config": {"workload": "driven zigzag ribbon 128x2048: disorder + F sin(Omega t) "
                                   "(c - L/2)/L, F = 0.5, Omega = 0.2, dt = 1, midpoint samples",
                       "M": M, "static_ms_per_step": s0.elapsed_time(s1) / K,
                       "l2": "working set in L2"},
            "roofline": None, "gpu_launches": gpu_launches, "clocks": clk}
    line.update(out)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    return 0


def run_armchair(args, world, rank, local):
    """Table 2 (Sec. 3.2): armchair ribbons of 10 x 1000 atoms with disorder W = 0.5 and 4 (one
    two-ribbon plan), the state on one central site, propagated to t = 10^4 with dt = 1, 10
    and 100; each propagation is timed once (time to solution), the rate is the sum of the
    matvecs over the sum of the times."""
    import torch

    import oracle
    import paper_0907_3022_gb300 as cb

    torch.cuda.set_device(local)
    prec = cb.CHEB_C64 if args.prec == "c64" else cb.CHEB_C128
    cdt = torch.complex64 if prec == cb.CHEB_C64 else torch.complex128
    rbs = [wl.ArmchairRibbon(disorder=w, stream=q) for q, w in enumerate((0.5, 4.0))]
    eps = torch.from_numpy(np.concatenate([rb.onsite() for rb in rbs])).to("cuda")
    desc, keep = cb.desc_armchair([rb.n_a for rb in rbs], [rb.length for rb in rbs], 1.0, eps)
    plan = cb.Plan(desc, [rb.bounds()[0] for rb in rbs], [rb.bounds()[1] for rb in rbs], 0.0,
                   prec, 1, keep=keep)
    x0 = np.concatenate([rb.packet() for rb in rbs])
    stream = torch.cuda.current_stream()
    runs, finals = {}, {}
    tot_mv, tot_ms, tot_steps = 0.0, 0.0, 0
    launches0 = plan.launches()
    clocks = Clocks(local)
    clocks.start()
    for dt in (1.0, 10.0, 100.0):
        nsteps = int(round(1e4 / dt))
        psi = torch.from_numpy(x0).to(cdt).to("cuda").contiguous()
        plan.evolve(psi, dt, 0)
        plan.autotune()
        plan.evolve(psi, dt, max(args.warmup, 3))
        psi.copy_(torch.from_numpy(x0).to(cdt))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.evolve(psi, dt, nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        Ms = [plan.block(q)["M"] for q in range(len(rbs))]
        mv = sum(Ms) * nsteps
        runs[str(int(dt))] = {"M": Ms, "steps": nsteps, "seconds_to_t1e4": ms / 1e3,
                              "matvec_steps_per_s": mv / (ms / 1e3)}
        finals[dt] = psi.cpu().numpy().astype(np.complex128)
        tot_mv += mv
        tot_ms += ms
        tot_steps += nsteps
    clk = clocks.stop()
    gpu_launches = plan.launches() - launches0
    acc = {"max_abs_diff_dt1_vs_dt100": float(np.max(np.abs(finals[1.0] - finals[100.0]))),
           "max_abs_diff_dt10_vs_dt100": float(np.max(np.abs(finals[10.0] - finals[100.0])))}
    out = {}
    if not args.lean:
        off = np.cumsum([0] + [rb.n_sites for rb in rbs])
        errs = []
        t0 = time.perf_counter()
        for q, rb in enumerate(rbs):
            a, b = oracle.rescale(*rb.bounds(), 0.0)
            C, _ = oracle.coeffs(a, b, 100.0)
            ref = oracle.honeycomb(rb.W, rb.L, 1.0, rb.onsite()).evolve(a, b, C, 100, rb.packet())
            errs.append(float(np.linalg.norm(finals[100.0][off[q]:off[q + 1]] - ref)
                              / np.linalg.norm(ref)))
        tcpu = time.perf_counter() - t0
        acc["rel_l2_vs_fp64_oracle_dt100"] = max(errs)
        if not args.no_cpu_baseline:
            mv100 = sum(runs["100"]["M"]) * 100
            out["cpu_baseline"] = {"value": mv100 / tcpu, "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(),
                                   "kind": "oracle", "sample": "both ribbons to t = 10^4 with "
                                   "dt = 100 (FP64 oracle, single thread)",
                                   "seconds_to_t1e4_dt100": tcpu}
    line = {"metric": METRIC, "value": tot_mv / (tot_ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": tot_steps, "warmup": max(args.warmup, 3), "ms_per_step": tot_ms / tot_steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64" if prec == cb.CHEB_C64 else "f64", "data": "synthetic",
            "config": {"workload": "Table 2: armchair ribbons 10 x 1000 atoms, W = 0.5 and 4, one "
                                   "central site, t = 10^4 with dt = 1, 10, 100",
                       "runs": runs, "l2": "working set in L2"},
            "roofline": None, "gpu_launches": gpu_launches, "clocks": clk, "accuracy": acc,
            "paper_context": "Table 2: one Xeon 5160 core, 378 / 97 / 45 s for dt = 1 / 10 / 100 "
                             "(its M = 104 / 264 / 1210 follow another cutoff)"}
    line.update(out)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    return 0


def run_polaron(args, world, rank, local):
    """The paper's polaron run (Sec. 3.3, Fig. 3): 18 sites, <= 11 phonons, D = 622,751,220;
    one step = one dt = 0.25 of the whole state; observables at the end of the timed region."""
    import torch

    import paper_0907_3022_gb300 as cb

    torch.cuda.set_device(local)
    pw = wl.Polaron()
    prec = cb.CHEB_C128 if args.prec == "c128" else cb.CHEB_C64
    d = torch.from_numpy(pw.delta()).to("cuda")
    g = torch.from_numpy(pw.gsite()).to("cuda")
    desc = cb.desc_holstein(pw.L, pw.nph, pw.periodic, pw.hop, pw.omega0, 1.0, delta=d, gsite=g,
                            matrix_free=args.matrix_free, sell_sigma=args.sell_sigma)
    lo, hi = pw.bounds()
    t0 = time.perf_counter()
    plan = cb.Plan(desc, [lo], [hi], pw.alpha, prec, 1, keep=(d, g))
    build_s = time.perf_counter() - t0
    cdt = torch.complex64 if prec == cb.CHEB_C64 else torch.complex128
    psi = torch.zeros(pw.dim, dtype=cdt, device="cuda")
    idx = torch.from_numpy(pw.packet_indices()).to("cuda")
    psi[idx] = torch.from_numpy(pw.electron_packet()).to(cdt).to("cuda")
    stream = torch.cuda.current_stream()
    plan.evolve(psi, pw.dt, 0)
    M = plan.block(0)["M"]
    plan.autotune()
    plan.evolve(psi, pw.dt, args.warmup)
    plan.sync()
    launches0 = plan.launches()
    clocks = Clocks(local)
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.evolve(psi, pw.dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    gpu_launches = plan.launches() - launches0
    plan.set_timing(True)
    plan.kernel_stats(reset=True)
    plan.evolve(psi, pw.dt, 1)
    kms, kcount, kbytes = plan.kernel_stats(reset=True)
    plan.set_timing(False)
    obs = {}
    for name, kind in (("density", cb.CHEB_OBS_HOL_DENSITY), ("phonons", cb.CHEB_OBS_HOL_PHONON),
                       ("chi", cb.CHEB_OBS_HOL_CHI)):
        out = torch.zeros(pw.L, dtype=torch.float64, device="cuda")
        plan.observables(psi, kind, 0.0, out)
        obs[name] = [round(float(x), 6) for x in out.cpu().numpy()]
    n2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.observables(psi, cb.CHEB_OBS_NORM2, 0.0, n2)
    peak, peak_kind = measured_peaks()
    dkey = "f64" if prec == cb.CHEB_C128 else "c64"
    per_unit = ALG_BYTES_PER_UNIT[("holstein-mf" if args.matrix_free else "holstein", dkey)]
    alg_per_launch = per_unit * pw.dim  # every launch forms one order for every row
    ms_per_launch = kms / max(kcount, 1)
    achieved = alg_per_launch / (ms_per_launch / 1e3) / 1e9
    traffic = None
    if args.matrix_free and (dkey, M) in POLARON_MF_DRAM_BYTES_PER_STEP:
        traffic = POLARON_MF_DRAM_BYTES_PER_STEP[(dkey, M)] / M
    steps_done = args.warmup + args.steps + 1
    line = {"metric": METRIC, "value": M * args.steps / (ms / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64" if prec == cb.CHEB_C64 else "f64",
            "data": "synthetic",
            "config": {"workload": "paper polaron run: 18 sites, <= 11 phonons, D = 622,751,220, "
                                   "dt = 0.25", "M": M, "plan_build_s": build_s,
                       "operator": "matrix-free" if args.matrix_free else "SELL-32",
                       "launch_shape": dict(zip(("threads", "sites_per_thread", "grid",
                                                 "vecs_per_thread"), plan.launch_shape())),
                       "l2": "inputs larger than L2"},
            "site_steps_per_s": M * pw.dim * args.steps / (ms / 1e3),
            "time_to_t20_s": ms / args.steps * pw.nsteps / 1e3,
            "roofline": {"bound": "alu" if prec == cb.CHEB_C128 else "hbm", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "kernel": ("k_rec_holmf<%s>" if args.matrix_free else "k_rec<%s,1,SellOp>")
                                   % ("double" if prec == cb.CHEB_C128 else "float"),
                         "peak_kind": f"{peak_kind} copy bandwidth", "launches": kcount,
                         "alg_bytes_per_launch": alg_per_launch, "alg_bytes_per_unit": per_unit,
                         "unit_definition": "one basis row and one Chebyshev order",
                         "kernel_bytes_per_launch": kbytes / max(kcount, 1),
                         "dram_achieved": (traffic / (ms_per_launch / 1e3) / 1e9) if traffic else None},
            "gpu_launches": gpu_launches, "clocks": clk,
            "physics": {"t": steps_done * pw.dt, "norm2": float(n2.item()), **obs},
            "paper_context": "Sec. 3.3: the same basis on 18 SGI Altix 4700 processors, ~60 GB, "
                             "< 500 CPU-hours to t ~ 14-20"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    try:
        if args.impl == "reference":
            if args.workload == "polaron":
                print(json.dumps({"impl": "reference", "unavailable": "the oracle would need "
                                  "~200 GB of host memory for D = 622,751,220"}))
                return 0
            if args.workload == "driven":
                print(json.dumps({"impl": "reference", "unavailable": "the oracle leg of the "
                                  "driven line is its cpu_baseline"}))
                return 0
            if args.workload == "armchair":
                print(json.dumps({"impl": "reference", "unavailable": "the oracle leg of the "
                                  "armchair line is its cpu_baseline (dt = 100)"}))
                return 0
            if args.workload != "ensemble":
                return run_reference_single(args, world, rank)
            return run_reference(args, world, rank)
        if args.workload == "polaron":
            return run_polaron(args, world, rank, local)
        if args.workload == "armchair":
            return run_armchair(args, world, rank, local)
        if args.workload == "driven":
            return run_driven(args, world, rank, local)
        if args.workload != "ensemble":
            return run_single(args, world, rank, local)
        if args.sweep:
            return run_sweep(args, local)
        return run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
