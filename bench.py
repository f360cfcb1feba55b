#!/usr/bin/env python
"""Benchmark: fast multiple-scattering products on the 100 000-patch workload.

Workload: interior (narrow escape) problem, N = 100 000 disk patches of radius
eps = 0.001 on a seeded jittered Fibonacci spiral (jitter 0.3 * sqrt(4 pi / N)),
K = 136 Zernike functions per patch (M = 15, 13.6 M unknowns), ID tolerance 1e-11,
incoming-grid tolerance 1e-8, cube-sphere tree. One step = one product y = A x of
the second-kind system (outgoing map, P2L onto incoming grids, direct sums, L2P,
Zernike transform) in the FP32 kernels that the mixed-precision solve iterates with.
The line also reports the FP64 and float-float product rates, the metric's solves to a
1e-8 relative residual (mixed, float-float and plain FP64, each with its recomputed true
residual and the density error against the FP64 solution), the 256-sphere batch, and the
mixed solves of the other N = 1e5 workloads (exterior, and 20 von Mises-Fisher clusters).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    torchrun --nproc-per-node N bench.py --gpus N ...   (independent replicas)
"""
from __future__ import annotations

import argparse
import faulthandler
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N=1e5 solve time to 1e-8 residual & matvecs/s, mixed vs FP64 on one GB300"
UNIT = "matvecs/s"
WORKLOAD = "interior narrow escape, N=100000 patches, eps=0.001, K=136, jittered Fibonacci layout, cube-sphere tree"
# Nominal work per pair evaluation used for flop rates: 3 sub, 3 mul/fma for d^2,
# rsqrt, log, ~4 for the kernel value, 1 fma accumulate ~ 20 flops (stated, not measured).
FLOPS_PER_PAIR = 20


# DRAM bytes per pair of the FP32 P2L kernel: dram__bytes_read.sum + dram__bytes_write.sum
# of one launch (169.9 + 15.5 MB) over its 1.4535e10 pairs, ncu capture of the packed pair
# loop at N = 2e4 of the same layout family (profiles/p2l_kernel_fp32_N2e4.md); the reads scale
# with the work items. Valid for the launch configuration that was captured (reported as null
# for any other).
P2L_CAPTURE = {"p2l_tile": 16, "item_patches": 16, "bytes_per_pair": 185.5e6 / 1.4535e10}


_T0 = time.time()


def _progress(msg):
    """One line per leg on stderr (the JSON line stays alone on stdout)."""
    print(f"[bench +{time.time() - _T0:.1f}s] {msg}", file=sys.stderr, flush=True)


def _workload_name(args, N):
    """The workload line: the metric's configuration, or the variant the flags select."""
    if args.mode == "interior" and args.layout == "fibonacci" and N == 100000:
        return WORKLOAD
    lay = "jittered Fibonacci layout" if args.layout == "fibonacci" else "20 von Mises-Fisher clusters (kappa=50)"
    kind = "interior narrow escape" if args.mode == "interior" else "exterior narrow capture"
    return f"{kind}, N={N} patches, eps=0.001, K=136, {lay}, cube-sphere tree"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(v, device="cpu"):
    """Largest per-rank value (the step time of the slowest replica); identity with one
    rank. device: where the process group's backend reduces (cuda for NCCL, cpu for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(v)
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(ms_per_step_max, world_size, units_per_step=1.0):
    """Whole-job throughput of independent replicas: the units all ranks processed per
    step over the slowest rank's step time."""
    return world_size * units_per_step * 1000.0 / ms_per_step_max


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"ncs_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
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
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1906_04209_gb300 import layouts as L, ncs

    ws, rank = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    centres, eps, mode, K = L.workload(3, layout=args.layout, N=args.patches)
    if args.mode == "exterior":
        mode = ncs.EXTERIOR
    N = len(centres)
    t0 = time.time()
    ctx = ncs.Context(eps, mode, K, method=ncs.METHOD_TREE, grid_tol=args.grid_tol, tensor_cores=args.tensor_cores)
    ctx.set_patches(centres)
    setup_s = time.time() - t0
    tuning = None
    if args.set_tuning:
        kv = dict(item.split("=") for item in args.set_tuning.split(","))
        ctx.set_tuning(**{k: (float(v) if k == "l2p_weight" else int(v)) for k, v in kv.items()})
        tuning = {"config": ctx.get_tuning(), "set": True}
    elif args.tune:
        _progress("tune")
        cfg, rep = ctx.tune(flags=3)
        tuning = {"config": cfg, "default_ms": round(rep["default_ms"], 3), "tuned_ms": round(rep["tuned_ms"], 3),
                  "trial_products": int(rep["trial_products"]), "error_vs_df64": rep["error"],
                  "seconds": round(rep["seconds"], 2)}
    info, tstats = ctx.info(), ctx.tree_stats()
    n = N * K
    g = torch.Generator(device="cuda").manual_seed(1234 + rank)
    x = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    prec = ncs.FP32 if args.precision == "fp32" else ncs.FP64

    def step(p=prec):
        ctx.matvec_dev(x.data_ptr(), y.data_ptr(), p, sp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-stage times of one product (the dominant kernel's duration for the roofline)
    stages32 = ctx.profile_matvec(x.data_ptr(), y.data_ptr(), prec, sp)

    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # P2L duration inside the timed region, measured on the launching stream
    e0.record(stream)
    n_launch0 = ncs.launch_count()
    for _ in range(args.steps):
        step()
    n_launches = ncs.launch_count() - n_launch0
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms_step = ms_total / args.steps
    ms_step = max_over_ranks(ms_step, device="cuda")
    value = replica_rate(ms_step, ws)

    # stage profile repeated inside a timed loop: the P2L share of each product
    p2l_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        p2l_ms.append(ctx.profile_matvec(x.data_ptr(), y.data_ptr(), prec, sp)["p2l"])
    p2l_avg = float(np.mean(p2l_ms))

    # end to end through the C ABI with host buffers (pinned), H2D + product + D2H
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    xh.copy_(x.cpu())
    yh = torch.empty(n, dtype=torch.float64).pin_memory()
    lib = ncs.load()
    import ctypes
    Dp = ctypes.POINTER(ctypes.c_double)
    ee = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ee):
        rc = lib.ncs_matvec(ctx.h, ctypes.cast(xh.data_ptr(), Dp), ctypes.cast(yh.data_ptr(), Dp), prec)
        assert rc == 0, ncs.load().ncs_last_error(ctx.h)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / ee, device="cuda")

    # FP64 product rate (fewer steps: the FP64 pipe is the bottleneck on this part)
    fma_peaks = {"fp64_tflops": round(ncs.fma_peak(ncs.FP64), 2), "fp32_tflops": round(ncs.fma_peak(ncs.FP32), 2),
                 "source": "ncs_fma_peak microkernel (independent FMA chains, best of 3 launches)"}
    fp64 = None
    if args.fp64_steps > 0:
        step(ncs.FP64)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.fp64_steps):
            step(ncs.FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64 = 1000.0 * args.fp64_steps / e0.elapsed_time(e1)

    df64 = None
    if args.df64_steps > 0:
        step(ncs.DF64)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.df64_steps):
            step(ncs.DF64)
        e1.record(stream)
        torch.cuda.synchronize()
        df64 = 1000.0 * args.df64_steps / e0.elapsed_time(e1)

    _progress("products done")
    solve = None
    if args.solve:
        solve = solve_legs(args, ctx, N, K, sp)

    batch = batch_leg(args) if (args.batch and rank == 0) else None
    others = other_workloads_leg(args) if (args.other_workloads and rank == 0 and args.patches is None) else None

    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # ALU roofline of the pair kernel: per pair the FP32 path issues mufu_per_pair MUFU
    # ops (an rsqrt unless the pair takes the Newton reciprocal square root on the FMA pipe,
    # a lg2 unless it takes the polynomial logarithm there); 152 SMs x 16 MUFU/clk cap it at
    # 16 / mufu_per_pair pairs/clk/SM. Two fixed bounds are reported beside it: the joint
    # MUFU + FMA-pipe bound over every share of the two offloads (9 FP32 operations per pair,
    # plus 7 per Newton rsqrt and 11 per polynomial log2, on 128 FMA lanes; the cheaper
    # rsqrt share b balances the pipes first: 16 / (2 - b) = 128 / (9 + 7 b) at b = 112/240,
    # 10.43 pairs/clk/SM), and the FP32 pipe at the nominal 20 flops per pair (128 lanes x 2
    # flops per clock).
    tuned_cfg = ctx.get_tuning()
    poly, rsq = tuned_cfg["p2l_poly"], tuned_cfg["p2l_rsq"]
    mufu_per_pair = 2.0 - (poly + rsq) / 16.0
    pair_peak = 152 * (16.0 / mufu_per_pair) * sm_max * 1e6 if prec == ncs.FP32 else None
    p2l_pairs = tstats["p2l_pairs"]
    achieved_pairs = p2l_pairs / (p2l_avg / 1000.0)
    roof = {
        "kernel": "p2l_kernel (interaction-list skeletons -> incoming grids)",
        "bound": "alu",
        "achieved": round(achieved_pairs * FLOPS_PER_PAIR / 1e12, 3),
        "peak": round(pair_peak * FLOPS_PER_PAIR / 1e12, 3) if pair_peak else None,
        "unit": "TFLOP/s",
        "frac": round(achieved_pairs / pair_peak, 4) if pair_peak else None,
        # DRAM bytes per launch: an ncu capture of this kernel on the N = 2e4 layout of the
        # same family (P2L_CAPTURE), scaled by the pair ratio; the arithmetic variants
        # (polynomial log, Newton rsqrt shares) move no data, so only the staging (patches per
        # tile and per work item) must match the capture (null otherwise and for other
        # precisions)
        "traffic": (round(P2L_CAPTURE["bytes_per_pair"] * p2l_pairs)
                    if prec == ncs.FP32 and all(tuned_cfg[k] == P2L_CAPTURE[k] for k in ("p2l_tile", "item_patches"))
                    else None),
        "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum at N=2e4, scaled by pairs",
        "pairs_per_launch": p2l_pairs,
        "ms_per_launch": round(p2l_avg, 3),
        "peak_source": "derived: 152 SMs x 16 MUFU/clk / %g MUFU per pair x %g MHz (%s clocks)" % (
            mufu_per_pair, sm_max, src),
        "frac_joint_mufu_fma": (round(achieved_pairs / (152 * (16.0 / (2.0 - 112.0 / 240.0)) * sm_max * 1e6), 4)
                                if prec == ncs.FP32 else None),
        "frac_fp32_pipe": (round(achieved_pairs * FLOPS_PER_PAIR / (152 * 256 * sm_max * 1e6), 4)
                           if prec == ncs.FP32 else None),
    }
    cpu = cpu_baseline(args, centres, eps, mode, K) if (rank == 0 and args.cpu_baseline) else None
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == ncs.FP32 else "f64",
        "data": "synthetic (seeded layout, random Gaussian input vector)",
        "config": {"workload": _workload_name(args, N), "N": N, "eps": eps, "K": K, "mode": args.mode,
                   "layout": args.layout, "p": info["p"], "Kstar": info["Kstar"], "levels": tstats["levels"],
                   "grid_tol": args.grid_tol, "tensor_cores": args.tensor_cores, "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "working set > L2 (skeleton offsets 200 MB, z 397 MB, grids per step)",
                   "setup_s": round(setup_s, 2)},
        "e2e": {"value": round(replica_rate(1000.0 * e2e_s, ws), 4), "unit": UNIT, "h2d_bytes_per_step": n * 8,
                "d2h_bytes_per_step": n * 8},
        "gpu_launches": n_launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk,
        "stages_ms": {k: round(v, 3) for k, v in stages32.items()},
        "fma_peaks": fma_peaks,
        "fp64_matvecs_per_s": round(fp64, 4) if fp64 else None,
        "df64_matvecs_per_s": round(df64, 4) if df64 else None,
        "pairs_per_step": tstats["p2l_pairs"] + tstats["direct_pairs"],
        "pair_rate_per_s": round((tstats["p2l_pairs"] + tstats["direct_pairs"]) * 1000.0 / ms_step, 1),
        "tuning": tuning,
        "solve": solve,
        "batch": batch,
        "other_workloads": others,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def solve_legs(args, ctx, N, K, sp):
    """The metric's solves of the same workload to a relative residual of args.solve_tol:
    mixed (FP32 inner GMRES on the inner tree, whose incoming grids are sized to the FP32
    products' accuracy + float-float refinement residuals on the product's tree), float-float (every
    product FP64-accurate on the FP32 pipes) and plain FP64 (every product on the FP64
    pipe). Each is timed around the ncs_solve call (densities copied back included); its
    true residual b - A x is then recomputed with one float-float product, outside the
    timed region, and the densities are compared with the FP64 solve's."""
    import torch

    from paper_1906_04209_gb300 import ncs

    P = ctx.operator()["P"]
    b = torch.tensor(np.tile(P.sum(axis=1), N), dtype=torch.float64, device="cuda")
    bn = float(torch.linalg.norm(b))
    legs = [("mixed", ncs.MIXED), ("df64", ncs.DF64)]
    if args.solve_fp64:
        legs.append(("fp64", ncs.FP64))
    out, fh = {}, {}
    for name, p in legs:
        _progress(f"solve {name}")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.solve(tol=args.solve_tol, precision=p, want_fhat=True, allow_noconv=True)
        sec = time.perf_counter() - t0
        st = ctx.solve_stats()
        xd = torch.from_numpy(r["fhat"]).to("cuda")
        yd = torch.empty_like(xd)
        ctx.matvec_dev(xd.data_ptr(), yd.data_ptr(), ncs.DF64, sp)
        torch.cuda.synchronize()
        true = float(torch.linalg.norm(b - yd)) / bn
        if name == "mixed":
            inf = ctx.info()
            inner = {"grid_tol": ncs.default_params().inner_grid_tol, "grid_points": inf["inner_grid_points"],
                     "pairs_per_product": inf["inner_tree_pairs"], "product_tree_grid_points": inf["grid_points"],
                     "product_tree_pairs": inf["tree_pairs"]}
        out[name] = {"seconds": round(sec, 3), "iterations": r["iterations"],
                     "gmres_steps": int(st["gmres_steps"]), "residual_products": int(st["residual_products"]),
                     "residual_updates": int(st["residual_updates"]), "graph_replays": int(st["graph_replays"]),
                     "mu": r["scalar"], "relres_reported": r["relres"], "relres_true": true, "rc": r["rc"]}
        if name == "mixed":
            out[name]["inner_tree"] = inner
        fh[name] = r["fhat"]
        del xd, yd
    ref = "fp64" if "fp64" in fh else "df64"
    fr = fh[ref]
    for name in fh:
        if name != ref:
            out[name]["density_err_vs_" + ref] = float(np.abs(fh[name] - fr).max() / np.abs(fr).max())
            out[name]["mu_relerr_vs_" + ref] = abs(out[name]["mu"] - out[ref]["mu"]) / abs(out[ref]["mu"])
    # every solution against a tight FP64-accurate one (float-float products to 1e-11,
    # untimed): two iterates that each meet 1e-8 differ by up to cond(A) x 1e-8, so the
    # error of each against the tight solution shows what the tolerance, not the precision,
    # leaves
    _progress("tight reference solve")
    rt = ctx.solve(tol=args.solve_tol * 1e-3, precision=ncs.DF64, want_fhat=True, allow_noconv=True)
    ft = rt["fhat"]
    out["tight_reference"] = {"precision": "df64", "tol": args.solve_tol * 1e-3, "relres": rt["relres"],
                              "iterations": rt["iterations"], "mu": rt["scalar"]}
    for name in fh:
        out[name]["density_err_vs_tight"] = float(np.abs(fh[name] - ft).max() / np.abs(ft).max())
        out[name]["mu_relerr_vs_tight"] = abs(out[name]["mu"] - rt["scalar"]) / abs(rt["scalar"])
    if "fp64" in out:
        out["speedup_mixed_over_fp64"] = round(out["fp64"]["seconds"] / out["mixed"]["seconds"], 2)
        out["speedup_df64_over_fp64"] = round(out["fp64"]["seconds"] / out["df64"]["seconds"], 2)
    out["speedup_mixed_over_df64"] = round(out["df64"]["seconds"] / out["mixed"]["seconds"], 2)
    out["tol"] = args.solve_tol
    # the paper's error measure for its large runs (eq. l2res): the relative L2 residual of
    # the mixed solution on a seeded random patch (untimed)
    ip = int(np.random.default_rng(1906).integers(N))
    _progress("patch residual")
    t0 = time.time()
    l2 = ctx.patch_residual(ip, fh["mixed"])
    out["mixed"]["patch_residual"] = {"patch": ip, "l2": l2, "seconds": round(time.time() - t0, 3)}
    return out


def other_workloads_leg(args):
    """The other N = 1e5 workloads of the metric's family (eps = 0.001, K = 136): exterior on
    the jittered Fibonacci layout, interior and exterior on 20 von Mises-Fisher clusters. Each
    gets its own context, tree and tuned launch configuration; reported: FP32 product time
    (CUDA events, 5 products after 2 warm-up) and the mixed solve to args.solve_tol with its
    true residual recomputed by a float-float product outside the timed region."""
    import torch

    from paper_1906_04209_gb300 import layouts as L, ncs
    out = {}
    for layout, mode in (("fibonacci", ncs.EXTERIOR), ("vmf", ncs.INTERIOR), ("vmf", ncs.EXTERIOR)):
        name = f"{'exterior' if mode == ncs.EXTERIOR else 'interior'}_{layout}"
        _progress(f"workload {name}")
        c, eps, _, K = L.workload(3, layout=layout)
        N = len(c)
        ctx = ncs.Context(eps, mode, K, method=ncs.METHOD_TREE)
        ctx.set_patches(c)
        cfg, rep = ctx.tune(flags=1)  # the pair-kernel variants (no tree rebuilds)
        x = torch.randn(N * K, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        sp = torch.cuda.current_stream().cuda_stream
        for _ in range(2):
            ctx.matvec_dev(x.data_ptr(), y.data_ptr(), ncs.FP32, sp)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            ctx.matvec_dev(x.data_ptr(), y.data_ptr(), ncs.FP32, sp)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.solve(tol=args.solve_tol, precision=ncs.MIXED, want_fhat=True, allow_noconv=True)
        sec = time.perf_counter() - t0
        P = ctx.operator()["P"]
        b = torch.tensor(np.tile(P.sum(axis=1), N), dtype=torch.float64, device="cuda")
        xd = torch.from_numpy(r["fhat"]).to("cuda")
        ctx.matvec_dev(xd.data_ptr(), y.data_ptr(), ncs.DF64, sp)
        torch.cuda.synchronize()
        true = float(torch.linalg.norm(b - y) / torch.linalg.norm(b))
        st = ctx.tree_stats()
        out[name] = {"N": N, "levels": st["levels"], "pairs_per_product": st["p2l_pairs"] + st["direct_pairs"],
                     "tuning": cfg, "ms_per_product": round(ms, 3), "mixed_solve_s": round(sec, 3),
                     "iterations": r["iterations"], "scalar": r["scalar"], "relres_true": true, "rc": r["rc"]}
        del x, y, xd, b
        ctx.close()
    return out


def batch_leg(args):
    """The batch workload: 256 independent spheres (N log-uniform in [50, 5000], eps in
    [0.005, 0.02], half interior, K = 128), each solved to args.solve_tol in mixed
    precision with its own precompute (spheres below the tree threshold in one grouped
    system per mode, the others on concurrent contexts with their own trees); wall time and
    aggregate products/s."""
    from paper_1906_04209_gb300 import layouts as L, ncs
    _progress("batch workload")
    work = L.batch_workload(args.batch_size)
    inst = [(c, e, m) for c, e, m, _ in work]
    K = work[0][3]
    _progress("batch solve")
    t0 = time.perf_counter()
    out = ncs.batch_solve(inst, K, tol=args.solve_tol, precision=ncs.MIXED)
    wall = time.perf_counter() - t0
    prods = int(np.sum(out["iterations"]))
    tmin = ncs.default_params().tree_min_patches
    return {"instances": len(inst), "patches": int(sum(len(c) for c, _, _ in inst)), "K": K,
            "grouped_instances": int(sum(len(c) < tmin for c, _, _ in inst)),
            "wall_s": round(wall, 3), "setup_s_summed": round(float(out["seconds"][0]), 3),
            "solve_s_summed": round(float(out["seconds"][1]), 3), "products": prods,
            "products_per_s": round(prods / wall, 2), "max_relres": float(np.max(out["relres"])),
            "all_converged": bool(np.all(out["status"] == 0))}


def cpu_baseline(args, centres, eps, mode, K, seconds=None):
    """The oracle as it stands (plain-C FP64 compressed sums, all host cores) on a
    bounded sample of target nodes, scaled to products per second."""
    from oracle import native, operator as O
    seconds = seconds or args.cpu_seconds
    pre = O.make_precompute(eps, mode, K, npan=8, nord=12, ntheta=40, tau=1e-10)
    N = len(centres)
    x = np.random.default_rng(5).standard_normal(N * K)
    rng = np.random.default_rng(6)
    # calibrate on a few targets, then time a sample sized to ~`seconds`
    t0 = time.time()
    native.rows(pre, centres, x, rng.choice(N, 8), rng.choice(pre.Kstar, 8))
    t_cal = time.time() - t0
    ns = int(max(8, min(4096, 8 * seconds / max(t_cal, 1e-3))))
    pat, nod = rng.choice(N, ns), rng.choice(pre.Kstar, ns)
    t0 = time.time()
    native.rows(pre, centres, x, pat, nod)
    dt = time.time() - t0
    value = (ns / (N * pre.Kstar)) / dt
    return {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{ns} of {N}x{pre.Kstar} Zernike-node outputs of one product (ID-direct sums, "
                      f"FP64, plain C with OpenMP), {dt:.1f} s, scaled to whole products"}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    from paper_1906_04209_gb300 import layouts as L
    centres, eps, mode, K = L.workload(3, layout=args.layout)
    per_step = []
    base = None
    for s in range(args.warmup + args.steps):
        r = cpu_baseline(args, centres, eps, mode, K, seconds=args.ref_seconds)
        base = r
        if s >= args.warmup:
            per_step.append(r["value"])
    value = float(np.mean(per_step))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "N": len(centres), "eps": eps, "K": K},
            "cpu_baseline": {"kind": "oracle", "cores": base["cores"], "sample": base["sample"], "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    faulthandler.enable()  # a crash in native code prints the Python stack to stderr
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--layout", default="fibonacci", choices=["fibonacci", "vmf"])
    ap.add_argument("--mode", default="interior", choices=["interior", "exterior"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--grid-tol", type=float, default=1e-8)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--df64-steps", type=int, default=2)
    ap.add_argument("--no-solve", dest="solve", action="store_false")
    ap.add_argument("--solve-tol", type=float, default=1e-8)
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--no-other-workloads", dest="other_workloads", action="store_false")
    # a fixed launch configuration instead of tuning (profiler captures of a chosen variant)
    ap.add_argument("--set-tuning", default=None, help="comma-separated key=value, e.g. p2l_poly=2,direct_poly=2")
    ap.add_argument("--batch-size", type=int, default=256)
    # a smaller layout of the same family (profiler captures only; the line names its N)
    ap.add_argument("--patches", type=int, default=None)
    ap.add_argument("--tensor-cores", type=int, default=1, choices=[0, 1])
    ap.add_argument("--no-solve-fp64", dest="solve_fp64", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
