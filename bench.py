#!/usr/bin/env python3
"""Benchmark of the LM-RS hot path on one GB300 (or N independent replicas).

Workload (default): the 200k-Gaussian scene -- SH degree 3 (coefficients
N(0, 0.2)), means from 32 anisotropic blobs, 24 views of 1024x672 on a
hemisphere, 10% of each tile's pixels sampled, 8 views per solve, 8 PCG
iterations per LM step, lambda 0.1 with diagonal damping.  A bench "step" is
one full LM step (sampling, projection, binning + sort, render, J^T W r,
diag, 8 damped-operator applications with the CG updates, step size and the
parameter update).  Reported metric: applications of (J^T W J + lambda D)
per second, i.e. 8 x LM steps / time, with all per-step work counted.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the
host cores instead (a bounded sample of the same workload).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "JᵀJv matvecs/s at 200k Gaussians (%HBM peak); fits/s & p99 fit latency vs plain"

WORKLOADS = {
    "moderate": dict(desc="LM steps with lambda*I damping (Eq. 8); 200k Gaussians, SH3, 8 of 24 views 1024x672, "
                          "10% per-tile sampling, 8 CG iters",
                     views_per_step=8, sample_frac=0.1, cg_iters=8, lam=0.1, damping_mode=0),
    "tiny": dict(desc="LM steps with lambda*I damping (Eq. 8); 1k Gaussians, SH0, 4 views 64x64, all pixels, "
                      "10 CG iters",
                 views_per_step=4, sample_frac=1.0, cg_iters=10, lam=1e-2, damping_mode=0),
    "large": dict(desc="LM steps with lambda*I damping (Eq. 8); 1.5M Gaussians, SH3, 12 of 100 views 1297x840 "
                       "(360 deg orbit, +-15 deg jitter), 25% per-tile sampling, BF16 per-sample caches, 8 CG iters",
                  views_per_step=12, sample_frac=0.25, cg_iters=8, lam=0.1, damping_mode=0, cache_bf16=1,
                  cpu_views=1),
    "fit": dict(desc="LM-RS fits of the 200k-Gaussian scene seen from 96 views 1024x672: 100 LM steps, 16 -> 32 "
                     "views and 5 -> 8 PCG iterations at step 50 (Sec. 5), 32 samples per 16x16 tile, lambda 0.1; "
                     "K-means view sampling (Sec. 4.3) against uniform, and the q_residual / q_Gaussian pixel "
                     "distributions; start = ground truth + N(0, 0.02)",
                n_views_total=96, n_steps=100, views=(16, 32), cg=(5, 8), switch=50, samples_per_tile=32, lam=0.1,
                eval_every=10),
    "ksweep": dict(desc="samples per 16x16 tile K in {26, 32, 64, 128, 256} on the 200k-Gaussian scene (8 of 24 "
                        "views 1024x672, SH3, 8 CG iters): operator and LM-step time vs K",
                   views_per_step=8, ks=(26, 32, 64, 128, 256), cg_iters=8, lam=0.1, damping_mode=0),
    "batched": dict(desc="64 independent fits: 5k-50k Gaussians (log-uniform), SH0, 4-16 views 256x256 each, "
                         "32 samples per 256-pixel tile, all views every step, 8 CG iters, 20 LM steps per fit",
                    samples_per_tile=32, cg_iters=8, lam=0.1, damping_mode=0, fit_steps=20,
                    tile_shapes=((16, 16), (32, 8), (8, 32))),
    "serving": dict(desc="fit requests with Poisson arrivals (mean 20/s): 2k-300k Gaussians (log-uniform), SH1, "
                         "8-32 views 512x512, all views every step, 32 samples per 256-pixel tile, 8 CG iters, "
                         "lambda*I damping; each fit runs until its full-frame PSNR over every camera is within "
                         "0.1 dB of its ground truth's (at most 60 steps); 120 GB admission budget",
                    samples_per_tile=32, cg_iters=8, lam=0.1, damping_mode=0, rate=20.0, requests=100,
                    max_steps=60, noise_sigma=0.02, psnr_slack_db=0.1, budget_bytes=120 << 30, max_active=8,
                    policy=1, full_frame_gate=1.25),
}


def make_scene(name, seed_offset=0):
    from paper_2504_12905_gb300 import synthetic as syn
    if name in ("moderate", "ksweep"):
        return syn.moderate_scene(seed=0x1A5E0001 + seed_offset)
    if name == "large":
        return syn.large_scene(seed=0x1A5E0002 + seed_offset)
    return syn.tiny_scene(seed=0x1A5E0000 + seed_offset)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# roofline models (the derivations are in the design notes)
# --------------------------------------------------------------------------
# FP32 FLOPs per (sample, Gaussian) pair composited before termination, from
# the formulas of the fused J^T W J raster kernel: forward pass with the
# tangent (offset, exponent, alpha, transmittance, colour and their
# tangents) 66, backward pass (the same primal, the colour cotangent, the 9
# feature cotangents, their warp sum) 63.
JTJ_FLOPS_PER_EVAL = 66 + 63
# float4 planes of the per-pair Jacobian cache for SH degree 0..3 (the SH
# basis values are recomputed from the view direction, not cached)
JAC_F4 = {0: 10, 1: 12, 2: 12, 3: 12}


def unit_peaks():
    """FP32, FP64, 2^x and atomic rates of this GPU, measured by the
    library's microbenchmarks (lmrs_measure_peaks), with its SM count."""
    from paper_2504_12905_gb300 import lmrs
    return lmrs.lmrs_measure_peaks()


def algorithmic_bytes(kernel, sizes):
    """Bytes each launch must move (every array once)."""
    Vis, P, nv, G = sizes["visible"], sizes["P"], sizes["views"], sizes["G"]
    deg = sizes["sh_degree"]
    jac = 16 * JAC_F4[deg]
    pg = P // G
    means = 12 * G if deg > 0 else 0  # the means, for the view direction of the SH basis
    if kernel == "k_prep_jvp":
        # rectangles of every pair; per visible pair the Jacobian, the 9-float
        # tangent written and the 9-float cotangent slot cleared; the PCG
        # direction p <- z + beta p formed in the same pass (z, p read; p written)
        return 16 * nv * G + Vis * (jac + 36 + 36) + 12 * P + means
    if kernel == "k_prep_vjp<dot>":
        # rectangles; per visible pair the Jacobian and the cotangents; p read,
        # Ap written, D read under diagonal damping
        d_read = 4 * P if sizes.get("damping_mode", 0) == 1 else 0
        return 16 * nv * G + Vis * (jac + 36) + 2 * 4 * P + d_read + means
    if kernel == "k_cg_update<true>":
        return 4 * P * 8  # p, Ap, M^-1, x, r read; x, r, z written
    return None


def source_hash(*names):
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2504_12905_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel's sources changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel)
    if not d or d.get("workload") != workload or d.get("source_hash") != source_hash(*d["sources"]):
        return None
    return d["dram_bytes_per_launch"]


class Replicas:
    """The ranks of a torchrun launch as independent replicas: the operator is
    a sum over views with no exchange step worth sharding on one node, so every
    rank runs its own fit.  A barrier around each timed region and the maximum
    of a rank-local time are the only traffic between ranks (NCCL on the GPU
    box; the tests use gloo on CPU)."""

    def __init__(self, rank, world, local_rank, backend="nccl"):
        self.rank, self.world = rank, world
        self.dist = None
        self.device = None
        if world > 1:
            import torch
            import torch.distributed as dist
            if backend == "nccl":
                self.device = torch.device("cuda", local_rank)
                dist.init_process_group(backend, device_id=self.device)
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x):
        """The maximum of a rank-local value over the ranks."""
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device if self.device is not None else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x):
        """The sum of a rank-local count over the ranks."""
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device if self.device is not None else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.barrier()
            self.dist.destroy_process_group()
            self.dist = None


def job_rate(units_per_rank, world, ms_max):
    """Whole-job throughput: the units all ranks processed (the same number on
    every rank) over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1000.0)


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2504_12905_gb300 import lmrs
    from paper_2504_12905_gb300 import synthetic as syn

    torch.cuda.set_device(local_rank)
    ranks = Replicas(rank, world, local_rank)
    wl = WORKLOADS[args.workload]
    sc = make_scene(args.workload, seed_offset=rank)
    G, deg = sc.n_gauss, sc.sh_degree
    nc = len(sc.cams)
    H, W = sc.height, sc.width
    # targets: renders of the perturbed parameters (through this library)
    rng = np.random.default_rng(1234 + rank)
    tparams = torch.from_numpy(syn.perturb(rng, sc.params)).cuda()
    targets = torch.zeros((nc, H, W, 3), dtype=torch.float32, device="cuda")
    tsc = lmrs.Scene(tparams, sc.cams, G, deg)
    for v0 in range(0, nc, 8):
        vs = list(range(v0, min(nc, v0 + 8)))
        lmrs.lmrs_preprocess(tsc.h, vs, 0)
        lmrs.lmrs_render(tsc.h, targets[v0:v0 + len(vs)])
    torch.cuda.synchronize()
    tsc.close()
    del tparams

    bf16 = wl.get("cache_bf16", 0)
    scene = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, G, deg, targets=targets,
                       sample_frac=wl["sample_frac"], lambda_=wl["lam"], damping_mode=wl["damping_mode"],
                       cg_iters=wl["cg_iters"], seed=0x5EED + rank, cache_bf16=bf16)
    h = scene.h
    vrng = np.random.default_rng(77 + rank)
    nvs = wl["views_per_step"]
    n_steps = args.warmup + args.steps
    views = [syn.view_subset(vrng, nc, nvs) for _ in range(n_steps + args.steps)]

    def barrier():
        torch.cuda.synchronize()
        ranks.barrier()

    # ---- peak rates of the units the raster kernels use (not timed) -----
    peaks = unit_peaks()

    # ---- warm-up -------------------------------------------------------
    for k in range(args.warmup):
        lmrs.lmrs_lm_step(h, views[k], k, stats=False)
    # grow the scene's buffers (tile lists, row lists, compact lists) to the
    # largest view set the timed and end-to-end steps will see, so no device
    # allocation falls inside a timed region; the timed steps still run every
    # kernel of their LM step
    for k in range(args.warmup, n_steps + args.steps):
        lmrs.lmrs_preprocess(h, views[k], k)
    barrier()

    # ---- timed region: K full LM steps, inputs resident ----------------
    vis_dev = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_idx = vis_dev.split(",")[local_rank] if vis_dev and not vis_dev.startswith("GPU") else str(local_rank)
    clocks = ClockSampler(smi_idx)
    launches0 = lmrs.lmrs_launch_count()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    last = None
    for k in range(args.warmup, n_steps):
        last = lmrs.lmrs_lm_step(h, views[k], k, stats=(k == n_steps - 1))
    e1.record()
    barrier()
    clock_info = clocks.stop()
    launches = lmrs.lmrs_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    ms_max = ranks.max(ms)
    matvecs = world * args.steps * wl["cg_iters"]
    value = job_rate(args.steps * wl["cg_iters"], world, ms_max)

    # ---- the same K steps again with an event pair around every launch ----
    # (per-kernel times for the shares and the roofline; the records cost host
    # time per launch, so the headline above is timed without them)
    lmrs.lmrs_get_timing(h)  # clear
    lmrs.lmrs_set_timing(h, True)
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    i0.record()
    for k in range(args.warmup, n_steps):
        lmrs.lmrs_lm_step(h, views[k], k, stats=False)
    i1.record()
    barrier()
    lmrs.lmrs_set_timing(h, False)
    ktimes = lmrs.lmrs_get_timing(h)
    ms_instr = i0.elapsed_time(i1)

    # sizes of the last step for the byte model, and the composited
    # evaluations per operator application averaged over the timed steps'
    # view sets (at the final parameters)
    evals, walked = [], []
    for k in range(args.warmup, n_steps):
        lmrs.lmrs_preprocess(h, views[k], k)
        lmrs.lmrs_render(h)
        evals.append(lmrs.lmrs_num_evaluations(h))
        walked.append(lmrs.lmrs_num_walked_entries(h))
    sizes = {"pairs": lmrs.lmrs_num_pairs(h), "visible": lmrs.lmrs_num_visible(h),
             "samples": lmrs.lmrs_num_samples(h), "view_tiles": nvs * scene.n_tiles, "P": scene.n_params,
             "views": nvs, "G": G, "sh_degree": deg, "evaluations_mean": int(np.mean(evals)),
             "walked_entries_mean": int(np.mean(walked)),
             "damping_mode": wl.get("damping_mode", 0)}

    # ---- (J^T W J + lambda diag(J^T W J)) v alone, at the current parameters
    cur = torch.empty(scene.n_params, dtype=torch.float32, device="cuda")
    lmrs.lmrs_get_params(h, cur)
    op = lmrs.Scene(cur, sc.cams, G, deg, targets=targets, sample_frac=wl["sample_frac"], lambda_=wl["lam"],
                    damping_mode=1, cg_iters=wl["cg_iters"], seed=0x5EED + rank, cache_bf16=bf16)
    lmrs.lmrs_preprocess(op.h, views[n_steps - 1], n_steps - 1)
    lmrs.lmrs_render(op.h)
    d_op = torch.empty(scene.n_params, dtype=torch.float32, device="cuda")
    lmrs.lmrs_jtj_diag(op.h, d_op)
    v = torch.randn(scene.n_params, device="cuda")
    out = torch.empty_like(v)
    for _ in range(3):
        lmrs.lmrs_jtjv(op.h, v, out)
    torch.cuda.synchronize()
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    m0.record()
    for _ in range(reps):
        lmrs.lmrs_jtjv(op.h, v, out)
    m1.record()
    torch.cuda.synchronize()
    matvec_ms = m0.elapsed_time(m1) / reps
    bf16_err = None
    if bf16:
        # The same quantities with FP32 caches (which match the FP64 oracle to
        # about 1e-6 on the 200k-Gaussian workload): the error the BF16 caches
        # add.  The cached final colour is read by the right-hand side's
        # back-scatter and by the diagonal; the operator recomputes the colour
        # in BF16 mode and differs only through D.
        op32 = lmrs.Scene(cur, sc.cams, G, deg, targets=targets, sample_frac=wl["sample_frac"], lambda_=wl["lam"],
                          damping_mode=1, cg_iters=wl["cg_iters"], seed=0x5EED + rank, cache_bf16=0)
        lmrs.lmrs_preprocess(op32.h, views[n_steps - 1], n_steps - 1)
        lmrs.lmrs_render(op32.h)
        d32 = torch.empty_like(d_op)
        lmrs.lmrs_jtj_diag(op32.h, d32)
        out32 = torch.empty_like(v)
        lmrs.lmrs_jtjv(op32.h, v, out32)
        b16, b32 = torch.empty_like(v), torch.empty_like(v)
        lmrs.lmrs_rhs(op.h, b16)
        lmrs.lmrs_rhs(op32.h, b32)
        torch.cuda.synchronize()

        def rel(a, b):
            return float(((a - b).norm() / b.norm()).item())

        bf16_err = {"rhs": rel(b16, b32), "diag": rel(d_op, d32), "operator": rel(out, out32),
                    "what": "normwise relative difference of J^T W r, diag(J^T W J) and the lambda*diag operator "
                            "with BF16 vs FP32 final-colour/transmittance caches (the operator sees the cache "
                            "only through D)"}
        op32.close()
        del out32, d32, b16, b32
    op.close()
    del cur, d_op

    # ---- end to end through the C-ABI with host buffers ---------------
    p_host = torch.empty(scene.n_params, dtype=torch.float32).pin_memory()
    lmrs.lmrs_get_params(h, p_host)
    barrier()
    t0 = time.perf_counter()
    for k in range(n_steps, n_steps + args.steps):
        lmrs.lmrs_set_params(h, p_host)          # host -> device, pinned
        lmrs.lmrs_lm_step(h, views[k], k, stats=False)
        lmrs.lmrs_get_params(h, p_host)          # device -> host, synchronises
    barrier()
    e2e_s = ranks.max(time.perf_counter() - t0)
    e2e = {"value": matvecs / e2e_s, "unit": "matvec/s", "h2d_bytes_per_step": 4 * scene.n_params,
           "d2h_bytes_per_step": 4 * scene.n_params}

    # ---- roofline of the dominant kernel ------------------------------
    # k_jtj is bound by FP32 / integer instruction issue (ALU), not by HBM:
    # algorithmic FLOPs = composited evaluations x FLOPs per evaluation,
    # against the FP32 FMA rate measured on this GPU
    peak_hbm, peak_kind = load_peaks()
    roof = None
    peak32 = peaks["fp32_tflops"]
    src32 = (f"measured: lmrs_measure_peaks FP32 FMA chains on {peaks['sm_count']} SMs "
             f"(nominal {peaks['sm_count']} x 128 lanes x 2 x {peaks['sm_clock_max_mhz']:.0f} MHz = "
             f"{peaks['sm_count'] * 256 * peaks['sm_clock_max_mhz'] * 1e-6:.1f})")
    if "k_jtj" in ktimes:
        n_l, tot = ktimes["k_jtj"]
        avg_s = tot / n_l / 1000.0
        flops = JTJ_FLOPS_PER_EVAL * sizes["evaluations_mean"]
        ach = flops / avg_s / 1e12
        roof = {"kernel": "k_jtj", "bound": "alu", "achieved": round(ach, 3), "peak": round(peak32, 2),
                "unit": "TFLOP/s", "frac": round(ach / peak32, 4),
                "traffic": profiled_traffic("k_jtj", args.workload),
                "peak_source": src32,
                "algorithmic_flops_per_launch": int(flops), "avg_launch_ms": round(tot / n_l, 4),
                "hbm_frac_of_measured": None}
        tr = roof["traffic"]
        if tr:
            roof["hbm_frac_of_measured"] = round(tr / avg_s / 1e9 / peak_hbm, 4)
    # the HBM-bound kernels of the PCG loop, against the measured copy bandwidth
    secondary = {}
    for kname in ("k_prep_jvp", "k_prep_vjp<dot>", "k_cg_update<true>"):
        if kname in ktimes:
            n_l, tot = ktimes[kname]
            byt = algorithmic_bytes(kname, sizes)
            ach = byt / (tot / n_l / 1000.0) / 1e9
            secondary[kname] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak_hbm, "unit": "GB/s",
                                "frac": round(ach / peak_hbm, 4), "peak_source": peak_kind,
                                "algorithmic_bytes_per_launch": int(byt), "avg_launch_ms": round(tot / n_l, 4)}
    # the whole operator application against the lower bound of the
    # algorithmic model: t_min = max(Q / HBM, F / FP32, exponentials / SFU,
    # atomics / L2 atomic rate), every rate measured on this GPU; the
    # back-scatter issues, per walked (work item, list entry), two 4-wide
    # and one scalar atomic add
    Q = 16 * sizes["P"] + 144 * sizes["visible"] + 4 * sizes["pairs"] + 20 * sizes["samples"] + \
        8 * sizes["view_tiles"]
    F = JTJ_FLOPS_PER_EVAL * sizes["evaluations_mean"]
    X = 2 * sizes["evaluations_mean"]
    Wk = sizes["walked_entries_mean"]
    t_parts = {"hbm_ms": Q / (peak_hbm * 1e9) * 1e3, "fp32_ms": F / (peak32 * 1e12) * 1e3,
               "sfu_ms": X / (peaks["ex2_gops"] * 1e9) * 1e3,
               "atomic_ms": (2 * Wk / peaks["red_v4_scattered_gops"] + Wk / peaks["atomic_scattered_gops"]) * 1e-9 * 1e3}
    t_min = max(t_parts.values())
    matvec_bound = {"Q_bytes": int(Q), "F_flops": int(F), "exponentials": int(X), "walked_entries": int(Wk),
                    "t_min_ms": round(t_min, 4), **{k: round(v, 4) for k, v in t_parts.items()},
                    "t_operator_ms": round(matvec_ms, 4), "frac": round(t_min / matvec_ms, 4),
                    "hbm_frac_of_measured": round(Q / (matvec_ms / 1e3) / 1e9 / peak_hbm, 4)}
    step_ms = ms_max / args.steps
    kshare = {k: {"launches": n, "ms": round(t, 3), "share": round(t / max(ms_instr, 1e-9), 4)}
              for k, (n, t) in sorted(ktimes.items(), key=lambda kv: -kv[1][1])}

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": "matvec/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 CG scalars)",
        "data": "synthetic (seeded; targets rendered from perturbed parameters)",
        "config": {"workload": f"{args.workload}: {wl['desc']}", "n_gauss": G, "sh_degree": deg,
                   "n_params": scene.n_params, "views_per_step": nvs, "image": f"{W}x{H}",
                   "cg_iters": wl["cg_iters"], "lambda": wl["lam"],
                   "damping": "LM steps: lambda*I (Eq. 8); matvec_only: lambda*diag(J^T W J)",
                   "sample_frac": wl["sample_frac"], "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (per-step working set > 129 MB)",
                   "lm_steps_per_s": round(1000.0 * args.steps / ms_max * world, 3),
                   "kernel_times": "per-kernel CUDA events on the library's stream over a second pass of "
                                   "the same K steps (%.3f ms per step with the records)" % (ms_instr / args.steps),
                   "matvec_only_ms": round(matvec_ms, 4), "matvec_only_per_s": round(1000.0 / matvec_ms, 2),
                   "sizes_last_step": sizes, "loss_last_step": None if last is None else last.loss,
                   "cache_bf16": bool(bf16), "bf16_cache_error": bf16_err, "operator_bound": matvec_bound,
                   "unit_peaks": {k: (round(v, 3) if isinstance(v, float) else v) for k, v in peaks.items()}},
        "roofline": roof, "rooflines_hbm": secondary, "kernels": kshare, "e2e": e2e, "gpu_launches": launches,
        "clocks": clock_info,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(sc, views[n_steps - 1], n_steps - 1, wl, budget_s=args.cpu_seconds)
    ranks.close()
    scene.close()
    return result


def run_fit(args, rank, world, local_rank):
    """Two LM-RS fits from the same start, K-means and uniform view draws,
    with the paper's schedules; full-frame PSNR over all 96 views."""
    import torch

    from paper_2504_12905_gb300 import lmrs
    from paper_2504_12905_gb300 import synthetic as syn

    torch.cuda.set_device(local_rank)
    wl = WORKLOADS["fit"]
    sc = syn.moderate_scene(seed=0x1A5E0001 + rank, n_views=wl["n_views_total"])
    G, deg, nc = sc.n_gauss, sc.sh_degree, len(sc.cams)
    targets = torch.zeros((nc, sc.height, sc.width, 3), dtype=torch.float32, device="cuda")
    gt = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, G, deg)
    for v0 in range(0, nc, 8):
        vs = list(range(v0, min(nc, v0 + 8)))
        lmrs.lmrs_preprocess(gt.h, vs, 0)
        lmrs.lmrs_render(gt.h, targets[v0:v0 + len(vs)])
    torch.cuda.synchronize()
    gt.close()
    start = syn.perturb(np.random.default_rng(99 + rank), sc.params, 0.02)
    vis_dev = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_idx = vis_dev.split(",")[local_rank] if vis_dev and not vis_dev.startswith("GPU") else str(local_rank)
    clocks = ClockSampler(smi_idx)
    out = {}
    launches0 = lmrs.lmrs_launch_count()
    clocks.start()
    # (view draws, pixel distribution, SSIM weight): K-means vs uniform views
    # with uniform pixels, K-means views with the two importance
    # distributions, and with the diagonal SSIM term at the paper's 0.2
    for mode, dist, ssim, name in ((1, 0, 0.0, "kmeans"), (0, 0, 0.0, "uniform"), (1, 1, 0.0, "kmeans_q_residual"),
                                   (1, 2, 0.0, "kmeans_q_gaussian"), (1, 0, 0.2, "kmeans_ssim")):
        scene = lmrs.Scene(torch.from_numpy(start).cuda(), sc.cams, G, deg, targets=targets,
                           samples_per_tile=wl["samples_per_tile"], lambda_=wl["lam"], damping_mode=0,
                           cg_iters=wl["cg"][0], seed=0x5EED + rank, sample_dist=dist, ssim_weight=ssim)
        psnr0 = -10.0 * math.log10(lmrs.lmrs_eval_mse(scene.h))
        t0 = time.perf_counter()
        recs = lmrs.lmrs_fit(scene.h, n_steps=wl["n_steps"], views_first=wl["views"][0], views_later=wl["views"][1],
                             cg_first=wl["cg"][0], cg_later=wl["cg"][1], switch_step=wl["switch"], view_mode=mode,
                             eval_every=wl["eval_every"], seed=0xF17 + rank)
        wall = time.perf_counter() - t0
        step_ms = sum(r.ms for r in recs)
        out[name] = {"psnr_start_db": round(psnr0, 3),
                     "psnr_curve_db": {r.step + 1: round(r.psnr, 3) for r in recs if r.mse_full >= 0},
                     "psnr_final_db": round(recs[-1].psnr, 3), "steps_ms_total": round(step_ms, 1),
                     "fit_wall_s_with_evals": round(wall, 2),
                     "matvecs_per_s": round(sum(r.cg_iters for r in recs) / (step_ms / 1e3), 2)}
        scene.close()
    clock_info = clocks.stop()
    launches = lmrs.lmrs_launch_count() - launches0
    km = out["kmeans"]
    return {
        "metric": METRIC, "value": km["matvecs_per_s"], "unit": "matvec/s", "n_gpus": 1, "steps": wl["n_steps"],
        "warmup": 0, "ms_per_step": round(km["steps_ms_total"] / wl["n_steps"], 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 CG scalars)",
        "data": "synthetic (seeded; targets = renders of the ground truth)",
        "config": {"workload": f"fit: {wl['desc']}", "value_is": "operator applications per second of the "
                   "K-means fit (all per-step work counted; the evaluations are excluded)",
                   "fits": out, "psnr_gain_kmeans_over_uniform_db": round(km["psnr_final_db"] -
                                                                           out["uniform"]["psnr_final_db"], 3),
                   "l2": "inputs larger than L2", "parallelism": "replicas x1"},
        "roofline": None, "gpu_launches": launches, "clocks": clock_info,
    }


def run_ksweep(args, rank, world, local_rank):
    """Operator and LM-step time against the per-tile sample count K (the
    throughput side of the paper's sampling ablation)."""
    import torch

    from paper_2504_12905_gb300 import lmrs
    from paper_2504_12905_gb300 import synthetic as syn

    torch.cuda.set_device(local_rank)
    wl = WORKLOADS["ksweep"]
    sc = make_scene("ksweep", seed_offset=rank)
    G, deg, nc = sc.n_gauss, sc.sh_degree, len(sc.cams)
    rng = np.random.default_rng(1234 + rank)
    tparams = torch.from_numpy(syn.perturb(rng, sc.params)).cuda()
    targets = torch.zeros((nc, sc.height, sc.width, 3), dtype=torch.float32, device="cuda")
    tsc = lmrs.Scene(tparams, sc.cams, G, deg)
    for v0 in range(0, nc, 8):
        vs = list(range(v0, min(nc, v0 + 8)))
        lmrs.lmrs_preprocess(tsc.h, vs, 0)
        lmrs.lmrs_render(tsc.h, targets[v0:v0 + len(vs)])
    torch.cuda.synchronize()
    tsc.close()
    vrng = np.random.default_rng(77 + rank)
    n_steps = args.warmup + args.steps
    views = [syn.view_subset(vrng, nc, wl["views_per_step"]) for _ in range(n_steps)]
    vis_dev = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_idx = vis_dev.split(",")[local_rank] if vis_dev and not vis_dev.startswith("GPU") else str(local_rank)
    clocks = ClockSampler(smi_idx)
    clocks.start()
    launches0 = lmrs.lmrs_launch_count()
    table = []
    for K in wl["ks"]:
        scene = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, G, deg, targets=targets, samples_per_tile=K,
                           lambda_=wl["lam"], damping_mode=wl["damping_mode"], cg_iters=wl["cg_iters"],
                           seed=0x5EED + rank)
        for k in range(args.warmup):
            lmrs.lmrs_lm_step(scene.h, views[k], k, stats=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(args.warmup, n_steps):
            lmrs.lmrs_lm_step(scene.h, views[k], k, stats=False)
        e1.record()
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / args.steps
        # the damped operator alone at the last step's samples
        op = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, G, deg, targets=targets, samples_per_tile=K,
                        lambda_=wl["lam"], damping_mode=1, cg_iters=wl["cg_iters"], seed=0x5EED + rank)
        lmrs.lmrs_preprocess(op.h, views[-1], n_steps - 1)
        lmrs.lmrs_render(op.h)
        lmrs.lmrs_jtj_diag(op.h)
        v = torch.randn(op.n_params, device="cuda")
        out = torch.empty_like(v)
        for _ in range(3):
            lmrs.lmrs_jtjv(op.h, v, out)
        torch.cuda.synchronize()
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        m0.record()
        for _ in range(20):
            lmrs.lmrs_jtjv(op.h, v, out)
        m1.record()
        torch.cuda.synchronize()
        mv_ms = m0.elapsed_time(m1) / 20
        table.append({"K": K, "samples": lmrs.lmrs_num_samples(op.h), "evaluations": lmrs.lmrs_num_evaluations(op.h),
                      "lm_step_ms": round(step_ms, 3), "matvec_ms": round(mv_ms, 4),
                      "matvecs_per_s_in_lm_steps": round(wl["cg_iters"] * 1000.0 / step_ms, 2)})
        op.close()
        scene.close()
    clock_info = clocks.stop()
    launches = lmrs.lmrs_launch_count() - launches0
    base = table[0]
    return {
        "metric": METRIC, "value": base["matvecs_per_s_in_lm_steps"], "unit": "matvec/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": base["lm_step_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 CG scalars)",
        "data": "synthetic (seeded; targets rendered from perturbed parameters)",
        "config": {"workload": f"ksweep: {wl['desc']}", "value_is": f"K = {base['K']}", "sweep": table,
                   "l2": "inputs larger than L2", "parallelism": "replicas x1"},
        "roofline": None, "gpu_launches": launches, "clocks": clock_info,
    }


def _psnr(lmrs, torch, scene_h, targets, n_views):
    """Mean PSNR (dB) of full-frame renders of every view against the targets."""
    H, W = targets.shape[1], targets.shape[2]
    out = []
    for v0 in range(0, n_views, 8):
        vs = list(range(v0, min(n_views, v0 + 8)))
        img = torch.empty((len(vs), H, W, 3), dtype=torch.float32, device="cuda")
        lmrs.lmrs_preprocess(scene_h, vs, 0)
        lmrs.lmrs_render(scene_h, img)
        lmrs.lmrs_synchronize(scene_h)  # the render ran on the scene's stream
        mse = ((img - targets[v0:v0 + len(vs)]) ** 2).mean(dim=(1, 2, 3))
        out += (-10.0 * torch.log10(mse.clamp_min(1e-12))).tolist()
    return float(np.mean(out))


def run_batched(args, rank, world, local_rank):
    """64 independent small fits: batched LM steps (one launch per PCG phase
    over all scenes, replayed as a CUDA graph) against the same fits run one
    scene at a time with lmrs_lm_step.  Ground truth: the drawn Gaussians;
    targets: their full-frame renders; each fit starts from the ground truth
    perturbed by N(0, 0.05) on every raw parameter."""
    import torch

    from paper_2504_12905_gb300 import lmrs
    from paper_2504_12905_gb300 import synthetic as syn

    torch.cuda.set_device(local_rank)
    ranks = Replicas(rank, world, local_rank)
    wl = WORKLOADS["batched"]
    scenes = syn.small_fit_scenes(seed=0x1A5E0003 + rank)
    n_sc = len(scenes)
    prng = np.random.default_rng(4321 + rank)
    targets, starts = [], []
    for sc in scenes:
        nc = len(sc.cams)
        t = torch.zeros((nc, sc.height, sc.width, 3), dtype=torch.float32, device="cuda")
        gt = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, sc.n_gauss, sc.sh_degree)
        for v0 in range(0, nc, 8):
            vs = list(range(v0, min(nc, v0 + 8)))
            lmrs.lmrs_preprocess(gt.h, vs, 0)
            lmrs.lmrs_render(gt.h, t[v0:v0 + len(vs)])
        gt.close()
        targets.append(t)
        starts.append(torch.from_numpy(syn.perturb(prng, sc.params)).cuda())
    torch.cuda.synchronize()
    views = [list(range(len(sc.cams))) for sc in scenes]
    cfg = dict(samples_per_tile=wl["samples_per_tile"], lambda_=wl["lam"], damping_mode=wl["damping_mode"],
               cg_iters=wl["cg_iters"], seed=0x5EED + rank)

    # ---- tile shape: autotuned on the scene of median size ----------------
    mid = int(np.argsort([sc.n_gauss for sc in scenes])[n_sc // 2])
    shapes = wl["tile_shapes"]
    tcfg = lmrs.lmrs_config_default(sh_degree=0, **cfg)
    best, tune_ms = lmrs.lmrs_autotune_tile(tcfg, scenes[mid].n_gauss, starts[mid], scenes[mid].cams, targets[mid],
                                            views[mid], shapes, reps=3)
    tw, th = shapes[best]
    cfg.update(tile_w=tw, tile_h=th)

    def make(i, stream):
        sc = scenes[i]
        return lmrs.Scene(starts[i], sc.cams, sc.n_gauss, sc.sh_degree, targets=targets[i], stream=stream, **cfg)

    def barrier():
        torch.cuda.synchronize()
        ranks.barrier()

    n_steps = args.warmup + args.steps
    vis_dev = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_idx = vis_dev.split(",")[local_rank] if vis_dev and not vis_dev.startswith("GPU") else str(local_rank)

    # ---- batched arm ------------------------------------------------------
    streams = [torch.cuda.Stream() for _ in range(n_sc)]
    bstream = torch.cuda.Stream()
    bsc = [make(i, streams[i].cuda_stream) for i in range(n_sc)]
    batch = lmrs.lmrs_batch_create([s.h for s in bsc], n_threads=8, stream=bstream.cuda_stream)
    lmrs.lmrs_batch_set_persistent(batch, 1 if args.pcg_launch == "persistent" else 0)
    for k in range(args.warmup):
        lmrs.lmrs_batch_lm_step(batch, views, [k] * n_sc, stats=False)
    barrier()
    clocks = ClockSampler(smi_idx)
    launches0 = lmrs.lmrs_launch_count()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bstream)
    for s in streams:
        s.wait_event(e0)  # every scene's setup starts after e0
    w0 = time.perf_counter()
    for k in range(args.warmup, n_steps):
        lmrs.lmrs_batch_lm_step(batch, views, [k] * n_sc, stats=False)
    e1.record(bstream)  # the last graph waits for every scene's setup
    barrier()
    wall_b = time.perf_counter() - w0
    clock_info = clocks.stop()
    launches = lmrs.lmrs_launch_count() - launches0
    ms_b = e0.elapsed_time(e1)
    psnr_b = [_psnr(lmrs, torch, s.h, targets[i], len(views[i])) for i, s in enumerate(bsc)]

    # ---- sequential arm: the same fits, one scene at a time ----------------
    sstream = torch.cuda.Stream()
    ssc = [make(i, sstream.cuda_stream) for i in range(n_sc)]
    psnr_0 = [_psnr(lmrs, torch, s.h, targets[i], len(views[i])) for i, s in enumerate(ssc)]
    for k in range(args.warmup):
        for i, s in enumerate(ssc):
            lmrs.lmrs_lm_step(s.h, views[i], k, stats=False)
    barrier()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(sstream)
    for k in range(args.warmup, n_steps):
        for i, s in enumerate(ssc):
            lmrs.lmrs_lm_step(s.h, views[i], k, stats=False)
    s1.record(sstream)
    barrier()
    ms_s = s0.elapsed_time(s1)
    psnr_s = [_psnr(lmrs, torch, s.h, targets[i], len(views[i])) for i, s in enumerate(ssc)]
    for s in ssc:
        s.close()

    # ---- end to end: pinned host parameters in and out every step ----------
    hosts = []
    for s in bsc:
        hp = torch.empty(s.n_params, dtype=torch.float32).pin_memory()
        lmrs.lmrs_get_params(s.h, hp)
        hosts.append(hp)
    barrier()
    t0 = time.perf_counter()
    for k in range(n_steps, n_steps + args.steps):
        for s, hp in zip(bsc, hosts):
            lmrs.lmrs_set_params(s.h, hp)
        lmrs.lmrs_batch_lm_step(batch, views, [k] * n_sc, stats=False)
        for s, hp in zip(bsc, hosts):
            lmrs.lmrs_get_params(s.h, hp)
    barrier()
    e2e_s = time.perf_counter() - t0
    lmrs.lmrs_batch_destroy(batch)
    for s in bsc:
        s.close()

    ms_b, ms_s, e2e_s = ranks.max(ms_b), ranks.max(ms_s), ranks.max(e2e_s)
    fits = world * n_sc * args.steps / wl["fit_steps"]
    P_tot = sum(sc.n_params for sc in scenes)
    result = {
        "metric": METRIC, "value": round(fits / (ms_b / 1000.0), 3), "unit": "fits/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_b / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 CG scalars)",
        "data": "synthetic (seeded; targets rendered from the drawn Gaussians, fits start from a perturbation)",
        "config": {"workload": f"batched: {wl['desc']}", "n_scenes": n_sc,
                   "n_gauss_total": int(sum(sc.n_gauss for sc in scenes)), "n_params_total": int(P_tot),
                   "views_total": int(sum(len(v) for v in views)), "cg_iters": wl["cg_iters"], "lambda": wl["lam"],
                   "damping": "lambda*I (Eq. 8)", "fit_steps": wl["fit_steps"],
                   "step": "one LM step of all 64 scenes", "parallelism": f"replicas x{world}",
                   "l2": "no flush: per-step working set of all scenes > 129 MB",
                   "tile_shape": f"{tw}x{th}",
                   "pcg_launch": ("one persistent cooperative launch per LM step (grid barriers between phases)"
                                  if args.pcg_launch == "persistent" else "CUDA graph of per-phase launches"),
                   "autotune_ms_per_step": {f"{a}x{b}": round(float(m), 4) for (a, b), m in zip(shapes, tune_ms)},
                   "sequential_fits_per_s": round(fits / (ms_s / 1000.0), 3),
                   "sequential_ms_per_step": round(ms_s / args.steps, 3),
                   "batched_over_sequential": round(ms_s / ms_b, 3),
                   "batched_wall_ms_per_step": round(1000.0 * wall_b / args.steps, 3),
                   "psnr_start_db": round(float(np.mean(psnr_0)), 3),
                   "psnr_after_db": {"batched": round(float(np.mean(psnr_b)), 3),
                                     "sequential": round(float(np.mean(psnr_s)), 3),
                                     "lm_steps": n_steps},
                   "max_psnr_gap_db": round(float(np.max(np.abs(np.array(psnr_b) - np.array(psnr_s)))), 4)},
        "roofline": None,
        "e2e": {"value": round(fits / e2e_s, 3), "unit": "fits/s", "h2d_bytes_per_step": 4 * P_tot,
                "d2h_bytes_per_step": 4 * P_tot},
        "gpu_launches": launches, "clocks": clock_info,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_batched(scenes, starts, targets, views, cfg, wl, args.cpu_seconds)
    ranks.close()
    return result


def _serving_inputs(lmrs, torch, syn, reqs, wl, rank):
    """Per request: ground-truth render + N(0, noise_sigma) noise as the
    targets (host), the stop loss (the ground truth's MSE against the
    targets, scaled by the PSNR slack) and the perturbed start (host)."""
    out = []
    for i, (t_arr, sc) in enumerate(reqs):
        nc = len(sc.cams)
        clean = torch.zeros((nc, sc.height, sc.width, 3), dtype=torch.float32, device="cuda")
        gt = lmrs.Scene(torch.from_numpy(sc.params).cuda(), sc.cams, sc.n_gauss, sc.sh_degree)
        for v0 in range(0, nc, 8):
            vs = list(range(v0, min(nc, v0 + 8)))
            lmrs.lmrs_preprocess(gt.h, vs, 0)
            lmrs.lmrs_render(gt.h, clean[v0:v0 + len(vs)])
        lmrs.lmrs_synchronize(gt.h)
        gt.close()
        gen = torch.Generator(device="cuda")
        gen.manual_seed(1000 * rank + i)
        tgt = clean + wl["noise_sigma"] * torch.randn(clean.shape, device="cuda", generator=gen)
        mse_gt = float(((tgt - clean) ** 2).mean().item())
        start = syn.perturb_appearance(np.random.default_rng([rank, i]), sc.params, sc.n_gauss, sc.sh_degree)
        out.append(dict(t=t_arr, sc=sc, targets=tgt.cpu().numpy(), start=start,
                        stop_loss=mse_gt * 10.0 ** (wl["psnr_slack_db"] / 10.0)))
        del clean, tgt
    torch.cuda.synchronize()
    return out


def _pct(x, q):
    return round(float(np.percentile(np.asarray(x), q)), 4) if len(x) else None


def run_serving(args, rank, world, local_rank):
    """Fit requests through the server (admission against the budget,
    continuous batching) and the same stream served one fit at a time with
    lmrs_lm_step; latency = finish - arrival."""
    import torch

    from paper_2504_12905_gb300 import lmrs
    from paper_2504_12905_gb300 import synthetic as syn

    torch.cuda.set_device(local_rank)
    ranks = Replicas(rank, world, local_rank)
    wl = dict(WORKLOADS["serving"])
    if args.max_active > 0:
        wl["max_active"] = args.max_active
    if args.policy >= 0:
        wl["policy"] = args.policy
    n_req = args.requests or wl["requests"]
    reqs = syn.serving_requests(seed=0x1A5E0004 + rank, n_requests=n_req + args.warmup, rate=wl["rate"])
    jobs = _serving_inputs(lmrs, torch, syn, reqs, wl, rank)
    warm, jobs = jobs[:args.warmup], jobs[args.warmup:]
    t_first = jobs[0]["t"]
    for j in jobs:
        j["t"] -= t_first
    cfgd = dict(samples_per_tile=wl["samples_per_tile"], lambda_=wl["lam"], damping_mode=wl["damping_mode"],
                cg_iters=wl["cg_iters"])

    def cfg_of(k, sc):
        return lmrs.lmrs_config_default(sh_degree=sc.sh_degree, seed=0x5EED + k, **cfgd)

    def barrier():
        torch.cuda.synchronize()
        ranks.barrier()

    # ---- server arm ---------------------------------------------------------
    srv = lmrs.lmrs_server_create(wl["budget_bytes"], max_active=wl["max_active"], setup_threads=8,
                                  policy=wl["policy"], stop_full_frame=1, full_frame_gate=wl["full_frame_gate"])
    wid = [lmrs.lmrs_server_submit(srv, cfg_of(k, j["sc"]), j["sc"].n_gauss, j["start"], j["sc"].cams, j["targets"],
                                   0, j["stop_loss"], wl["max_steps"]) for k, j in enumerate(warm)]
    for w in wid:
        lmrs.lmrs_server_wait(srv, w, 600.0)
    barrier()
    vis_dev = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_idx = vis_dev.split(",")[local_rank] if vis_dev and not vis_dev.startswith("GPU") else str(local_rank)
    clocks = ClockSampler(smi_idx)
    launches0 = lmrs.lmrs_launch_count()
    clocks.start()
    t0 = time.perf_counter()
    ids = []
    for k, j in enumerate(jobs):
        delay = t0 + j["t"] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        ids.append(lmrs.lmrs_server_submit(srv, cfg_of(k, j["sc"]), j["sc"].n_gauss, j["start"], j["sc"].cams,
                                           j["targets"], 0, j["stop_loss"], wl["max_steps"]))
    infos = []
    for jid in ids:
        status, info = lmrs.lmrs_server_wait(srv, jid, 1800.0)
        infos.append(info)
    wall_srv = time.perf_counter() - t0
    clock_info = clocks.stop()
    launches = lmrs.lmrs_launch_count() - launches0
    sstats = lmrs.lmrs_server_get_stats(srv)
    lmrs.lmrs_server_destroy(srv)
    ok = [i for i in infos if i.state == lmrs.JOB_DONE]
    lat_srv = [i.t_done - i.t_submit for i in ok]
    span_srv = max(i.t_done for i in infos) - min(i.t_submit for i in infos)

    # ---- plain arm: one fit at a time, in arrival order ----------------------
    sstream = torch.cuda.Stream()
    lat_plain, conv_plain, steps_plain = [], 0, []
    t0 = time.perf_counter()
    for k, j in enumerate(jobs):
        delay = t0 + j["t"] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        sc = j["sc"]
        tg = torch.from_numpy(j["targets"]).to("cuda", non_blocking=False)
        scene = lmrs.Scene(j["start"], sc.cams, sc.n_gauss, sc.sh_degree, targets=tg, stream=sstream.cuda_stream,
                           seed=0x5EED + k, **cfgd)
        views = list(range(len(sc.cams)))
        conv = False
        for step in range(wl["max_steps"]):
            st = lmrs.lmrs_lm_step(scene.h, views, step)
            # the server's rule: full-frame MSE after the step, checked once
            # the sampled loss is within the gate
            if st.loss <= wl["full_frame_gate"] * j["stop_loss"] and lmrs.lmrs_eval_mse(scene.h) <= j["stop_loss"]:
                conv = True
                break
        out = np.empty(scene.n_params, np.float32)
        lmrs.lmrs_get_params(scene.h, out)
        scene.close()
        del tg
        lat_plain.append(time.perf_counter() - t0 - j["t"])
        conv_plain += int(conv)
        steps_plain.append(step + 1)
    wall_plain = time.perf_counter() - t0
    barrier()

    n = len(jobs)
    # whole-job rates over the slowest rank's span (every rank serves its own stream)
    span_srv_max, wall_plain_max = ranks.max(span_srv), ranks.max(wall_plain)
    fits_srv = ranks.sum(len(ok)) / span_srv_max
    fits_plain = job_rate(n, world, wall_plain_max * 1000.0)
    h2d = int(np.mean([j["targets"].nbytes + j["start"].nbytes for j in jobs]))
    d2h = int(np.mean([j["start"].nbytes for j in jobs]))
    est = np.array([i.footprint_est for i in ok], np.float64)
    peak = np.array([i.footprint_peak for i in ok], np.float64)
    result = {
        "metric": METRIC, "value": round(fits_srv, 3), "unit": "fits/s", "n_gpus": world, "steps": n,
        "warmup": len(warm), "ms_per_step": round(1000.0 * span_srv / max(len(ok), 1), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 CG scalars)",
        "data": "synthetic (seeded; targets = ground-truth renders + N(0, 0.02^2) noise)",
        "config": {"workload": f"serving: {wl['desc']}", "requests": n, "rate_per_s": wl["rate"],
                   "step": "one fit request (a bench step = one request)",
                   "n_gauss_mean": int(np.mean([j["sc"].n_gauss for j in jobs])),
                   "views_mean": round(float(np.mean([len(j["sc"].cams) for j in jobs])), 2),
                   "budget_gb": wl["budget_bytes"] / 2**30, "max_active": wl["max_active"],
                   "bytes_peak_gb": round(sstats.bytes_peak / 2**30, 3),
                   "footprint_peak_over_estimate": {"max": round(float((peak / est).max()), 3),
                                                    "mean": round(float((peak / est).mean()), 3)} if len(ok) else None,
                   "latency_s": {"p50": _pct(lat_srv, 50), "p99": _pct(lat_srv, 99), "max": _pct(lat_srv, 100)},
                   "converged": sum(i.converged for i in ok), "failed": n - len(ok),
                   "steps_mean": round(float(np.mean([i.steps for i in ok])), 2) if ok else None,
                   "scheduler_iterations": sstats.iterations,
                   "plain": {"fits_per_s": round(fits_plain, 3),
                             "latency_s": {"p50": _pct(lat_plain, 50), "p99": _pct(lat_plain, 99)},
                             "converged": conv_plain, "steps_mean": round(float(np.mean(steps_plain)), 2)},
                   "server_over_plain": round(fits_srv / fits_plain, 3),
                   "offered_load_over_plain_capacity": round(wl["rate"] / fits_plain, 2),
                   "policy": "least estimated work first" if wl["policy"] == 1 else "FIFO",
                   "stop_rule": (f"full-frame MSE over every camera <= the ground truth's MSE x 10^(0.1/10), "
                                 f"checked when the sampled loss is within {wl['full_frame_gate']}x of it; "
                                 f"both arms"),
                   "parallelism": f"replicas x{world}", "l2": "no flush: per-step working set > 129 MB",
                   "wall_s": {"server": round(wall_srv, 2), "plain": round(wall_plain, 2)}},
        "roofline": None,
        "e2e": {"value": round(fits_srv, 3), "unit": "fits/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "clocks": clock_info,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t, m, dt = _oracle_fit_step_time([j["sc"] for j in jobs], [j["start"] for j in jobs],
                                         [j["targets"] for j in jobs], [list(range(len(j["sc"].cams))) for j in jobs],
                                         {**cfgd, "seed": 0x5EED}, {"fit_steps": 0}, args.cpu_seconds)
        spf = float(np.mean([i.steps for i in ok])) if ok else wl["max_steps"]
        result["cpu_baseline"] = {
            "value": round(1.0 / (spf * t), 6), "unit": "fits/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one FP64 LM step on each of the first {m} requests ({dt:.1f} s); fits/s = 1 / "
                      f"({spf:.1f} steps per fit, the server's mean, x mean seconds per step)"}
    ranks.close()
    return result


def _oracle_fit_step_time(scenes, starts, targets, views, cfg, wl, budget_s):
    """The FP64 oracle's LM step on scenes 0, 1, ... until budget_s; returns
    (mean seconds per scene-step, scenes done, seconds)."""
    import oracle
    ocfg = {k: v for k, v in cfg.items()}
    times = []
    t_all = time.perf_counter()
    for i, sc in enumerate(scenes):
        tgt = targets[i].cpu().numpy() if hasattr(targets[i], "cpu") else targets[i]
        p0 = starts[i].cpu().numpy() if hasattr(starts[i], "cpu") else starts[i]
        o = oracle.OracleScene(p0, sc.cams, sc.n_gauss, sc.sh_degree, targets=tgt, **ocfg)
        t0 = time.perf_counter()
        o.lm_step(views[i], wl["fit_steps"] // 2)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all >= budget_s:
            break
    return float(np.mean(times)), len(times), time.perf_counter() - t_all


def cpu_baseline_batched(scenes, starts, targets, views, cfg, wl, budget_s):
    import oracle
    t, n, dt = _oracle_fit_step_time(scenes, starts, targets, views, cfg, wl, budget_s)
    return {"value": round(1.0 / (wl["fit_steps"] * t), 5), "unit": "fits/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"one FP64 LM step on each of the first {n} of the {len(scenes)} scenes ({dt:.1f} s); "
                      f"fits/s = 1 / ({wl['fit_steps']} x mean seconds per scene-step)"}


def cpu_baseline(sc, views, step, wl, budget_s=20.0):
    """The FP64 oracle as it stands: J^T W J v over the same scene and views,
    repeated until budget_s (at least once); value in operator applications
    per second."""
    import oracle
    o = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, sc.sh_degree, sample_frac=wl["sample_frac"],
                           lambda_=wl["lam"], damping_mode=1, seed=0x5EED)
    n_all = len(views)
    if wl.get("cpu_views"):
        views = list(views)[:wl["cpu_views"]]  # the operator's cost is linear in the views
    o.begin_step(list(views), step)
    v = np.random.default_rng(0).standard_normal(o.n_params)
    D = np.zeros(o.n_params)  # the damping term is one axpy; the product is J^T W J v
    n, t0 = 0, time.perf_counter()
    while True:
        o.apply(v, D)
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    scale = len(views) / n_all
    return {"value": round(n / dt * scale, 5), "unit": "matvec/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} operator application(s) J^T W J v over {len(views)} of the {n_all} sampled views of "
                      f"the same scene ({o.n_samples} samples), FP64, {dt:.1f} s"
                      + (f"; scaled by {scale:.4f} to the full operator" if scale < 1 else "")}


def run_reference_batched(args):
    """The oracle on the batched workload: each bench step is one FP64 LM
    step of one of the 64 scenes (in turn); fits/s = 1 / (20 x mean step
    time).  Targets are noise: the cost of a step depends on the Gaussians
    and the sampling, not on the target values."""
    import oracle
    from paper_2504_12905_gb300 import synthetic as syn
    wl = WORKLOADS["batched"]
    scenes = syn.small_fit_scenes()
    prng = np.random.default_rng(4321)
    cfg = dict(samples_per_tile=wl["samples_per_tile"], lambda_=wl["lam"], damping_mode=wl["damping_mode"],
               cg_iters=wl["cg_iters"], seed=0x5EED)
    times = []
    for k in range(args.warmup + args.steps):
        sc = scenes[k % len(scenes)]
        p0 = syn.perturb(prng, sc.params)
        tgt = syn.noise_targets(prng, len(sc.cams), sc.height, sc.width)
        o = oracle.OracleScene(p0, sc.cams, sc.n_gauss, sc.sh_degree, targets=tgt, **cfg)
        t0 = time.perf_counter()
        o.lm_step(list(range(len(sc.cams))), k)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = 1.0 / (wl["fit_steps"] * t)
    cores = oracle.num_threads()
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "fits/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * t, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": f"batched: {wl['desc']}", "parallelism": "host cores"},
            "cpu_baseline": {"value": round(value, 5), "unit": "fits/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step one LM step of one scene (scenes in turn), "
                                       f"fits/s = 1 / ({wl['fit_steps']} x mean step time)"},
            "e2e": {"value": round(value, 5), "unit": "fits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference(args):
    import oracle
    if args.workload == "batched":
        return run_reference_batched(args)
    wl = WORKLOADS[args.workload]
    sc = make_scene(args.workload)
    from paper_2504_12905_gb300 import synthetic as syn
    vrng = np.random.default_rng(77)
    nc = len(sc.cams)
    o = oracle.OracleScene(sc.params, sc.cams, sc.n_gauss, sc.sh_degree, sample_frac=wl["sample_frac"],
                           lambda_=wl["lam"], damping_mode=1, seed=0x5EED)
    v = np.random.default_rng(0).standard_normal(o.n_params)
    D = np.zeros(o.n_params)
    # each step: one operator application on one of the sampled views (a
    # bounded sample of the workload); the metric scales it to full steps
    per_step_views = 1
    total = 0.0
    for k in range(args.warmup + args.steps):
        vs = syn.view_subset(vrng, nc, wl["views_per_step"])[:per_step_views]
        o.begin_step(list(vs), k)
        t0 = time.perf_counter()
        o.apply(v, D)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            total += dt
    frac = per_step_views / wl["views_per_step"]
    value = args.steps * frac / total
    cores = oracle.num_threads()
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "matvec/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * total / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": f"{args.workload}: {wl['desc']}", "parallelism": "host cores"},
            "cpu_baseline": {"value": round(value, 4), "unit": "matvec/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step one operator application over 1 of the {wl['views_per_step']} "
                                       f"views (scaled by {frac:.3f} of an application)"},
            "e2e": {"value": round(value, 4), "unit": "matvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="moderate")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=0, help="serving workload: number of timed requests")
    ap.add_argument("--max-active", type=int, default=0, help="serving workload: resident jobs at most (0: default)")
    ap.add_argument("--policy", type=int, default=-1, help="serving workload: 0 FIFO, 1 least work first")
    ap.add_argument("--pcg-launch", choices=["persistent", "graph"], default="persistent",
                    help="batched workload: the PCG of all scenes in one persistent launch per LM step "
                         "(default), or a CUDA graph of per-phase launches")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        print("bench: at least 3 warm-up steps are required", file=sys.stderr)
        args.warmup = 3
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    run = {"batched": run_batched, "serving": run_serving, "ksweep": run_ksweep, "fit": run_fit}.get(args.workload,
                                                                                                   run_ours)
    res = run(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
