"""Benchmark: ProxSkip time to a 1e-4 relative objective gap on one GB300, beside
PGD with the same prox, and the fused FGP kernel's bandwidth against its roofline.

Headline workload (one "step" = one solve): 2D TV deblurring, 1024 x 1024 phantom
of 40 random ellipses, 9x9 Gaussian blur (sigma 2, reflective boundary), noise
sigma 0.01, alpha 0.02, gamma = 1/||A||^2 = 1, 50 FGP iterations per prox, at most
1000 outer iterations, FP32 iterates and dual.  The step is one ProxSkip solve
(p = 0.5, Philox seed 0) from x_0 = b until (F(x_k) - F*)/F* <= 1e-4.  F* is the
FP64 oracle's reference optimum of this problem (tests/golden/fstar_deblur2d_1024.json,
written by a script that calls only the oracle); a long GPU FISTA run is made too
and its agreement with F* reported.

Outside the timed region the line also carries: PGD, FISTA and ProxSkip at the
other probabilities with the same prox; the expensive-prox regime (200 inner
iterations); and the other workloads where the method's targets are decided --
denoise3d_512 (FGP bandwidth against the HBM roofline, 512^3, FP32 / BF16 / Q15
dual), batch2d_256 (256 uneven problems in one batched solve against a loop of
single solves) and ct2d_512 (PDHG against PDHGSkip-2 and PDHGSkip-1).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-extras]
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

METRIC = "ProxSkip time-to-1e-4 gap vs PGD on one GB300; FGP TB/s vs HBM peak"
TARGET = 1e-4
P_SKIP = 0.5
P_OTHERS = (0.1, 0.05)
F_STAR_ITERS, F_STAR_INNER = 3000, 100
# Bytes of one dual component per pixel for each dual storage type.
DUAL_BYTES = {"f32": 4, "bf16": 2, "f16": 2, "q15": 2}
WORKLOAD = ("deblur2d_1024: 1024x1024, 40 ellipses, 9x9 Gaussian sigma 2, noise 0.01, alpha 0.02, gamma 1, "
            "ProxSkip p 0.5 seed 0, 50 FGP iterations per prox, stop at relative objective gap 1e-4 "
            "(max 1000 iterations)")
# DRAM bytes (read + write) per launch of an inner-iteration kernel from one ncu
# capture of `dram__bytes_read.sum + dram__bytes_write.sum`.  Each record describes
# only the kernel sources and launch configuration it was taken on: the bench line
# carries it only while the hash of those sources (and the configuration) match.
FGP_TRAFFIC = {"config": [5, 2, 104], "bytes": 20195840,
               "sources": ["common.cuh", "fgp_rb.cuh", "fgp_tb.cu"],
               "sha256": "7dafce1aec9a07fdd0483c5eb416d9acad51838b822cd5265c8f481ed5a03bd9"}
# 3D: per momentum launch of the default kernel, captured on a 320^3 volume
# (inputs larger than L2) and scaled by the voxel count to 512^3.
_FGP3_SRC = {"sources": ["common.cuh", "tma.cuh", "fgp3d.cu"],
             "sha256": "cf831402f604485ec8c42bd514da6902281b4a93b3b78c8ce0754a2e0158cbbf"}
FGP3_TRAFFIC = {"f32": dict(_FGP3_SRC, bytes=5397339439),
                "bf16": dict(_FGP3_SRC, bytes=2951982612),
                "q15": dict(_FGP3_SRC, bytes=2961351639)}
# Iterations this workload's ProxSkip solve needs to reach the target on the GPU
# (its trace: 265 iterations to the 1e-4 gap against the oracle's F*); the reference
# arm extrapolates the oracle to them, counting the prox calls among them from the
# coin schedule.
REF_ITERS_DEFAULT = 265
FSTAR_GOLDEN = os.path.join(ROOT, "tests", "golden", "fstar_deblur2d_1024.json")
FSTAR_CT_GOLDEN = os.path.join(ROOT, "tests", "golden", "fstar_ct2d_512.json")


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value, device=None):
    """The largest value over the ranks of the default process group (the value
    itself without one): replicas are timed by their slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback (6.8 TB/s, no MEASURED_PEAKS.json)"


def _sources_hash(names):
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2411_00688_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _fgp_traffic(fgp_cfg):
    """The recorded DRAM traffic per launch, or None when the kernel or its
    configuration differs from the one it was measured on."""
    if _sources_hash(FGP_TRAFFIC["sources"]) != FGP_TRAFFIC["sha256"] or list(fgp_cfg) != FGP_TRAFFIC["config"]:
        return None
    return FGP_TRAFFIC["bytes"]


def _fgp3_traffic(dual):
    rec = FGP3_TRAFFIC.get(dual)
    if not rec or _sources_hash(rec["sources"]) != rec["sha256"]:
        return None
    return rec["bytes"]


def fgp_algo_bytes(n_iter, units, ndim, dual="f32"):
    """Algorithmic HBM bytes of n_iter FGP iterations over `units` pixels or voxels
    (nothing cached between iterations): each reads z (FP32) and p_k and writes
    p_{k+1} (ndim components each); from the third on it also reads p_{k-1} for
    the momentum term, whose weight is zero in the first two because t restarts
    at 1 with every prox call.  2D FP32: 20 and 28 B per pixel; 3D FP32: 28 and
    40 B per voxel; 3D 16-bit: 16 and 22 B per voxel."""
    p = ndim * DUAL_BYTES[dual]
    return units * (n_iter * (4 + 2 * p) + max(n_iter - 2, 0) * p)


def _golden_f_star():
    if not os.path.exists(FSTAR_GOLDEN):
        return None
    with open(FSTAR_GOLDEN) as f:
        return json.load(f)


def ct_f_star(f_gpu, path=FSTAR_CT_GOLDEN):
    """F* of the CT workload: the FP64 oracle's (committed, written by
    tests/golden/make_fstar_ct2d_512.py) when present, else the GPU's long PDHG
    run; returns (F*, where it came from, the agreement record)."""
    if os.path.exists(path):
        with open(path) as f:
            rec = json.load(f)
        fs = float(rec["f_star"])
        return fs, "FP64 oracle (tests/golden/fstar_ct2d_512.json)", {
            "gpu_pdhg_min": f_gpu, "rel_diff": (f_gpu - fs) / fs}
    return f_gpu, "PDHG, 4000 iterations, 100 inner, same GPU", None


def _workload_inputs():
    from synth.configs import DeblurConfig
    cfg = DeblurConfig()
    return cfg, cfg.phantom().astype(np.float32), cfg.noise().astype(np.float32)


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _flush_l2(buf):
    buf.add_(1.0)  # touches 256 MB (> 129 MB L2)


def _events(stream):
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _make_ctx(tvs, device, stream):
    """A context launching on the benchmark's own (non-default) torch stream, so
    that CUDA events recorded there bracket its work."""
    import ctypes as C
    from paper_2411_00688_gb300 import _lib as L
    ctx = tvs.Context.__new__(tvs.Context)
    ctx._h = C.c_void_p()
    L.check(L.lib().tvs_create(C.byref(ctx._h), device, C.c_void_p(stream.cuda_stream)))
    ctx.device = device
    return ctx


def _rec(tr, t_s=None):
    reached = bool(tr.reached)
    return {"reached": reached, "iterations": (tr.reached_iter + 1) if reached else tr.iters_run,
            "prox_calls": tr.prox_calls, "time_s": t_s if t_s is not None else tr.solve_ms * 1e-3,
            "time_to_target_s": tr.time_to_target_s if reached else None}


def _timed_once(stream, fn, prep=None):
    """fn() once after a warm-up call, timed with CUDA events on `stream`;
    prep() (untimed) runs before each of the two calls."""
    import torch
    if prep:
        prep()
    fn()
    if prep:
        prep()
    torch.cuda.synchronize()
    e0, e1 = _events(stream)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) * 1e-3


# ---------------------------------------------------------------- extra workloads
def extra_denoise3d(tvs, ctx, stream, hbm_peak, peak_kind):
    """512^3 TV denoising (alpha 0.05): FGP time per inner iteration and its
    bandwidth against the HBM peak for each dual storage (the volume and its duals,
    3.5-9.7 GB, are far larger than L2), from tv_prox on the benchmark's stream with
    n + 2 inner iterations minus 2, so that every timed iteration carries the
    momentum read."""
    import torch
    from synth.configs import Denoise3DConfig
    cfg = Denoise3DConfig()
    vol = cfg.phantom()
    vol += cfg.noise()
    with torch.cuda.stream(stream):
        b = torch.from_numpy(vol).cuda()
        u = torch.empty_like(b)
    del vol
    N = cfg.N
    out = {"workload": f"denoise3d_512: {N}^3, 60 ellipsoids, noise 0.05, alpha 0.05 (prox step lambda 0.5 as "
                       f"ProxSkip p = 0.1 takes it)", "peak": hbm_peak, "peak_kind": peak_kind}
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "q15": torch.int16}
    n_it = 8
    for dual in ("f32", "bf16", "q15"):
        with torch.cuda.stream(stream):
            state = torch.zeros((3, N, N, N), dtype=tdt[dual], device="cuda")
        torch.cuda.synchronize()

        def prox(n):
            tvs.tv_prox(ctx, b, u, cfg.alpha / cfg.p, n, dual=dual, dual_state=state)

        def med(n, reps=3):
            prox(n)
            ts = []
            for _ in range(reps):
                e0, e1 = _events(stream)
                e0.record(stream)
                prox(n)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e-3)
            return statistics.median(ts)
        # iterations 3 .. n_it + 2, all with momentum: prox(n_it + 2) minus prox(2)
        per_it = (med(n_it + 2) - med(2)) / n_it
        per_launch = (fgp_algo_bytes(n_it + 2, N ** 3, 3, dual) - fgp_algo_bytes(2, N ** 3, 3, dual)) / n_it
        achieved = per_launch / per_it / 1e9
        out[dual] = {"kernel": "fgp3d_tma2_kernel (z-marching, planes by TMA tile loads, packed FP32x2, "
                               "2 columns x 4 rows per lane)", "us_per_inner_iteration": per_it * 1e6,
                     "bytes_per_launch": per_launch, "achieved_gbs": achieved,
                     "frac": achieved / hbm_peak, "traffic": _fgp3_traffic(dual)}
        del state
        torch.cuda.empty_cache()
    del b, u
    torch.cuda.empty_cache()
    return out


def extra_batch(tvs, ctx, stream, rank, world):
    """batch2d_256: 256 uneven problems, one batched solve against a loop of single
    solves (200 iterations, 50 inner, FP32 and Q15 dual); with several ranks each
    solves its share of the problems (LPT split by pixels, no exchange)."""
    import torch
    from paper_2411_00688_gb300.shard import lpt_shards
    from synth.configs import BatchConfig
    cfg = BatchConfig()
    specs = cfg.specs()
    mine = lpt_shards([sp["H"] * sp["W"] for sp in specs], world)[rank]
    specs = [specs[i] for i in mine]
    probs, bs = [], []
    with torch.cuda.stream(stream):
        for sp in specs:
            truth = torch.from_numpy(cfg.phantom(sp).astype(np.float32)).cuda()
            noise = torch.from_numpy(cfg.noise(sp).astype(np.float32)).cuda()
            if sp["kind"] == "deblur":
                opp = tvs.Problem(ctx, truth, sp["alpha"], op="blur", blur_sigma=sp["blur_sigma"])
                clean = torch.empty_like(truth)
                tvs.tvs_op_apply(opp, truth, clean)
                opp.close()
                b = (clean + noise).contiguous()
                probs.append(tvs.Problem(ctx, b, sp["alpha"], op="blur", blur_sigma=sp["blur_sigma"]))
            else:
                b = (truth + noise).contiguous()
                probs.append(tvs.Problem(ctx, b, sp["alpha"]))
            bs.append(b)
    torch.cuda.synchronize()
    ps = [sp["p"] for sp in specs]
    seeds = [sp["seed"] for sp in specs]
    K, N = cfg.max_iter, cfg.n_inner

    with torch.cuda.stream(stream):
        xs = [torch.empty_like(b) for b in bs]

    def reset():
        with torch.cuda.stream(stream):
            for x, b in zip(xs, bs):
                x.copy_(b)

    def batched(dual):
        return tvs.proxskip_solve_batch(ctx, probs, xs, [1.0] * len(probs), ps, seeds, K, N, dual=dual)

    def loop():
        return [tvs.proxskip_solve(pr, x, 1.0, p, s, K, N)[1] for pr, x, p, s in zip(probs, xs, ps, seeds)]

    _, t_b = _timed_once(stream, lambda: batched("f32"), reset)
    _, t_q = _timed_once(stream, lambda: batched("q15"), reset)
    _, t_l = _timed_once(stream, loop, reset)
    t_b, t_q, t_l = (max_over_ranks(t, device="cuda") for t in (t_b, t_q, t_l))
    for pr in probs:
        pr.close()
    return {"workload": "batch2d_256: 256 problems, sides log-uniform in [64, 1024], half denoising, half "
                        "deblurring, own alpha/p/seed each, 200 iterations, 50 inner",
            "problems": len(specs) * world if world > 1 else len(specs), "ranks": world,
            "pixels_this_rank": sum(sp["H"] * sp["W"] for sp in specs),
            "batched_s": t_b, "batched_q15_s": t_q, "loop_s": t_l, "speedup": t_l / t_b}


def extra_ct(tvs, ctx, stream):
    """ct2d_512: 512^2 phantom, 720 angles x 725 bins, Poisson counts, alpha 0.5.
    PDHG against PDHGSkip-2 (p 0.7, 0.5, 0.2) and PDHGSkip-1 (p 0.7, 0.2), time to
    the 1e-4 gap with F* from the FP64 oracle (a long PDHG run on the same GPU
    without it, reported beside it in either case), at the step sizes
    and inner iteration count where PDHG is fastest in a sweep of sigma/tau in
    {1, 1/2, 1/4, 1/16} and 100 / 200 / 500 inner iterations (sigma = tau,
    sigma tau ||A||^2 = 0.98, 200 inner); and the projector pair's time."""
    import torch
    from synth.configs import CTConfig
    cfg = CTConfig()
    N = cfg.N
    mk = dict(op="ct", shape=(N, N), n_angles=cfg.n_angles, n_det=cfg.n_det, pixel_size=1.0 / N,
              det_spacing=1.0 / N)
    with torch.cuda.stream(stream):
        truth = torch.from_numpy(cfg.phantom().astype(np.float32)).cuda()
        zeros_sino = torch.zeros((cfg.n_angles, cfg.n_det), device="cuda")
        clean = torch.empty_like(zeros_sino)
    op = tvs.Problem(ctx, zeros_sino, cfg.alpha, **mk)
    tvs.tvs_op_apply(op, truth, clean)
    counts = cfg.counts(clean.cpu().numpy().astype(np.float64))
    with torch.cuda.stream(stream):
        b = torch.from_numpy((-np.log(np.maximum(counts, 1.0) / cfg.photons)).astype(np.float32)).cuda()
        x0 = torch.zeros((N, N), device="cuda")
        y = torch.empty_like(zeros_sino)
        z = torch.empty_like(x0)
    prob = tvs.Problem(ctx, b, cfg.alpha, **mk)
    # ||A||^2 by the power method on the GPU operator pair
    with torch.cuda.stream(stream):
        v = torch.rand((N, N), device="cuda")
        v /= v.norm()
    L = 0.0
    for _ in range(60):
        tvs.tvs_op_apply(prob, v, y)
        tvs.tvs_op_apply(prob, y, z, adjoint=True)
        with torch.cuda.stream(stream):
            L = float((v * z).sum())
            v = z / z.norm()
    # projector pair
    _, t_fwd = _timed_once(stream, lambda: tvs.tvs_op_apply(prob, x0, y))
    _, t_bwd = _timed_once(stream, lambda: tvs.tvs_op_apply(prob, y, z, adjoint=True))
    st = 0.99 / math.sqrt(L)
    sg = ta = st
    _, _, ref = tvs.pdhg_solve(prob, x0.clone(), zeros_sino.clone(), st, st, 4000, 100)
    f_star, f_from, f_check = ct_f_star(float(np.nanmin(ref.objective)))
    runs = {"pdhg": lambda: tvs.pdhg_solve(prob, x0.clone(), zeros_sino.clone(), sg, ta, cfg.max_iter, 200,
                                           f_star=f_star, target=TARGET)}
    for p in (0.7, 0.5, 0.2):
        runs[f"pdhgskip2_p{p}"] = (lambda p=p: tvs.pdhgskip_solve(
            prob, x0.clone(), zeros_sino.clone(), sg, ta, p, cfg.seed, cfg.max_iter, 200, f_star=f_star,
            target=TARGET))
    for p in (0.7, 0.2):
        runs[f"pdhgskip1_p{p}"] = (lambda p=p: tvs.pdhgskip1_solve(
            prob, x0.clone(), zeros_sino.clone(), sg, ta, p, cfg.seed, cfg.max_iter, 200, f_star=f_star,
            target=TARGET))
    out = {"workload": "ct2d_512: 512^2, 720 angles, 725 bins, 1e4 photons, alpha 0.5; sigma = tau "
                       "(sigma tau ||A||^2 = 0.98), 200 inner iterations",
           "norm_A_sq": L, "f_star": f_star, "f_star_from": f_from, "f_star_check": f_check,
           "projector_us": t_fwd * 1e6, "backprojector_us": t_bwd * 1e6}
    for name, fn in runs.items():
        (*_, tr), t = _timed_once(stream, fn)
        out[name] = _rec(tr, t)
    ref_t = out["pdhg"]["time_to_target_s"]
    for name in list(runs):
        if name != "pdhg" and out[name]["reached"] and ref_t:
            out[name]["speedup_vs_pdhg"] = ref_t / out[name]["time_to_target_s"]
    prob.close()
    op.close()
    return out


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import paper_2411_00688_gb300 as tvs

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    ctx = _make_ctx(tvs, local, stream)

    cfg, truth, noise = _workload_inputs()
    H, W = truth.shape
    with torch.cuda.stream(stream):
        t_truth = torch.from_numpy(truth).cuda()
        clean = torch.empty_like(t_truth)
    stream.synchronize()
    op_prob = tvs.Problem(ctx, t_truth, cfg.alpha, op="blur", blur_sigma=cfg.blur_sigma)
    tvs.tvs_op_apply(op_prob, t_truth, clean)
    op_prob.close()
    with torch.cuda.stream(stream):
        b = (clean + torch.from_numpy(noise).cuda()).contiguous()
    torch.cuda.synchronize()
    prob = tvs.Problem(ctx, b, cfg.alpha, op="blur", blur_sigma=cfg.blur_sigma)
    gamma = 1.0  # ||A||^2 = 1 for the normalised reflective blur

    # reference optimum: the oracle's (committed), cross-checked by a long GPU FISTA
    # run (not timed)
    golden = _golden_f_star()
    _, fista_tr = tvs.fista_solve(prob, b.clone(), gamma, F_STAR_ITERS, F_STAR_INNER)
    f_gpu = float(np.nanmin(fista_tr.objective))
    if golden is not None:
        f_star, f_from = float(golden["f_star"]), "FP64 oracle (tests/golden/fstar_deblur2d_1024.json)"
    else:
        f_star, f_from = f_gpu, "GPU FISTA, 3000 iterations, 100 inner (no oracle value committed)"
    # the FP32 iterates floor the GPU's objective about 1.5e-6 above the FP64
    # optimum (rounding spreads values of flat regions, which TV then counts)
    f_check = {"f_star": f_star, "from": f_from, "gpu_fista_min": f_gpu,
               "rel_diff": abs(f_gpu - f_star) / f_star, "agree_to_1e-5": abs(f_gpu - f_star) <= 1e-5 * f_star}

    def solve(kind, x, p=P_SKIP):
        if kind == "proxskip":
            return tvs.proxskip_solve(prob, x, gamma, p, cfg.seed, cfg.max_iter, cfg.n_inner,
                                      f_star=f_star, target=TARGET)
        return tvs.pgd_solve(prob, x, gamma, cfg.max_iter, cfg.n_inner, f_star=f_star, target=TARGET)

    with torch.cuda.stream(stream):
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        x = torch.empty_like(b)

    def timed(kind, steps):
        times, traces = [], []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                _flush_l2(flush)
                x.copy_(b)
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            e0, e1 = _events(stream)
            e0.record(stream)
            _, tr = solve(kind, x)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            traces.append(tr)
        return times, traces

    # PGD beside it (same prox, same target), after its own warm-up
    timed("pgd", 1)
    pgd_times, pgd_tr = timed("pgd", max(1, min(args.steps, 2)))

    timed("proxskip", args.warmup)
    torch.cuda.nvtx.range_push("timed")   # lets a profiler restrict itself to the timed solves
    with ClockSampler(local) as clk:
        ps_times, ps_tr = timed("proxskip", args.steps)
    clocks = clk.summary()
    torch.cuda.nvtx.range_pop()

    def reset_x():
        with torch.cuda.stream(stream):
            x.copy_(b)

    def one(fn):
        (_, tr), t = _timed_once(stream, fn, reset_x)
        r = _rec(tr, t)
        r["best_rel_gap"] = float(np.nanmin((tr.objective - f_star) / f_star))
        return r

    # the other probabilities of the workload, one solve each (outside the timed region)
    per_p = {str(pp): one(lambda pp=pp: solve("proxskip", x, pp)) for pp in (P_SKIP,) + P_OTHERS}
    # the small-p regime with an expensive prox (200 inner iterations for every solver)
    n200 = {
        "pgd": one(lambda: tvs.pgd_solve(prob, x, gamma, cfg.max_iter, 200, f_star=f_star, target=TARGET)),
        "proxskip_p0.1": one(lambda: tvs.proxskip_solve(prob, x, gamma, 0.1, cfg.seed, cfg.max_iter, 200,
                                                        f_star=f_star, target=TARGET)),
    }
    if n200["pgd"]["reached"] and n200["proxskip_p0.1"]["reached"]:
        n200["speedup_vs_pgd"] = n200["pgd"]["time_s"] / n200["proxskip_p0.1"]["time_s"]
    # FISTA with the same warm-started prox (the paper's main comparator)
    fista = one(lambda: tvs.fista_solve(prob, x, gamma, cfg.max_iter, cfg.n_inner, f_star=f_star, target=TARGET))

    # FGP kernel duration with CUDA events on the launching stream: tv_prox with
    # N inner iterations minus tv_prox with none, per launch.
    with torch.cuda.stream(stream):
        z = b.clone()
        u = torch.empty_like(z)
        state = torch.zeros((2, H, W), dtype=torch.float32, device="cuda")

    def prox_time(n_iter, reps=5):
        tvs.tv_prox(ctx, z, u, gamma / P_SKIP * cfg.alpha, n_iter, dual_state=state)
        best = []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                _flush_l2(flush)
            torch.cuda.synchronize()
            e0, e1 = _events(stream)
            e0.record(stream)
            tvs.tv_prox(ctx, z, u, gamma / P_SKIP * cfg.alpha, n_iter, dual_state=state)
            e1.record(stream)
            torch.cuda.synchronize()
            best.append(e0.elapsed_time(e1) * 1e-3)
        return statistics.median(best)

    fgp_cfg = tvs.tvs_fgp_config(ctx, (H, W))
    n_fgp = cfg.n_inner
    launches_per_prox = -(-n_fgp // fgp_cfg[0])
    fgp_launch_s = (prox_time(n_fgp) - prox_time(0)) / launches_per_prox
    in_solve = [t.fgp_ms / t.fgp_launches for t in ps_tr if t.fgp_launches > 0]
    fgp_in_solve_s = statistics.median(in_solve) * 1e-3 if in_solve else None
    hbm_peak, peak_kind = _peaks()
    bytes_per_launch = fgp_algo_bytes(n_fgp, H * W, 2) / launches_per_prox
    achieved = bytes_per_launch / fgp_launch_s / 1e9

    # end to end through the C ABI with pinned host buffers: H2D of b and x_0,
    # D2H of the result, every step
    b_host = torch.empty((H, W), dtype=torch.float32, pin_memory=True)
    b_host.copy_(b.cpu())
    x_host = torch.empty((H, W), dtype=torch.float32, pin_memory=True)
    b_np, x_np = b_host.numpy(), x_host.numpy()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            _flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob.set_data(b_np)
        x_np[...] = b_np
        tvs.proxskip_solve(prob, x_np, gamma, P_SKIP, cfg.seed, cfg.max_iter, cfg.n_inner,
                           f_star=f_star, target=TARGET)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_times.append(t1 - t0)

    ms_per_step = max_over_ranks(1e3 * statistics.mean(ps_times), device="cuda")
    last = ps_tr[-1]
    # kernels per iteration: the fused step kernel + 1 reduction; per prox: the
    # start stamp, the blocked inner launches and the finalisation (which writes the
    # end stamp); per solve: start stamp + final objective (2)
    launches = sum(tr.iters_run * 2 + tr.prox_calls * 2 + tr.fgp_launches + 3 for tr in ps_tr)
    result = {
        "metric": METRIC,
        "value": ms_per_step / 1e3,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps (256 MB write)"},
        "f_star": f_check,
        "time_to_target_device_s": statistics.mean(t.time_to_target_s for t in ps_tr),
        "iterations_to_target": last.reached_iter + 1 if last.reached else None,
        "outer_iterations_per_s": (last.reached_iter + 1) / last.time_to_target_s
        if last.reached and last.time_to_target_s > 0 else None,
        "prox_calls": last.prox_calls,
        "reached": all(t.reached for t in ps_tr),
        "pgd_time_to_target_s": statistics.mean(pgd_times) if all(t.reached for t in pgd_tr) else None,
        "pgd_iterations_to_target": pgd_tr[-1].reached_iter + 1 if pgd_tr[-1].reached else None,
        "speedup_vs_pgd": (statistics.mean(pgd_times) / statistics.mean(ps_times))
        if all(t.reached for t in pgd_tr) else None,
        "proxskip_by_p": per_p,
        "inner_200": n200,
        "fista": fista,
        # the 1024^2 image and its duals (about 40 MB) stay in L2 across the inner
        # iterations and the kernel runs 4 of them per launch in registers: the
        # algorithmic bytes per second are effective L2/register throughput (DRAM
        # traffic is about a fifth of them), stated against the HBM copy peak for
        # scale only -- no L2 peak is measured here; the HBM roofline is judged on
        # the 512^3 volume (roofline_hbm)
        "roofline": {"bound": "l2", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": _fgp_traffic(fgp_cfg),
                     "kernel": ("fgp2d_rb_kernel" if fgp_cfg[2] >= 100 else "fgp2d_tb_kernel")
                               + f"<float> ({fgp_cfg[0]} inner iterations per launch, config {list(fgp_cfg)})",
                     "bytes_per_launch": bytes_per_launch, "launch_us": fgp_launch_s * 1e6,
                     "peak_kind": peak_kind + "; HBM copy peak, for scale: the working set is L2-resident",
                     "launch_us_in_solve": fgp_in_solve_s * 1e6 if fgp_in_solve_s else None},
        "e2e": {"value": statistics.mean(e2e_times), "unit": "s",
                "h2d_bytes_per_step": 2 * H * W * 4, "d2h_bytes_per_step": H * W * 4},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    prob.close()
    del z, u, state, flush
    torch.cuda.empty_cache()
    if not args.no_extras:
        result["denoise3d_512"] = extra_denoise3d(tvs, ctx, stream, hbm_peak, peak_kind)
        result["roofline_hbm"] = dict(result["denoise3d_512"]["f32"], bound="hbm", unit="GB/s",
                                      peak=hbm_peak, peak_kind=peak_kind,
                                      achieved=result["denoise3d_512"]["f32"]["achieved_gbs"])
        result["batch2d_256"] = extra_batch(tvs, ctx, stream, rank, world)
        result["ct2d_512"] = extra_ct(tvs, ctx, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(cfg, truth, noise, args.ref_iters)
    if rank == 0:
        print(json.dumps(result))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- oracle timing
def _oracle_problem(cfg, truth, noise):
    from oracle import c, operators
    w = operators.gaussian_weights(cfg.blur_sigma, cfg.blur_radius)
    b = c.blur(truth.astype(np.float64), w) + noise.astype(np.float64)
    return w, b


def oracle_sample(cfg, truth, noise, iters_target, sample_iters=16):
    """The FP64 oracle on this workload, sampled: the first `sample_iters`
    iterations of its ProxSkip solve (p = 0.5, the true coins) with the C
    transcription on every host core, and the same iterations with every coin 0 to
    separate gradient steps from prox calls; extrapolated to `iters_target`
    iterations and the prox calls the coin schedule puts among them.  Also one
    gradient step and one prox of the numpy oracle on one core."""
    from oracle import c, coin, operators, solvers, tv
    w, b = _oracle_problem(cfg, truth, noise)
    coins = coin.schedule(cfg.seed, P_SKIP, max(iters_target, sample_iters))
    t0 = time.perf_counter()
    run = c.fb_solve("proxskip", b, cfg.alpha, 1.0, sample_iters, cfg.n_inner, w=w, p=P_SKIP,
                     coins=coins[:sample_iters])
    t1 = time.perf_counter()
    c.fb_solve("proxskip", b, cfg.alpha, 1.0, sample_iters, cfg.n_inner, w=w, p=P_SKIP,
               coins=[0] * sample_iters)
    t2 = time.perf_counter()
    t_step = (t2 - t1) / sample_iters
    t_prox = max((t1 - t0) - (t2 - t1), 0.0) / max(run["prox_calls"], 1)
    prox_target = int(sum(coins[:iters_target]))
    # numpy oracle, one core: one gradient step (with objective) and one prox
    prob = solvers.Problem(operators.blur_op(cfg.blur_sigma, cfg.blur_radius), b, cfg.alpha, b.shape)
    t3 = time.perf_counter()
    x_hat = b - prob.grad_f(b)
    prob.objective(x_hat)
    t4 = time.perf_counter()
    tv.fgp_prox(x_hat, cfg.alpha / P_SKIP, cfg.n_inner)
    t5 = time.perf_counter()
    return {"c_all_cores": {"threads": c.threads(), "step_s": t_step, "prox_s": t_prox,
                            "value": iters_target * t_step + prox_target * t_prox,
                            "sample_s": t2 - t0},
            "numpy_1_core": {"step_s": t4 - t3, "prox_s": t5 - t4,
                             "value": iters_target * (t4 - t3) + prox_target * (t5 - t4),
                             "sample_s": t5 - t3},
            "iters": iters_target, "prox_calls": prox_target, "sample_iters": sample_iters,
            "wall_s": t5 - t0}


def cpu_baseline(cfg, truth, noise, iters_target):
    s = oracle_sample(cfg, truth, noise, iters_target)
    ca, npy = s["c_all_cores"], s["numpy_1_core"]
    return {"value": ca["value"], "unit": "s", "cores": ca["threads"], "kind": "oracle",
            "extrapolated": True,
            "sample": (f"FP64 oracle, C transcription on {ca['threads']} host threads: the first "
                       f"{s['sample_iters']} ProxSkip iterations of this workload ({ca['sample_s']:.1f} s; "
                       f"{ca['step_s'] * 1e3:.0f} ms per gradient step, {ca['prox_s'] * 1e3:.0f} ms per "
                       f"50-iteration prox), extrapolated to {s['iters']} iterations and {s['prox_calls']} "
                       f"prox calls"),
            "numpy_1_core": {"value": npy["value"], "cores": 1,
                             "sample": f"one gradient step ({npy['step_s']:.2f} s) and one prox "
                                       f"({npy['prox_s']:.2f} s) of the numpy oracle, extrapolated alike"}}


def run_reference(args):
    """The reference arm: the FP64 oracle (no reference code exists for a paper),
    rank 0 only.  Each step times a bounded sample of the workload (see
    oracle_sample); `value` is the sample extrapolated to the whole solve,
    `ms_per_step` the wall time each step actually took."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    cfg, truth, noise = _workload_inputs()
    vals, walls, last = [], [], None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        last = oracle_sample(cfg, truth, noise, args.ref_iters)
        t1 = time.perf_counter()
        if i >= args.warmup:
            vals.append(last["c_all_cores"]["value"])
            walls.append(t1 - t0)
    value = statistics.mean(vals)
    ca = last["c_all_cores"]
    sample = (f"per step: the first {last['sample_iters']} ProxSkip iterations of the workload by the FP64 "
              f"oracle's C transcription on {ca['threads']} host threads (and the same with every coin 0, "
              f"and one step and one prox of the numpy oracle on 1 core), extrapolated to {last['iters']} "
              f"iterations and {last['prox_calls']} prox calls")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "extrapolated": True,
        "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps (256 MB write)"},
        "cpu_baseline": {"value": value, "unit": "s", "cores": ca["threads"], "kind": "oracle", "sample": sample,
                         "numpy_1_core_value": last["numpy_1_core"]["value"]},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the 3D, batch and CT records")
    ap.add_argument("--ref-iters", type=int, default=REF_ITERS_DEFAULT,
                    help="iterations the oracle's time is extrapolated to (the GPU solve's count)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
