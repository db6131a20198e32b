"""Time-to-target measurements of the synthetic workloads other than the
benchmark's headline one (python -m paper_2411_00688_gb300.workloads NAME ...).

  denoise2d_256  ProxSkip p = 0.1 vs PGD, 100 inner iterations, <= 500 iterations
  ct2d_512       PDHGSkip-2 and PDHGSkip-1 p in {0.2, 0.05} vs PDHG, <= 2000 iterations, at sigma = tau with 50
                 inner iterations and at sigma = tau / 4 with 200; explicit preconditioned PDHG
                 (closed-form proxes) <= 20000 iterations
  deblur2d_1024  PGD, FISTA and ProxSkip p in {0.5, 0.1, 0.05} at 50, 100 and 200 inner
                 iterations (<= 1000 iterations); explicit preconditioned PDHG <= 20000
  denoise3d_512  ProxSkip p = 0.1 vs PGD, 30 inner, <= 200 iterations (FP32 / BF16 / FP16 dual)
  batch2d_256    256 uneven problems: one batched solve vs a loop of single solves
  table1_deblur2d_1024  Table 1's solvers (FISTA-100, ISTA-10, ProxSkip-10 p = 0.5, ProxSkip-100
                 p = 0.05) to a 1e-5 relative distance from u*
  dual_huber_200x300    ProjGD, AProjGD and ProxSkip on Dual-Huber-ROF (Section 2.2)
  iteration_split_deblur2d_1024  device time of skipped and prox outer iterations of the
                 ProxSkip solve (trace timestamps), p = 0.5 and 0.02
  batch_dual_error      the batched workload with each 16-bit dual storage against FP32:
                 problems over 2e-3 relative l2, worst cases, largest PSNR change

Each prints one JSON line per solver: iterations and prox calls to a 1e-4
relative objective gap, device time to the target and wall time of the solve.
F* is the smallest objective of a long reference run on the same GPU
(FISTA for forward-backward problems, PDHG for CT), made first.
"""

from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

TARGET = 1e-4


def _ctx():
    import paper_2411_00688_gb300 as tvs
    return tvs, tvs.Context(0)


def _solve_record(name, tr, wall_s, f_star, **extra):
    gaps = (tr.objective - f_star) / f_star if len(tr.objective) else np.array([np.nan])
    its = (tr.reached_iter + 1) if tr.reached else tr.iters_run
    rec = {"solver": name, "reached": tr.reached, "iterations": its,
           "iterations_per_s": its / (tr.time_to_target_s if tr.reached and tr.time_to_target_s > 0
                                      else max(tr.solve_ms * 1e-3, 1e-12)),
           "prox_calls": tr.prox_calls, "time_to_target_s": tr.time_to_target_s if tr.reached else None,
           "wall_s": wall_s, "final_rel_gap": float(gaps[-1]), "best_rel_gap": float(np.nanmin(gaps))}
    rec.update(extra)
    return rec


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def denoise2d_256():
    import torch
    from synth.configs import DenoiseConfig
    tvs, ctx = _ctx()
    cfg = DenoiseConfig()
    b = torch.from_numpy((cfg.phantom() + cfg.noise()).astype(np.float32)).cuda()
    prob = tvs.Problem(ctx, b, cfg.alpha)
    _, ref = tvs.fista_solve(prob, b.clone(), cfg.gamma, 3000, 200)
    f_star = float(np.nanmin(ref.objective))
    out = []
    for name, fn in [
        ("pgd", lambda: tvs.pgd_solve(prob, b.clone(), cfg.gamma, cfg.max_iter, cfg.n_inner, f_star=f_star, target=TARGET)),
        ("proxskip_p0.1", lambda: tvs.proxskip_solve(prob, b.clone(), cfg.gamma, cfg.p, cfg.seed, cfg.max_iter,
                                                     cfg.n_inner, f_star=f_star, target=TARGET)),
    ]:
        fn()  # warm-up (graph capture paths, autotuner)
        (_, tr), wall = _timed(fn)
        out.append(_solve_record(name, tr, wall, f_star, workload=cfg.name))
    return out


def _power_norm_sq(tvs, prob, shape, meas_shape, iters=100):
    import torch
    x = torch.randn(shape, device="cuda")
    x /= x.norm()
    y = torch.empty(meas_shape, device="cuda")
    z = torch.empty(shape, device="cuda")
    lam = 0.0
    for _ in range(iters):
        tvs.tvs_op_apply(prob, x, y)
        tvs.tvs_op_apply(prob, y, z, adjoint=True)
        lam = float((x * z).sum())
        x = z / z.norm()
    return lam


def ct2d_512():
    import torch
    from synth.configs import CTConfig
    tvs, ctx = _ctx()
    cfg = CTConfig()
    N = cfg.N
    truth = torch.from_numpy(cfg.phantom().astype(np.float32)).cuda()
    mk = dict(op="ct", shape=(N, N), n_angles=cfg.n_angles, n_det=cfg.n_det, pixel_size=1.0 / N,
              det_spacing=1.0 / N)
    zeros_sino = torch.zeros((cfg.n_angles, cfg.n_det), device="cuda")
    op = tvs.Problem(ctx, zeros_sino, cfg.alpha, **mk)
    clean = torch.empty_like(zeros_sino)
    tvs.tvs_op_apply(op, truth, clean)
    counts = cfg.counts(clean.cpu().numpy().astype(np.float64))
    b = torch.from_numpy((-np.log(np.maximum(counts, 1.0) / cfg.photons)).astype(np.float32)).cuda()
    prob = tvs.Problem(ctx, b, cfg.alpha, **mk)
    L = _power_norm_sq(tvs, prob, (N, N), (cfg.n_angles, cfg.n_det))
    st = 0.99 / math.sqrt(L)
    x0 = torch.zeros((N, N), device="cuda")
    _, _, ref = tvs.pdhg_solve(prob, x0.clone(), zeros_sino.clone(), st, st, 6000, 100)
    f_star = float(np.nanmin(ref.objective))
    out = []
    # the configuration's setting (sigma = tau, 50 inner iterations) and a second
    # one with a smaller primal step (sigma = tau / 4, sigma tau ||A||^2 = 0.98) and
    # 200 inner iterations, where the larger prox steps lambda = sigma alpha / p of
    # PDHGSkip-2 are solved accurately enough to reach the target
    for ratio, n_inner in ((1.0, cfg.n_inner), (0.25, 200)):
        sg, ta = st * math.sqrt(ratio), st / math.sqrt(ratio)
        runs = [("pdhg", lambda sg=sg, ta=ta, ni=n_inner: tvs.pdhg_solve(
            prob, x0.clone(), zeros_sino.clone(), sg, ta, cfg.max_iter, ni, f_star=f_star, target=TARGET))]
        for p in cfg.ps:
            runs.append((f"pdhgskip_p{p}", lambda p=p, sg=sg, ta=ta, ni=n_inner: tvs.pdhgskip_solve(
                prob, x0.clone(), zeros_sino.clone(), sg, ta, p, cfg.seed, cfg.max_iter, ni, f_star=f_star,
                target=TARGET)))
            # PDHGSkip-1 also skips both projector applications when theta_k = 0
            runs.append((f"pdhgskip1_p{p}", lambda p=p, sg=sg, ta=ta, ni=n_inner: tvs.pdhgskip1_solve(
                prob, x0.clone(), zeros_sino.clone(), sg, ta, p, cfg.seed, cfg.max_iter, ni, f_star=f_star,
                target=TARGET)))
        for name, fn in runs:
            fn()
            (_, _, tr), wall = _timed(fn)
            out.append(_solve_record(name, tr, wall, f_star, workload=cfg.name, norm_A_sq=L, sigma=sg, tau=ta,
                                     n_inner=n_inner))
    out.append(_explicit(tvs, prob, x0, zeros_sino, f_star, cfg.name))
    return out


def ct2d_512_sweep():
    """PDHG against PDHGSkip-2 and PDHGSkip-1 (p = 0.2, 0.05) on the CT workload over
    the step split sigma = tau * ratio (sigma tau ||A||^2 = 0.98) and the inner
    iteration count: time to the 1e-4 gap (F* from a long PDHG run), iterations and
    prox calls; the projector pair's time beside it."""
    import torch
    from synth.configs import CTConfig
    tvs, ctx = _ctx()
    cfg = CTConfig()
    N = cfg.N
    truth = torch.from_numpy(cfg.phantom().astype(np.float32)).cuda()
    mk = dict(op="ct", shape=(N, N), n_angles=cfg.n_angles, n_det=cfg.n_det, pixel_size=1.0 / N,
              det_spacing=1.0 / N)
    zeros_sino = torch.zeros((cfg.n_angles, cfg.n_det), device="cuda")
    op = tvs.Problem(ctx, zeros_sino, cfg.alpha, **mk)
    clean = torch.empty_like(zeros_sino)
    tvs.tvs_op_apply(op, truth, clean)
    counts = cfg.counts(clean.cpu().numpy().astype(np.float64))
    b = torch.from_numpy((-np.log(np.maximum(counts, 1.0) / cfg.photons)).astype(np.float32)).cuda()
    prob = tvs.Problem(ctx, b, cfg.alpha, **mk)
    L = _power_norm_sq(tvs, prob, (N, N), (cfg.n_angles, cfg.n_det))
    st = 0.99 / math.sqrt(L)
    x0 = torch.zeros((N, N), device="cuda")
    _, _, ref = tvs.pdhg_solve(prob, x0.clone(), zeros_sino.clone(), st, st, 6000, 100)
    f_star = float(np.nanmin(ref.objective))
    out = []
    for ratio in (1.0, 0.25, 0.0625):
        sg, ta = st * math.sqrt(ratio), st / math.sqrt(ratio)
        for n_inner in (50, 200, 500):
            runs = [("pdhg", lambda: tvs.pdhg_solve(prob, x0.clone(), zeros_sino.clone(), sg, ta, cfg.max_iter,
                                                    n_inner, f_star=f_star, target=TARGET))]
            for p in cfg.ps:
                runs.append((f"pdhgskip2_p{p}", lambda p=p: tvs.pdhgskip_solve(
                    prob, x0.clone(), zeros_sino.clone(), sg, ta, p, cfg.seed, cfg.max_iter, n_inner,
                    f_star=f_star, target=TARGET)))
                runs.append((f"pdhgskip1_p{p}", lambda p=p: tvs.pdhgskip1_solve(
                    prob, x0.clone(), zeros_sino.clone(), sg, ta, p, cfg.seed, cfg.max_iter, n_inner,
                    f_star=f_star, target=TARGET)))
            for name, fn in runs:
                fn()
                (_, _, tr), wall = _timed(fn)
                out.append(_solve_record(name, tr, wall, f_star, workload="ct2d_512", ratio=ratio,
                                         n_inner=n_inner))
    return out


def _explicit(tvs, prob, x0, y0, f_star, name, K=20000):
    def run():
        return tvs.pdhg_explicit_solve(prob, x0.clone(), y0.clone(), None, K, f_star=f_star, target=TARGET)
    run()
    (_, _, _, tr), wall = _timed(run)
    return _solve_record("pdhg_explicit", tr, wall, f_star, workload=name,
                         ms_per_iteration=tr.solve_ms / max(tr.iters_run, 1))


def deblur2d_1024():
    import torch
    from synth.configs import DeblurConfig
    tvs, ctx = _ctx()
    cfg = DeblurConfig()
    truth = torch.from_numpy(cfg.phantom().astype(np.float32)).cuda()
    noise = torch.from_numpy(cfg.noise().astype(np.float32)).cuda()
    prob = tvs.Problem(ctx, truth, cfg.alpha, op="blur", blur_sigma=cfg.blur_sigma)
    b = torch.empty_like(truth)
    tvs.tvs_op_apply(prob, truth, b)
    b = (b + noise).contiguous()
    prob.set_data(b)
    _, ref = tvs.fista_solve(prob, b.clone(), 1.0, 3000, 100)  # gamma = 1/||A||^2 = 1
    f_star = float(np.nanmin(ref.objective))
    out = []
    # ProxSkip at every probability of the configuration and PGD / FISTA with the
    # same prox, at the configuration's 50 inner iterations and at 100 and 200 (a
    # more accurate prox is what the small-p runs need at lambda = gamma alpha / p)
    for n_inner in (cfg.n_inner, 100, 200):
        runs = [("pgd", lambda ni=n_inner: tvs.pgd_solve(prob, b.clone(), 1.0, cfg.max_iter, ni, f_star=f_star,
                                                           target=TARGET)),
                ("fista", lambda ni=n_inner: tvs.fista_solve(prob, b.clone(), 1.0, cfg.max_iter, ni, f_star=f_star,
                                                               target=TARGET))]
        for p in cfg.ps:
            runs.append((f"proxskip_p{p}", lambda p=p, ni=n_inner: tvs.proxskip_solve(
                prob, b.clone(), 1.0, p, cfg.seed, cfg.max_iter, ni, f_star=f_star, target=TARGET)))
        for name, fn in runs:
            fn()
            (_, tr), wall = _timed(fn)
            out.append(_solve_record(name, tr, wall, f_star, workload=cfg.name, n_inner=n_inner))
    out.append(_explicit(tvs, prob, b, torch.zeros_like(b), f_star, cfg.name))
    return out


def iteration_split_deblur2d_1024():
    """Where an outer iteration's time goes in the ProxSkip solve of the deblurring
    workload (50 inner iterations, no stopping target): from the trace's device
    timestamps, the median time between the objective records of two consecutive
    skipped iterations and of two consecutive prox iterations (whose records run
    beside the inner iterations, so only two records made the same way are
    compared), with the inner iterations' time per prox call; at p = 0.5 (the
    benchmark's probability) and at p = 0.02 (almost every iteration skipped)."""
    import statistics
    import torch
    from synth.configs import DeblurConfig
    tvs, ctx = _ctx()
    cfg = DeblurConfig()
    truth = torch.from_numpy(cfg.phantom().astype(np.float32)).cuda()
    noise = torch.from_numpy(cfg.noise().astype(np.float32)).cuda()
    prob = tvs.Problem(ctx, truth, cfg.alpha, op="blur", blur_sigma=cfg.blur_sigma)
    b = torch.empty_like(truth)
    tvs.tvs_op_apply(prob, truth, b)
    b = (b + noise).contiguous()
    prob.set_data(b)
    out = []
    for p, K in ((0.5, 300), (0.02, 600)):
        for _ in range(3):  # the last of three solves (graphs captured, clocks up)
            _, tr = tvs.proxskip_solve(prob, b.clone(), 1.0, p, cfg.seed, K, cfg.n_inner)
        t, c, n = tr.t_s, tr.coins, tr.iters_run
        skip = [t[k + 1] - t[k] for k in range(n - 1) if c[k] == 0 and c[k + 1] == 0]
        prox = [t[k + 1] - t[k] for k in range(n - 1) if c[k] == 1 and c[k + 1] == 1]
        out.append({"workload": cfg.name, "p": p, "iterations": n, "prox_calls": tr.prox_calls,
                    "solve_ms": tr.solve_ms,
                    "skipped_iteration_us": statistics.median(skip) * 1e6 if skip else None,
                    "prox_iteration_us": statistics.median(prox) * 1e6 if prox else None,
                    "inner_us_per_prox": tr.fgp_ms / max(tr.prox_calls, 1) * 1e3})
    return out


def denoise3d_512(duals=("f32", "bf16", "f16", "q15")):
    import torch
    from synth.configs import Denoise3DConfig
    tvs, ctx = _ctx()
    cfg = Denoise3DConfig()
    vol = cfg.phantom()
    vol += cfg.noise()
    b = torch.from_numpy(vol).cuda()
    del vol
    prob = tvs.Problem(ctx, b, cfg.alpha)
    _, ref = tvs.fista_solve(prob, b.clone(), cfg.gamma, 400, 60)
    f_star = float(np.nanmin(ref.objective))
    out = []
    for dual in duals:
        for name, fn in [
            ("pgd", lambda: tvs.pgd_solve(prob, b.clone(), cfg.gamma, cfg.max_iter, cfg.n_inner, dual=dual,
                                          f_star=f_star, target=TARGET)),
            ("proxskip_p0.1", lambda: tvs.proxskip_solve(prob, b.clone(), cfg.gamma, cfg.p, cfg.seed, cfg.max_iter,
                                                         cfg.n_inner, dual=dual, f_star=f_star, target=TARGET)),
        ]:
            (_, tr), wall = _timed(fn)
            per_it = tr.fgp_ms / max(tr.fgp_launches, 1) * 1e-3
            bpv = 40 if dual == "f32" else 22
            out.append(_solve_record(name, tr, wall, f_star, workload=cfg.name, dual=dual,
                                     fgp_launch_us=per_it * 1e6,
                                     fgp_gbs=bpv * cfg.N ** 3 / per_it / 1e9 if per_it > 0 else None))
    return out


def table1_deblur2d_1024():
    """Table 1's comparison on the synthetic 1024^2 deblurring problem: time to a
    relative distance ||x_k - u*|| / ||u*|| of 1e-4 and 1e-5 (the paper's error
    measure and target, Section 3.1) for FISTA-100, ISTA-10 (= PGD), ProxSkip-10
    with p = 0.5 and ProxSkip-100 with p = 0.05, every prox warm-started, 5000
    iterations each.  u* is a long FISTA run (4000 iterations, 200 inner) on the
    same GPU."""
    import torch
    from synth.configs import DeblurConfig
    tvs, ctx = _ctx()
    cfg = DeblurConfig()
    truth = torch.from_numpy(cfg.phantom().astype(np.float32)).cuda()
    noise = torch.from_numpy(cfg.noise().astype(np.float32)).cuda()
    prob = tvs.Problem(ctx, truth, cfg.alpha, op="blur", blur_sigma=cfg.blur_sigma)
    b = torch.empty_like(truth)
    tvs.tvs_op_apply(prob, truth, b)
    b = (b + noise).contiguous()
    prob.set_data(b)
    u_star, ref = tvs.fista_solve(prob, b.clone(), 1.0, 4000, 200)
    u_star = u_star.clone()
    prob.set_reference(u_star)
    K = 5000
    rows = [("fista_100", lambda: tvs.fista_solve(prob, b.clone(), 1.0, K, 100)),
            ("ista_10", lambda: tvs.pgd_solve(prob, b.clone(), 1.0, K, 10)),
            ("proxskip_10_p0.5", lambda: tvs.proxskip_solve(prob, b.clone(), 1.0, 0.5, cfg.seed, K, 10)),
            ("proxskip_100_p0.05", lambda: tvs.proxskip_solve(prob, b.clone(), 1.0, 0.05, cfg.seed, K, 100))]
    out = []
    for name, fn in rows:
        fn()
        (_, tr), wall = _timed(fn)
        d = tr.rel_dist
        rec = {"workload": "table1_deblur2d_1024", "solver": name, "iterations_run": tr.iters_run,
               "wall_s": wall, "best_rel_dist": float(np.nanmin(d))}
        for tgt in (1e-4, 1e-5):
            hit = np.nonzero(d <= tgt)[0]
            k = int(hit[0]) if len(hit) else None
            rec[f"to_{tgt:g}"] = {"reached": k is not None, "iterations": (k + 1) if k is not None else None,
                                  "prox_calls": int(np.sum(tr.coins[: k + 1])) if k is not None else None,
                                  "time_s": float(tr.t_s[k]) if k is not None else None}
        out.append(rec)
    for tgt in ("to_0.0001", "to_1e-05"):
        t_f = out[0][tgt]["time_s"]
        for r in out:
            if t_f and r[tgt]["time_s"]:
                r[tgt]["faster_than_fista_pct"] = 100.0 * (t_f - r[tgt]["time_s"]) / t_f
    return out


def dual_huber_200x300(target=1e-6):
    """Section 2.2's comparison: Dual-Huber-ROF (alpha 0.55, eps 0.1) on a 200 x 300
    shapes image with noise 0.05, ProjGD, AProjGD and ProxSkip (p = 0.04767), step
    1/L with L = 8 + eps/alpha, at most 5000 iterations, time until the relative
    error ||u_k - u*|| / ||u*|| of u = b + div q is <= target (the paper's measure).
    u* from a 40000-iteration AProjGD run."""
    import torch
    from synth import phantoms
    tvs, ctx = _ctx()
    H, W, alpha, eps = 200, 300, 0.55, 0.1
    b = torch.from_numpy((phantoms.shapes_phantom_2d(H, W, 12, 7100)
                          + phantoms.gaussian_noise((H, W), 0.05, 7101)).astype(np.float32)).cuda()
    gamma = 1.0 / (8.0 + eps / alpha)
    q = torch.zeros((2, H, W), device="cuda")
    u_star = torch.empty((H, W), device="cuda")
    tvs.dual_rof_solve(ctx, b, q, alpha, gamma, 40000, eps=eps, accelerated=True, u=u_star)
    runs = [("projgd", dict()), ("aprojgd", dict(accelerated=True)), ("proxskip_p0.04767", dict(p=0.04767, seed=1))]
    out = []
    for name, kw in runs:
        def fn(kw=kw):
            return tvs.dual_rof_solve(ctx, b, torch.zeros((2, H, W), device="cuda"), alpha, gamma, 5000, eps=eps,
                                      u_ref=u_star, target_dist=target, **kw)
        fn()
        (_, _, tr), wall = _timed(fn)
        k = tr.reached_iter if tr.reached else None
        out.append({"workload": "dual_huber_200x300", "solver": name, "target_rel_dist": target,
                    "reached": bool(tr.reached), "iterations": (k + 1) if k is not None else tr.iters_run,
                    "prox_calls": int(np.sum(tr.coins[: k + 1])) if k is not None else tr.prox_calls,
                    "time_to_target_s": tr.time_to_target_s if tr.reached else None,
                    "best_rel_dist": float(np.nanmin(tr.rel_dist)), "wall_s": wall})
    return out


def _batch(n_problems=None, K=None, batch_only=False, dual="f32"):
    import torch
    from synth.configs import BatchConfig
    tvs, ctx = _ctx()
    cfg = BatchConfig()
    specs = cfg.specs()[: n_problems or cfg.n_problems]
    K = K or cfg.max_iter
    probs, bs = [], []
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
    ps = [sp["p"] for sp in specs]
    seeds = [sp["seed"] for sp in specs]
    npx = sum(sp["H"] * sp["W"] for sp in specs)

    def batched():
        xs = [b.clone() for b in bs]
        return tvs.proxskip_solve_batch(ctx, probs, xs, [1.0] * len(probs), ps, seeds, K, cfg.n_inner, dual=dual)

    def loop():
        trs = []
        for pr, b, p, s in zip(probs, bs, ps, seeds):
            trs.append(tvs.proxskip_solve(pr, b.clone(), 1.0, p, s, K, cfg.n_inner, dual=dual)[1])
        return trs

    batched()
    _, t_batch = _timed(batched)
    if batch_only:
        return [{"workload": cfg.name, "problems": len(specs), "pixels": npx, "iterations": K,
                 "n_inner": cfg.n_inner, "batched_s": t_batch}]
    loop()
    _, t_loop = _timed(loop)
    return [{"workload": cfg.name, "dual": dual, "problems": len(specs), "pixels": npx, "iterations": K,
             "n_inner": cfg.n_inner, "batched_s": t_batch, "loop_s": t_loop, "speedup": t_loop / t_batch}]


def batch_dual_error():
    """The batched workload (256 problems, 200 iterations, 50 inner) solved with each
    16-bit dual storage and with FP32: per storage, how many problems' iterates are
    more than 2e-3 (relative l2) from the FP32 ones, the two worst with their prox
    step lambda = gamma alpha / p, and the largest PSNR change against the phantom."""
    import torch
    from synth.configs import BatchConfig
    tvs, ctx = _ctx()
    cfg = BatchConfig()
    specs = cfg.specs()
    probs, bs, truths = [], [], []
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
        truths.append(truth)
    ps = [sp["p"] for sp in specs]
    seeds = [sp["seed"] for sp in specs]

    def solve(dual):
        xs = [b.clone() for b in bs]
        tvs.proxskip_solve_batch(ctx, probs, xs, [1.0] * len(probs), ps, seeds, cfg.max_iter, cfg.n_inner,
                                 dual=dual)
        return [x.double() for x in xs]

    def psnr(x, t):
        mse = float(((x - t.double()) ** 2).mean())
        peak = float(t.abs().max())
        return 10.0 * math.log10(peak * peak / mse) if mse > 0 and peak > 0 else float("inf")

    ref = solve("f32")
    ref_psnr = [psnr(x, t) for x, t in zip(ref, truths)]
    out = []
    for dual in ("bf16", "f16", "q15"):
        xs = solve(dual)
        rows = []
        for i, (x, r) in enumerate(zip(xs, ref)):
            rel = float(torch.linalg.norm(x - r) / torch.linalg.norm(r))
            dpsnr = abs(psnr(x, truths[i]) - ref_psnr[i])
            rows.append((rel, specs[i]["alpha"] / ps[i], specs[i]["H"], specs[i]["W"], dpsnr))
        worst = sorted(rows, reverse=True)[:2]
        out.append({"workload": cfg.name, "dual": dual, "problems": len(rows),
                    "over_2e-3": sum(1 for r in rows if r[0] > 2e-3),
                    "worst": [{"rel_l2": w[0], "lambda": w[1], "shape": [w[2], w[3]]} for w in worst],
                    "max_dpsnr_db": max(r[4] for r in rows)})
    for pr in probs:
        pr.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["denoise2d_256", "ct2d_512", "denoise3d_512", "batch2d_256",
                                         "deblur2d_1024", "table1_deblur2d_1024", "dual_huber_200x300",
                                         "ct2d_512_sweep", "iteration_split_deblur2d_1024",
                                         "batch_dual_error"])
    ap.add_argument("--problems", type=int, default=None)
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--batch-only", action="store_true", help="batch2d_256: time the batched solve only")
    ap.add_argument("--dual", default="f32", choices=["f32", "bf16", "f16", "q15"], help="batch2d_256: dual storage")
    args = ap.parse_args(argv)
    if args.workload == "batch2d_256":
        recs = _batch(args.problems, args.iters, args.batch_only, args.dual)
    else:
        recs = {"denoise2d_256": denoise2d_256, "ct2d_512": ct2d_512, "denoise3d_512": denoise3d_512,
                "deblur2d_1024": deblur2d_1024, "table1_deblur2d_1024": table1_deblur2d_1024,
                "dual_huber_200x300": dual_huber_200x300, "ct2d_512_sweep": ct2d_512_sweep,
                "iteration_split_deblur2d_1024": iteration_split_deblur2d_1024,
                "batch_dual_error": batch_dual_error}[args.workload]()
    for r in recs:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
