"""Small driver for profiling the inner TV-prox kernels with ncu.

Runs ``tv_prox`` (the fused FGP iterations and the finalisation) on a seeded
random image of the requested size, a few times, so that a profiler can capture
single launches of the kernel of interest:

    python -m paper_2411_00688_gb300.prof --shape 4096 4096 --iters 8 --reps 3
    python -m paper_2411_00688_gb300.prof --shape 256 256 256 --iters 4 --dual bf16
    python -m paper_2411_00688_gb300.prof --ct 512 720 725 --reps 3
    python -m paper_2411_00688_gb300.prof --step 1024 1024 --iters 64 --reps 3

It prints the per-iteration time measured with CUDA events on the launching
stream (not meaningful under a profiler).  --ct N ANGLES BINS instead applies the
parallel-beam projector and backprojector of an N x N unit-square geometry.
--step H W runs PGD without inner iterations on an H x W 9x9-blur problem, so that
the fused forward-backward step kernel (one launch per iteration, with the
objective reduction beside it) can be captured, and prints the device time per
outer iteration.
"""

from __future__ import annotations

import argparse
import ctypes as C
import statistics


def main(argv=None):
    import torch

    import paper_2411_00688_gb300 as tvs
    from paper_2411_00688_gb300 import _lib as L

    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", type=int, nargs="+", default=[4096, 4096])
    ap.add_argument("--iters", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--lam", type=float, default=0.2)
    ap.add_argument("--dual", default="f32", choices=["f32", "bf16", "f16", "q15"])
    ap.add_argument("--ct", type=int, nargs=3, default=None, metavar=("N", "ANGLES", "BINS"))
    ap.add_argument("--step", type=int, nargs=2, default=None, metavar=("H", "W"))
    args = ap.parse_args(argv)
    if args.ct:
        return _ct(args, tvs, L)
    if args.step:
        return _step(args, tvs, L)

    stream = torch.cuda.Stream()
    ctx = tvs.Context.__new__(tvs.Context)
    ctx._h = C.c_void_p()
    L.check(L.lib().tvs_create(C.byref(ctx._h), torch.cuda.current_device(), C.c_void_p(stream.cuda_stream)))
    ctx.device = torch.cuda.current_device()
    shape = tuple(args.shape)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    z = (torch.rand(shape, device="cuda", generator=g) > 0.5).float() + 0.2 * torch.randn(
        shape, device="cuda", generator=g)
    u = torch.empty_like(z)
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16, "q15": torch.int16}[args.dual]
    state = torch.zeros((len(shape),) + shape, dtype=dt, device="cuda")
    times = []
    for _ in range(args.reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tvs.tv_prox(ctx, z, u, args.lam, args.iters, dual=args.dual, dual_state=state)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / max(args.iters, 1))
    print(f"shape {shape} dual {args.dual}: {statistics.median(times) * 1e3:.2f} us per inner iteration "
          f"(incl. finalisation)")
    ctx.close()


def _ct(args, tvs, L):
    import torch
    N, na, nd = args.ct
    stream = torch.cuda.Stream()
    ctx = tvs.Context.__new__(tvs.Context)
    ctx._h = C.c_void_p()
    L.check(L.lib().tvs_create(C.byref(ctx._h), torch.cuda.current_device(), C.c_void_p(stream.cuda_stream)))
    ctx.device = torch.cuda.current_device()
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    x = torch.rand((N, N), device="cuda", generator=g)
    y = torch.rand((na, nd), device="cuda", generator=g)
    prob = tvs.Problem(ctx, y, 0.0, op="ct", shape=(N, N), n_angles=na, n_det=nd, pixel_size=1.0 / N,
                       det_spacing=1.0 / N)
    ax = torch.empty_like(y)
    aty = torch.empty_like(x)
    for name, src, dst, adj in (("projector", x, ax, False), ("backprojector", y, aty, True)):
        times = []
        for _ in range(args.reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tvs.tvs_op_apply(prob, src, dst, adjoint=adj)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        print(f"{name} {N}^2, {na} angles, {nd} bins: {statistics.median(times) * 1e3:.1f} us")
    prob.close()
    ctx.close()


def _step(args, tvs, L):
    import torch
    H, W = args.step
    stream = torch.cuda.Stream()
    ctx = tvs.Context.__new__(tvs.Context)
    ctx._h = C.c_void_p()
    L.check(L.lib().tvs_create(C.byref(ctx._h), torch.cuda.current_device(), C.c_void_p(stream.cuda_stream)))
    ctx.device = torch.cuda.current_device()
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    b = torch.rand((H, W), device="cuda", generator=g)
    prob = tvs.Problem(ctx, b, 0.02, op="blur", blur_sigma=2.0)
    per_it = []
    for _ in range(args.reps):
        _, tr = tvs.pgd_solve(prob, b.clone(), 1.0, args.iters, 0)
        per_it.append(tr.solve_ms / max(tr.iters_run, 1))
    print(f"blur step {H}x{W}: {statistics.median(per_it) * 1e3:.2f} us per outer iteration")
    prob.close()
    ctx.close()


if __name__ == "__main__":
    main()
