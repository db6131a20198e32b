"""Writes fstar_ct2d_512.json: the reference optimum F* of the 512 x 512 CT
workload, computed by the FP64 oracle only (its C transcription, oracle/tvo.c,
which the tests hold to the numpy oracle at 1e-12).

Problem (Eq. 5, Section 3.3): min_x 1/2 ||A x - b||^2 + alpha TV(x) with A the
parallel-beam projector in Joseph's discretisation (unit square, 720 angles on
[0, pi), 725 bins of pixel width), alpha = 0.5, and b = -log(max(I, 1) / 1e4) from
seeded Poisson counts I of mean 1e4 exp(-A u_true), u_true the seeded 10-ellipse
phantom stored as float32 (the values the GPU side receives), A u_true formed in
FP64 by the oracle, b stored as float32 as the GPU side stores it.  The counts are
drawn from the oracle's projection; the GPU side draws them from its own, and the
two differ in a handful of the 522 000 rays (the script reports how many differ
when the projection is only rounded to float32).

||A||^2 comes from the power method on A^T A; F* is the smallest objective of a
long implicit PDHG run (the paper's reference solver, Section 4.1: Algorithm 6 at
p = 1, sigma = tau = 0.99 / ||A||, 100 warm-started inner iterations per prox,
x_0 = 0, y_0 = 0), accepted when over the last `window` iterations the objective's
spread (max - min) is below `settle` times F (1e-7 by default, three orders of
magnitude below the 1e-4 relative gap it serves).  (FISTA with the same inexact
prox does not settle here: at alpha = 0.5 its prox step is large, and the
momentum carries the prox errors; its objective rose from 362.9 at 50 iterations
to 383.6 at 2000.)

Usage: python tests/golden/make_fstar_ct2d_512.py [--iters K] [--window M] [--settle S]
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "fstar_ct2d_512.json")


def main():
    from oracle import c, operators, power
    from synth.configs import CTConfig

    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=4000)
    ap.add_argument("--inner", type=int, default=100)
    ap.add_argument("--window", type=int, default=500)
    ap.add_argument("--settle", type=float, default=1e-7)
    ap.add_argument("--power-iters", type=int, default=100)
    args = ap.parse_args()

    cfg = CTConfig()
    geom = operators.ParallelBeam.unit_square(cfg.N, cfg.n_angles, cfg.n_det)
    truth = cfg.phantom().astype(np.float32).astype(np.float64)
    clean = c.joseph(truth, geom)
    counts = cfg.counts(clean)
    differ = int((counts != cfg.counts(clean.astype(np.float32).astype(np.float64))).sum())
    b = (-np.log(np.maximum(counts, 1.0) / cfg.photons)).astype(np.float32).astype(np.float64)
    t0 = time.time()
    L = power.power_method(lambda x: c.joseph(c.joseph(x, geom), geom, adjoint=True), (cfg.N, cfg.N),
                           args.power_iters)
    st = 0.99 / np.sqrt(L)
    out = c.ct_pdhg(b, cfg.alpha, st, st, args.iters, args.inner, geom)
    wall = time.time() - t0
    F = np.asarray(out["objective"])
    tail = F[-args.window:]
    spread = float((tail.max() - tail.min()) / tail.min())
    rec = {
        "workload": "ct2d_512",
        "f_star": float(F.min()),
        "norm_A_sq": float(L),
        "solver": f"implicit PDHG, sigma = tau = 0.99 / ||A||, {args.inner} inner FGP iterations per prox "
                  f"(warm start), {args.iters} iterations, from x_0 = 0, y_0 = 0",
        "settled": {"window": args.window, "relative_spread": spread, "threshold": args.settle,
                    "accepted": spread < args.settle},
        "objective_at": {str(k): float(F[k - 1]) for k in (50, 100, 200, 500, 1000, 2000, 3000, args.iters)
                         if k <= len(F)},
        "counts_differing_at_float32_projection": differ,
        "threads": c.threads(),
        "wall_s": wall,
        "command": "python tests/golden/make_fstar_ct2d_512.py "
                   f"--iters {args.iters} --window {args.window} --settle {args.settle}",
    }
    if not rec["settled"]["accepted"]:
        with open(OUT + ".rejected", "w") as f:
            json.dump(rec, f, indent=1)
        raise SystemExit(f"not settled: spread {spread:.3e} over the last {args.window} iterations")
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
