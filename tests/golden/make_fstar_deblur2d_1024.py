"""Writes fstar_deblur2d_1024.json: the reference optimum F* of the 1024 x 1024
deblurring workload, computed by the FP64 oracle only (its C transcription,
oracle/tvo.c, which the tests hold to the numpy oracle at 1e-12).

Problem (Eq. 5): min_x 1/2 ||A x - b||^2 + alpha TV(x) with A the 9 x 9 Gaussian
blur of sigma 2 (half-sample symmetric boundary), alpha = 0.02, and
b = A u_true + noise, u_true the seeded 40-ellipse phantom and the seeded noise of
sigma 0.01 stored as float32 (the values the GPU side receives), A u_true formed
in FP64.

F* is the smallest objective of a long FISTA run (Algorithm 3, gamma = 1/||A||^2
= 1, 100 warm-started inner iterations per prox), the paper's way of making
reference solutions by running a solver far past the tolerance of interest
(Section 4.1).  It is accepted when the objective has settled: over the last
`window` iterations its spread (max - min) is below `settle` times F (1e-8 by
default, four orders of magnitude below the 1e-4 relative gap it serves).

Usage: python tests/golden/make_fstar_deblur2d_1024.py [--iters K] [--window M] [--settle S]
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

OUT = os.path.join(HERE, "fstar_deblur2d_1024.json")


def main():
    from oracle import c, operators
    from synth.configs import DeblurConfig

    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--inner", type=int, default=100)
    ap.add_argument("--window", type=int, default=500)
    ap.add_argument("--settle", type=float, default=1e-8)
    args = ap.parse_args()

    cfg = DeblurConfig()
    truth = cfg.phantom().astype(np.float32).astype(np.float64)
    noise = cfg.noise().astype(np.float32).astype(np.float64)
    w = operators.gaussian_weights(cfg.blur_sigma, cfg.blur_radius)
    b = c.blur(truth, w) + noise
    t0 = time.time()
    out = c.fb_solve("fista", b, cfg.alpha, 1.0, args.iters, args.inner, w=w)
    wall = time.time() - t0
    F = np.asarray(out["objective"])
    tail = F[-args.window:]
    spread = float((tail.max() - tail.min()) / tail.min())
    f_star = float(F.min())
    rec = {
        "workload": "deblur2d_1024",
        "f_star": f_star,
        "solver": f"FISTA, gamma 1, {args.inner} inner FGP iterations per prox (warm start), "
                  f"{args.iters} iterations, from x_0 = b",
        "settled": {"window": args.window, "relative_spread": spread, "threshold": args.settle,
                    "accepted": spread < args.settle},
        "objective_at": {str(k): float(F[k - 1]) for k in (50, 100, 200, 500, 1000, 2000, args.iters)
                         if k <= len(F)},
        "threads": c.threads(),
        "wall_s": wall,
        "command": "python tests/golden/make_fstar_deblur2d_1024.py "
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
