"""A problem keeps the CUDA graphs of its last solve of each solver family and
replays them when the next solve bakes in the same values.  Whatever the cache
does, every solve must compute what a solve on a fresh problem computes: repeated
solves, solves whose parameters change in between (step, probability, inner
count, dual storage, target, a reference solution set and removed, a trace that
grows), and the primal-dual solvers the same way."""

import math

import numpy as np
import pytest

from oracle import operators
from synth import phantoms
from tests._util import cuda, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tvs():
    import paper_2411_00688_gb300 as tvs
    return tvs


@pytest.fixture(scope="module")
def ctx(tvs):
    c = tvs.Context(0)
    yield c
    c.close()


def _b(shape=(40, 52), seed=3):
    truth = phantoms.shapes_phantom_2d(shape[0], shape[1], 5, seed)
    clean = operators.blur(truth, operators.gaussian_weights(2.0, 4))
    return (clean + phantoms.gaussian_noise(shape, 0.01, seed + 1)).astype(np.float32)


def _fresh(tvs, ctx, b, fn):
    prob = tvs.Problem(ctx, cuda(b), 0.03, op="blur", blur_sigma=2.0)
    try:
        x, tr = fn(prob, cuda(b))
        return host(x), tr
    finally:
        prob.close()


RUNS = [
    ("proxskip", dict(gamma=1.0, p=0.4, seed=2, K=12, N=7)),
    ("proxskip", dict(gamma=1.0, p=0.4, seed=2, K=12, N=7)),          # same key: replay
    ("proxskip", dict(gamma=0.8, p=0.4, seed=2, K=12, N=7)),          # step changed
    ("proxskip", dict(gamma=0.8, p=0.3, seed=5, K=12, N=7)),          # probability and seed
    ("proxskip", dict(gamma=0.8, p=0.3, seed=5, K=30, N=9)),          # longer trace, inner count
    ("pgd", dict(gamma=1.0, K=10, N=7)),
    ("fista", dict(gamma=1.0, K=10, N=7)),
    ("proxskip", dict(gamma=1.0, p=0.4, seed=2, K=12, N=7, dual="q15")),
    ("proxskip", dict(gamma=1.0, p=0.4, seed=2, K=12, N=7)),
]


def _call(tvs, kind, prm, prob, x):
    kw = {"dual": prm.get("dual", "f32")}
    if kind == "proxskip":
        return tvs.proxskip_solve(prob, x, prm["gamma"], prm["p"], prm["seed"], prm["K"], prm["N"], **kw)
    fn = tvs.pgd_solve if kind == "pgd" else tvs.fista_solve
    return fn(prob, x, prm["gamma"], prm["K"], prm["N"], **kw)


def test_repeated_forward_backward_solves_equal_fresh_solves(tvs, ctx):
    b = _b()
    prob = tvs.Problem(ctx, cuda(b), 0.03, op="blur", blur_sigma=2.0)
    try:
        for kind, prm in RUNS:
            x, tr = _call(tvs, kind, prm, prob, cuda(b))
            ref, rtr = _fresh(tvs, ctx, b, lambda pr, x0: _call(tvs, kind, prm, pr, x0))
            np.testing.assert_array_equal(host(x), ref)
            np.testing.assert_array_equal(tr.objective, rtr.objective)
            assert list(tr.coins) == list(rtr.coins)
    finally:
        prob.close()


def test_reference_and_target_changes_are_seen(tvs, ctx):
    """Setting or removing a reference solution, or changing the stopping target,
    changes what the captured iterations record: the next solve must see it."""
    b = _b(seed=9)
    prob = tvs.Problem(ctx, cuda(b), 0.03, op="blur", blur_sigma=2.0)
    try:
        x1, t1 = tvs.proxskip_solve(prob, cuda(b), 1.0, 0.5, 1, 15, 6)
        assert np.all(np.isnan(t1.rel_dist))
        prob.set_reference(cuda(host(x1).astype(np.float32)))
        _, t2 = tvs.proxskip_solve(prob, cuda(b), 1.0, 0.5, 1, 15, 6)
        assert np.all(np.isfinite(t2.rel_dist)) and t2.rel_dist[-1] == 0.0
        f_end = float(t2.objective[-1])
        _, t3 = tvs.proxskip_solve(prob, cuda(b), 1.0, 0.5, 1, 15, 6, f_star=f_end * (1 - 1e-3), target=1e-2)
        assert t3.reached and t3.reached_iter >= 0
        prob.set_reference(None)
        _, t4 = tvs.proxskip_solve(prob, cuda(b), 1.0, 0.5, 1, 15, 6)
        assert np.all(np.isnan(t4.rel_dist)) and t4.iters_run == 15
        np.testing.assert_array_equal(t4.objective, t1.objective)
    finally:
        prob.close()


@pytest.mark.parametrize("solver", ["pdhg", "pdhgskip", "pdhgskip1"])
def test_repeated_primal_dual_solves_equal_fresh_solves(tvs, ctx, solver):
    b = _b((36, 36), seed=11)
    fn = getattr(tvs, f"{solver}_solve")

    def run(prob, x0, sigma):
        y0 = cuda(np.zeros_like(b))
        args = (prob, x0, y0, sigma, 0.9 / sigma)
        if solver != "pdhg":
            args = args + (0.4, 3)
        x, y, tr = fn(*args, 10, 6)
        return x, tr

    prob = tvs.Problem(ctx, cuda(b), 0.03, op="blur", blur_sigma=2.0)
    try:
        for sigma in (0.9, 0.9, 0.6, 0.9):
            x, tr = run(prob, cuda(b), sigma)
            ref, rtr = _fresh(tvs, ctx, b, lambda pr, x0: run(pr, x0, sigma))
            np.testing.assert_array_equal(host(x), ref)
            np.testing.assert_array_equal(tr.objective, rtr.objective)
    finally:
        prob.close()
