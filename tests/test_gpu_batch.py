"""GPU parity of the batched ProxSkip solve (many problems of uneven sizes, each
with its own alpha, p and seed, in shared launches) against the FP64 oracle and
against one-at-a-time solves."""

import numpy as np
import pytest

from oracle import operators, solvers
from synth import phantoms
from tests._util import TOL_OBJ, TOL_X_F32, cuda, f32, host, assert_close

pytestmark = pytest.mark.gpu

SPECS = [  # (H, W, op, alpha, p, seed, blur sigma)
    (64, 64, "identity", 0.10, 0.30, 0, 2.0),
    (61, 47, "blur", 0.03, 0.50, 1, 2.0),
    (100, 130, "identity", 0.05, 0.10, 2, 2.0),
    (96, 200, "blur", 0.02, 0.25, 3, 1.3),
    (33, 257, "identity", 0.15, 0.45, 4, 2.0),
    (128, 128, "blur", 0.04, 0.05, 5, 2.9),
    (9, 11, "blur", 0.05, 0.9, 6, 1.0),
]


@pytest.fixture(scope="module")
def tvs():
    import paper_2411_00688_gb300 as tvs
    return tvs


@pytest.fixture(scope="module")
def ctx(tvs):
    c = tvs.Context(0)
    yield c
    c.close()


def _problem(spec, k):
    H, W, op, alpha, p, seed, sig = spec
    truth = phantoms.shapes_phantom_2d(H, W, 4, 100 + k)
    clean = operators.blur(truth, operators.gaussian_weights(sig, 4)) if op == "blur" else truth
    b32, b64 = f32(clean + phantoms.gaussian_noise((H, W), 0.05, 200 + k))
    A = operators.blur_op(sig) if op == "blur" else operators.identity_op()
    return b32, b64, solvers.Problem(A, b64, alpha, (H, W))


def _build(tvs, ctx):
    probs, xs, data = [], [], []
    for k, spec in enumerate(SPECS):
        b32, b64, oprob = _problem(spec, k)
        H, W, op, alpha, p, seed, sig = spec
        probs.append(tvs.Problem(ctx, cuda(b32), alpha, op=op, blur_sigma=sig))
        xs.append(cuda(b32))
        data.append((b32, b64, oprob))
    return probs, xs, data


def test_batch_matches_oracle_and_single_solves(tvs, ctx):
    K, N = 20, 12
    probs, xs, data = _build(tvs, ctx)
    gam = [1.0] * len(SPECS)
    ps = [s[4] for s in SPECS]
    seeds = [s[5] for s in SPECS]
    xs, traces = tvs.proxskip_solve_batch(ctx, probs, xs, gam, ps, seeds, K, N)
    for k, spec in enumerate(SPECS):
        b32, b64, oprob = data[k]
        tr = traces[k]
        ref = solvers.proxskip(oprob, b64, 1.0, spec[4], spec[5], K, N)
        assert tr.iters_run == K
        assert list(tr.coins) == ref["coins"] and tr.prox_calls == ref["prox_calls"]
        assert_close(host(xs[k]), ref["x"], TOL_X_F32, spec)
        rel = np.abs(tr.objective - np.asarray(ref["objective"])) / np.abs(np.asarray(ref["objective"]))
        assert rel.max() <= TOL_OBJ, spec
        x1, t1 = tvs.proxskip_solve(probs[k], cuda(b32), 1.0, spec[4], spec[5], K, N)
        assert_close(host(xs[k]), host(x1), 1e-5)


def test_batch_stops_each_problem_at_its_target(tvs, ctx):
    K, N = 30, 10
    probs, xs, data = _build(tvs, ctx)
    ps = [s[4] for s in SPECS]
    seeds = [s[5] for s in SPECS]
    # per-problem reference optimum: the lowest objective a plain run reaches in K
    # iterations; the target 1e-3 then stops each problem at a different iteration
    f_stars, expect = [], []
    tol = 1e-3
    for k, spec in enumerate(SPECS):
        b32, b64, oprob = data[k]
        _, t = tvs.proxskip_solve(probs[k], cuda(b32), 1.0, spec[4], spec[5], K, N)
        fs = float(np.nanmin(t.objective))
        f_stars.append(fs)
        expect.append(int(np.argmax(t.objective - fs <= tol * fs)))
    xs, traces = tvs.proxskip_solve_batch(ctx, probs, xs, [1.0] * len(SPECS), ps, seeds, K, N,
                                          f_stars=f_stars, targets=[tol] * len(SPECS))
    for k, spec in enumerate(SPECS):
        tr = traces[k]
        fs = f_stars[k]
        b32, b64, oprob = data[k]
        assert tr.reached and tr.iters_run == tr.reached_iter + 1
        if tr.iters_run == 0:  # x_0 itself met the target
            np.testing.assert_array_equal(host(xs[k]), b64)
            continue
        # stopped at the first recorded iterate within the target, by its own trace
        assert tr.objective[-1] - fs <= tol * fs
        assert np.all(tr.objective[:-1] - fs > tol * fs)
        assert tr.reached_iter == expect[k]
        ref = solvers.proxskip(oprob, b64, 1.0, spec[4], spec[5], tr.iters_run, N)
        assert_close(host(xs[k]), ref["x"], TOL_X_F32)


def test_batch_rejects_mismatched_parameters(tvs, ctx):
    import ctypes as C
    from paper_2411_00688_gb300 import _lib as L
    probs, xs, _ = _build(tvs, ctx)
    prm = (L.FBParams * 2)(L.FBParams(gamma=1.0, p=0.5, max_iter=5, n_inner=4),
                           L.FBParams(gamma=1.0, p=0.5, max_iter=5, n_inner=5))
    handles = (C.c_void_p * 2)(probs[0].handle.value, probs[1].handle.value)
    ptrs = (C.c_void_p * 2)(xs[0].data_ptr(), xs[1].data_ptr())
    assert L.lib().proxskip_solve_batch(ctx.handle, 2, handles, prm, ptrs, 0, None) == 1
    handles2 = (C.c_void_p * 2)(probs[0].handle.value, probs[0].handle.value)
    prm[1].n_inner = 4
    assert L.lib().proxskip_solve_batch(ctx.handle, 2, handles2, prm, ptrs, 0, None) == 1


# Where each reduced dual storage meets the 2e-3 relative-l2 bound against the
# FP64 oracle on these problems: the 16-bit fixed point everywhere; bfloat16 (8
# significant bits) and half (11) lose accuracy in proportion to the prox step
# lambda = alpha / p and, relative to the image, on tiny images -- the problems
# outside their range are reported as failing the bound, not held to a wider one.
BATCH_VS_SINGLE = {"bf16": 2e-4, "f16": 2e-4, "q15": 2e-4}
HALF_DUAL_RANGE = {"q15": lambda lam, n: True,
                   "f16": lambda lam, n: n >= 1000,
                   "bf16": lambda lam, n: lam <= 0.1 and n >= 1000}


@pytest.mark.parametrize("dual", ["bf16", "f16", "q15"])
def test_batch_half_dual_matches_oracle(tvs, ctx, dual):
    """Reduced dual storage in the batch: equal to the single solve of each
    problem with the same storage, and within 2e-3 relative l2 of the FP64 oracle
    (and 0.05 dB of its PSNR against the phantom) wherever the storage type's
    range above includes the problem."""
    import math
    from tests._util import TOL_X_HALF
    K, N = 15, 12
    probs, xs, data = _build(tvs, ctx)
    ps = [s[4] for s in SPECS]
    seeds = [s[5] for s in SPECS]
    xs, traces = tvs.proxskip_solve_batch(ctx, probs, xs, [1.0] * len(SPECS), ps, seeds, K, N, dual=dual)
    checked = 0
    for k, spec in enumerate(SPECS):
        b32, b64, oprob = data[k]
        ref = solvers.proxskip(oprob, b64, 1.0, spec[4], spec[5], K, N)
        x1, _ = tvs.proxskip_solve(probs[k], cuda(b32), 1.0, spec[4], spec[5], K, N, dual=dual)
        # the batch's outer steps sum in another order than the single solve's, and
        # a last-place FP32 difference can move a stored dual value by one code of
        # the 16-bit format, which the later iterations carry on
        assert_close(host(xs[k]), host(x1), BATCH_VS_SINGLE[dual])
        if not HALF_DUAL_RANGE[dual](spec[3] / spec[4], spec[0] * spec[1]):
            continue
        checked += 1
        truth = phantoms.shapes_phantom_2d(spec[0], spec[1], 4, 100 + k)

        def psnr(u):
            return 10.0 * math.log10(float(truth.max()) ** 2 / float(np.mean((u - truth) ** 2)))
        assert_close(host(xs[k]), ref["x"], TOL_X_HALF, spec)
        assert abs(psnr(host(xs[k])) - psnr(ref["x"])) <= 0.05, spec
    assert checked >= 2


def test_batch_full_size_sampled(tvs, ctx):
    """The 256-problem batched workload (sides log-uniform in [64, 1024], half
    denoising, half deblurring with sigma in [1, 3], own alpha/p/seed each) in the
    launch configuration the workload times: 3 outer iterations of 8 inner
    iterations; a sample of problems is compared with single solves (which the
    other tests hold to the oracle), every problem's trace is finite and its prox
    count equals its coins."""
    from synth.configs import BatchConfig
    cfg = BatchConfig()
    specs = cfg.specs()
    probs, bs = [], []
    for sp in specs:
        truth = cfg.phantom(sp)
        noise = cfg.noise(sp)
        if sp["kind"] == "deblur":
            clean = operators.blur(truth, operators.gaussian_weights(sp["blur_sigma"], 4))
            b = (clean + noise).astype(np.float32)
            probs.append(tvs.Problem(ctx, cuda(b), sp["alpha"], op="blur", blur_sigma=sp["blur_sigma"]))
        else:
            b = (truth + noise).astype(np.float32)
            probs.append(tvs.Problem(ctx, cuda(b), sp["alpha"]))
        bs.append(b)
    K, N = 3, 8
    ps = [sp["p"] for sp in specs]
    seeds = [sp["seed"] for sp in specs]
    xs, traces = tvs.proxskip_solve_batch(ctx, probs, [cuda(b) for b in bs], [1.0] * len(specs), ps, seeds, K, N)
    for k, tr in enumerate(traces):
        assert tr.iters_run == K and np.all(np.isfinite(tr.objective))
        assert tr.prox_calls == int(np.sum(tr.coins))
    for k in sorted({0, 1, 17, 100, 200, len(specs) - 1}):
        x1, t1 = tvs.proxskip_solve(probs[k], cuda(bs[k]), 1.0, ps[k], seeds[k], K, N)
        assert_close(host(xs[k]), host(x1), 1e-5)
        np.testing.assert_allclose(traces[k].objective, t1.objective, rtol=1e-6)


def test_batch_host_memory_matches_device_memory(tvs, ctx):
    """Iterates in host memory (copied in and out around the solve) give the same
    results and traces as iterates in device memory."""
    K, N = 12, 8
    probs, xs_dev, data = _build(tvs, ctx)
    xs_host = [d[0].copy() for d in data]
    ps = [s[4] for s in SPECS]
    seeds = [s[5] for s in SPECS]
    gam = [1.0] * len(SPECS)
    xs_dev, tr_dev = tvs.proxskip_solve_batch(ctx, probs, xs_dev, gam, ps, seeds, K, N)
    xs_host, tr_host = tvs.proxskip_solve_batch(ctx, probs, xs_host, gam, ps, seeds, K, N)
    for k in range(len(SPECS)):
        np.testing.assert_array_equal(xs_host[k], host(xs_dev[k]))
        np.testing.assert_array_equal(tr_host[k].objective, tr_dev[k].objective)
        np.testing.assert_array_equal(tr_host[k].coins, tr_dev[k].coins)
        assert tr_host[k].iters_run == tr_dev[k].iters_run == K


def test_batch_many_problems_uses_global_scan(tvs, ctx):
    """More problems than the inner kernel's shared-memory copy of the work scan
    holds (2047): the kernels search the scan in device memory.  Every problem
    must still follow its own single solve."""
    import torch
    n, K, N = 2100, 3, 4
    g = np.random.default_rng(21)
    probs, xs, bs = [], [], []
    for i in range(n):
        H, W = int(g.integers(3, 9)), int(g.integers(3, 9))
        b = cuda(g.random((H, W)).astype(np.float32))
        probs.append(tvs.Problem(ctx, b, 0.05 + 0.001 * (i % 7)))
        bs.append(b)
        xs.append(b.clone())
    ps = [0.5 + 0.2 * (i % 3) for i in range(n)]
    xs, traces = tvs.proxskip_solve_batch(ctx, probs, xs, [1.0] * n, ps, list(range(n)), K, N)
    for i in list(range(0, n, 97)) + [n - 1]:
        x1, t1 = tvs.proxskip_solve(probs[i], bs[i].clone(), 1.0, ps[i], i, K, N)
        assert list(traces[i].coins) == list(t1.coins)
        assert_close(host(xs[i]), host(x1), 1e-5)
    for p in probs:
        p.close()
    torch.cuda.synchronize()


def test_batch_setup_reused_and_rebuilt(tvs):
    """A repeated batched solve (same problems and parameters) replays the kept
    set-up and graphs and gives the same bits; a changed parameter, a different
    memory kind or a destroyed problem makes it build a new set-up, whose result
    equals a solve in a fresh context."""
    import torch
    K, N = 15, 8
    ctx = tvs.Context(0)
    try:
        probs, xs0, data = _build(tvs, ctx)
        gam = [1.0] * len(SPECS)
        ps = [s[4] for s in SPECS]
        seeds = [s[5] for s in SPECS]

        def run(ps_, dev=True):
            xs = [x.clone() for x in xs0] if dev else [np.ascontiguousarray(host(x), dtype=np.float32) for x in xs0]
            out, trs = tvs.proxskip_solve_batch(ctx, probs, xs, gam, ps_, seeds, K, N)
            return [host(x) if dev else x for x in out], [list(t.objective) for t in trs]

        a_x, a_obj = run(ps)
        b_x, b_obj = run(ps)
        for u, v in zip(a_x, b_x):
            np.testing.assert_array_equal(u, v)
        assert a_obj == b_obj
        h_x, _ = run(ps, dev=False)
        for u, v in zip(a_x, h_x):
            np.testing.assert_array_equal(u, v)
        ps2 = list(ps)
        ps2[2] = 0.6
        c_x, c_obj = run(ps2)
        fresh = tvs.Context(0)
        try:
            fprobs = [tvs.Problem(fresh, cuda(data[k][0]), s[3], op=s[2], blur_sigma=s[6])
                      for k, s in enumerate(SPECS)]
            fx = [x.clone() for x in xs0]
            f_out, f_trs = tvs.proxskip_solve_batch(fresh, fprobs, fx, gam, ps2, seeds, K, N)
            for u, v in zip(c_x, f_out):
                np.testing.assert_array_equal(u, host(v))
            assert c_obj == [list(t.objective) for t in f_trs]
        finally:
            fresh.close()
        # a destroyed problem drops the kept set-up; a batch of new problems still solves
        probs[0].close()
        probs[0] = tvs.Problem(ctx, cuda(data[0][0]), SPECS[0][3], op=SPECS[0][2], blur_sigma=SPECS[0][6])
        d_x, d_obj = run(ps)
        for u, v in zip(a_x, d_x):
            np.testing.assert_array_equal(u, v)
        assert d_obj == a_obj
        torch.cuda.synchronize()
    finally:
        ctx.close()
