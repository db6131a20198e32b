"""GPU parity of the outer solvers (PGD, FISTA, ProxSkip, PDHG, PDHGSkip-2)
against the FP64 oracle: same seeded inputs, same coin schedule, final iterate
within 1e-4 relative l2 and every recorded objective within 1e-6 relative."""

import math

import numpy as np
import pytest

from oracle import coin, operators, solvers
from oracle.power import power_method
from synth import configs, phantoms
from tests._util import TOL_OBJ, TOL_X_F32, TOL_X_HALF, cuda, f32, host, assert_close

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


def _data(shape, op, seed, noise):
    truth = phantoms.shapes_phantom_2d(shape[0], shape[1], 6, seed)
    if op == "blur":
        clean = operators.blur(truth, operators.gaussian_weights(2.0, 4))
    else:
        clean = truth
    return f32(clean + phantoms.gaussian_noise(shape, noise, seed + 1))


def _check(trace, ref, x_gpu, tol_x=TOL_X_F32):
    assert list(trace.coins) == list(ref["coins"])
    assert trace.prox_calls == ref["prox_calls"]
    assert_close(x_gpu, ref["x"], tol_x)
    obj = np.asarray(ref["objective"])
    rel = np.abs(trace.objective - obj) / np.abs(obj)
    assert rel.max() <= TOL_OBJ, rel.max()


@pytest.mark.parametrize("op,shape", [("identity", (64, 80)), ("blur", (61, 47)), ("blur", (128, 128))])
@pytest.mark.parametrize("solver", ["pgd", "proxskip", "fista"])
def test_fb_solvers_small(tvs, ctx, op, shape, solver):
    b32, b64 = _data(shape, op, 11, 0.05)
    alpha, gamma, p, seed, K, N = 0.04, 1.0, 0.3, 7, 30, 20
    prob = tvs.Problem(ctx, cuda(b32), alpha, op=op, blur_sigma=2.0)
    A = operators.identity_op() if op == "identity" else operators.blur_op(2.0)
    oprob = solvers.Problem(A, b64, alpha, shape)
    x = cuda(b32)
    if solver == "pgd":
        x, tr = tvs.pgd_solve(prob, x, gamma, K, N)
        ref = solvers.pgd(oprob, b64, gamma, K, N)
    elif solver == "fista":
        x, tr = tvs.fista_solve(prob, x, gamma, K, N)
        ref = solvers.fista(oprob, b64, gamma, K, N)
    else:
        x, tr = tvs.proxskip_solve(prob, x, gamma, p, seed, K, N)
        ref = solvers.proxskip(oprob, b64, gamma, p, seed, K, N)
    _check(tr, ref, host(x))


def test_proxskip_3d_small(tvs, ctx):
    g = np.random.default_rng(3)
    shape = (12, 20, 33)
    b32, b64 = f32((g.random(shape) > 0.5) * 1.0 + 0.1 * g.standard_normal(shape))
    prob = tvs.Problem(ctx, cuda(b32), 0.08)
    x, tr = tvs.proxskip_solve(prob, cuda(b32), 1.0, 0.4, 3, 15, 10)
    ref = solvers.proxskip(solvers.Problem(operators.identity_op(), b64, 0.08, shape), b64, 1.0, 0.4, 3, 15, 10)
    _check(tr, ref, host(x))


def test_proxskip_nonneg_and_host_memory(tvs, ctx):
    """Host (numpy) buffers go through the same path; the non-negativity constraint."""
    b32, b64 = _data((40, 52), "blur", 21, 0.05)
    b32 = b32 - np.float32(0.2)
    b64 = b32.astype(np.float64)
    prob = tvs.Problem(ctx, b32, 0.03, op="blur", blur_sigma=2.0, nonneg=True)
    x = b32.copy()
    x, tr = tvs.proxskip_solve(prob, x, 1.0, 0.5, 4, 20, 15)
    ref = solvers.proxskip(solvers.Problem(operators.blur_op(2.0), b64, 0.03, (40, 52), nonneg=True),
                           b64, 1.0, 0.5, 4, 20, 15)
    _check(tr, ref, x.astype(np.float64))


def _psnr(u, truth):
    """10 log10(max(u_true)^2 / MSE) against the ground-truth phantom."""
    return 10.0 * math.log10(float(truth.max()) ** 2 / float(np.mean((u - truth) ** 2)))


@pytest.mark.parametrize("dual", ["bf16", "f16", "q15"])
def test_proxskip_half_dual(tvs, ctx, dual):
    """BF16/FP16 dual storage: final iterate within 2e-3 relative l2 of the FP64
    oracle and its PSNR against the phantom within 0.05 dB of the oracle's."""
    b32, b64 = _data((96, 96), "blur", 31, 0.02)
    truth = phantoms.shapes_phantom_2d(96, 96, 6, 31)
    prob = tvs.Problem(ctx, cuda(b32), 0.03, op="blur", blur_sigma=2.0)
    x, tr = tvs.proxskip_solve(prob, cuda(b32), 1.0, 0.3, 2, 25, 20, dual=dual)
    ref = solvers.proxskip(solvers.Problem(operators.blur_op(2.0), b64, 0.03, (96, 96)), b64, 1.0, 0.3, 2, 25, 20)
    assert_close(host(x), ref["x"], TOL_X_HALF)
    assert abs(_psnr(host(x), truth) - _psnr(ref["x"], truth)) <= 0.05


@pytest.mark.parametrize("op,alpha,p", [("blur", 0.2, 0.05), ("blur", 0.2, 0.1), ("identity", 0.1, 0.3),
                                        ("identity", 0.2, 0.05)])
def test_proxskip_q15_dual_large_lambda(tvs, ctx, op, alpha, p):
    """16-bit fixed-point dual at large prox steps (lambda = alpha / p up to 4, the
    top of the batched workload's range): final iterate within 2e-3 relative l2 of
    the FP64 oracle and PSNR within 0.05 dB of the oracle's."""
    from oracle import coin
    shape = (100, 140)
    b32, b64 = _data(shape, op, 31, 0.01 if op == "blur" else 0.1)
    truth = phantoms.shapes_phantom_2d(shape[0], shape[1], 6, 31)
    seed = next(s for s in range(100) if sum(coin.schedule(s, p, 25)) >= 3)
    prob = tvs.Problem(ctx, cuda(b32), alpha, op=op, blur_sigma=2.0)
    x, tr = tvs.proxskip_solve(prob, cuda(b32), 1.0, p, seed, 25, 20, dual="q15")
    A = operators.blur_op(2.0) if op == "blur" else operators.identity_op()
    ref = solvers.proxskip(solvers.Problem(A, b64, alpha, shape), b64, 1.0, p, seed, 25, 20)
    assert tr.prox_calls == ref["prox_calls"] >= 3
    assert_close(host(x), ref["x"], TOL_X_HALF)
    assert abs(_psnr(host(x), truth) - _psnr(ref["x"], truth)) <= 0.05


def test_proxskip_p1_equals_pgd_on_gpu(tvs, ctx):
    b32, _ = _data((50, 50), "blur", 41, 0.02)
    prob = tvs.Problem(ctx, cuda(b32), 0.03, op="blur", blur_sigma=2.0)
    x1, t1 = tvs.pgd_solve(prob, cuda(b32), 1.0, 12, 10)
    x2, t2 = tvs.proxskip_solve(prob, cuda(b32), 1.0, 1.0, 9, 12, 10)
    assert_close(host(x2), host(x1), 1e-5)
    assert t2.prox_calls == 12


def _ct_setup(N, na, nd, seed, alpha, nonneg=False):
    geom = operators.ParallelBeam.unit_square(N, na, nd)
    truth = phantoms.ellipses_phantom_2d(N, 5, seed, intensity=(0.0, 0.5))
    clean = operators.joseph_forward(truth, geom)
    b32, b64 = f32(clean + phantoms.gaussian_noise(clean.shape, 0.002, seed + 1))
    A = operators.ct_op(geom)
    L = power_method(lambda x: A.adjoint(A.forward(x)), (N, N), 100)
    return geom, b32, b64, solvers.Problem(A, b64, alpha, (N, N), nonneg), L


@pytest.mark.parametrize("skip", [False, True])
def test_pd_solvers_ct_small(tvs, ctx, skip):
    N, na, nd = 48, 60, 69
    geom, b32, b64, oprob, L = _ct_setup(N, na, nd, 51, 0.002)
    st = 0.99 / math.sqrt(L)
    prob = tvs.Problem(ctx, cuda(b32), 0.002, op="ct", shape=(N, N), n_angles=na, n_det=nd,
                       pixel_size=1.0 / N, det_spacing=1.0 / N)
    x0 = np.zeros((N, N), dtype=np.float32)
    y0 = np.zeros((na, nd), dtype=np.float32)
    K, NI, p, seed = 25, 15, 0.3, 6
    if skip:
        x, y, tr = tvs.pdhgskip_solve(prob, cuda(x0), cuda(y0), st, st, p, seed, K, NI)
        ref = solvers.pdhgskip2(oprob, x0.astype(np.float64), y0.astype(np.float64), st, st, p, seed, K, NI)
    else:
        x, y, tr = tvs.pdhg_solve(prob, cuda(x0), cuda(y0), st, st, K, NI)
        ref = solvers.pdhg(oprob, x0.astype(np.float64), y0.astype(np.float64), st, st, K, NI)
    _check(tr, ref, host(x))
    assert_close(host(y), ref["y"], TOL_X_F32)


@pytest.mark.parametrize("p", [1.0, 0.3])
def test_pdhgskip1_ct_small(tvs, ctx, p):
    N, na, nd = 48, 60, 69
    geom, b32, b64, oprob, L = _ct_setup(N, na, nd, 52, 0.002)
    st = 0.99 / math.sqrt(L)
    prob = tvs.Problem(ctx, cuda(b32), 0.002, op="ct", shape=(N, N), n_angles=na, n_det=nd,
                       pixel_size=1.0 / N, det_spacing=1.0 / N)
    x0 = np.zeros((N, N), dtype=np.float32)
    y0 = np.zeros((na, nd), dtype=np.float32)
    x, y, tr = tvs.pdhgskip1_solve(prob, cuda(x0), cuda(y0), st, st, p, 7, 25, 15)
    ref = solvers.pdhgskip1(oprob, x0.astype(np.float64), y0.astype(np.float64), st, st, p, 7, 25, 15)
    _check(tr, ref, host(x))
    assert_close(host(y), ref["y"], TOL_X_F32)


@pytest.mark.parametrize("op", ["identity", "blur"])
def test_pdhgskip1_image_operators(tvs, ctx, op):
    b32, b64 = _data((45, 58), op, 62, 0.05)
    A = operators.identity_op() if op == "identity" else operators.blur_op(2.0)
    oprob = solvers.Problem(A, b64, 0.04, (45, 58))
    prob = tvs.Problem(ctx, cuda(b32), 0.04, op=op, blur_sigma=2.0)
    y0 = np.zeros_like(b32)
    x, y, tr = tvs.pdhgskip1_solve(prob, cuda(b32), cuda(y0), 0.9, 0.9, 0.4, 8, 20, 12)
    ref = solvers.pdhgskip1(oprob, b64, y0.astype(np.float64), 0.9, 0.9, 0.4, 8, 20, 12)
    _check(tr, ref, host(x))


@pytest.mark.parametrize("op", ["identity", "blur"])
def test_pdhgskip_image_operators(tvs, ctx, op):
    b32, b64 = _data((45, 58), op, 61, 0.05)
    A = operators.identity_op() if op == "identity" else operators.blur_op(2.0)
    oprob = solvers.Problem(A, b64, 0.04, (45, 58))
    prob = tvs.Problem(ctx, cuda(b32), 0.04, op=op, blur_sigma=2.0)
    y0 = np.zeros_like(b32)
    x, y, tr = tvs.pdhgskip_solve(prob, cuda(b32), cuda(y0), 0.9, 0.9, 0.4, 8, 20, 12)
    ref = solvers.pdhgskip2(oprob, b64, y0.astype(np.float64), 0.9, 0.9, 0.4, 8, 20, 12)
    _check(tr, ref, host(x))


def test_ct_nonneg_proxskip(tvs, ctx):
    """ProxSkip on the CT operator with the non-negativity constraint."""
    N, na, nd = 32, 40, 47
    geom, b32, b64, oprob, L = _ct_setup(N, na, nd, 71, 0.002, nonneg=True)
    gamma = 1.0 / L
    prob = tvs.Problem(ctx, cuda(b32), 0.002, op="ct", shape=(N, N), n_angles=na, n_det=nd,
                       pixel_size=1.0 / N, det_spacing=1.0 / N, nonneg=True)
    x0 = np.zeros((N, N), dtype=np.float32)
    x, tr = tvs.proxskip_solve(prob, cuda(x0), gamma, 0.3, 5, 20, 10)
    ref = solvers.proxskip(oprob, x0.astype(np.float64), gamma, 0.3, 5, 20, 10)
    _check(tr, ref, host(x))


def test_deblur_full_size_prefix(tvs, ctx):
    """1024 x 1024 deblurring workload (9x9 Gaussian sigma 2, alpha 0.02, 50 inner
    iterations, p = 0.5) in the configuration the benchmark times: 4 outer iterations
    compared with the oracle."""
    cfg = configs.DeblurConfig()
    truth = cfg.phantom()
    w = operators.gaussian_weights(cfg.blur_sigma, cfg.blur_radius)
    b32, b64 = f32(operators.blur(truth, w) + cfg.noise())
    prob = tvs.Problem(ctx, cuda(b32), cfg.alpha, op="blur", blur_sigma=cfg.blur_sigma)
    K = 4
    x, tr = tvs.proxskip_solve(prob, cuda(b32), 1.0, 0.5, cfg.seed, K, cfg.n_inner)
    ref = solvers.proxskip(solvers.Problem(operators.blur_op(cfg.blur_sigma), b64, cfg.alpha, b64.shape),
                           b64, 1.0, 0.5, cfg.seed, K, cfg.n_inner)
    _check(tr, ref, host(x))


def test_pdhgskip_ct_full_size_prefix(tvs, ctx):
    """The CT workload at its full size -- 512^2 image, 720 angles x 725 bins,
    alpha 0.5, sigma = tau/4 with sigma tau ||A||^2 = 0.98 -- in the configuration
    the benchmark times: PDHGSkip-2 (p = 0.2, a seed whose first iterations evaluate
    the prox), 2 outer iterations of 10 inner iterations, every iterate compared
    whole with the oracle (its projector pair takes most of a minute here)."""
    from oracle import coin
    cfg = configs.CTConfig()
    N = cfg.N
    geom = operators.ParallelBeam.unit_square(N, cfg.n_angles, cfg.n_det)
    truth = cfg.phantom()
    clean = operators.joseph_forward(truth, geom)
    counts = cfg.counts(clean)
    b32, b64 = f32(-np.log(np.maximum(counts, 1.0) / cfg.photons))
    st = 0.99 / math.sqrt(1.3578)            # ||A||^2 of this geometry by the power method
    sg, ta = 0.5 * st, 2.0 * st
    p, K, NI = 0.2, 2, 10
    seed = next(s for s in range(100) if coin.schedule(s, p, K) == [1, 1])
    prob = tvs.Problem(ctx, cuda(b32), cfg.alpha, op="ct", shape=(N, N), n_angles=cfg.n_angles, n_det=cfg.n_det,
                       pixel_size=1.0 / N, det_spacing=1.0 / N)
    x0 = np.zeros((N, N), dtype=np.float32)
    y0 = np.zeros((cfg.n_angles, cfg.n_det), dtype=np.float32)
    x, y, tr = tvs.pdhgskip_solve(prob, cuda(x0), cuda(y0), sg, ta, p, seed, K, NI)
    oprob = solvers.Problem(operators.ct_op(geom), b64, cfg.alpha, (N, N))
    ref = solvers.pdhgskip2(oprob, x0.astype(np.float64), y0.astype(np.float64), sg, ta, p, seed, K, NI,
                            record=False)
    assert list(tr.coins) == [1, 1] and tr.prox_calls == 2
    assert_close(host(x), ref["x"], TOL_X_F32)
    assert_close(host(y), ref["y"], TOL_X_F32)
    prob.close()


def test_proxskip_3d_prefix_256(tvs, ctx):
    """3D denoising at 256^3 (60 ellipsoids on the volume's grid, noise 0.05, alpha
    0.05, p 0.1, 30 inner iterations as the 512^3 workload): 3 outer iterations with
    a seed whose coins evaluate the prox, compared whole with the oracle's C
    transcription (the numpy oracle would take minutes at this size)."""
    from oracle import c as oc
    from oracle import coin
    N, alpha, p, K, NI = 256, 0.05, 0.1, 3, 30
    vol = phantoms.ellipsoids_phantom_3d(N, 60, 4000) + phantoms.gaussian_noise((N,) * 3, 0.05, 4001,
                                                                                 dtype=np.float32)
    b32 = np.ascontiguousarray(vol.astype(np.float32))
    seed = next(s for s in range(1000) if coin.schedule(s, p, K) == [1, 0, 1])
    prob = tvs.Problem(ctx, cuda(b32), alpha)
    x, tr = tvs.proxskip_solve(prob, cuda(b32), 1.0, p, seed, K, NI)
    ref = oc.fb_solve("proxskip", b32.astype(np.float64), alpha, 1.0, K, NI, p=p, coins=coin.schedule(seed, p, K))
    assert list(tr.coins) == [1, 0, 1]
    assert_close(host(x), ref["x"], TOL_X_F32)
    obj = np.asarray(ref["objective"])
    assert (np.abs(tr.objective - obj) / np.abs(obj)).max() <= TOL_OBJ
    prob.close()


def test_denoise_full_size(tvs, ctx):
    """256 x 256 denoising workload (alpha 0.1, p 0.1, 100 inner iterations), 40 iterations."""
    cfg = configs.DenoiseConfig()
    b32, b64 = f32(cfg.phantom() + cfg.noise())
    prob = tvs.Problem(ctx, cuda(b32), cfg.alpha)
    K = 40
    x, tr = tvs.proxskip_solve(prob, cuda(b32), cfg.gamma, cfg.p, cfg.seed, K, cfg.n_inner)
    ref = solvers.proxskip(solvers.Problem(operators.identity_op(), b64, cfg.alpha, b64.shape), b64,
                           cfg.gamma, cfg.p, cfg.seed, K, cfg.n_inner)
    _check(tr, ref, host(x))


def test_solver_edge_cases(tvs, ctx):
    b32, b64 = _data((20, 24), "blur", 81, 0.02)
    prob = tvs.Problem(ctx, cuda(b32), 0.05, op="blur", blur_sigma=2.0)
    x, tr = tvs.proxskip_solve(prob, cuda(b32), 1.0, 0.5, 1, 0, 10)      # no iterations
    assert tr.iters_run == 0 and np.array_equal(host(x), b64)
    x, tr = tvs.proxskip_solve(prob, cuda(b32), 1.0, 0.5, 1, 6, 0)      # no inner iterations
    ref = solvers.proxskip(solvers.Problem(operators.blur_op(2.0), b64, 0.05, (20, 24)), b64, 1.0, 0.5, 1, 6, 0)
    _check(tr, ref, host(x))
    prob0 = tvs.Problem(ctx, cuda(b32), 0.0, op="blur", blur_sigma=2.0)  # alpha = 0: no prox
    x, tr = tvs.pgd_solve(prob0, cuda(b32), 1.0, 5, 10)
    ref = solvers.pgd(solvers.Problem(operators.blur_op(2.0), b64, 0.0, (20, 24)), b64, 1.0, 5, 10)
    _check(tr, ref, host(x))
    for bad in (0.0, 1.5, float("nan")):
        with pytest.raises(tvs.TVSError):
            tvs.proxskip_solve(prob, cuda(b32), 1.0, bad, 1, 5, 5)
    with pytest.raises(tvs.TVSError):
        tvs.pgd_solve(prob, cuda(b32), -1.0, 5, 5)


def test_target_stops_early(tvs, ctx):
    """With f* given, the solve stops within a few iterations after the gap target."""
    b32, b64 = _data((64, 64), "identity", 91, 0.1)
    prob = tvs.Problem(ctx, cuda(b32), 0.1)
    _, full = tvs.pgd_solve(prob, cuda(b32), 1.0, 200, 30)
    f_star = float(np.min(full.objective))
    x, tr = tvs.pgd_solve(prob, cuda(b32), 1.0, 200, 30, f_star=f_star, target=1e-3)
    assert tr.reached
    k = tr.reached_iter
    assert (tr.objective[k] - f_star) <= 1e-3 * f_star
    assert np.all(tr.objective[:k] - f_star > 1e-3 * f_star)
    assert tr.iters_run <= k + 1 + 10
    assert tr.time_to_target_s > 0


def test_resume_equals_uninterrupted_proxskip(tvs, ctx):
    """K iterations + a resumed run of K more (k0 = K) equals one run of 2K iterations."""
    b32, _ = _data((64, 80), "blur", 101, 0.02)
    prob = tvs.Problem(ctx, cuda(b32), 0.03, op="blur", blur_sigma=2.0)
    K = 12
    xa, ta = tvs.proxskip_solve(prob, cuda(b32), 1.0, 0.4, 17, 2 * K, 10)
    xb, tb = tvs.proxskip_solve(prob, cuda(b32), 1.0, 0.4, 17, K, 10)
    xc, tc = tvs.proxskip_solve(prob, xb, 1.0, 0.4, 17, K, 10, resume=True, k0=K)
    np.testing.assert_array_equal(host(xc), host(xa))
    assert list(tb.coins) + list(tc.coins) == list(ta.coins)
    np.testing.assert_allclose(np.concatenate([tb.objective, tc.objective]), ta.objective, rtol=1e-12)


def test_chunk_graphs_equal_single_iteration_graphs(tvs, ctx):
    """A solve of 13 iterations runs three four-iteration chunk graphs and one
    single-iteration graph; 13 resumed solves of one iteration each run only
    single-iteration graphs.  Both give the same iterates, bit for bit, for every
    solver family whose outer loop launches chunks (ProxSkip, PGD, PDHGSkip-2,
    PDHGSkip-1)."""
    b32, _ = _data((48, 56), "blur", 102, 0.02)
    prob = tvs.Problem(ctx, cuda(b32), 0.03, op="blur", blur_sigma=2.0)
    K, N = 13, 6
    xa, ta = tvs.proxskip_solve(prob, cuda(b32), 1.0, 0.4, 23, K, N)
    x = cuda(b32)
    coins = []
    for k in range(K):
        x, t = tvs.proxskip_solve(prob, x, 1.0, 0.4, 23, 1, N, resume=k > 0, k0=k)
        coins += list(t.coins)
    np.testing.assert_array_equal(host(x), host(xa))
    assert coins == list(ta.coins)
    # PGD (every coin 1) against PGD in pieces: the warm dual carries over as resume keeps it
    xa, _ = tvs.pgd_solve(prob, cuda(b32), 1.0, K, N)
    x = cuda(b32)
    for k in range(K):
        x, _ = tvs.pgd_solve(prob, x, 1.0, 1, N, resume=k > 0, k0=k)
    np.testing.assert_array_equal(host(x), host(xa))
    Nc, na, nd = 32, 40, 45
    geom, c32, c64, oprob, L = _ct_setup(Nc, na, nd, 56, 0.002)
    st = 0.99 / math.sqrt(L)
    cprob = tvs.Problem(ctx, cuda(c32), 0.002, op="ct", shape=(Nc, Nc), n_angles=na, n_det=nd,
                        pixel_size=1.0 / Nc, det_spacing=1.0 / Nc)
    z = np.zeros((Nc, Nc), dtype=np.float32)
    y0 = np.zeros((na, nd), dtype=np.float32)
    for fn in (tvs.pdhgskip_solve, tvs.pdhgskip1_solve):
        xa, ya, _ = fn(cprob, cuda(z), cuda(y0), st, st, 0.5, 4, K, N)
        x, y = cuda(z), cuda(y0)
        for k in range(K):
            x, y, _ = fn(cprob, x, y, st, st, 0.5, 4, 1, N, resume=k > 0, k0=k)
        np.testing.assert_array_equal(host(x), host(xa))
        np.testing.assert_array_equal(host(y), host(ya))


def test_resume_equals_uninterrupted_pdhgskip(tvs, ctx):
    N, na, nd = 40, 48, 57
    geom, b32, b64, oprob, L = _ct_setup(N, na, nd, 55, 0.002)
    st = 0.99 / math.sqrt(L)
    prob = tvs.Problem(ctx, cuda(b32), 0.002, op="ct", shape=(N, N), n_angles=na, n_det=nd,
                       pixel_size=1.0 / N, det_spacing=1.0 / N)
    z = np.zeros((N, N), dtype=np.float32)
    y0 = np.zeros((na, nd), dtype=np.float32)
    K = 10
    for fn in (tvs.pdhgskip_solve, tvs.pdhgskip1_solve):
        xa, ya, ta = fn(prob, cuda(z), cuda(y0), st, st, 0.3, 9, 2 * K, 8)
        xb, yb, tb = fn(prob, cuda(z), cuda(y0), st, st, 0.3, 9, K, 8)
        xc, yc, tc = fn(prob, xb, yb, st, st, 0.3, 9, K, 8, resume=True, k0=K)
        np.testing.assert_array_equal(host(xc), host(xa))
        np.testing.assert_array_equal(host(yc), host(ya))
        np.testing.assert_allclose(np.concatenate([tb.objective, tc.objective]), ta.objective, rtol=1e-12)


def test_resume_rejected_for_fista(tvs, ctx):
    b32, _ = _data((20, 20), "identity", 5, 0.05)
    prob = tvs.Problem(ctx, cuda(b32), 0.05)
    with pytest.raises(tvs.TVSError) as e:
        tvs.fista_solve(prob, cuda(b32), 1.0, 5, 5, resume=True, k0=5)
    assert e.value.status == 6


@pytest.mark.parametrize("solver", ["proxskip", "fista", "pdhgskip", "pdhgskip1"])
def test_reference_distance_trace_and_stop(tvs, ctx, solver):
    """With a reference u*, the trace records ||x_{k+1} - u*|| / ||u*|| (checked on
    the returned iterate) and target_rel_dist stops the solve at the first
    iterate within it."""
    b32, b64 = _data((48, 56), "blur", 111, 0.02)
    prob = tvs.Problem(ctx, cuda(b32), 0.03, op="blur", blur_sigma=2.0)
    ref = solvers.fista(solvers.Problem(operators.blur_op(2.0), b64, 0.03, (48, 56)), b64, 1.0, 150, 30,
                        record=False)["x"]
    u32, _ = f32(ref)
    prob.set_reference(cuda(u32))
    y0 = cuda(np.zeros_like(b32))

    def run(**kw):
        if solver == "proxskip":
            x, tr = tvs.proxskip_solve(prob, cuda(b32), 1.0, 0.5, 3, 40, 20, **kw)
        elif solver == "fista":
            x, tr = tvs.fista_solve(prob, cuda(b32), 1.0, 40, 20, **kw)
        elif solver == "pdhgskip":
            x, _, tr = tvs.pdhgskip_solve(prob, cuda(b32), y0.clone(), 0.9, 0.9, 0.5, 3, 40, 20, **kw)
        else:
            x, _, tr = tvs.pdhgskip1_solve(prob, cuda(b32), y0.clone(), 0.9, 0.9, 0.5, 3, 40, 20, **kw)
        return host(x), tr

    x, tr = run()
    assert np.all(np.isfinite(tr.rel_dist))
    d_last = np.linalg.norm(x - u32.astype(np.float64)) / np.linalg.norm(u32.astype(np.float64))
    assert abs(tr.rel_dist[-1] - d_last) <= 1e-5 * d_last
    target = float(np.quantile(tr.rel_dist, 0.5))
    x2, tr2 = run(target_dist=target)
    assert tr2.reached and tr2.rel_dist[tr2.reached_iter] <= target
    assert np.all(tr2.rel_dist[:tr2.reached_iter] > target)
    prob.set_reference(None)


@pytest.mark.parametrize("solver", ["pgd", "proxskip", "pdhg"])
def test_divergence_reported(tvs, ctx, solver):
    """A step far above 2/L makes the iteration diverge; the device reduction sees
    the non-finite objective, stops the solve and the call returns TVS_ENUMERIC."""
    b32, _ = _data((40, 40), "blur", 3, 0.05)
    prob = tvs.Problem(ctx, cuda(b32), 0.02, op="blur", blur_sigma=2.0)
    with pytest.raises(tvs.TVSError) as e:
        if solver == "pgd":
            tvs.pgd_solve(prob, cuda(b32), 200.0, 500, 5)
        elif solver == "proxskip":
            tvs.proxskip_solve(prob, cuda(b32), 200.0, 0.5, 1, 500, 5)
        else:
            tvs.pdhg_solve(prob, cuda(b32), cuda(np.zeros_like(b32)), 50.0, 50.0, 500, 5)
    assert e.value.status == 4
