"""GPU parity of explicit, diagonally preconditioned PDHG (the explicit formulation
of Section 3.2, the paper's reference-solution solver) against the FP64 oracle:
every iterate component within 1e-4 relative l2, every recorded objective within
1e-6 relative; solving in pieces reproduces one long solve exactly."""

import numpy as np
import pytest

from oracle import operators, solvers
from synth import phantoms
from tests._util import TOL_OBJ, TOL_X_F32, cuda, f32, host, assert_close

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


def _case(tvs, ctx, op, shape, alpha, nonneg=False, seed=5):
    H, W = shape
    if op == "ct":
        na, nd = 24, 2 * W + 3
        geom = operators.ParallelBeam.unit_square(W, na, nd)
        truth = phantoms.ellipses_phantom_2d(W, 4, seed, intensity=(0.0, 0.5))
        clean = operators.joseph_forward(truth, geom)
        A = operators.ct_op(geom)
        b32, b64 = f32(clean + phantoms.gaussian_noise(clean.shape, 0.002, seed + 1))
        prob = tvs.Problem(ctx, cuda(b32), alpha, op="ct", shape=shape, n_angles=na, n_det=nd,
                           pixel_size=1.0 / W, det_spacing=1.0 / W, nonneg=nonneg)
        x0 = np.zeros(shape, dtype=np.float32)
    else:
        truth = phantoms.shapes_phantom_2d(H, W, 5, seed)
        if op == "blur":
            A = operators.blur_op(1.5)
            clean = A.forward(truth)
        else:
            A = operators.identity_op()
            clean = truth
        b32, b64 = f32(clean + phantoms.gaussian_noise(shape, 0.05, seed + 1))
        prob = tvs.Problem(ctx, cuda(b32), alpha, op=op, blur_sigma=1.5, nonneg=nonneg)
        x0 = b32.copy()
    oprob = solvers.Problem(A, b64, alpha, shape, nonneg)
    return prob, oprob, x0, b32


def _run(tvs, prob, x0, b32, K, **kw):
    x = cuda(x0)
    y = cuda(np.zeros(b32.shape, dtype=np.float32))
    q = cuda(np.zeros((2,) + x0.shape, dtype=np.float32))
    x, y, q, tr = tvs.pdhg_explicit_solve(prob, x, y, q, K, **kw)
    return host(x), host(y), host(q), tr


@pytest.mark.parametrize("op,shape,alpha,nonneg", [
    ("identity", (37, 53), 0.1, False),
    ("identity", (1, 17), 0.2, False),
    ("blur", (70, 45), 0.03, False),
    ("blur", (64, 64), 0.03, True),
    ("ct", (40, 40), 0.002, False),
    ("ct", (33, 33), 0.002, True),
])
def test_explicit_pdhg_matches_oracle(tvs, ctx, op, shape, alpha, nonneg):
    K = 60
    prob, oprob, x0, b32 = _case(tvs, ctx, op, shape, alpha, nonneg)
    x, y, q, tr = _run(tvs, prob, x0, b32, K)
    ref = solvers.pdhg_explicit(oprob, x0.astype(np.float64), K=K)
    assert tr.iters_run == K and tr.prox_calls == K
    assert_close(x, ref["x"], TOL_X_F32)
    assert_close(y, ref["y"], TOL_X_F32)
    assert_close(q, ref["q"], TOL_X_F32)
    obj = np.asarray(ref["objective"])
    assert (np.abs(tr.objective - obj) / np.abs(obj)).max() <= TOL_OBJ
    if nonneg:
        assert x.min() >= 0.0
    assert np.sqrt((q * q).sum(axis=0)).max() <= alpha * (1 + 1e-6)


def test_explicit_pdhg_steps_scale(tvs, ctx):
    """sigma and tau scale the preconditioned steps; sigma tau > 1 is rejected."""
    prob, oprob, x0, b32 = _case(tvs, ctx, "blur", (48, 40), 0.03)
    x, y, q, tr = _run(tvs, prob, x0, b32, 30, sigma=2.0, tau=0.5)
    ref = solvers.pdhg_explicit(oprob, x0.astype(np.float64), K=30, sigma=2.0, tau=0.5)
    assert_close(x, ref["x"], TOL_X_F32)
    assert_close(q, ref["q"], TOL_X_F32)
    from paper_2411_00688_gb300 import TVSError
    with pytest.raises(TVSError):
        _run(tvs, prob, x0, b32, 5, sigma=2.0, tau=0.6)


def test_explicit_pdhg_in_pieces_equals_one_solve(tvs, ctx):
    prob, oprob, x0, b32 = _case(tvs, ctx, "ct", (32, 32), 0.002, seed=9)
    x, y, q, tr = _run(tvs, prob, x0, b32, 40)
    xa = cuda(x0)
    ya = cuda(np.zeros(b32.shape, dtype=np.float32))
    qa = cuda(np.zeros((2, 32, 32), dtype=np.float32))
    xa, ya, qa, t1 = tvs.pdhg_explicit_solve(prob, xa, ya, qa, 25)
    xa, ya, qa, t2 = tvs.pdhg_explicit_solve(prob, xa, ya, qa, 15)
    np.testing.assert_array_equal(host(xa), x)
    np.testing.assert_array_equal(host(ya), y)
    np.testing.assert_array_equal(host(qa), q)
    np.testing.assert_array_equal(np.concatenate([t1.objective, t2.objective]), tr.objective)


def test_explicit_pdhg_host_memory_and_no_q(tvs, ctx):
    prob, oprob, x0, b32 = _case(tvs, ctx, "identity", (50, 70), 0.08)
    xd, yd, qd, td = _run(tvs, prob, x0, b32, 20)
    xh = x0.copy()
    yh = np.zeros(b32.shape, dtype=np.float32)
    xh, yh, _, th = tvs.pdhg_explicit_solve(prob, xh, yh, None, 20)
    np.testing.assert_array_equal(xh, xd)
    np.testing.assert_array_equal(yh, yd)
    np.testing.assert_array_equal(th.objective, td.objective)


def test_explicit_pdhg_alpha_zero_is_least_squares(tvs, ctx):
    """alpha = 0: q stays 0 and x tends to the least-squares solution (b for A = I)."""
    prob, oprob, x0, b32 = _case(tvs, ctx, "identity", (20, 30), 0.0)
    x, y, q, tr = _run(tvs, prob, np.zeros_like(x0), b32, 200)
    assert np.all(q == 0.0)
    assert_close(x, b32.astype(np.float64), 1e-5)


def test_explicit_pdhg_stops_at_target(tvs, ctx):
    prob, oprob, x0, b32 = _case(tvs, ctx, "blur", (64, 48), 0.03)
    _, _, _, ref = _run(tvs, prob, x0, b32, 400)
    f_star = float(np.nanmin(ref.objective))
    target = 1e-3
    k_expect = int(np.argmax(ref.objective - f_star <= target * f_star))
    _, _, _, tr = _run(tvs, prob, x0, b32, 400, f_star=f_star, target=target)
    assert tr.reached and tr.reached_iter == k_expect
    assert tr.iters_run < 400
