"""Pins of the oracle's outer solvers (Algorithms 2, 3, 4, 5, 6, implicit PDHG and
explicit, diagonally preconditioned PDHG).

* ProxSkip with p = 1 is PGD and PDHGSkip-2 with p = 1 is PDHG (the prox argument
  x^ - gamma h equals x - gamma grad f(x)): compared iterate for iterate against the
  separately written PGD / PDHG.
* After every executed prox (no constraint) h = alpha div p_N, since
  h + (p/gamma)(x+ - x^) = (p/gamma) lam div p_N with lam = (gamma/p) alpha.
* Between prox events h does not change.
* All solvers reach the closed-form two-pixel minimiser, and on a small deblurring
  problem PGD, FISTA and PDHG agree on the minimum.
* Explicit PDHG: its step sizes are the reciprocal row and column sums of the dense
  block matrix [A; D] and satisfy the norm bound of Pock and Chambolle's Lemma 2; it
  reaches the two-pixel minimiser, the optimality (KKT) conditions of Eq. 5, and the
  minimisers of the implicit solvers.
"""

import math

import numpy as np
import pytest

from oracle import coin, operators, solvers, tv


def _deblur_problem(n=12, seed=0, alpha=0.05, nonneg=False):
    g = np.random.default_rng(seed)
    truth = np.zeros((n, n))
    truth[2:7, 3:9] = 1.0
    truth[6:10, 1:5] = 0.5
    A = operators.blur_op(1.5)
    b = A.forward(truth) + 0.01 * g.standard_normal((n, n))
    return solvers.Problem(A, b, alpha, (n, n), nonneg)


def _denoise_problem(n=10, seed=1, alpha=0.1):
    g = np.random.default_rng(seed)
    truth = np.zeros((n, n))
    truth[3:8, 2:6] = 1.0
    b = truth + 0.1 * g.standard_normal((n, n))
    return solvers.Problem(operators.identity_op(), b, alpha, (n, n))


def _ct_problem(N=12, seed=2, alpha=0.02):
    geom = operators.ParallelBeam.unit_square(N, 16, 17)
    A = operators.ct_op(geom)
    g = np.random.default_rng(seed)
    truth = np.zeros((N, N))
    truth[3:9, 4:8] = 0.4
    b = A.forward(truth) + 0.001 * g.standard_normal((16, 17))
    return solvers.Problem(A, b, alpha, (N, N)), geom


@pytest.mark.parametrize("make", [_deblur_problem, _denoise_problem])
def test_proxskip_p1_equals_pgd(make):
    prob = make()
    a = solvers.pgd(prob, prob.b, 1.0, 25, 7)
    b = solvers.proxskip(prob, prob.b, 1.0, 1.0, 3, 25, 7)
    assert b["prox_calls"] == 25
    np.testing.assert_allclose(b["x"], a["x"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(b["objective"], a["objective"], rtol=1e-12)


def test_pdhgskip_p1_equals_pdhg():
    prob, geom = _ct_problem()
    L = 0.0
    # sigma = tau = 0.99/||A||
    from oracle.power import power_method
    L = power_method(lambda x: prob.A.adjoint(prob.A.forward(x)), prob.shape, 300)
    st = 0.99 / math.sqrt(L)
    y0 = np.zeros_like(prob.b)
    a = solvers.pdhg(prob, np.zeros(prob.shape), y0, st, st, 20, 6)
    b = solvers.pdhgskip2(prob, np.zeros(prob.shape), y0, st, st, 1.0, 5, 20, 6)
    np.testing.assert_allclose(b["x"], a["x"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(b["y"], a["y"], rtol=0, atol=1e-12)


def test_pdhgskip1_p1_equals_pdhg():
    """Algorithm 5 with p = 1 (omega = 0, every coin 1) is PDHG: x_{k+1} = prox(...) and
    K(x_{k+1} + x^_k) = K(2 x_{k+1} - x_k)."""
    prob, geom = _ct_problem()
    from oracle.power import power_method
    L = power_method(lambda x: prob.A.adjoint(prob.A.forward(x)), prob.shape, 300)
    st = 0.99 / math.sqrt(L)
    y0 = np.zeros_like(prob.b)
    a = solvers.pdhg(prob, np.zeros(prob.shape), y0, st, st, 20, 6)
    b = solvers.pdhgskip1(prob, np.zeros(prob.shape), y0, st, st, 1.0, 5, 20, 6)
    np.testing.assert_allclose(b["x"], a["x"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(b["y"], a["y"], rtol=0, atol=1e-12)


def test_pdhgskip1_skipped_iterations_keep_x():
    """With theta_k = 0 the primal iterate does not move (x^ = 0), only y does."""
    prob, _ = _ct_problem()
    p, seed = 0.3, 8
    sched = coin.schedule(seed, p, 12)
    xs = [solvers.pdhgskip1(prob, np.zeros(prob.shape), np.zeros_like(prob.b), 0.3, 0.3, p, seed, k, 5,
                            record=False)["x"] for k in range(1, 13)]
    for k in range(1, 12):
        if not sched[k]:
            np.testing.assert_array_equal(xs[k], xs[k - 1])


@pytest.mark.parametrize("p", [0.5, 0.2])
def test_proxskip_control_variate_identity(p):
    prob = _deblur_problem(seed=3)
    gamma = 1.0
    seen = []

    def check(k, x, h, dual):
        seen.append(k)
        np.testing.assert_allclose(h, prob.alpha * tv.div(dual), rtol=0, atol=1e-12)

    out = solvers.proxskip(prob, prob.b, gamma, p, 11, 40, 5, on_prox=check)
    assert len(seen) == out["prox_calls"] == sum(out["coins"]) > 0
    assert out["coins"] == coin.schedule(11, p, 40)


def test_pdhgskip_control_variate_identity():
    prob, _ = _ct_problem()
    seen = []

    def check(k, x, h, dual):
        seen.append(k)
        np.testing.assert_allclose(h, prob.alpha * tv.div(dual), rtol=0, atol=1e-12)

    out = solvers.pdhgskip2(prob, np.zeros(prob.shape), np.zeros_like(prob.b), 0.3, 0.3, 0.3, 4, 30, 5,
                            on_prox=check)
    assert len(seen) == out["prox_calls"] > 0


def test_h_constant_between_prox_events():
    prob = _denoise_problem()
    p, seed, K = 0.3, 21, 30
    sched = coin.schedule(seed, p, K)
    hs = []
    for k in range(1, K + 1):
        hs.append(solvers.proxskip(prob, prob.b, 1.0, p, seed, k, 4, record=False)["h"])
    for k in range(1, K):
        if not sched[k]:
            np.testing.assert_array_equal(hs[k], hs[k - 1])


def _two_pixel(b1, b2, alpha):
    if abs(b1 - b2) <= 2 * alpha:
        return np.array([[(b1 + b2) / 2] * 2])
    s = math.copysign(1.0, b2 - b1)
    return np.array([[b1 + s * alpha, b2 - s * alpha]])


@pytest.mark.parametrize("b1,b2,alpha", [(0.0, 1.0, 0.2), (0.4, 0.5, 0.1)])
def test_solvers_reach_two_pixel_minimiser(b1, b2, alpha):
    """A = I on a 1 x 2 image: the minimiser of Eq. 5 is the two-pixel TV prox of b."""
    b = np.array([[b1, b2]])
    prob = solvers.Problem(operators.identity_op(), b, alpha, (1, 2))
    expect = _two_pixel(b1, b2, alpha)
    x0 = np.zeros_like(b)
    outs = [
        solvers.pgd(prob, x0, 1.0, 30, 60)["x"],
        solvers.fista(prob, x0, 0.5, 200, 60)["x"],
        solvers.proxskip(prob, x0, 0.5, 0.5, 1, 400, 60)["x"],
        solvers.pdhg(prob, x0, np.zeros_like(b), 0.5, 0.5, 600, 60)["x"],
        solvers.pdhgskip2(prob, x0, np.zeros_like(b), 0.5, 0.5, 0.5, 2, 1500, 60)["x"],
        solvers.pdhgskip1(prob, x0, np.zeros_like(b), 0.5, 0.5, 0.5, 3, 3000, 60)["x"],
    ]
    for x in outs:
        np.testing.assert_allclose(x, expect, atol=1e-7)


def test_deblur_solvers_agree_on_minimum():
    """PGD, FISTA and PDHG (three different iterations) reach the same minimum value."""
    prob = _deblur_problem(n=10, alpha=0.03)
    x0 = prob.b.copy()
    f_pgd = solvers.pgd(prob, x0, 1.0, 1500, 30)["objective"][-1]
    f_fista = solvers.fista(prob, x0, 1.0, 600, 30)["objective"][-1]
    f_pdhg = solvers.pdhg(prob, x0, np.zeros_like(prob.b), 0.99, 0.99, 3000, 30)["objective"][-1]
    assert abs(f_pgd - f_fista) <= 1e-8 * f_fista
    assert abs(f_pdhg - f_fista) <= 1e-8 * f_fista


def test_pdhg_residual_decreases():
    """The PDHG fixed-point residual, averaged over windows, decreases."""
    from oracle.power import power_method
    prob, _ = _ct_problem(N=10)
    L = power_method(lambda x: prob.A.adjoint(prob.A.forward(x)), prob.shape, 300)
    st = 0.95 / math.sqrt(L)
    res = []

    def rec(k, x, y, xn, yn):
        res.append(np.linalg.norm((x - xn) / st - prob.A.adjoint(y - yn))
                   + np.linalg.norm((y - yn) / st - prob.A.forward(x - xn)))

    solvers.pdhg(prob, np.zeros(prob.shape), np.zeros_like(prob.b), st, st, 60, 20, record=False, on_iter=rec)
    w = np.array(res).reshape(6, 10).mean(axis=1)
    assert np.all(np.diff(w) < 0)


def test_objective_closed_form():
    """F(x) = 1/2 ||A x - b||^2 + alpha TV(x) on a step image with A = I, b = 0."""
    x = np.zeros((5, 8))
    x[:, 3:] = 2.0
    prob = solvers.Problem(operators.identity_op(), np.zeros_like(x), 0.1, x.shape)
    assert prob.objective(x) == pytest.approx(0.5 * 4.0 * 25 + 0.1 * 2.0 * 5, rel=1e-15)


# ---------------------------------------------------------------- Dual-ROF (light prox)
def test_dual_rof_projgd_reaches_rof_solution():
    """Chambolle's projected gradient on Dual-ROF: u = b + div q converges to the TV
    prox of b, pinned by the 1D exact solver on a single row (isotropic = 1D there)."""
    from tests.test_oracle_tv import _exact_1d_tv_prox
    z = np.random.default_rng(31).standard_normal(9)
    out = solvers.dual_rof_projgd(z[None, :], 0.3, 1.0 / 8.0, 20000)
    np.testing.assert_allclose(out["u"].ravel(), _exact_1d_tv_prox(z, 0.3), atol=1e-8)


def test_dual_rof_proxskip_p1_equals_projgd():
    b = np.random.default_rng(32).standard_normal((9, 12))
    a = solvers.dual_rof_projgd(b, 0.2, 1.0 / 8.0, 40)
    c = solvers.dual_rof_proxskip(b, 0.2, 1.0 / 8.0, 1.0, 4, 40)
    np.testing.assert_allclose(c["q"], a["q"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("eps", [0.0, 0.1])
def test_dual_rof_proxskip_converges(eps):
    """ProxSkip on (Huber-)Dual-ROF reaches the projected-gradient fixed point."""
    b = np.random.default_rng(33).standard_normal((8, 10))
    ref = solvers.dual_rof_projgd(b, 0.25, 1.0 / 8.0, 20000, eps=eps, record=False)
    out = solvers.dual_rof_proxskip(b, 0.25, 1.0 / 8.0, 0.3, 5, 20000, eps=eps, record=False)
    np.testing.assert_allclose(out["u"], ref["u"], atol=1e-6)
    assert np.sqrt((out["q"] ** 2).sum(axis=0)).max() <= 0.25 * (1 + 1e-12)


def test_huber_dual_rof_closed_form_two_pixel():
    """Dual-Huber-ROF on two pixels: F(q) = 1/2 (q + b1)^2 + 1/2 (b2 - q)^2 + eps/(2a) q^2
    with |q| <= a (the single horizontal difference) has the closed-form minimiser
    q* = clip((b2 - b1) / (2 + eps/a), -a, a)."""
    b1, b2, a, eps = 0.1, 0.9, 0.3, 0.1
    b = np.array([[b1, b2]])
    out = solvers.dual_rof_projgd(b, a, 1.0 / 8.0, 5000, eps=eps, record=False)
    q_star = np.clip((b2 - b1) / (2 + eps / a), -a, a)
    assert abs(out["q"][1, 0, 0] - q_star) < 1e-10


# ---------------------------------------------------------------- explicit PDHG
def _dense(fn, in_shape):
    """Matrix of a linear map, one unit vector at a time."""
    n = int(np.prod(in_shape))
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(np.asarray(fn(e.reshape(in_shape))).ravel())
    return np.stack(cols, axis=1)


def _explicit_cases():
    ct, _ = _ct_problem(N=6)  # 16 angles x 17 bins on a 6 x 6 image: some rays miss it
    return [_denoise_problem(n=5), _deblur_problem(n=6), ct]


@pytest.mark.parametrize("case", range(3))
def test_explicit_preconditioners_satisfy_lemma(case):
    """T and Sigma are the reciprocal column and row sums of |K|, K = [A; D], taken
    from the dense matrix, and ||Sigma^1/2 K T^1/2||_2 <= 1 (Pock and Chambolle 2011,
    Lemma 2), which is what makes sigma = tau = 1 a convergent step."""
    prob = _explicit_cases()[case]
    A = _dense(prob.A.forward, prob.shape)
    Dm = _dense(tv.grad, prob.shape)
    assert A.min() >= 0.0  # |A| = A for every operator here
    Kd = np.vstack([A, Dm])
    T, S_A, S_D = solvers.pdhg_explicit_preconditioners(prob)
    col = np.abs(Kd).sum(axis=0)
    np.testing.assert_allclose(T.ravel(), 1.0 / col, rtol=1e-13)
    row = np.abs(A).sum(axis=1)
    live = row > 0
    np.testing.assert_allclose(S_A.ravel()[live], 1.0 / row[live], rtol=1e-13)
    assert np.all(S_A.ravel()[~live] == 1.0)
    drow = np.abs(Dm).sum(axis=1)
    assert set(np.unique(drow)) <= {0.0, 2.0} and S_D == 0.5
    sig = np.concatenate([np.broadcast_to(S_A, prob.b.shape).ravel(), np.full(Dm.shape[0], S_D)])
    M = np.sqrt(sig)[:, None] * Kd * np.sqrt(T.ravel())[None, :]
    assert np.linalg.norm(M, 2) <= 1.0 + 1e-12


@pytest.mark.parametrize("b1,b2,alpha", [(0.0, 1.0, 0.2), (0.4, 0.5, 0.1)])
def test_explicit_pdhg_reaches_two_pixel_minimiser(b1, b2, alpha):
    b = np.array([[b1, b2]])
    prob = solvers.Problem(operators.identity_op(), b, alpha, (1, 2))
    out = solvers.pdhg_explicit(prob, np.zeros_like(b), K=400, record=False)
    np.testing.assert_allclose(out["x"], _two_pixel(b1, b2, alpha), atol=1e-9)


def _kkt(prob, x, q):
    """Optimality of Eq. 5 at (x, q) with no constraint: A^T(Ax - b) - div q = 0,
    |q_i| <= alpha, and q_i = alpha (Dx)_i / |(Dx)_i| wherever (Dx)_i != 0."""
    stat = prob.A.adjoint(prob.A.forward(x) - prob.b) - tv.div(q)
    g = tv.grad(x)
    nrm = np.sqrt((g * g).sum(axis=0))
    qn = np.sqrt((q * q).sum(axis=0))
    big = nrm > 1e-6
    align = np.abs(q[:, big] - prob.alpha * g[:, big] / nrm[big]).max() if big.any() else 0.0
    return np.abs(stat).max(), qn.max() - prob.alpha, align


@pytest.mark.parametrize("make,K", [(_denoise_problem, 20000), (_deblur_problem, 4000)])
def test_explicit_pdhg_satisfies_optimality(make, K):
    prob = make()
    out = solvers.pdhg_explicit(prob, prob.b.copy(), K=K, record=False)
    stat, excess, align = _kkt(prob, out["x"], out["q"])
    assert stat <= 1e-7 and excess <= 1e-12 and align <= 1e-5


def test_explicit_pdhg_agrees_with_implicit_solvers():
    """Same minimum value as FISTA with the FGP prox on a small deblurring problem,
    and, with the non-negativity constraint on a small tomography problem, the
    minimiser of implicit PDHG (explicit PDHG converges at the slower O(1/k) rate
    there, hence the looser bound)."""
    prob = _deblur_problem(n=10, alpha=0.03)
    f_fista = solvers.fista(prob, prob.b.copy(), 1.0, 300, 30)["objective"][-1]
    f_exp = solvers.pdhg_explicit(prob, prob.b.copy(), K=4000)["objective"][-1]
    assert abs(f_exp - f_fista) <= 1e-7 * f_fista
    ct, _ = _ct_problem(N=8, alpha=0.01)
    ct.nonneg = True
    from oracle.power import power_method
    L = power_method(lambda x: ct.A.adjoint(ct.A.forward(x)), ct.shape, 300)
    st = 0.99 / math.sqrt(L)
    imp = solvers.pdhg(ct, np.zeros(ct.shape), np.zeros_like(ct.b), st, st, 800, 40)
    out = solvers.pdhg_explicit(ct, np.zeros(ct.shape), K=1500)
    assert out["x"].min() >= 0.0
    assert np.linalg.norm(out["x"] - imp["x"]) <= 2e-5 * np.linalg.norm(imp["x"])
    f_imp = imp["objective"][-1]
    assert -1e-9 <= (out["objective"][-1] - f_imp) / f_imp <= 2e-6
