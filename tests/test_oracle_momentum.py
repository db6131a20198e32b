"""Finite-N pins of the oracle's accelerated iterations: the inner AProjGD/FGP
solver of the TV prox (ProjGD plus the FISTA momentum of Algorithm 3, run for a
fixed number of iterations with a warm start, Sections 2.2 and 3.1) and the outer
FISTA solver (Algorithm 3).

Every GPU parity test compares fixed-N iterates with these two functions, so their
trajectories (not only their limits) are pinned here:

* t_1 = 1 makes the first two momentum coefficients zero, so one and two FGP
  iterations are plain projected-gradient steps: they must equal the separately
  written ProjGD route (on the lambda-scaled dual, Section 2.1), and a run split into
  calls of two iterations (the momentum restarting every call) must equal ProjGD run
  straight through.
* On two pixels (and two voxels) in the regime where the ball projection is
  inactive, every iteration is affine in the previous ones; the iterates are
  written out by hand with the momentum coefficients in closed form
  (t_2 = (1 + sqrt 5)/2, ...), not by re-running the recurrence.
* Beck and Teboulle's bound for the accelerated method on the dual,
  F(p_N) - F(p*) <= 2 L ||p_0 - p*||^2 / (N + 1)^2 with L = 8 lambda^2, is checked
  with every quantity certified (||p*||^2 bounded by the count of dual entries that
  can be non-zero, F(p*) bounded through weak duality); plain ProjGD breaks it on
  the same instance.
* FISTA's first extrapolation coefficient is zero, so two FISTA steps equal two PGD
  steps bit for bit; on two pixels with an exact prox the next steps are written out
  by hand.

Finally, a set of plausible mistakes (wrong or missing momentum coefficient, wrong
sign, frozen t, lost warm start, final u from the extrapolated point, wrong step,
gradient at the wrong point) is planted into copies of the oracle functions, and
each mutant must fail at least one of these pins.
"""

import inspect
import math
import textwrap

import numpy as np
import pytest

from oracle import operators, solvers, tv

# Momentum coefficients in closed form.  With t_1 = 1 and t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2:
#   t_2 = (1 + sqrt 5)/2, t_2^2 = (3 + sqrt 5)/2, so 1 + 4 t_2^2 = 7 + 2 sqrt 5;
#   t_3 = (1 + s7)/2 with s7 = sqrt(7 + 2 sqrt 5), t_3^2 = (8 + 2 sqrt 5 + 2 s7)/4,
#   so 1 + 4 t_3^2 = 9 + 2 sqrt 5 + 2 s7 and t_4 = (1 + sqrt(9 + 2 sqrt 5 + 2 s7))/2.
# beta_k = (t_k - 1)/t_{k+1}, so beta_1 = 0 and beta_2, beta_3 are:
SQ5 = math.sqrt(5.0)
S7 = math.sqrt(7.0 + 2.0 * SQ5)
S9 = math.sqrt(9.0 + 2.0 * SQ5 + 2.0 * S7)
BETA2 = (SQ5 - 1.0) / (1.0 + S7)
BETA3 = (S7 - 1.0) / (1.0 + S9)


def test_closed_form_coefficients():
    """The closed forms above against decimal values worked out by hand
    (t_2 = 1.6180340 is the golden ratio, t_3 = 2.1935271, t_4 = 2.7497913)."""
    assert (1.0 + S7) / 2.0 == pytest.approx(2.1935271, abs=1e-7)
    assert (1.0 + S9) / 2.0 == pytest.approx(2.7497913, abs=1e-7)
    assert BETA2 == pytest.approx(0.6180340 / 2.1935271, abs=1e-7)
    assert BETA3 == pytest.approx(1.1935271 / 2.7497913, abs=1e-7)


# ----------------------------------------------------------------- pins (FGP)
def _pin_first_two_are_projgd(fgp):
    g = np.random.default_rng(11)
    for shape, lam in [((7, 9), 0.3), ((7, 9), 0.02), ((3, 4, 5), 0.2), ((5, 1, 6), 0.03)]:
        z = g.standard_normal(shape)
        p0 = tv.project_unit_ball(g.standard_normal((len(shape),) + shape))
        for warm in (None, p0):
            for n in (1, 2):
                u, p = fgp(z, lam, n, warm)
                u_ref, p_ref = tv.projgd_prox(z, lam, n, warm)
                np.testing.assert_allclose(u, u_ref, rtol=0, atol=1e-13)
                np.testing.assert_allclose(p, p_ref, rtol=0, atol=1e-13)


def _pin_restart_every_call(fgp):
    g = np.random.default_rng(12)
    for shape, lam in [((6, 8), 0.25), ((4, 3, 5), 0.1)]:
        z = g.standard_normal(shape)
        p = None
        for _ in range(3):               # three calls of two iterations ...
            u, p = fgp(z, lam, 2, p)
        u_ref, p_ref = tv.projgd_prox(z, lam, 6)   # ... are six ProjGD steps
        np.testing.assert_allclose(u, u_ref, rtol=0, atol=1e-13)
        np.testing.assert_allclose(p, p_ref, rtol=0, atol=1e-13)


def _two_pixel_expected(d, lam, n, a):
    """Iterates of the unclipped two-pixel (two-voxel) dual, by hand.

    With z = (z0, z0 + d), the only free dual entry q sits on the first pixel;
    u = (z0 + lam r, z0 + d - lam r), D u = d - 2 lam r, and the dual step with
    constant a = 4 ndim gives p = (1 - 2/a) r + c, c = d/(a lam).  Starting from
    p_0 = 0 = r_1:
      p_1 = c;  r_2 = p_1 (beta_1 = 0);  p_2 = (2 - 2/a) c;
      r_3 = p_2 + beta_2 (p_2 - p_1);  p_3 = (1 - 2/a) r_3 + c;
      r_4 = p_3 + beta_3 (p_3 - p_2);  p_4 = (1 - 2/a) r_4 + c.
    """
    c = d / (a * lam)
    m = 1.0 - 2.0 / a
    p1 = c
    p2 = m * p1 + c
    p3 = m * (p2 + BETA2 * (p2 - p1)) + c
    p4 = m * (p3 + BETA3 * (p3 - p2)) + c
    return [p1, p2, p3, p4][n - 1]


def _pin_two_pixel_unrolled(fgp):
    z0, d, lam = 0.2, 0.3, 0.25
    # 2D: a 1 x 2 image, q in the horizontal plane at pixel 0; a = 8, c = 0.15
    for n in (1, 2, 3, 4):
        q = _two_pixel_expected(d, lam, n, 8.0)
        assert abs(q) < 1.0                 # the projection stays inactive
        u, p = fgp(np.array([[z0, z0 + d]]), lam, n)
        np.testing.assert_allclose(p[1, 0, 0], q, rtol=0, atol=1e-14)
        np.testing.assert_allclose(p[1, 0, 1], 0.0, atol=0)
        np.testing.assert_allclose(p[0], 0.0, atol=0)
        np.testing.assert_allclose(u.ravel(), [z0 + lam * q, z0 + d - lam * q], rtol=0, atol=1e-14)
    # the same pair along columns
    for n in (3, 4):
        q = _two_pixel_expected(d, lam, n, 8.0)
        u, p = fgp(np.array([[z0], [z0 + d]]), lam, n)
        np.testing.assert_allclose(p[0, 0, 0], q, rtol=0, atol=1e-14)
        np.testing.assert_allclose(u.ravel(), [z0 + lam * q, z0 + d - lam * q], rtol=0, atol=1e-14)
    # 3D: two voxels along the slowest axis, a = 12
    for n in (1, 2, 3, 4):
        q = _two_pixel_expected(d, lam, n, 12.0)
        z = np.array([z0, z0 + d]).reshape(2, 1, 1)
        u, p = fgp(z, lam, n)
        np.testing.assert_allclose(p[0, 0, 0, 0], q, rtol=0, atol=1e-14)
        np.testing.assert_allclose(u.ravel(), [z0 + lam * q, z0 + d - lam * q], rtol=0, atol=1e-14)


def _dual_F(z, lam, p):
    w = z + lam * tv.div(p)
    return 0.5 * float(np.sum(w * w))


def _rate_instance():
    """A 1 x 64 ramp: a chain whose dual converges slowly under plain ProjGD."""
    z = np.linspace(0.0, 1.0, 64)[None, :]
    lam = 0.5
    _, p_long = tv.fgp_prox(z, lam, 20000)
    gap = tv.rof_gap(z, lam, p_long)
    assert 0.0 <= gap < 1e-12
    F_lo = _dual_F(z, lam, p_long) - gap      # F(p*) >= F(p_long) - gap (weak duality)
    R2 = z.shape[1] - 1                        # ||p_0 - p*||^2 <= 63 (|p_i| <= 1, 63 free entries)
    return z, lam, F_lo, R2


RATE_N = (1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233)


def _rate_ratios(prox, z, lam, F_lo, R2):
    L = 8.0 * lam * lam
    out = []
    for N in RATE_N:
        _, p = prox(z, lam, N)
        out.append((_dual_F(z, lam, p) - F_lo) / (2.0 * L * R2 / (N + 1) ** 2))
    return np.array(out)


def _pin_beck_teboulle(fgp):
    z, lam, F_lo, R2 = _rate_instance()
    assert np.all(_rate_ratios(fgp, z, lam, F_lo, R2) <= 1.0)


PINS_FGP = [_pin_first_two_are_projgd, _pin_restart_every_call, _pin_two_pixel_unrolled,
            _pin_beck_teboulle]


@pytest.mark.parametrize("pin", PINS_FGP, ids=lambda f: f.__name__[5:])
def test_fgp_pins(pin):
    pin(tv.fgp_prox)


def test_projgd_breaks_the_accelerated_rate():
    """The rate pin separates the accelerated method from plain ProjGD: on the same
    instance ProjGD exceeds the O(1/N^2) bound (its own rate is O(1/N))."""
    z, lam, F_lo, R2 = _rate_instance()
    r = _rate_ratios(lambda z, lam, n: tv.projgd_prox(z, lam, n), z, lam, F_lo, R2)
    assert r.max() > 5.0


# ----------------------------------------------------------------- pins (FISTA)
def _two_pixel_problem():
    return solvers.Problem(operators.identity_op(), np.array([[0.0, 1.0]]), 0.1, (1, 2))


def _pin_fista_two_steps_are_pgd(fista):
    g = np.random.default_rng(13)
    A = operators.blur_op(1.2)
    b = A.forward(np.kron(np.eye(3), np.ones((3, 3)))) + 0.01 * g.standard_normal((9, 9))
    prob = solvers.Problem(A, b, 0.03, (9, 9))
    a = solvers.pgd(prob, b, 0.9, 2, 6)
    f = fista(prob, b, 0.9, 2, 6)
    np.testing.assert_array_equal(f["x"], a["x"])
    np.testing.assert_array_equal(f["objective"], a["objective"])


def _pin_fista_two_pixel_unrolled(fista):
    """A = I, b = (0, 1), alpha = 0.1, gamma = 1/2 (lam = 0.05), x_0 = y_0 = b.

    prox argument v = y - gamma (y - b) = (y_0 / 2, (y_1 + 1)/2); while its two
    entries differ by more than 2 lam the exact two-pixel prox moves each lam toward
    the other, so with e = first entry (the second is 1 - e): e_{k+1} = y_k / 2 + lam,
    y_{k+1} = e_{k+1} + beta (e_{k+1} - e_k), beta = 0, BETA2, BETA3 in turn."""
    prob = _two_pixel_problem()
    lam = 0.05
    e1 = 0.0 / 2 + lam
    y1 = e1
    e2 = y1 / 2 + lam
    y2 = e2 + BETA2 * (e2 - e1)
    e3 = y2 / 2 + lam
    y3 = e3 + BETA3 * (e3 - e2)
    e4 = y3 / 2 + lam
    for K, e in [(1, e1), (2, e2), (3, e3), (4, e4)]:
        out = fista(prob, prob.b, 0.5, K, 200)
        np.testing.assert_allclose(out["x"].ravel(), [e, 1.0 - e], rtol=0, atol=1e-13)
    assert (e1, e2) == pytest.approx((0.05, 0.075))


PINS_FISTA = [_pin_fista_two_steps_are_pgd, _pin_fista_two_pixel_unrolled]


@pytest.mark.parametrize("pin", PINS_FISTA, ids=lambda f: f.__name__[5:])
def test_fista_pins(pin):
    pin(solvers.fista)


# ----------------------------------------------------------------- planted mistakes
def _mutant(func, old, new):
    """A copy of ``func`` with one source fragment replaced, compiled in the
    function's own module namespace (the oracle itself is not modified)."""
    src = textwrap.dedent(inspect.getsource(func))
    assert src.count(old) == 1, f"mutation target not found once: {old!r}"
    ns = dict(inspect.getmodule(func).__dict__)
    exec(compile(src.replace(old, new), f"<mutant {func.__name__}>", "exec"), ns)
    return ns[func.__name__]


FGP_MUTANTS = {
    "beta_t_over_tnew": ("((t - 1.0) / t_new)", "(t / t_new)"),
    "no_momentum": ("((t - 1.0) / t_new)", "0.0"),
    "momentum_sign": ("(p_new - p_prev)", "(p_prev - p_new)"),
    "t_frozen": ("        t = t_new\n", "        t = t\n"),
    "t_recurrence": ("4.0 * t * t", "4.0 * t"),
    "warm_start_lost": ("r = p.copy()", "r = np.zeros_like(p)"),
    "u_from_extrapolated": ("div(p_prev), nonneg)\n    return", "div(r), nonneg)\n    return"),
    "step_without_lambda": ("grad(u) / (L * lam)", "grad(u) / L"),
    "step_constant": ("L = dual_step_constant(d)", "L = 8.0"),
}


@pytest.mark.parametrize("name", sorted(FGP_MUTANTS))
def test_fgp_mutants_fail_a_pin(name):
    old, new = FGP_MUTANTS[name]
    bad = _mutant(tv.fgp_prox, old, new)
    failed = []
    for pin in PINS_FGP:
        try:
            pin(bad)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"planted mistake {name} passes every FGP pin"


FISTA_MUTANTS = {
    "beta_t_over_tnew": ("((t - 1.0) / t_new)", "(t / t_new)"),
    "extrapolation_sign": ("(x_new - x)", "(x - x_new)"),
    "t_frozen": ("x, t = x_new, t_new", "x, t = x_new, t"),
    "gradient_at_x": ("y - gamma * prob.grad_f(y)", "y - gamma * prob.grad_f(x)"),
    "prox_from_x": ("y - gamma * prob.grad_f(y)", "x - gamma * prob.grad_f(x)"),
}


@pytest.mark.parametrize("name", sorted(FISTA_MUTANTS))
def test_fista_mutants_fail_a_pin(name):
    old, new = FISTA_MUTANTS[name]
    bad = _mutant(solvers.fista, old, new)
    failed = []
    for pin in PINS_FISTA:
        try:
            pin(bad)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"planted mistake {name} passes every FISTA pin"


# ----------------------------------------------------------------- pins (AProjGD on Dual-ROF)
def _pin_aprojgd_first_two_are_projgd(aprojgd):
    """y_0 = q_0 and the first extrapolation coefficient is zero: one and two
    AProjGD steps are ProjGD steps, bit for bit."""
    g = np.random.default_rng(14)
    b = g.standard_normal((7, 9))
    for eps in (0.0, 0.1):
        for K in (1, 2):
            a = solvers.dual_rof_projgd(b, 0.2, 1.0 / 8.0, K, eps=eps)
            c = aprojgd(b, 0.2, 1.0 / 8.0, K, eps=eps)
            np.testing.assert_array_equal(c["q"], a["q"])
            np.testing.assert_array_equal(c["objective"], a["objective"])


def _pin_aprojgd_two_pixel_unrolled(aprojgd):
    """Dual-Huber-ROF on two pixels b = (0.1, 0.3), alpha = 0.3, eps = 0.1, gamma = 1/8:
    the single dual entry q has grad F(q) = (2 + eps/alpha) q - (b_2 - b_1), so while
    |q| < alpha a step is y -> m y + c with m = 1 - (2 + eps/alpha)/8 and c = 0.2/8:
      q_1 = c, y_1 = q_1;  q_2 = m y_1 + c, y_2 = q_2 + beta_2 (q_2 - q_1);
      q_3 = m y_2 + c, y_3 = q_3 + beta_3 (q_3 - q_2);  q_4 = m y_3 + c."""
    b = np.array([[0.1, 0.3]])
    a, eps = 0.3, 0.1
    m, c = 1.0 - (2.0 + eps / a) / 8.0, 0.2 / 8.0
    q1 = c
    q2 = m * q1 + c
    y2 = q2 + BETA2 * (q2 - q1)
    q3 = m * y2 + c
    y3 = q3 + BETA3 * (q3 - q2)
    q4 = m * y3 + c
    for K, q in [(1, q1), (2, q2), (3, q3), (4, q4)]:
        assert abs(q) < a
        out = aprojgd(b, a, 1.0 / 8.0, K, eps=eps)
        np.testing.assert_allclose(out["q"][1, 0, 0], q, rtol=0, atol=1e-15)
        np.testing.assert_allclose(out["u"].ravel(), [0.1 + q, 0.3 - q], rtol=0, atol=1e-15)


def _pin_aprojgd_beck_teboulle(aprojgd):
    """F(q_K) - F* <= 2 L ||q_0 - q*||^2 / (K + 1)^2 with L = 8 (the step 1/8) on a
    64-pixel ramp, alpha = 0.5: ||q*||^2 <= 63 alpha^2, and F* >= 1/2 ||b||^2 - P(u)
    for any u (weak duality with the ROF primal P), here u from a long run."""
    z = np.linspace(0.0, 1.0, 64)[None, :]
    alpha = 0.5
    u_long, _ = tv.fgp_prox(z, alpha, 20000)
    F_lo = 0.5 * float(np.sum(z * z)) - tv.rof_primal(u_long, z, alpha)
    R2 = 63 * alpha * alpha
    for K in RATE_N:
        F = aprojgd(z, alpha, 1.0 / 8.0, K)["objective"][-1]
        assert F - F_lo <= 2.0 * 8.0 * R2 / (K + 1) ** 2


PINS_APROJGD = [_pin_aprojgd_first_two_are_projgd, _pin_aprojgd_two_pixel_unrolled, _pin_aprojgd_beck_teboulle]


@pytest.mark.parametrize("pin", PINS_APROJGD, ids=lambda f: f.__name__[5:])
def test_aprojgd_pins(pin):
    pin(solvers.dual_rof_aprojgd)


def test_projgd_breaks_the_accelerated_rate_on_dual_rof():
    with pytest.raises(AssertionError):
        _pin_aprojgd_beck_teboulle(lambda b, a, g, K, eps=0.0: solvers.dual_rof_projgd(b, a, g, K, eps=eps))


APROJGD_MUTANTS = {
    "beta_t_over_tnew": ("((t - 1.0) / t_new)", "(t / t_new)"),
    "no_momentum": ("((t - 1.0) / t_new)", "0.0"),
    "extrapolation_sign": ("(q_new - q)", "(q - q_new)"),
    "t_frozen": ("q, t = q_new, t_new", "q, t = q_new, t"),
    "gradient_at_q": ("_dual_rof_grad(y, b", "_dual_rof_grad(q, b"),
}


@pytest.mark.parametrize("name", sorted(APROJGD_MUTANTS))
def test_aprojgd_mutants_fail_a_pin(name):
    old, new = APROJGD_MUTANTS[name]
    bad = _mutant(solvers.dual_rof_aprojgd, old, new)
    failed = []
    for pin in PINS_APROJGD:
        try:
            pin(bad)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"planted mistake {name} passes every AProjGD pin"
