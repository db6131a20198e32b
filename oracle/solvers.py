"""Outer solvers for min_u 1/2 ||A u - b||^2 + alpha TV(u)  (Eq. 5), FP64 oracle.

f(x) = 1/2 ||A x - b||^2 (gradient A^T (A x - b)), g = alpha TV (+ the indicator of
x >= 0 when ``nonneg``).  Every prox of g is the warm-started fixed-iteration inner
solver ``tv.fgp_prox`` (Section 3.1); each solver keeps one dual field across its
prox calls.  Coins come from ``coin.coin``.

Each solver returns a dict with the final iterates, the objective F(x_{k+1}) after
every outer iteration, the coin of every iteration and the number of prox calls.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import coin as coin_mod
from . import tv
from .operators import LinearOp


@dataclass
class Problem:
    """min_u 1/2 ||A u - b||^2 + alpha TV(u) [+ indicator(u >= 0)]."""
    A: LinearOp
    b: np.ndarray
    alpha: float
    shape: tuple
    nonneg: bool = False

    def grad_f(self, x):
        return self.A.adjoint(self.A.forward(x) - self.b)

    def objective(self, x):
        r = self.A.forward(x) - self.b
        return 0.5 * float(np.sum(r * r)) + self.alpha * tv.tv(x)


def _prox_g(prob: Problem, v, step, n_inner, dual):
    """prox_{step * g}(v) with g = alpha TV: FGP with lam = step * alpha."""
    return tv.fgp_prox(v, step * prob.alpha, n_inner, dual, prob.nonneg)


def pgd(prob: Problem, x0, gamma, K, n_inner, record=True):
    """Algorithm 2: x_{k+1} = prox_{gamma g}(x_k - gamma grad f(x_k))."""
    x = np.array(x0, dtype=np.float64)
    dual = None
    obj = []
    for _ in range(K):
        x, dual = _prox_g(prob, x - gamma * prob.grad_f(x), gamma, n_inner, dual)
        if record:
            obj.append(prob.objective(x))
    return dict(x=x, dual=dual, objective=obj, coins=[1] * K, prox_calls=K)


def proxskip(prob: Problem, x0, gamma, p, seed, K, n_inner, h0=None, record=True,
             on_prox=None):
    """Algorithm 4 (ProxSkip).

    x^_{k+1} = x_k - gamma (grad f(x_k) - h_k);
    if theta_k = 1: x_{k+1} = prox_{(gamma/p) g}(x^_{k+1} - (gamma/p) h_k)
    else:          x_{k+1} = x^_{k+1};
    h_{k+1} = h_k + (p/gamma)(x_{k+1} - x^_{k+1}).
    ``on_prox(k, x, h, dual)`` is called after each executed prox (for tests).
    """
    x = np.array(x0, dtype=np.float64)
    h = np.zeros_like(x) if h0 is None else np.array(h0, dtype=np.float64)
    dual = None
    obj, coins = [], []
    n_prox = 0
    for k in range(K):
        x_hat = x - gamma * (prob.grad_f(x) - h)
        theta = coin_mod.coin(seed, p, k)
        coins.append(theta)
        if theta:
            x_new, dual = _prox_g(prob, x_hat - (gamma / p) * h, gamma / p, n_inner, dual)
            n_prox += 1
        else:
            x_new = x_hat
        h = h + (p / gamma) * (x_new - x_hat)
        x = x_new
        if theta and on_prox is not None:
            on_prox(k, x, h, dual)
        if record:
            obj.append(prob.objective(x))
    return dict(x=x, h=h, dual=dual, objective=obj, coins=coins, prox_calls=n_prox)


def fista(prob: Problem, x0, gamma, K, n_inner, record=True):
    """Algorithm 3 (FISTA) in Beck and Teboulle's form.

    x_{k+1} = prox_{gamma g}(y_k - gamma grad f(y_k)); t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2;
    y_{k+1} = x_{k+1} + ((t_k - 1)/t_{k+1}) (x_{k+1} - x_k); y_0 = x_0, t_0 = 1.
    """
    x = np.array(x0, dtype=np.float64)
    y = x.copy()
    t = 1.0
    dual = None
    obj = []
    for _ in range(K):
        x_new, dual = _prox_g(prob, y - gamma * prob.grad_f(y), gamma, n_inner, dual)
        t_new = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        y = x_new + ((t - 1.0) / t_new) * (x_new - x)
        x, t = x_new, t_new
        if record:
            obj.append(prob.objective(x))
    return dict(x=x, dual=dual, objective=obj, coins=[1] * K, prox_calls=K)


def prox_fconj(v, tau, b):
    """prox_{tau f*}(v) for f = 1/2 ||. - b||^2, through Moreau's identity.

    prox_{tau f*}(v) = v - tau prox_{f/tau}(v / tau), and prox_{f/tau}(w) minimises
    1/2 ||x - w||^2 + (1/(2 tau)) ||x - b||^2, i.e. x = (tau w + b) / (tau + 1).
    """
    w = v / tau
    return v - tau * (tau * w + b) / (tau + 1.0)


def pdhg(prob: Problem, x0, y0, sigma, tau, K, n_inner, record=True, on_iter=None):
    """Implicit PDHG for f(K x) + g(x) with K = A, f = 1/2 ||. - b||^2, g = alpha TV.

    Written with the step naming of Algorithm 6 (sigma primal, tau dual):
    x_{k+1} = prox_{sigma g}(x_k - sigma K^T y_k); x-bar = 2 x_{k+1} - x_k;
    y_{k+1} = prox_{tau f*}(y_k + tau K x-bar).
    ``on_iter(k, x_k, y_k, x_{k+1}, y_{k+1})`` is called after every iteration (for tests).
    """
    x = np.array(x0, dtype=np.float64)
    y = np.array(y0, dtype=np.float64)
    dual = None
    obj = []
    for _ in range(K):
        x_new, dual = _prox_g(prob, x - sigma * prob.A.adjoint(y), sigma, n_inner, dual)
        x_bar = 2.0 * x_new - x
        y_new = prox_fconj(y + tau * prob.A.forward(x_bar), tau, prob.b)
        if on_iter is not None:
            on_iter(_, x, y, x_new, y_new)
        x, y = x_new, y_new
        if record:
            obj.append(prob.objective(x))
    return dict(x=x, y=y, dual=dual, objective=obj, coins=[1] * K, prox_calls=K)


def pdhgskip2(prob: Problem, x0, y0, sigma, tau, p, seed, K, n_inner, h0=None,
              record=True, on_prox=None):
    """Algorithm 6 (PDHGSkip-2), with the index reading
    h_{k+1} = h_k + (p/sigma)(x_{k+1} - x^_k) and y_{k+1} = prox_{tau f*}(y_k + tau K x-bar_{k+1}):

    x^_k = x_k - sigma (K^T y_k - h_k);
    if theta_k = 1: x_{k+1} = prox_{(sigma/p) g}(x^_k - (sigma/p) h_k) else x_{k+1} = x^_k;
    x-bar_{k+1} = 2 x_{k+1} - x_k.
    """
    x = np.array(x0, dtype=np.float64)
    y = np.array(y0, dtype=np.float64)
    h = np.zeros_like(x) if h0 is None else np.array(h0, dtype=np.float64)
    dual = None
    obj, coins = [], []
    n_prox = 0
    for k in range(K):
        x_hat = x - sigma * (prob.A.adjoint(y) - h)
        theta = coin_mod.coin(seed, p, k)
        coins.append(theta)
        if theta:
            x_new, dual = _prox_g(prob, x_hat - (sigma / p) * h, sigma / p, n_inner, dual)
            n_prox += 1
        else:
            x_new = x_hat
        x_bar = 2.0 * x_new - x
        y = prox_fconj(y + tau * prob.A.forward(x_bar), tau, prob.b)
        h = h + (p / sigma) * (x_new - x_hat)
        x = x_new
        if theta and on_prox is not None:
            on_prox(k, x, h, dual)
        if record:
            obj.append(prob.objective(x))
    return dict(x=x, y=y, h=h, dual=dual, objective=obj, coins=coins, prox_calls=n_prox)


def pdhgskip1(prob: Problem, x0, y0, sigma, tau, p, seed, K, n_inner, record=True):
    """Algorithm 5 (PDHGSkip-1, Condat's skipping PDHG) with omega + 1 = 1/p (Section 3.2).

    x^_k = B_p(prox_{sigma g}(x_k - sigma K^T y_k) - x_k), where B_p(v) = v / p when
    theta_k = 1 and 0 otherwise (the prox is evaluated only when theta_k = 1);
    x_{k+1} = x_k + x^_k / (1 + omega);
    y_{k+1} = prox_{tau f*}(y_k + tau K (x_{k+1} + x^_k)).
    """
    x = np.array(x0, dtype=np.float64)
    y = np.array(y0, dtype=np.float64)
    omega = 1.0 / p - 1.0
    dual = None
    obj, coins = [], []
    n_prox = 0
    for k in range(K):
        theta = coin_mod.coin(seed, p, k)
        coins.append(theta)
        if theta:
            u, dual = _prox_g(prob, x - sigma * prob.A.adjoint(y), sigma, n_inner, dual)
            x_hat = (u - x) / p
            n_prox += 1
        else:
            x_hat = np.zeros_like(x)
        x_new = x + x_hat / (1.0 + omega)
        y = prox_fconj(y + tau * prob.A.forward(x_new + x_hat), tau, prob.b)
        x = x_new
        if record:
            obj.append(prob.objective(x))
    return dict(x=x, y=y, dual=dual, objective=obj, coins=coins, prox_calls=n_prox)


# ---------------------------------------------------------------- explicit PDHG
def difference_column_counts(shape):
    """Entries of D in each pixel's column, sum_i |D_ij|: per axis a, pixel j enters
    the difference at j (when j_a < n_a - 1) and the one at j - e_a (when j_a > 0)."""
    cnt = np.zeros(shape, dtype=np.float64)
    for a, n_a in enumerate(shape):
        idx = np.arange(n_a).reshape([-1 if b == a else 1 for b in range(len(shape))])
        cnt += (idx < n_a - 1).astype(np.float64) + (idx > 0).astype(np.float64)
    return cnt


def pdhg_explicit_preconditioners(prob: Problem):
    """Diagonal step sizes of Pock and Chambolle (ICCV 2011), Lemma 2 with exponent 1,
    for the block operator K = [A; D] of the explicit formulation (Section 3.2):
    T_j = 1 / sum_i |K_ij| per pixel and Sigma_i = 1 / sum_j |K_ij| per dual entry.

    Every operator here has non-negative entries (blur weights, Joseph weights, the
    identity), so |A| 1 = A 1 and |A|^T 1 = A^T 1.  A row of D holds -1 and +1, or
    nothing on the last slice of its axis: all D rows take Sigma = 1/2 (a smaller
    step than 1/0 on the empty rows, which keeps the bound of the lemma).  An empty
    row of A or an empty column of K takes 1: the matching entries of K are zero,
    so the bound does not involve them.
    Returns (T, Sigma_A, Sigma_D)."""
    col = prob.A.adjoint(np.ones(prob.b.shape)) + difference_column_counts(prob.shape)
    row = prob.A.forward(np.ones(prob.shape))
    T = np.where(col > 0, 1.0 / np.where(col > 0, col, 1.0), 1.0)
    S_A = np.where(row > 0, 1.0 / np.where(row > 0, row, 1.0), 1.0)
    return T, S_A, 0.5


def pdhg_explicit(prob: Problem, x0, y0=None, q0=None, K=100, sigma=1.0, tau=1.0, record=True):
    """Explicit PDHG with diagonal preconditioning, the solver behind the paper's
    reference solutions u* (Section 4.1) in the explicit form of Section 3.2:
    K = [A; D], f(v, w) = 1/2 ||v - b||^2 + alpha sum_i |w_i|_2 (separable), g = 0 or
    the indicator of x >= 0; every prox is closed-form.  With T, Sigma from
    ``pdhg_explicit_preconditioners`` scaled by sigma (primal) and tau (dual),
    sigma * tau <= 1, and the step naming of Algorithm 6:

        x_{k+1} = P_X(x_k - sigma T (A^T y_k - div q_k))        (K^T (y, q) = A^T y - div q)
        x-bar   = 2 x_{k+1} - x_k
        y_{k+1} = (y_k + tau S_A (A x-bar - b)) / (1 + tau S_A)  (prox of the conjugate of 1/2||. - b||^2)
        q_{k+1} = P_alpha(q_k + tau S_D D x-bar)                  (prox of the conjugate of alpha |.|_{2,1})
    """
    x = np.array(x0, dtype=np.float64)
    y = np.zeros(prob.b.shape) if y0 is None else np.array(y0, dtype=np.float64)
    q = np.zeros((x.ndim,) + x.shape) if q0 is None else np.array(q0, dtype=np.float64)
    T, S_A, S_D = pdhg_explicit_preconditioners(prob)
    obj = []
    for _ in range(K):
        x_new = x - sigma * T * (prob.A.adjoint(y) - tv.div(q))
        if prob.nonneg:
            x_new = np.maximum(x_new, 0.0)
        x_bar = 2.0 * x_new - x
        s_a = tau * S_A
        y = (y + s_a * (prob.A.forward(x_bar) - prob.b)) / (1.0 + s_a)
        if prob.alpha > 0:
            q = tv.project_ball(q + (tau * S_D) * tv.grad(x_bar), prob.alpha)
        else:  # the ball of radius 0
            q = np.zeros_like(q)
        x = x_new
        if record:
            obj.append(prob.objective(x))
    return dict(x=x, y=y, q=q, objective=obj, coins=[1] * K, prox_calls=K)


# ---------------------------------------------------------------- light-prox case
def dual_rof_objective(q, b, alpha, eps=0.0):
    """F(q) = 1/2 ||div q + b||^2 + (eps / (2 alpha)) ||q||^2 (Eq. 6 / Eq. 8 without
    their constant term)."""
    w = tv.div(q) + b
    val = 0.5 * float(np.sum(w * w))
    if eps > 0.0:
        val += eps / (2.0 * alpha) * float(np.sum(q * q))
    return val


def _dual_rof_grad(q, b, alpha, eps):
    """Gradient of F: -D(div q + b) + (eps / alpha) q  (div = -D^T)."""
    g = -tv.grad(tv.div(q) + b)
    if eps > 0.0:
        g = g + (eps / alpha) * q
    return g


def dual_rof_projgd(b, alpha, gamma, K, eps=0.0, q0=None, record=True):
    """Projected gradient on Dual-ROF (Section 2.1) or Dual-Huber-ROF (Section 2.2):
    q_{k+1} = P_C(q_k - gamma grad F(q_k)), P_C the pointwise projection onto the
    alpha-ball (Eq. 7).  The primal iterate is u_k = b + div q_k."""
    b = np.asarray(b, dtype=np.float64)
    q = np.zeros((b.ndim,) + b.shape) if q0 is None else np.array(q0, dtype=np.float64)
    obj = []
    for _ in range(K):
        q = tv.project_ball(q - gamma * _dual_rof_grad(q, b, alpha, eps), alpha)
        if record:
            obj.append(dual_rof_objective(q, b, alpha, eps))
    return dict(q=q, u=b + tv.div(q), objective=obj, coins=[1] * K, prox_calls=K)


def dual_rof_aprojgd(b, alpha, gamma, K, eps=0.0, q0=None, record=True):
    """AProjGD on Dual-ROF / Dual-Huber-ROF (Section 2.2): the projected gradient
    step of Algorithm 2 taken from the extrapolated point of Algorithm 3 (FISTA,
    Beck and Teboulle's form):

        q_{k+1} = P_C(y_k - gamma grad F(y_k));  t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2;
        y_{k+1} = q_{k+1} + ((t_k - 1) / t_{k+1}) (q_{k+1} - q_k);  y_0 = q_0, t_0 = 1.

    The objective is recorded at q_{k+1}; the primal iterate is u_k = b + div q_k."""
    b = np.asarray(b, dtype=np.float64)
    q = np.zeros((b.ndim,) + b.shape) if q0 is None else np.array(q0, dtype=np.float64)
    y = q.copy()
    t = 1.0
    obj = []
    for _ in range(K):
        q_new = tv.project_ball(y - gamma * _dual_rof_grad(y, b, alpha, eps), alpha)
        t_new = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        y = q_new + ((t - 1.0) / t_new) * (q_new - q)
        q, t = q_new, t_new
        if record:
            obj.append(dual_rof_objective(q, b, alpha, eps))
    return dict(q=q, u=b + tv.div(q), objective=obj, coins=[1] * K, prox_calls=K)


def dual_rof_proxskip(b, alpha, gamma, p, seed, K, eps=0.0, record=True):
    """Algorithm 4 on Dual-ROF / Dual-Huber-ROF: f = F, g = indicator of C, so the
    prox is P_C (prox of an indicator does not depend on the step)."""
    b = np.asarray(b, dtype=np.float64)
    q = np.zeros((b.ndim,) + b.shape)
    h = np.zeros_like(q)
    obj, coins = [], []
    n_prox = 0
    for k in range(K):
        q_hat = q - gamma * (_dual_rof_grad(q, b, alpha, eps) - h)
        theta = coin_mod.coin(seed, p, k)
        coins.append(theta)
        if theta:
            q_new = tv.project_ball(q_hat - (gamma / p) * h, alpha)
            n_prox += 1
        else:
            q_new = q_hat
        h = h + (p / gamma) * (q_new - q_hat)
        q = q_new
        if record:
            obj.append(dual_rof_objective(q, b, alpha, eps))
    return dict(q=q, h=h, u=b + tv.div(q), objective=obj, coins=coins, prox_calls=n_prox)
