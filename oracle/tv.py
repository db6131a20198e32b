"""Finite differences, divergence, isotropic TV and the TV prox (FP64 oracle).

Conventions (Eq. 5 and Section 2.1):
* ``grad(u)`` is the forward-difference operator D with Neumann boundary: component
  ``a`` differentiates along array axis ``a`` and is zero on the last slice of that
  axis.  For an image (H, W) the components are (D_y, D_x); a volume adds a third.
* ``div`` is the negative adjoint, div = -D^T (Section 2.1).
* TV(u) = sum over pixels of the Euclidean norm of (Du)_i (isotropic, Eq. 5).

The TV prox prox_{lam TV}(z) (Eq. 3 with R = TV) is computed on the dual: with
u = z + lam div p and |p_i| <= 1, the dual objective is 1/2 ||z + lam div p||^2,
whose gradient in p is -lam D u, with Lipschitz constant lam^2 ||D||^2 <= 8 lam^2
in 2D (12 lam^2 in 3D).  The projected gradient step is therefore
p <- P_B(p + D u / (8 lam)), the ProjGD iteration of Section 2.1 written for the
unit-ball dual p = q / lam, and its accelerated form (AProjGD, Section 2.2) adds the
FISTA momentum of Algorithm 3.  P_B projects each pixel's vector onto the unit ball,
the pointwise form of P_C in Eq. 7.
"""

from __future__ import annotations

import math

import numpy as np


def _sl(ndim, axis, s):
    out = [slice(None)] * ndim
    out[axis] = s
    return tuple(out)


def grad(u: np.ndarray) -> np.ndarray:
    """Forward differences with Neumann boundary; shape (u.ndim, *u.shape)."""
    u = np.asarray(u, dtype=np.float64)
    g = np.zeros((u.ndim,) + u.shape, dtype=np.float64)
    for a in range(u.ndim):
        g[a][_sl(u.ndim, a, slice(0, -1))] = (u[_sl(u.ndim, a, slice(1, None))]
                                              - u[_sl(u.ndim, a, slice(0, -1))])
    return g


def div(p: np.ndarray) -> np.ndarray:
    """Discrete divergence div = -D^T (Section 2.1).

    (div p)_i = sum_a ( p_a[i] * [i_a < n_a - 1] - p_a[i - e_a] * [i_a > 0] ).
    """
    p = np.asarray(p, dtype=np.float64)
    d = p.shape[0]
    out = np.zeros(p.shape[1:], dtype=np.float64)
    for a in range(d):
        q = p[a]
        out[_sl(d, a, slice(0, -1))] += q[_sl(d, a, slice(0, -1))]
        out[_sl(d, a, slice(1, None))] -= q[_sl(d, a, slice(0, -1))]
    return out


def tv(u: np.ndarray) -> float:
    """Isotropic total variation sum_i |(Du)_i|_2 (Eq. 5)."""
    g = grad(u)
    return float(np.sum(np.sqrt(np.sum(g * g, axis=0))))


def project_unit_ball(q: np.ndarray) -> np.ndarray:
    """Pointwise projection of each pixel's vector onto the unit Euclidean ball.

    q_i / max(1, |q_i|_2): Eq. 7 with the ball radius scaled to one.
    """
    nrm = np.sqrt(np.sum(q * q, axis=0))
    return q / np.maximum(1.0, nrm)[None]


def project_ball(q: np.ndarray, radius: float) -> np.ndarray:
    """P_C of Eq. 7 read as alpha * q_i / max(alpha, |q_i|_2)."""
    nrm = np.sqrt(np.sum(q * q, axis=0))
    return radius * q / np.maximum(radius, nrm)[None]


def dual_step_constant(ndim: int) -> float:
    """Upper bound 4 * ndim on ||D||^2 used as the dual Lipschitz constant."""
    return 4.0 * ndim


def _project_x(u, nonneg):
    return np.maximum(u, 0.0) if nonneg else u


def fgp_prox(z, lam, n_iter, p0=None, nonneg=False):
    """prox_{lam TV}(z) by ``n_iter`` accelerated dual projected-gradient iterations.

    This is the AProjGD inner solver run for a fixed number of iterations with a warm
    start (Section 3.1): ``p0`` is the dual returned by the previous call (zeros when
    None); the momentum restarts (t = 1) on every call.  With ``nonneg`` the primal
    candidate is clipped at zero (the non-negativity constraint of Section 3.3),
    u = max(z + lam div r, 0).

    Returns (u, p_N): u = P_X(z + lam div p_N) and the final dual field.
    """
    z = np.asarray(z, dtype=np.float64)
    d = z.ndim
    p = np.zeros((d,) + z.shape) if p0 is None else np.array(p0, dtype=np.float64)
    if lam == 0.0:
        return _project_x(z.copy(), nonneg), p
    L = dual_step_constant(d)
    r = p.copy()          # r_1 = p_0
    p_prev = p.copy()     # p_0
    t = 1.0               # t_1
    for _ in range(n_iter):
        u = _project_x(z + lam * div(r), nonneg)
        p_new = project_unit_ball(r + grad(u) / (L * lam))
        t_new = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        r = p_new + ((t - 1.0) / t_new) * (p_new - p_prev)
        p_prev = p_new
        t = t_new
    u = _project_x(z + lam * div(p_prev), nonneg)
    return u, p_prev


def projgd_prox(z, lam, n_iter, p0=None):
    """prox_{lam TV}(z) by plain dual projected gradient (ProjGD of Section 2.1).

    q_{k+1} = P_C(q_k + gamma D(div q_k + z)) with gamma = 1/8 (1/12 in 3D) on the
    lam-ball dual q = lam p, then u = z + div q.  Used only as a second, independent
    route to the same prox.
    """
    z = np.asarray(z, dtype=np.float64)
    d = z.ndim
    q = np.zeros((d,) + z.shape) if p0 is None else lam * np.array(p0, dtype=np.float64)
    gamma = 1.0 / dual_step_constant(d)
    for _ in range(n_iter):
        q = project_ball(q + gamma * grad(div(q) + z), lam)
    return z + div(q), q / lam if lam > 0 else q


def rof_primal(u, z, lam):
    """ROF primal 1/2 ||u - z||^2 + lam TV(u)."""
    return 0.5 * float(np.sum((u - z) ** 2)) + lam * tv(u)


def rof_dual(p, z, lam):
    """ROF dual value 1/2 ||z||^2 - 1/2 ||z + lam div p||^2 for |p_i| <= 1.

    (Eq. 6 up to the sign of its constant term, for the unit-ball dual.)
    """
    w = z + lam * div(p)
    return 0.5 * float(np.sum(z * z)) - 0.5 * float(np.sum(w * w))


def rof_gap(z, lam, p):
    """Duality gap P(u) - D(p) at u = z + lam div p (zero exactly at the optimum)."""
    u = z + lam * div(p)
    return rof_primal(u, z, lam) - rof_dual(p, z, lam)
