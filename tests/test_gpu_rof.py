"""GPU parity of the light-prox solvers (projected gradient, its accelerated form
AProjGD and ProxSkip on Dual-ROF / Dual-Huber-ROF) against the FP64 oracle."""

import numpy as np
import pytest

from oracle import solvers
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


def _b(shape, seed):
    return f32(phantoms.shapes_phantom_2d(shape[0], shape[1], 5, seed)
               + phantoms.gaussian_noise(shape, 0.05, seed + 1))


@pytest.mark.parametrize("shape,p,eps", [((37, 53), 1.0, 0.0), ((64, 96), 0.3, 0.0), ((50, 41), 0.1, 0.1),
                                         ((1, 17), 0.5, 0.0)])
def test_dual_rof_matches_oracle(tvs, ctx, shape, p, eps):
    import torch
    b32, b64 = _b(shape, 7) if min(shape) > 4 else f32(np.random.default_rng(1).standard_normal(shape))
    alpha, gamma, K, seed = 0.3, 1.0 / 8.0, 60, 9
    q = torch.zeros((2,) + shape, device="cuda")
    u = torch.empty(shape, device="cuda")
    q, u, tr = tvs.dual_rof_solve(ctx, cuda(b32), q, alpha, gamma, K, p=p, seed=seed, eps=eps, u=u)
    if p == 1.0:
        ref = solvers.dual_rof_projgd(b64, alpha, gamma, K, eps=eps)
    else:
        ref = solvers.dual_rof_proxskip(b64, alpha, gamma, p, seed, K, eps=eps)
    assert list(tr.coins) == list(ref["coins"])
    assert_close(host(q), ref["q"], TOL_X_F32)
    assert_close(host(u), ref["u"], TOL_X_F32)
    obj = np.asarray(ref["objective"])
    assert (np.abs(tr.objective - obj) / np.abs(obj)).max() <= TOL_OBJ


def test_dual_rof_host_buffers_and_invalid(tvs, ctx):
    b32, b64 = _b((20, 30), 3)
    q = np.zeros((2, 20, 30), dtype=np.float32)
    q, _, tr = tvs.dual_rof_solve(ctx, b32, q, 0.2, 0.125, 30, p=0.5, seed=2)
    ref = solvers.dual_rof_proxskip(b64, 0.2, 0.125, 0.5, 2, 30)
    assert_close(q, ref["q"], TOL_X_F32)
    with pytest.raises(tvs.TVSError):
        tvs.dual_rof_solve(ctx, b32, q, -0.2, 0.125, 30)


@pytest.mark.parametrize("shape,eps,K", [((37, 53), 0.0, 60), ((50, 41), 0.1, 75), ((1, 17), 0.0, 40),
                                         ((129, 67), 0.1, 7)])
def test_dual_rof_aprojgd_matches_oracle(tvs, ctx, shape, eps, K):
    """AProjGD (Section 2.2): the extrapolation coefficients of every iteration come
    from a device table through the recorded-iteration counter, over the three
    rotating dual buffers; iterates and every recorded objective against the oracle."""
    import torch
    b32, b64 = _b(shape, 8) if min(shape) > 4 else f32(np.random.default_rng(2).standard_normal(shape))
    alpha, gamma = 0.3, 1.0 / (8.0 + eps / 0.3)
    q = torch.zeros((2,) + shape, device="cuda")
    u = torch.empty(shape, device="cuda")
    q, u, tr = tvs.dual_rof_solve(ctx, cuda(b32), q, alpha, gamma, K, eps=eps, u=u, accelerated=True)
    ref = solvers.dual_rof_aprojgd(b64, alpha, gamma, K, eps=eps)
    assert tr.iters_run == K and tr.prox_calls == K
    assert_close(host(q), ref["q"], TOL_X_F32)
    assert_close(host(u), ref["u"], TOL_X_F32)
    obj = np.asarray(ref["objective"])
    assert (np.abs(tr.objective - obj) / np.abs(obj)).max() <= TOL_OBJ


def test_dual_rof_aprojgd_invalid_with_skipping(tvs, ctx):
    b32, _ = _b((20, 30), 3)
    q = np.zeros((2, 20, 30), dtype=np.float32)
    with pytest.raises(tvs.TVSError):
        tvs.dual_rof_solve(ctx, b32, q, 0.2, 0.125, 30, p=0.5, accelerated=True)


@pytest.mark.parametrize("p,accel", [(1.0, False), (0.3, False), (1.0, True)])
def test_dual_rof_reference_distance(tvs, ctx, p, accel):
    """With a reference u*, the trace records ||u_{k+1} - u*|| / ||u*|| for
    u = b + div q (the error measure of Sections 2.1-2.2), also on the iterations
    ProxSkip skips; and a distance target stops the solve."""
    import torch
    shape = (37, 53)
    b32, b64 = _b(shape, 12)
    alpha, gamma, K, seed = 0.3, 1.0 / 8.0, 25, 4
    u_ref32, u_ref64 = f32(b64 * 0.9 + 0.05)
    q = torch.zeros((2,) + shape, device="cuda")
    _, _, tr = tvs.dual_rof_solve(ctx, cuda(b32), q, alpha, gamma, K, p=p, seed=seed, accelerated=accel,
                                  u_ref=cuda(u_ref32))
    dist = []
    for k in range(1, K + 1):
        if accel:
            out = solvers.dual_rof_aprojgd(b64, alpha, gamma, k)
        elif p == 1.0:
            out = solvers.dual_rof_projgd(b64, alpha, gamma, k)
        else:
            out = solvers.dual_rof_proxskip(b64, alpha, gamma, p, seed, k)
        dist.append(np.linalg.norm(out["u"] - u_ref64) / np.linalg.norm(u_ref64))
    np.testing.assert_allclose(tr.rel_dist, dist, rtol=1e-5)
    target = dist[K // 2]
    q = torch.zeros((2,) + shape, device="cuda")
    _, _, tr2 = tvs.dual_rof_solve(ctx, cuda(b32), q, alpha, gamma, K, p=p, seed=seed, accelerated=accel,
                                   u_ref=cuda(u_ref32), target_dist=target * (1 + 1e-6))
    first = next(k for k, d in enumerate(dist) if d <= target * (1 + 1e-6))
    assert tr2.reached and tr2.reached_iter == first
