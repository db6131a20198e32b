"""GPU parity of the light-prox solvers (projected gradient and ProxSkip on
Dual-ROF / Dual-Huber-ROF) against the FP64 oracle."""

import numpy as np
import pytest

from oracle import solvers
from synth import phantoms
from tests._util import TOL_OBJ, TOL_X_F32, cuda, f32, host, rel_l2

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
    assert rel_l2(host(q), ref["q"]) <= TOL_X_F32
    assert rel_l2(host(u), ref["u"]) <= TOL_X_F32
    obj = np.asarray(ref["objective"])
    assert (np.abs(tr.objective - obj) / np.abs(obj)).max() <= TOL_OBJ


def test_dual_rof_host_buffers_and_invalid(tvs, ctx):
    b32, b64 = _b((20, 30), 3)
    q = np.zeros((2, 20, 30), dtype=np.float32)
    q, _, tr = tvs.dual_rof_solve(ctx, b32, q, 0.2, 0.125, 30, p=0.5, seed=2)
    ref = solvers.dual_rof_proxskip(b64, 0.2, 0.125, 0.5, 2, 30)
    assert rel_l2(q, ref["q"]) <= TOL_X_F32
    with pytest.raises(tvs.TVSError):
        tvs.dual_rof_solve(ctx, b32, q, -0.2, 0.125, 30)
