"""GPU parity of the forward operators, the objective and the coin."""

import math

import numpy as np
import pytest

from oracle import coin, operators, solvers
from synth import phantoms
from tests._util import cuda, f32, host, assert_close

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


@pytest.mark.parametrize("shape,sigma", [((1, 1), 2.0), ((5, 3), 1.0), ((37, 64), 2.0), ((1024, 1024), 2.0),
                                         ((130, 70), 2.9)])
def test_blur_matches_oracle(tvs, ctx, shape, sigma):
    import torch
    g = np.random.default_rng(0)
    x32, x64 = f32(g.standard_normal(shape))
    prob = tvs.Problem(ctx, x32, 0.0, op="blur", blur_sigma=sigma)
    xt = cuda(x32)
    yt = torch.empty_like(xt)
    tvs.tvs_op_apply(prob, xt, yt)
    ref = operators.blur(x64, operators.gaussian_weights(sigma, 4))
    assert_close(host(yt), ref, 1e-6)
    tvs.tvs_op_apply(prob, xt, yt, adjoint=True)
    assert_close(host(yt), operators.blur_adjoint(x64, operators.gaussian_weights(sigma, 4)), 1e-6)


@pytest.mark.parametrize("N,na,nd", [(16, 24, 23), (64, 90, 91), (31, 40, 45)])
def test_projector_matches_oracle(tvs, ctx, N, na, nd):
    import torch
    geom = operators.ParallelBeam.unit_square(N, na, nd)
    g = np.random.default_rng(1)
    x32, x64 = f32(g.standard_normal((N, N)))
    y32, y64 = f32(g.standard_normal((na, nd)))
    prob = tvs.Problem(ctx, y32, 0.0, op="ct", shape=(N, N), n_angles=na, n_det=nd,
                       pixel_size=1.0 / N, det_spacing=1.0 / N)
    xt, yt = cuda(x32), cuda(y32)
    ax = torch.empty_like(yt)
    aty = torch.empty_like(xt)
    tvs.tvs_op_apply(prob, xt, ax)
    tvs.tvs_op_apply(prob, yt, aty, adjoint=True)
    assert_close(host(ax), operators.joseph_forward(x64, geom), 1e-5)
    assert_close(host(aty), operators.joseph_adjoint(y64, geom), 1e-5)
    lhs = float(np.sum(host(ax) * y64))
    rhs = float(np.sum(x64 * host(aty)))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_projector_full_size(tvs, ctx):
    """512 x 512 image, 720 angles, 725 bins: the CT workload's projector."""
    import torch
    N, na, nd = 512, 720, 725
    geom = operators.ParallelBeam.unit_square(N, na, nd)
    x32, x64 = f32(phantoms.ellipses_phantom_2d(N, 10, 3000, intensity=(0.0, 0.5)))
    g = np.random.default_rng(2)
    y32, y64 = f32(g.standard_normal((na, nd)))
    prob = tvs.Problem(ctx, y32, 0.0, op="ct", shape=(N, N), n_angles=na, n_det=nd,
                       pixel_size=1.0 / N, det_spacing=1.0 / N)
    xt, yt = cuda(x32), cuda(y32)
    ax = torch.empty_like(yt)
    aty = torch.empty_like(xt)
    tvs.tvs_op_apply(prob, xt, ax)
    tvs.tvs_op_apply(prob, yt, aty, adjoint=True)
    assert_close(host(ax), operators.joseph_forward(x64, geom), 1e-5)
    # the adjoint at sampled pixels (the oracle's scatter is slow at full size):
    # compare through the dot test and a few pixels: (A^T y)_ij = <A e_ij, y>
    lhs = float(np.sum(host(ax) * y64))
    rhs = float(np.sum(x64 * host(aty)))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    at = host(aty)
    rng = np.random.default_rng(3)
    for _ in range(3):
        i, j = rng.integers(0, N, size=2)
        e = np.zeros((N, N))
        e[i, j] = 1.0
        col = operators.joseph_forward(e, geom)
        assert abs(at[i, j] - float(np.sum(col * y64))) <= 1e-4 * (1.0 + abs(at[i, j]))


@pytest.mark.parametrize("op", ["identity", "blur", "ct"])
def test_objective_matches_oracle(tvs, ctx, op):
    N = 48
    g = np.random.default_rng(4)
    x32, x64 = f32(phantoms.shapes_phantom_2d(N, N, 5, 9) + 0.05 * g.standard_normal((N, N)))
    if op == "ct":
        geom = operators.ParallelBeam.unit_square(N, 60, 69)
        A = operators.ct_op(geom)
        b32, b64 = f32(g.standard_normal((60, 69)) * 0.1)
        prob = tvs.Problem(ctx, b32, 0.07, op="ct", shape=(N, N), n_angles=60, n_det=69,
                           pixel_size=1.0 / N, det_spacing=1.0 / N)
    else:
        A = operators.identity_op() if op == "identity" else operators.blur_op(2.0)
        b32, b64 = f32(g.standard_normal((N, N)) * 0.1)
        prob = tvs.Problem(ctx, b32, 0.07, op=op, blur_sigma=2.0)
    ref = solvers.Problem(A, b64, 0.07, (N, N)).objective(x64)
    got = tvs.tvs_objective(prob, cuda(x32))
    assert abs(got - ref) <= 1e-6 * abs(ref)


def _fp32_terms_objective(x, b, alpha):
    """F(x) for A = I with every per-pixel term rounded to FP32 as the kernels form
    it (0.5 r^2 and sqrt(fma(dy, dy, dx^2))), summed exactly enough in FP64."""
    r = (x - b).astype(np.float32)
    data = (np.float32(0.5) * (r * r)).astype(np.float64)
    dy = np.zeros_like(x)
    dx = np.zeros_like(x)
    dy[:-1] = x[1:] - x[:-1]
    dx[:, :-1] = x[:, 1:] - x[:, :-1]
    dx2 = (dx * dx).astype(np.float32)
    inner = (dy.astype(np.float64) ** 2 + dx2.astype(np.float64)).astype(np.float32)
    tv = np.sqrt(inner).astype(np.float64)
    return math.fsum(data.ravel()) + alpha * math.fsum(tv.ravel())


def test_objective_sums_are_fp64_accurate(tvs, ctx):
    """The block partial sums (compensated FP32 pairs) and their final reduction
    reproduce the exactly summed FP32 terms of a 2000 x 3000 objective to 1e-11."""
    g = np.random.default_rng(12)
    x = g.standard_normal((2000, 3000)).astype(np.float32)
    b = (g.standard_normal((2000, 3000)) * 0.5).astype(np.float32)
    prob = tvs.Problem(ctx, cuda(b), 0.3)
    got = tvs.tvs_objective(prob, cuda(x))
    ref = _fp32_terms_objective(x, b, 0.3)
    assert abs(got - ref) <= 1e-11 * abs(ref)


def test_coin_host_and_device_match_oracle(tvs, ctx):
    for seed in [0, 1, 3, 2**40 + 7, 2**64 - 1, 123456789]:
        for p in (0.05, 0.1, 0.5, 1.0):
            ref = coin.schedule(seed, p, 2000)
            dev = tvs.tvs_coin_schedule_device(ctx, seed, p, 0, 2000)
            assert list(dev) == ref
            assert [tvs.tvs_coin(seed, p, k) for k in range(2000)] == ref
    assert list(tvs.tvs_coin_schedule_device(ctx, 9, 0.3, 10**12, 300)) == \
        [coin.coin(9, 0.3, 10**12 + k) for k in range(300)]
    assert tvs.tvs_coin(0, 0.0, 0) == -1 and tvs.tvs_coin(0, 1.5, 0) == -1


def test_nonfinite_measurement_rejected(tvs, ctx):
    b = np.zeros((8, 8), dtype=np.float32)
    b[3, 4] = np.nan
    with pytest.raises(tvs.TVSError) as e:
        tvs.Problem(ctx, b, 0.1)
    assert e.value.status == 4


@pytest.mark.parametrize("det_ratio", [0.6, 1.7])
def test_projector_other_detector_spacing(tvs, ctx, det_ratio):
    """Bins narrower / wider than a pixel: the backprojector's candidate window widens."""
    import torch
    N, na, nd = 24, 30, 41
    geom = operators.ParallelBeam(N, na, nd, 1.0 / N, det_ratio / N)
    g = np.random.default_rng(5)
    x32, x64 = f32(g.standard_normal((N, N)))
    y32, y64 = f32(g.standard_normal((na, nd)))
    prob = tvs.Problem(ctx, y32, 0.0, op="ct", shape=(N, N), n_angles=na, n_det=nd,
                       pixel_size=1.0 / N, det_spacing=det_ratio / N)
    xt, yt = cuda(x32), cuda(y32)
    ax = torch.empty_like(yt)
    aty = torch.empty_like(xt)
    tvs.tvs_op_apply(prob, xt, ax)
    tvs.tvs_op_apply(prob, yt, aty, adjoint=True)
    assert_close(host(ax), operators.joseph_forward(x64, geom), 1e-5)
    assert_close(host(aty), operators.joseph_adjoint(y64, geom), 1e-5)
