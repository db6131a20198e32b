"""GPU parity of the TV prox (fused FGP kernels) against the FP64 oracle."""

import numpy as np
import pytest

from oracle import tv
from synth import phantoms
from tests._util import TOL_X_F32, TOL_X_HALF, cuda, f32, host, assert_close

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


def _z(shape, seed):
    g = np.random.default_rng(seed)
    if len(shape) == 2 and min(shape) >= 8:
        base = phantoms.shapes_phantom_2d(shape[0], shape[1], 5, seed)
    else:
        base = np.zeros(shape)
    return base + 0.2 * g.standard_normal(shape)


def _run(tvs, ctx, z32, lam, n_iter, dual="f32", state=None, nonneg=False):
    import torch
    zt = cuda(z32)
    ut = torch.empty_like(zt)
    tvs.tv_prox(ctx, zt, ut, lam, n_iter, dual=dual, dual_state=state, nonneg=nonneg)
    return host(ut)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (2, 2), (33, 47), (100, 130), (256, 256)])
@pytest.mark.parametrize("lam,n_iter", [(0.05, 1), (0.3, 2), (0.15, 37)])
def test_prox_2d_cold(tvs, ctx, shape, lam, n_iter):
    z32, z64 = f32(_z(shape, 1))
    u_ref, _ = tv.fgp_prox(z64, lam, n_iter)
    u = _run(tvs, ctx, z32, lam, n_iter)
    assert_close(u, u_ref, TOL_X_F32)


@pytest.mark.parametrize("n_iter", [0, 3])
def test_prox_lambda_zero_and_no_iterations(tvs, ctx, n_iter):
    z32, z64 = f32(_z((19, 23), 2))
    np.testing.assert_array_equal(_run(tvs, ctx, z32, 0.0, n_iter), z64)
    if n_iter == 0:
        np.testing.assert_array_equal(_run(tvs, ctx, z32, 0.2, 0), z64)


def test_prox_2d_warm_start_and_nonneg(tvs, ctx):
    import torch
    shape = (70, 61)
    z32, z64 = f32(_z(shape, 3))
    lam = 0.2
    state = torch.zeros((2,) + shape, dtype=torch.float32, device="cuda")
    p_ref = None
    for call in range(3):
        u_ref, p_ref = tv.fgp_prox(z64, lam, 10 + call, p_ref)
        u = _run(tvs, ctx, z32, lam, 10 + call, state=state)
        assert_close(u, u_ref, TOL_X_F32)
        assert_close(host(state), p_ref, TOL_X_F32)
    u_ref, _ = tv.fgp_prox(z64 - 0.3, lam, 25, nonneg=True)
    z32b, _ = f32(z64 - 0.3)
    u = _run(tvs, ctx, z32b, lam, 25, nonneg=True)
    assert u.min() >= 0.0
    assert_close(u, u_ref, TOL_X_F32)


@pytest.mark.parametrize("dual", ["bf16", "f16", "q15"])
def test_prox_half_dual(tvs, ctx, dual):
    z32, z64 = f32(_z((128, 96), 4))
    u_ref, _ = tv.fgp_prox(z64, 0.1, 50)
    assert_close(_run(tvs, ctx, z32, 0.1, 50, dual=dual), u_ref, TOL_X_HALF)


@pytest.mark.parametrize("shape", [(9, 11), (96, 96), (33, 257), (5, 7, 9)])
@pytest.mark.parametrize("lam", [0.05, 0.5, 2.0, 4.0])
def test_prox_q15_dual_across_lambda(tvs, ctx, shape, lam):
    """The 16-bit fixed-point dual keeps the prox within the reduced-storage bound
    (2e-3 relative l2 of the FP64 oracle) over the prox steps lambda = gamma alpha / p
    of the batched workload (alpha in [0.01, 0.2], p in [0.05, 0.5]), cold and
    warm-started."""
    import torch
    z64 = _z(shape, 9)
    if len(shape) == 3:   # blocks on a background of 0.5: the prox does not collapse to ~0
        z64 = 0.5 + 0.2 * z64 + (np.indices(shape).sum(axis=0) % 7 > 3)
    z32, z64 = f32(z64)
    u_ref, p_ref = tv.fgp_prox(z64, lam, 50)
    state = torch.zeros((len(shape),) + shape, dtype=torch.int16, device="cuda")
    assert_close(_run(tvs, ctx, z32, lam, 50, dual="q15", state=state), u_ref, TOL_X_HALF)
    u_ref2, _ = tv.fgp_prox(z64 + 0.01, lam, 30, p_ref)
    z32b, _ = f32(z64 + 0.01)
    assert_close(_run(tvs, ctx, z32b, lam, 30, dual="q15", state=state), u_ref2, TOL_X_HALF)


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 4, 5), (17, 33, 40), (40, 9, 70)])
def test_prox_3d(tvs, ctx, shape):
    g = np.random.default_rng(5)
    z32, z64 = f32(g.standard_normal(shape))
    u_ref, _ = tv.fgp_prox(z64, 0.1, 12)
    assert_close(_run(tvs, ctx, z32, 0.1, 12), u_ref, TOL_X_F32)


def test_prox_full_size_2d(tvs, ctx):
    """1024 x 1024, 50 iterations (the deblurring workload's prox), whole image."""
    z32, z64 = f32(phantoms.ellipses_phantom_2d(1024, 40, 2000) + phantoms.gaussian_noise((1024, 1024), 0.05, 3))
    lam = 0.2
    u_ref, p_ref = tv.fgp_prox(z64, lam, 50)
    u = _run(tvs, ctx, z32, lam, 50)
    assert_close(u, u_ref, TOL_X_F32)
    assert abs(u.sum() - z64.sum()) <= 1e-5 * np.abs(z64).sum()


def test_prox_3d_properties_large(tvs, ctx):
    """256^3 volume: properties that hold at any size (mean preservation, and the
    ROF duality gap of the returned dual is small and non-negative), plus a
    128^3 sub-problem compared whole with the oracle."""
    import torch
    N = 256
    vol = phantoms.ellipsoids_phantom_3d(N, 20, 4000) + phantoms.gaussian_noise((N,) * 3, 0.05, 4001,
                                                                                  dtype=np.float32)
    z32 = np.ascontiguousarray(vol.astype(np.float32))
    zt = cuda(z32)
    ut = torch.empty_like(zt)
    state = torch.zeros((3,) + z32.shape, dtype=torch.float32, device="cuda")
    tvs.tv_prox(ctx, zt, ut, 0.05, 30, dual_state=state)
    u = ut.double()
    assert abs(u.sum().item() - zt.double().sum().item()) <= 1e-5 * zt.double().abs().sum().item()
    assert torch.sqrt((state.double() ** 2).sum(0)).max().item() <= 1.0 + 1e-6
    sub32 = np.ascontiguousarray(z32[:128, 64:192, 32:160])
    u_ref, _ = tv.fgp_prox(sub32.astype(np.float64), 0.05, 30)
    assert_close(_run(tvs, ctx, sub32, 0.05, 30), u_ref, TOL_X_F32)


def test_prox_invalid_arguments(tvs, ctx):
    import torch
    z = torch.zeros((8, 8), device="cuda")
    u = torch.zeros((8, 8), device="cuda")
    with pytest.raises(tvs.TVSError):
        tvs.tv_prox(ctx, z, u, -1.0, 5)
    with pytest.raises(tvs.TVSError):
        tvs.tv_prox(ctx, z, u, float("nan"), 5)
    with pytest.raises(tvs.TVSError):
        tvs.tv_prox(ctx, z, z, 0.1, 5)


@pytest.mark.parametrize("shape,dual", [((130, 97), "f32"), ((20, 33, 17), "f32"), ((130, 97), "bf16"),
                                        ((130, 97), "q15")])
def test_prox_gap_matches_oracle(tvs, ctx, shape, dual):
    """The ROF duality gap of the dual tv_prox leaves equals the oracle's P(u) - D(p)
    on the same dual, is non-negative and shrinks as the prox converges (with a
    reduced dual the rounded |p_i| may exceed 1 by an ulp, so only the first two
    checks apply there, and the gap levels off at the storage precision)."""
    import torch
    z32, z64 = f32(_z(shape, 7))
    lam = 0.2
    zt = cuda(z32)
    ut = torch.empty_like(zt)
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "q15": torch.int16}[dual]
    state = torch.zeros((len(shape),) + shape, dtype=dt, device="cuda")
    gaps = []
    for n_iter in (3, 30, 300):
        state.zero_()
        tvs.tv_prox(ctx, zt, ut, lam, n_iter, dual=dual, dual_state=state)
        g = tvs.tv_prox_gap(ctx, zt, lam, state, dual=dual)
        if dual == "q15":   # the fixed-point code i stands for i * float32(1/32767)
            p64 = (state.cpu().numpy().astype(np.float32) * np.float32(1.0 / 32767.0)).astype(np.float64)
        else:
            p64 = state.float().cpu().numpy().astype(np.float64)
        ref = tv.rof_gap(z64, lam, p64)
        if dual == "f32":
            assert g >= 0.0
        # FP32 evaluation of u = z + lam div p: absolute error ~ n * lam * 1e-7 * |D u|
        assert abs(g - ref) <= 1e-4 * ref + 1e-6 * z64.size * lam, (n_iter, g, ref)
        gaps.append(g)
    assert gaps[1] < gaps[0]
    if dual == "f32":
        assert gaps[2] < gaps[1]


def test_prox_3d_full_size_sampled(tvs, ctx):
    """512^3, the 3D denoising workload's size, in the launch configuration of its
    solves (z-marching kernel): 4 inner iterations, sampled voxels compared with
    the oracle run on a 15^3 crop around each (after N iterations u at a voxel
    depends on z within N + 2 voxels, so a crop of radius N + 3, clipped at the
    volume's own faces, reproduces it)."""
    import torch
    N, n_iter, lam, rad = 512, 4, 0.05, 7
    g = np.random.default_rng(11)
    z32 = g.standard_normal((N, N, N), dtype=np.float32)
    z32[100:300, 50:400, 200:500] += 1.0
    zt = cuda(z32)
    ut = torch.empty_like(zt)
    tvs.tv_prox(ctx, zt, ut, lam, n_iter)
    samples = [(0, 0, 0), (511, 511, 511), (0, 255, 300), (137, 13, 0), (255, 255, 255), (400, 511, 29),
               (63, 64, 65), (99, 301, 199), (300, 49, 500), (511, 0, 256)]
    for (k, i, j) in samples:
        lo = [max(0, c - rad) for c in (k, i, j)]
        hi = [min(N, c + rad + 1) for c in (k, i, j)]
        crop = z32[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]].astype(np.float64)
        u_ref, _ = tv.fgp_prox(crop, lam, n_iter)
        ref = u_ref[k - lo[0], i - lo[1], j - lo[2]]
        got = float(ut[k, i, j].item())
        assert abs(got - ref) <= 1e-5 * (1.0 + abs(ref)), ((k, i, j), got, ref)
