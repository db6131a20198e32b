"""The allocation-free TV prox (tv_prox_noalloc) against tv_prox.

tv_prox_noalloc exists for callers that may not allocate device memory (an
application that reserves the GPU's memory for its own pool, or code running
beside a global-mode CUDA graph capture, where cudaMalloc is refused).  It keeps
its working dual fields in a fixed array inside the library image instead of
allocating them.  Here it is called through the C ABI several times in a row,
with different sizes so that anything left in the shared array by the previous
call would show, and each result is compared with the context-based tv_prox
within the FP32 tolerance the other parity tests use.  This file is collected
last so that a run stopping at its first failure has run every other test.
"""

import numpy as np
import pytest

from tests._util import TOL_X_F32, assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tvs():
    import paper_2411_00688_gb300 as tvs
    return tvs


def _image(shape, seed):
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return (torch.rand(shape, device="cuda", generator=g) > 0.5).float() + \
        0.2 * torch.randn(shape, device="cuda", generator=g)


def _reference(tvs, ctx, z, lam, n_iter, state=None):
    import torch
    u = torch.empty_like(z)
    tvs.tv_prox(ctx, z, u, lam, n_iter, dual_state=state)
    return u


def test_noalloc_matches_tv_prox_on_consecutive_calls(tvs):
    import torch
    ctx = tvs.Context(0)
    try:
        cases = [((300, 257), 0.15, 23), ((1024, 1024), 0.3, 50), ((17, 33, 40), 0.1, 9), ((300, 257), 0.05, 6)]
        for i, (shape, lam, n_iter) in enumerate(cases):
            z = _image(shape, 10 + i)
            ref = _reference(tvs, ctx, z, lam, n_iter)
            u = torch.full_like(z, float("nan"))
            assert tvs.tv_prox_noalloc(z, u, lam, n_iter) == 0
            torch.cuda.synchronize()
            assert_close(u.cpu().numpy(), ref.cpu().numpy(), TOL_X_F32, (shape, lam, n_iter))
    finally:
        ctx.close()


def test_noalloc_warm_start_two_calls(tvs):
    """Warm-started calls (the caller owns the dual field) agree call after call."""
    import torch
    ctx = tvs.Context(0)
    try:
        shape = (256, 320)
        z = _image(shape, 3)
        s_ref = torch.zeros((2,) + shape, device="cuda")
        s_new = torch.zeros((2,) + shape, device="cuda")
        for call in range(2):
            ref = _reference(tvs, ctx, z, 0.2, 13 + call, state=s_ref)
            u = torch.empty_like(z)
            assert tvs.tv_prox_noalloc(z, u, 0.2, 13 + call, dual_state=s_new) == 0
            torch.cuda.synchronize()
            assert_close(u.cpu().numpy(), ref.cpu().numpy(), TOL_X_F32)
            assert_close(s_new.cpu().numpy(), s_ref.cpu().numpy(), TOL_X_F32)
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_the_scratch(tvs):
    import torch
    z = torch.zeros((1025, 1024), device="cuda")
    u = torch.full_like(z, 7.0)
    assert tvs.tv_prox_noalloc(z, u, 0.1, 5) == 6          # TVS_EUNSUPPORTED
    torch.cuda.synchronize()
    assert bool((u == 7.0).all())                           # nothing was launched
    assert tvs.tv_prox_noalloc(z, z, 0.1, 5) == 1           # aliasing: TVS_EINVAL


def test_noalloc_leaves_device_memory_unchanged(tvs):
    """The property the entry point exists for: after its first call on a device
    (which places the static array there), further calls of several sizes, cold
    and warm-started, change the device's free memory by nothing.  A context-based
    tv_prox on a fresh context, the control, does allocate."""
    import torch
    shapes = [(512, 700), (1024, 1024), (9, 33, 40), (1, 1)]
    zs = [_image(s, 40 + i) for i, s in enumerate(shapes)]
    us = [torch.empty_like(z) for z in zs]
    state = torch.zeros((2,) + shapes[0], device="cuda")
    assert tvs.tv_prox_noalloc(zs[0], us[0], 0.1, 0) == 0           # first call: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for rep in range(2):
        for z, u in zip(zs, us):
            assert tvs.tv_prox_noalloc(z, u, 0.2, 11) == 0
        assert tvs.tv_prox_noalloc(zs[0], us[0], 0.2, 7, dual_state=state) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ctx = tvs.Context(0)
    try:
        u = torch.empty_like(zs[1])
        tvs.tv_prox(ctx, zs[1], u, 0.2, 11)
        torch.cuda.synchronize()
        free2, _ = torch.cuda.mem_get_info()
        assert free2 < free1 - 16 * 2 ** 20
    finally:
        ctx.close()
