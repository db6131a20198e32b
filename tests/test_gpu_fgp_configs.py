"""Every inner-kernel configuration the autotuner or the environment can select
computes the same iterates: the 2D ones TVS_FGP_CONFIG forces per context (the
one-iteration kernel, the shared-memory blocked kernels and the register-blocked
ones, one and two columns per lane), and the 3D ones TVS_FGP3D_CFG / TVS_FGP3D
select per launch (z-marching variants with register loads or with TMA
staging, forced on volumes small enough that the automatic choice would take
the tiled kernel, and the tiled kernel).  The 3D shapes give the z-marching
variants CTAs whose region lies inside the volume and CTAs that meet each face;
the TMA variants run where the row pitch is a multiple of 16 bytes (the last two
shapes) and fall back to register loads elsewhere (the first).

With an FP32, BF16 or FP16 dual every configuration agrees with the reference
kernel bit for bit; with the 16-bit fixed point the blocked kernels keep each
iteration's rounded value in a register while the one-iteration kernel stores
and reloads it, so stored codes may differ by a few units after tens of
iterations (each code is 1/32767).  Each configuration also meets the oracle
bound (1e-4 relative l2 with FP32, 2e-3 with 16-bit storage) on its own.
"""

import os

import numpy as np
import pytest

from oracle import tv
from tests._util import TOL_X_F32, TOL_X_HALF, assert_close, cuda, f32, host

pytestmark = pytest.mark.gpu

CFG_2D = ["1", "2,2,4", "3,2,4", "4,2,4", "4,2,5", "4,1,5", "6,2,6", "8,2,6", "2,2,104", "4,1,105", "4,2,105",
          "4,2,108", "4,1,108", "6,2,108", "3,2,106", "4,2,104", "4,1,106", "5,2,104"]
CFG_3D = ["1,2,64", "1,4,64", "2,2,64", "1,2,32", "2,2,32", "2,4,32", "tma:1,2,64", "tma:1,2,32", "tma:1,4,64",
          "tma:2,2,64", "tma:2,2,32", "tma:2,4,32", "tma3:1,2,64", "tma3:2,2,32", "tile"]
DUALS = ["f32", "bf16", "f16", "q15"]
ENV_3D = ("TVS_FGP3D_CFG", "TVS_FGP3D", "TVS_FGP3D_STAGES")


@pytest.fixture(scope="module")
def tvs():
    import paper_2411_00688_gb300 as tvs
    return tvs


def _torch_dtype(dual):
    import torch
    return {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16, "q15": torch.int16}[dual]


def _inputs(shapes, seed):
    g = np.random.default_rng(seed)
    return [f32((g.random(s) > 0.5) + 0.2 * g.standard_normal(s)) for s in shapes]


def _run(tvs, ctx, z32, dual, n1, n2, lam):
    """A cold prox of n1 iterations, then one warm-started from its dual, of n2."""
    import torch
    z = cuda(z32)
    st = torch.zeros((z.ndim,) + tuple(z.shape), dtype=_torch_dtype(dual), device="cuda")
    u1, u2 = torch.empty_like(z), torch.empty_like(z)
    tvs.tv_prox(ctx, z, u1, lam, n1, dual=dual, dual_state=st)
    tvs.tv_prox(ctx, z + 0.01, u2, lam, n2, dual=dual, dual_state=st)
    # the stored dual as raw bits (numpy has no bfloat16)
    raw = st if dual == "f32" else st.view(torch.int16)
    return host(u1), host(u2), raw.cpu().numpy()


def _compare(runs, ref_key, dual):
    r1, r2, rst = runs[ref_key]
    for key, (u1, u2, st) in runs.items():
        if dual == "q15":
            assert np.abs(st.astype(np.int64) - rst.astype(np.int64)).max() <= 16, key
            assert np.abs(u1 - r1).max() <= 1e-3 and np.abs(u2 - r2).max() <= 1e-3, key
        else:
            np.testing.assert_array_equal(u1, r1, err_msg=str(key))
            np.testing.assert_array_equal(u2, r2, err_msg=str(key))
            np.testing.assert_array_equal(st, rst, err_msg=str(key))


@pytest.mark.parametrize("dual", DUALS)
def test_2d_configurations_agree(tvs, dual):
    shapes = [(67, 130), (256, 200), (9, 11), (130, 67)]
    zs = _inputs(shapes, 3)
    lam, n1, n2 = 0.15, 23, 10
    ref0 = tv.fgp_prox(zs[0][1], lam, n1)[0]
    runs = {}
    old = os.environ.get("TVS_FGP_CONFIG")
    try:
        for cfg in CFG_2D:
            os.environ["TVS_FGP_CONFIG"] = cfg
            ctx = tvs.Context(0)
            try:
                for si, (z32, _) in enumerate(zs):
                    runs[(cfg, si)] = _run(tvs, ctx, z32, dual, n1, n2, lam)
            finally:
                ctx.close()
            assert_close(runs[(cfg, 0)][0], ref0, TOL_X_F32 if dual == "f32" else TOL_X_HALF, cfg)
    finally:
        if old is None:
            os.environ.pop("TVS_FGP_CONFIG", None)
        else:
            os.environ["TVS_FGP_CONFIG"] = old
    for si in range(len(shapes)):
        _compare({k: v for k, v in runs.items() if k[1] == si}, ("1", si), dual)


@pytest.mark.parametrize("dual", DUALS)
def test_3d_variants_agree(tvs, dual):
    shapes = [(17, 33, 70), (5, 9, 40), (20, 100, 144)]
    zs = _inputs(shapes, 4)
    lam, n1, n2 = 0.1, 7, 4
    ref0 = tv.fgp_prox(zs[0][1], lam, n1)[0]
    runs = {}
    saved = {k: os.environ.get(k) for k in ENV_3D}
    ctx = tvs.Context(0)
    try:
        for var in ["default"] + CFG_3D:
            for k in ENV_3D:
                os.environ.pop(k, None)
            if var == "tile":
                os.environ["TVS_FGP3D"] = "tile"
            elif var.startswith("tma"):
                kind, cfg = var.split(":")
                os.environ["TVS_FGP3D"] = "tma"
                os.environ["TVS_FGP3D_CFG"] = cfg
                if kind == "tma3":
                    os.environ["TVS_FGP3D_STAGES"] = "3"
            elif var != "default":
                os.environ["TVS_FGP3D"] = "zm"
                os.environ["TVS_FGP3D_CFG"] = var
            for si, (z32, _) in enumerate(zs):
                runs[(var, si)] = _run(tvs, ctx, z32, dual, n1, n2, lam)
            assert_close(runs[(var, 0)][0], ref0, TOL_X_F32 if dual == "f32" else TOL_X_HALF, var)
    finally:
        ctx.close()
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    for si in range(len(shapes)):
        _compare({k: v for k, v in runs.items() if k[1] == si}, ("default", si), dual)
