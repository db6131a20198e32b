"""Failure paths, made to fail on the host: no GPU fault, trap or hang is caused.

* TVS_FAULT_INJECT=alloc:N makes the N-th device allocation fail as if the device
  were out of memory (the library makes no CUDA call for it).  Every allocation of
  a problem's creation and of a prox call is failed in turn: the call returns
  TVS_ENOMEM, the context holds exactly the bytes it held before, and the same
  call succeeds once the injection is lifted.
* TVS_SOLVE_TIMEOUT_MS bounds a solve's host loop: a long solve stops at the limit
  and returns TVS_ETIMEDOUT, and the context stays usable.
"""

import os

import numpy as np
import pytest

from tests._util import cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tvs():
    import paper_2411_00688_gb300 as tvs
    return tvs


@pytest.fixture()
def clean_env():
    yield
    os.environ.pop("TVS_FAULT_INJECT", None)
    os.environ.pop("TVS_SOLVE_TIMEOUT_MS", None)


def _image(shape=(96, 80), seed=1):
    return np.random.default_rng(seed).random(shape).astype(np.float32)


@pytest.mark.parametrize("op", ["identity", "blur", "ct"])
def test_problem_creation_survives_every_failed_allocation(tvs, clean_env, op):
    ctx = tvs.Context(0)
    try:
        b = _image((48, 48)) if op != "ct" else _image((30, 70))
        kw = dict(op=op, blur_sigma=2.0)
        if op == "ct":
            kw.update(shape=(48, 48), n_angles=30, n_det=70, pixel_size=1 / 48, det_spacing=1 / 48)
        base = ctx.device_bytes()
        failures = 0
        for n in range(1, 60):
            os.environ["TVS_FAULT_INJECT"] = f"alloc:{n}"
            try:
                prob = tvs.Problem(ctx, cuda(b), 0.05, **kw)
            except tvs.TVSError as e:
                assert e.status == 2, e          # TVS_ENOMEM
                assert ctx.device_bytes() == base
                failures += 1
                continue
            # n is past the last allocation: creation succeeded
            prob.close()
            break
        else:
            pytest.fail("problem creation never got past the injected failures")
        assert failures >= 8
        os.environ.pop("TVS_FAULT_INJECT")
        prob = tvs.Problem(ctx, cuda(b), 0.05, **kw)
        prob.close()
        assert ctx.device_bytes() == base
    finally:
        ctx.close()


def test_prox_scratch_failure_then_success(tvs, clean_env):
    import torch
    ctx = tvs.Context(0)
    try:
        z = cuda(_image((128, 128)))
        u = torch.empty_like(z)
        base = ctx.device_bytes()
        os.environ["TVS_FAULT_INJECT"] = "alloc:1"
        with pytest.raises(tvs.TVSError) as ei:
            tvs.tv_prox(ctx, z, u, 0.1, 8)
        assert ei.value.status == 2
        assert ctx.device_bytes() == base
        os.environ.pop("TVS_FAULT_INJECT")
        tvs.tv_prox(ctx, z, u, 0.1, 8)
        assert torch.isfinite(u).all()
    finally:
        ctx.close()


@pytest.mark.parametrize("solver", ["proxskip", "pdhg", "pdhgskip1"])
def test_solve_time_limit(tvs, clean_env, solver):
    ctx = tvs.Context(0)
    try:
        b = cuda(_image((256, 256), 3))
        prob = tvs.Problem(ctx, b, 0.05, op="blur", blur_sigma=2.0)
        os.environ["TVS_SOLVE_TIMEOUT_MS"] = "5"
        with pytest.raises(tvs.TVSError) as ei:
            if solver == "proxskip":
                tvs.proxskip_solve(prob, b.clone(), 1.0, 0.5, 1, 200000, 20)
            elif solver == "pdhg":
                import torch
                tvs.pdhg_solve(prob, b.clone(), torch.zeros_like(b), 0.9, 0.9, 200000, 20)
            else:
                import torch
                tvs.pdhgskip1_solve(prob, b.clone(), torch.zeros_like(b), 0.9, 0.9, 0.5, 1, 200000, 20)
        assert ei.value.status == 5      # TVS_ETIMEDOUT
        os.environ.pop("TVS_SOLVE_TIMEOUT_MS")
        x, tr = tvs.proxskip_solve(prob, b.clone(), 1.0, 0.5, 1, 10, 5)
        assert tr.iters_run == 10
        prob.close()
    finally:
        ctx.close()
