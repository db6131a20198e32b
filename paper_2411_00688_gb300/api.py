"""Python binding of the C ABI: argument marshalling only.

Every computation runs in libtvs.so.  Arrays may be torch CUDA tensors (device
pointers) or numpy float32 arrays (host pointers; the library copies them in and
out).  Functions keep the names of the C entry points.
"""

from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np

from . import _lib as L


def _torch():
    import torch  # imported lazily: host-only users need numpy only
    return torch


def _is_cuda_tensor(a) -> bool:
    try:
        torch = _torch()
    except ImportError:
        return False
    return isinstance(a, torch.Tensor) and a.is_cuda


def _sync_torch():
    torch = _torch()
    if torch.cuda.is_available():
        torch.cuda.current_stream().synchronize()


def _arr(a, what):
    """(pointer, mem kind, keep-alive object) for a float32 array."""
    if _is_cuda_tensor(a):
        torch = _torch()
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError(f"{what}: CUDA tensors must be contiguous float32")
        return a.data_ptr(), L.MEM_DEVICE, a
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise ValueError(f"{what}: numpy arrays must be C-contiguous float32")
        return a.ctypes.data, L.MEM_HOST, a
    raise TypeError(f"{what}: expected a CUDA tensor or a numpy float32 array")


class Context:
    """tvs_ctx on one device with a private stream."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        L.check(L.lib().tvs_create(C.byref(self._h), int(device), None))
        self.device = device

    @property
    def handle(self):
        return self._h

    def device_bytes(self) -> int:
        return int(L.lib().tvs_device_bytes(self._h))

    def close(self):
        if self._h:
            L.lib().tvs_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class SolveTrace:
    objective: np.ndarray
    coins: np.ndarray
    t_s: np.ndarray
    iters_run: int
    prox_calls: int
    reached: bool
    reached_iter: int
    time_to_target_s: float
    solve_ms: float
    fgp_ms: float
    fgp_launches: int
    fgp_pixel_iters: int
    rel_dist: np.ndarray


class _TraceBuffers:
    def __init__(self, cap):
        self.obj = np.full(cap, np.nan)
        self.coins = np.zeros(cap, dtype=np.uint8)
        self.ts = np.full(cap, np.nan)
        self.dist = np.full(cap, np.nan)


def _new_trace(cap):
    buf = _TraceBuffers(cap)
    tr = L.Trace()
    tr.cap = cap
    tr.objective = buf.obj.ctypes.data_as(C.POINTER(C.c_double))
    tr.coins = buf.coins.ctypes.data_as(C.POINTER(C.c_ubyte))
    tr.t_s = buf.ts.ctypes.data_as(C.POINTER(C.c_double))
    tr.rel_dist = buf.dist.ctypes.data_as(C.POINTER(C.c_double))
    return tr, buf


def _finish_trace(tr, buf):
    n = tr.iters_run
    return SolveTrace(buf.obj[:n].copy(), buf.coins[:n].copy(), buf.ts[:n].copy(), tr.iters_run, tr.prox_calls,
                      bool(tr.reached), tr.reached_iter, tr.time_to_target_s, tr.solve_ms, tr.fgp_ms,
                      tr.fgp_launches, tr.fgp_pixel_iters, buf.dist[:n].copy())


class Problem:
    """tvs_problem: min_u 1/2 ||A u - b||^2 + alpha TV(u) [+ u >= 0]."""

    def __init__(self, ctx: Context, b, alpha: float, op: str = "identity", shape=None,
                 nonneg: bool = False, blur_sigma: float = 2.0, blur_radius: int = 4,
                 n_angles: int = 0, n_det: int = 0, pixel_size: float = 0.0,
                 det_spacing: float = 0.0):
        self.ctx = ctx
        d = L.ProblemDesc()
        if op == "ct":
            if shape is None:
                raise ValueError("CT problems need the image shape")
            img_shape = tuple(shape)
        else:
            img_shape = tuple(b.shape) if shape is None else tuple(shape)
        self.shape = img_shape
        if len(img_shape) == 2:
            d.ndim, d.nz, d.ny, d.nx = 2, 1, img_shape[0], img_shape[1]
        elif len(img_shape) == 3:
            d.ndim, d.nz, d.ny, d.nx = 3, img_shape[0], img_shape[1], img_shape[2]
        else:
            raise ValueError("images are 2D or 3D")
        d.alpha = float(alpha)
        d.nonneg = int(bool(nonneg))
        kinds = {"identity": L.OP_IDENTITY, "blur": L.OP_GAUSS_BLUR, "ct": L.OP_PARALLEL_BEAM}
        d.op.kind = kinds[op]
        d.op.blur_radius = int(blur_radius)
        d.op.blur_sigma = float(blur_sigma)
        d.op.n_angles = int(n_angles)
        d.op.n_det = int(n_det)
        d.op.pixel_size = float(pixel_size)
        d.op.det_spacing = float(det_spacing)
        self.op = op
        self.alpha = float(alpha)
        self.meas_shape = (n_angles, n_det) if op == "ct" else img_shape
        self._desc = d
        ptr, mem, keep = _arr(b, "b")
        if mem == L.MEM_DEVICE:
            _sync_torch()
        self._h = C.c_void_p()
        L.check(L.lib().tvs_problem_create(ctx.handle, C.byref(d), C.c_void_p(ptr), mem, C.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def set_reference(self, u_ref):
        """Reference solution u*: solves then record ||x_k - u*|| / ||u*|| (None removes it)."""
        if u_ref is None:
            L.check(L.lib().tvs_problem_set_reference(self._h, None, L.MEM_DEVICE))
            return
        ptr, mem, keep = _arr(u_ref, "u_ref")
        if mem == L.MEM_DEVICE:
            _sync_torch()
        L.check(L.lib().tvs_problem_set_reference(self._h, C.c_void_p(ptr), mem))

    def set_data(self, b):
        ptr, mem, keep = _arr(b, "b")
        if mem == L.MEM_DEVICE:
            _sync_torch()
        L.check(L.lib().tvs_problem_set_data(self._h, C.c_void_p(ptr), mem))

    def close(self):
        # a closed context has already destroyed its problems
        if self._h and self.ctx.handle:
            L.lib().tvs_problem_destroy(self._h)
        self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tvs_op_apply(prob: Problem, x, y, adjoint: bool = False):
    """y = A x or A^T x (device tensors)."""
    _sync_torch()
    L.check(L.lib().tvs_op_apply(prob.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                 int(bool(adjoint))))
    return y


def tvs_objective(prob: Problem, x) -> float:
    _sync_torch()
    out = C.c_double()
    L.check(L.lib().tvs_objective(prob.handle, C.c_void_p(x.data_ptr()), C.byref(out)))
    return out.value


_DUAL_TORCH = {"f32": "float32", "bf16": "bfloat16", "f16": "float16", "q15": "int16"}


def _prox_args(z, u, dual, dual_state):
    """Checked C arguments of the TV-prox entry points: (dims, ndim, dual pointer).

    z and u: contiguous float32 CUDA tensors of one 2D (H, W) or 3D (D, H, W) shape
    on the current device; dual_state (optional): a contiguous tensor of the dual
    type with shape (ndim,) + z.shape on the same device."""
    torch = _torch()
    if dual not in L.DUAL:
        raise ValueError(f"dual must be one of {sorted(L.DUAL)}")
    for name, t in (("z", z), ("u", u)):
        if not _is_cuda_tensor(t) or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor")
    shape = tuple(z.shape)
    if len(shape) not in (2, 3):
        raise ValueError("z must be 2D or 3D")
    if tuple(u.shape) != shape:
        raise ValueError("u must have z's shape")
    dev = torch.cuda.current_device()
    if z.device.index != dev or u.device.index != dev:
        raise ValueError("z and u must be on the current CUDA device")
    ds = None
    if dual_state is not None:
        want = getattr(torch, _DUAL_TORCH[dual])
        if (not _is_cuda_tensor(dual_state) or dual_state.dtype != want or not dual_state.is_contiguous()
                or tuple(dual_state.shape) != (len(shape),) + shape or dual_state.device.index != dev):
            raise ValueError(f"dual_state: expected a contiguous {want} CUDA tensor of shape "
                             f"{(len(shape),) + shape} on the current device")
        ds = C.c_void_p(dual_state.data_ptr())
    dims = (C.c_int * 3)(*(list(reversed(shape)) + [1] * (3 - len(shape))))
    return dims, len(shape), ds


def tv_prox(ctx: Context, z, u, lam: float, n_iter: int, dual: str = "f32", dual_state=None,
            nonneg: bool = False):
    """u = prox_{lam TV}(z) on device tensors (2D (H, W) or 3D (D, H, W))."""
    dims, ndim, ds = _prox_args(z, u, dual, dual_state)
    _sync_torch()
    L.check(L.lib().tv_prox(ctx.handle, ndim, dims, C.c_void_p(z.data_ptr()),
                            C.c_void_p(u.data_ptr()), float(lam), int(n_iter), L.DUAL[dual], ds,
                            int(bool(nonneg))))
    return u


def tv_prox_gap(ctx: Context, z, lam: float, dual_state, dual: str = "f32") -> float:
    """ROF duality gap G = P(u) - D(p) of the dual p = dual_state (as tv_prox leaves
    it) for prox_{lam TV}(z), u = z + lam div p.  z and dual_state: CUDA tensors."""
    shape = tuple(z.shape)
    if len(shape) not in (2, 3):
        raise ValueError("z must be 2D or 3D")
    dims = (C.c_int * 3)(*(list(reversed(shape)) + [1] * (3 - len(shape))))
    _sync_torch()
    out = C.c_double()
    L.check(L.lib().tv_prox_gap(ctx.handle, len(shape), dims, C.c_void_p(z.data_ptr()), float(lam), L.DUAL[dual],
                                C.c_void_p(dual_state.data_ptr()), C.byref(out)))
    return out.value


def tvs_fgp_config(ctx: Context, shape, dual: str = "f32"):
    """(iterations per launch, columns per lane, rows per warp [+100 register-blocked])
    of the inner kernel the context uses for this image shape (autotuned once)."""
    if len(shape) == 2:
        dims = (C.c_int * 3)(shape[1], shape[0], 1)
    else:
        dims = (C.c_int * 3)(shape[2], shape[1], shape[0])
    out = (C.c_int * 3)()
    L.check(L.lib().tvs_fgp_config(ctx.handle, len(shape), dims, L.DUAL[dual], out))
    return tuple(out)


def tv_prox_noalloc(z, u, lam: float, n_iter: int, dual: str = "f32", dual_state=None,
                    nonneg: bool = False) -> int:
    """u = prox_{lam TV}(z) through the allocation-free entry point.

    For callers that may not allocate device memory: no context is used and the
    library allocates nothing (its working dual fields sit in a fixed device
    array of TVS_NOALLOC_SCRATCH_BYTES).  Runs on torch's current stream and
    returns the raw tvs_status (0 on success; 6 when the image needs more scratch
    than the fixed array holds).
    """
    torch = _torch()
    if z.data_ptr() == u.data_ptr():
        return L.TVS_EINVAL
    dims, ndim, ds = _prox_args(z, u, dual, dual_state)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return int(L.lib().tv_prox_noalloc(ndim, dims, C.c_void_p(z.data_ptr()), C.c_void_p(u.data_ptr()),
                                       float(lam), int(n_iter), L.DUAL[dual], ds, int(bool(nonneg)), stream))


def _fb(fn_name, prob, x, gamma, max_iter, n_inner, p=1.0, seed=0, dual="f32", f_star=0.0,
        target=0.0, every=1, resume=False, k0=0, target_dist=0.0):
    prm = L.FBParams(gamma=float(gamma), p=float(p), seed=int(seed) & ((1 << 64) - 1),
                     max_iter=int(max_iter), n_inner=int(n_inner), dual=L.DUAL[dual],
                     f_star=float(f_star), target_rel_gap=float(target), objective_every=int(every),
                     resume=int(bool(resume)), k0=int(k0), target_rel_dist=float(target_dist))
    ptr, mem, keep = _arr(x, "x")
    if mem == L.MEM_DEVICE:
        _sync_torch()
    tr, buf = _new_trace(max(int(max_iter), 1))
    L.check(getattr(L.lib(), fn_name)(prob.handle, C.byref(prm), C.c_void_p(ptr), mem, C.byref(tr)))
    return x, _finish_trace(tr, buf)


def pgd_solve(prob, x, gamma, max_iter, n_inner, **kw):
    """PGD (Algorithm 2); x holds x_0 on entry and the final iterate on return."""
    return _fb("pgd_solve", prob, x, gamma, max_iter, n_inner, **kw)


def fista_solve(prob, x, gamma, max_iter, n_inner, **kw):
    """FISTA (Algorithm 3)."""
    return _fb("fista_solve", prob, x, gamma, max_iter, n_inner, **kw)


def proxskip_solve(prob, x, gamma, p, seed, max_iter, n_inner, **kw):
    """ProxSkip (Algorithm 4)."""
    return _fb("proxskip_solve", prob, x, gamma, max_iter, n_inner, p=p, seed=seed, **kw)


def proxskip_solve_batch(ctx: Context, probs, xs, gammas, ps, seeds, max_iter, n_inner, dual="f32",
                         f_stars=None, targets=None):
    """ProxSkip on many independent problems in shared launches (proxskip_solve_batch).

    probs: list of Problem; xs: matching list of CUDA tensors (x_0 in, result out);
    gammas, ps, seeds (and optionally f_stars, targets): per-problem lists.
    Returns (xs, [SolveTrace])."""
    n = len(probs)
    prm = (L.FBParams * n)()
    for i in range(n):
        prm[i] = L.FBParams(gamma=float(gammas[i]), p=float(ps[i]), seed=int(seeds[i]) & ((1 << 64) - 1),
                            max_iter=int(max_iter), n_inner=int(n_inner), dual=L.DUAL[dual],
                            f_star=float(f_stars[i]) if f_stars is not None else 0.0,
                            target_rel_gap=float(targets[i]) if targets is not None else 0.0,
                            objective_every=1)
    mems = set()
    ptrs = (C.c_void_p * n)()
    keep = []
    for i, x in enumerate(xs):
        ptr, mem, k = _arr(x, f"x[{i}]")
        ptrs[i] = ptr
        mems.add(mem)
        keep.append(k)
    if len(mems) != 1:
        raise ValueError("all x must live in the same memory")
    mem = mems.pop()
    if mem == L.MEM_DEVICE:
        _sync_torch()
    handles = (C.c_void_p * n)(*[p.handle.value for p in probs])
    cap = max(int(max_iter), 1)
    tr = (L.Trace * n)()
    keep_tr = []
    for i in range(n):
        t, buf = _new_trace(cap)
        tr[i] = t
        keep_tr.append(buf)
    L.check(L.lib().proxskip_solve_batch(ctx.handle, n, handles, prm, ptrs, mem, tr))
    return xs, [_finish_trace(tr[i], keep_tr[i]) for i in range(n)]


def _pd(fn_name, prob, x, y, sigma, tau, max_iter, n_inner, p=1.0, seed=0, dual="f32", f_star=0.0,
        target=0.0, every=1, resume=False, k0=0, target_dist=0.0):
    prm = L.PDParams(sigma=float(sigma), tau=float(tau), p=float(p), seed=int(seed) & ((1 << 64) - 1),
                     max_iter=int(max_iter), n_inner=int(n_inner), dual=L.DUAL[dual],
                     f_star=float(f_star), target_rel_gap=float(target), objective_every=int(every),
                     resume=int(bool(resume)), k0=int(k0), target_rel_dist=float(target_dist))
    px, mem, kx = _arr(x, "x")
    py, mem_y, ky = _arr(y, "y")
    if mem != mem_y:
        raise ValueError("x and y must live in the same memory")
    if mem == L.MEM_DEVICE:
        _sync_torch()
    tr, buf = _new_trace(max(int(max_iter), 1))
    L.check(getattr(L.lib(), fn_name)(prob.handle, C.byref(prm), C.c_void_p(px), C.c_void_p(py), mem,
                                      C.byref(tr)))
    return x, y, _finish_trace(tr, buf)


def pdhg_solve(prob, x, y, sigma, tau, max_iter, n_inner, **kw):
    """Implicit PDHG (PDHGSkip-2 with p = 1)."""
    return _pd("pdhg_solve", prob, x, y, sigma, tau, max_iter, n_inner, **kw)


def pdhgskip_solve(prob, x, y, sigma, tau, p, seed, max_iter, n_inner, **kw):
    """PDHGSkip-2 (Algorithm 6)."""
    return _pd("pdhgskip_solve", prob, x, y, sigma, tau, max_iter, n_inner, p=p, seed=seed, **kw)


def pdhgskip1_solve(prob, x, y, sigma, tau, p, seed, max_iter, n_inner, **kw):
    """PDHGSkip-1 (Algorithm 5, omega + 1 = 1/p)."""
    return _pd("pdhgskip1_solve", prob, x, y, sigma, tau, max_iter, n_inner, p=p, seed=seed, **kw)


def pdhg_explicit_solve(prob, x, y, q=None, max_iter=100, sigma=1.0, tau=1.0, f_star=0.0, target=0.0,
                        every=1, target_dist=0.0):
    """Explicit PDHG with diagonal preconditioning (the explicit formulation of
    Section 3.2; the paper's solver for reference solutions).  x (image), y
    (measurement size) and the optional q (2, H, W) carry the iterates in and out."""
    prm = L.PDXParams(sigma=float(sigma), tau=float(tau), max_iter=int(max_iter), f_star=float(f_star),
                      target_rel_gap=float(target), objective_every=int(every),
                      target_rel_dist=float(target_dist))
    px, mem, kx = _arr(x, "x")
    py, mem_y, ky = _arr(y, "y")
    pq, mem_q = None, mem
    if q is not None:
        pq, mem_q, kq = _arr(q, "q")
    if len({mem, mem_y, mem_q}) != 1:
        raise ValueError("x, y and q must live in the same memory")
    if mem == L.MEM_DEVICE:
        _sync_torch()
    tr, buf = _new_trace(max(int(max_iter), 1))
    L.check(L.lib().pdhg_explicit_solve(prob.handle, C.byref(prm), C.c_void_p(px), C.c_void_p(py),
                                        C.c_void_p(pq) if pq is not None else None, mem, C.byref(tr)))
    return x, y, q, _finish_trace(tr, buf)


def dual_rof_solve(ctx: Context, b, q, alpha, gamma, max_iter, p=1.0, seed=0, eps=0.0, u=None,
                   f_star=0.0, target=0.0, accelerated=False, u_ref=None, target_dist=0.0):
    """Projected gradient (p = 1), AProjGD (p = 1, accelerated) or ProxSkip on
    Dual-ROF / Dual-Huber-ROF.

    b: image (H, W); q: dual field (2, H, W), initial value in, final out; u: optional
    output for b + div q; u_ref: optional reference solution (the trace then records
    ||u_k - u*|| / ||u*||, and target_dist > 0 stops on it).  All CUDA tensors or all
    numpy float32 arrays."""
    pr, mem_r = (None, None)
    if u_ref is not None:
        pr, mem_r, kr = _arr(u_ref, "u_ref")
    prm = L.RofParams(alpha=float(alpha), eps=float(eps), gamma=float(gamma), p=float(p),
                      seed=int(seed) & ((1 << 64) - 1), max_iter=int(max_iter), f_star=float(f_star),
                      target_rel_gap=float(target), accelerated=int(bool(accelerated)),
                      u_ref=C.c_void_p(pr) if pr is not None else None, target_rel_dist=float(target_dist))
    pb, mem, kb = _arr(b, "b")
    pq, mem_q, kq = _arr(q, "q")
    pu, mem_u = (None, mem)
    if u is not None:
        pu, mem_u, ku = _arr(u, "u")
    if len({mem, mem_q, mem_u} | ({mem_r} if mem_r is not None else set())) != 1:
        raise ValueError("b, q, u and u_ref must live in the same memory")
    if mem == L.MEM_DEVICE:
        _sync_torch()
    H, W = b.shape
    dims = (C.c_int * 2)(W, H)
    tr, buf = _new_trace(max(int(max_iter), 1))
    L.check(L.lib().dual_rof_solve(ctx.handle, dims, C.c_void_p(pb), C.byref(prm), C.c_void_p(pq),
                                   C.c_void_p(pu) if pu is not None else None, mem, C.byref(tr)))
    return q, u, _finish_trace(tr, buf)


def tvs_coin(seed: int, p: float, k: int) -> int:
    return int(L.lib().tvs_coin(int(seed) & ((1 << 64) - 1), float(p), int(k)))


def tvs_coin_schedule_device(ctx: Context, seed: int, p: float, k0: int, K: int) -> np.ndarray:
    out = np.zeros(int(K), dtype=np.uint8)
    L.check(L.lib().tvs_coin_schedule_device(ctx.handle, int(seed) & ((1 << 64) - 1), float(p),
                                             int(k0), int(K), out.ctypes.data_as(C.c_void_p)))
    return out


def gaussian_blur_norm_sq() -> float:
    """||A||^2 of the normalised, reflect-boundary Gaussian blur (exactly 1)."""
    return 1.0


def pd_steps(norm_A_sq: float, ratio: float = 1.0, safety: float = 0.99):
    """sigma, tau with sigma tau ||A||^2 = safety^2 (sigma / tau = ratio)."""
    nrm = math.sqrt(norm_A_sq)
    return safety * math.sqrt(ratio) / nrm, safety / (math.sqrt(ratio) * nrm)
