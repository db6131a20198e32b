"""ctypes access to ``tvo.c``, the C transcription of the oracle (test and
measurement infrastructure only, like the rest of this package).

``tvo.c`` restates in plain FP64 C, with OpenMP over image rows, what ``tv.py``
(D, div, TV, the AProjGD TV prox), ``operators.py`` (the Gaussian blur and the
Joseph projector, each with its scattered adjoint) and ``solvers.py`` (PGD, FISTA,
ProxSkip, with the blur, the identity or the projector as A) compute; the tests in
``tests/test_oracle_c.py`` hold it to the numpy oracle at 1e-12.  It exists for the
full-size runs the numpy code is too slow for.  ``build()`` compiles it with gcc
into ``oracle/_build/<machine>/libtvo.so``.
"""

from __future__ import annotations

import ctypes as C
import os
import platform
import shutil
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tvo.c")
_LIB = os.path.join(_HERE, "_build", platform.machine(), "libtvo.so")
_lib = None

_D = C.POINTER(C.c_double)
_L = C.POINTER(C.c_long)


def build(force: bool = False) -> str:
    """Compile tvo.c (gcc, -O2, OpenMP, no floating-point contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the oracle's C transcription")
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp"
    subprocess.run([cc, "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.tvo_fgp_prox.argtypes = [C.c_int, _L, _D, C.c_double, C.c_int, _D, C.c_int, _D]
        _lib.tvo_fgp_prox.restype = C.c_int
        _lib.tvo_grad.argtypes = [C.c_int, _L, _D, _D]
        _lib.tvo_div.argtypes = [C.c_int, _L, _D, _D]
        _lib.tvo_tv.argtypes = [C.c_int, _L, _D, _D]
        _lib.tvo_tv.restype = C.c_double
        _lib.tvo_blur.argtypes = [C.c_long, C.c_long, _D, C.c_int, _D, _D, C.c_int]
        _lib.tvo_objective.argtypes = [C.c_int, _L, _D, C.c_int, _D, C.c_double, _D]
        _lib.tvo_objective.restype = C.c_double
        _lib.tvo_fb_solve.argtypes = [C.c_int, C.c_int, _L, _D, C.c_int, _D, C.c_double, C.c_int,
                                      C.c_double, C.c_double, C.POINTER(C.c_ubyte), C.c_int, C.c_int, _D,
                                      _D, _D, C.c_double, C.c_double, C.POINTER(C.c_int)]
        _lib.tvo_fb_solve.restype = C.c_int
        _lib.tvo_max_threads.restype = C.c_int
        _lib.tvo_joseph.argtypes = [C.c_long, C.c_long, C.c_long, C.c_double, C.c_double, _D, _D, C.c_int]
        _lib.tvo_ct_fb_solve.argtypes = [C.c_int, C.c_long, C.c_long, C.c_long, C.c_double, C.c_double, _D,
                                         C.c_double, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_ubyte),
                                         C.c_int, C.c_int, _D, _D, _D, C.c_double, C.c_double,
                                         C.POINTER(C.c_int)]
        _lib.tvo_ct_fb_solve.restype = C.c_int
        _lib.tvo_ct_pdhg.argtypes = [C.c_long, C.c_long, C.c_long, C.c_double, C.c_double, _D, C.c_double,
                                     C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, _D, _D, _D, _D]
        _lib.tvo_ct_pdhg.restype = C.c_int
    return _lib


def threads() -> int:
    """Threads the C transcription's OpenMP passes use."""
    return int(lib().tvo_max_threads())


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(_D)


def _shape(shape):
    return (C.c_long * len(shape))(*shape)


def grad(u):
    u = _f64(u)
    g = np.empty((u.ndim,) + u.shape)
    lib().tvo_grad(u.ndim, _shape(u.shape), _ptr(u), _ptr(g))
    return g


def div(p):
    p = _f64(p)
    out = np.empty(p.shape[1:])
    lib().tvo_div(p.shape[0], _shape(p.shape[1:]), _ptr(p), _ptr(out))
    return out


def tv(u):
    u = _f64(u)
    g = np.empty((u.ndim,) + u.shape)
    return float(lib().tvo_tv(u.ndim, _shape(u.shape), _ptr(u), _ptr(g)))


def fgp_prox(z, lam, n_iter, p0=None, nonneg=False):
    """As ``tv.fgp_prox``: (u, p_N)."""
    z = _f64(z)
    p = np.zeros((z.ndim,) + z.shape) if p0 is None else np.array(p0, dtype=np.float64, order="C")
    u = np.empty_like(z)
    if lib().tvo_fgp_prox(z.ndim, _shape(z.shape), _ptr(z), float(lam), int(n_iter), _ptr(p),
                          int(bool(nonneg)), _ptr(u)):
        raise MemoryError("tvo_fgp_prox")
    return u, p


def blur(u, w, adjoint=False):
    """A u (or A^T u) for the separable taps w, as ``operators.blur`` / ``blur_adjoint``."""
    u = _f64(u)
    w = _f64(w)
    out = np.empty_like(u)
    lib().tvo_blur(u.shape[0], u.shape[1], _ptr(w), (len(w) - 1) // 2, _ptr(u), _ptr(out), int(bool(adjoint)))
    return out


def joseph(u, geom, adjoint=False):
    """A u (sinogram, n_angles x n_det) or A^T y (image) for an ``operators.ParallelBeam``
    geometry, as ``operators.joseph_forward`` / ``joseph_adjoint``."""
    u = _f64(u)
    N, na, nd = geom.N, geom.n_angles, geom.n_det
    out = np.empty((N, N) if adjoint else (na, nd))
    lib().tvo_joseph(N, na, nd, float(geom.pixel_size), float(geom.det_spacing), _ptr(u), _ptr(out),
                     int(bool(adjoint)))
    return out


def objective(b, alpha, x, w=None):
    """1/2 ||A x - b||^2 + alpha TV(x), A the blur with taps w (identity when None)."""
    b, x = _f64(b), _f64(x)
    wa = _f64(w if w is not None else [1.0])
    R = 0 if w is None else (len(w) - 1) // 2
    return float(lib().tvo_objective(x.ndim, _shape(x.shape), _ptr(wa), R, _ptr(b), float(alpha), _ptr(x)))


_KIND = {"pgd": 0, "fista": 1, "proxskip": 2}


def fb_solve(kind, b, alpha, gamma, K, n_inner, x0=None, w=None, p=1.0, coins=None, nonneg=False,
             f_star=0.0, target=0.0, dual=None, record=True):
    """PGD / FISTA / ProxSkip on 1/2 ||A x - b||^2 + alpha TV(x) (A: blur taps w or the
    identity), as ``solvers.pgd`` / ``fista`` / ``proxskip``; ProxSkip takes its coins
    as a list.  With f_star > 0 the solve stops after the first iteration with
    (F - f_star)/f_star <= target.  Returns a dict like the numpy solvers' (plus
    ``iters_run``)."""
    b = _f64(b)
    x = _f64(b if x0 is None else x0).copy()
    wa = _f64(w if w is not None else [1.0])
    R = 0 if w is None else (len(w) - 1) // 2
    d = np.zeros((b.ndim,) + b.shape) if dual is None else np.array(dual, dtype=np.float64, order="C")
    c = np.ones(max(K, 1), dtype=np.uint8) if coins is None else np.ascontiguousarray(coins, dtype=np.uint8)
    obj = np.full(max(K, 1), np.nan)
    nprox = C.c_int(0)
    ran = lib().tvo_fb_solve(_KIND[kind], b.ndim, _shape(b.shape), _ptr(wa), R, _ptr(b), float(alpha),
                             int(bool(nonneg)), float(gamma), float(p), c.ctypes.data_as(C.POINTER(C.c_ubyte)),
                             int(K), int(n_inner), _ptr(x), _ptr(d), _ptr(obj) if record else None,
                             float(f_star), float(target), C.byref(nprox))
    if ran < 0:
        raise MemoryError("tvo_fb_solve")
    return dict(x=x, dual=d, objective=list(obj[:ran]) if record else [], coins=list(c[:ran]),
                prox_calls=int(nprox.value), iters_run=int(ran))


def ct_fb_solve(kind, b, alpha, gamma, K, n_inner, geom, x0=None, p=1.0, coins=None, nonneg=False,
                f_star=0.0, target=0.0, dual=None, record=True):
    """``fb_solve`` with A the parallel-beam projector of ``geom`` (b: the sinogram;
    x_0 = 0 unless given)."""
    b = _f64(b)
    N = geom.N
    x = np.zeros((N, N)) if x0 is None else _f64(x0).copy()
    d = np.zeros((2, N, N)) if dual is None else np.array(dual, dtype=np.float64, order="C")
    c = np.ones(max(K, 1), dtype=np.uint8) if coins is None else np.ascontiguousarray(coins, dtype=np.uint8)
    obj = np.full(max(K, 1), np.nan)
    nprox = C.c_int(0)
    ran = lib().tvo_ct_fb_solve(_KIND[kind], N, geom.n_angles, geom.n_det, float(geom.pixel_size),
                                float(geom.det_spacing), _ptr(b), float(alpha), int(bool(nonneg)), float(gamma),
                                float(p), c.ctypes.data_as(C.POINTER(C.c_ubyte)), int(K), int(n_inner), _ptr(x),
                                _ptr(d), _ptr(obj) if record else None, float(f_star), float(target),
                                C.byref(nprox))
    if ran < 0:
        raise MemoryError("tvo_ct_fb_solve")
    return dict(x=x, dual=d, objective=list(obj[:ran]) if record else [], coins=list(c[:ran]),
                prox_calls=int(nprox.value), iters_run=int(ran))


def ct_pdhg(b, alpha, sigma, tau, K, n_inner, geom, x0=None, y0=None, nonneg=False, record=True):
    """``solvers.pdhg`` with K the parallel-beam projector of ``geom`` (x_0 = 0 and
    y_0 = 0 unless given).  Returns a dict like the numpy solver's."""
    b = _f64(b)
    N = geom.N
    x = np.zeros((N, N)) if x0 is None else _f64(x0).copy()
    y = np.zeros(b.shape) if y0 is None else _f64(y0).copy()
    d = np.zeros((2, N, N))
    obj = np.full(max(K, 1), np.nan)
    ran = lib().tvo_ct_pdhg(N, geom.n_angles, geom.n_det, float(geom.pixel_size), float(geom.det_spacing),
                            _ptr(b), float(alpha), int(bool(nonneg)), float(sigma), float(tau), int(K),
                            int(n_inner), _ptr(x), _ptr(y), _ptr(d), _ptr(obj) if record else None)
    if ran < 0:
        raise MemoryError("tvo_ct_pdhg")
    return dict(x=x, y=y, dual=d, objective=list(obj[:ran]) if record else [], iters_run=int(ran))
