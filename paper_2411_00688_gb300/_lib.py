"""ctypes declarations mirroring include/tvs.h and the loader of libtvs.so.

The library is built in-tree by ``paper_2411_00688_gb300.build`` (or
``__graft_entry__.build()``).  There is no fallback: if the library is missing or
fails to load, importing the binding raises.
"""

from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtvs.so")

TVS_OK, TVS_EINVAL, TVS_ENOMEM, TVS_ECUDA, TVS_ENUMERIC, TVS_ETIMEDOUT, TVS_EUNSUPPORTED = range(7)
STATUS_NAMES = {0: "TVS_OK", 1: "TVS_EINVAL", 2: "TVS_ENOMEM", 3: "TVS_ECUDA", 4: "TVS_ENUMERIC",
                5: "TVS_ETIMEDOUT", 6: "TVS_EUNSUPPORTED"}
OP_IDENTITY, OP_GAUSS_BLUR, OP_PARALLEL_BEAM = 0, 1, 2
DUAL = {"f32": 0, "bf16": 1, "f16": 2, "q15": 3}
MEM_DEVICE, MEM_HOST = 0, 1


class OpDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("blur_radius", C.c_int), ("blur_sigma", C.c_double),
                ("n_angles", C.c_int), ("n_det", C.c_int), ("pixel_size", C.c_double),
                ("det_spacing", C.c_double)]


class ProblemDesc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("alpha", C.c_double), ("nonneg", C.c_int), ("op", OpDesc)]


class FBParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("p", C.c_double), ("seed", C.c_uint64),
                ("max_iter", C.c_int), ("n_inner", C.c_int), ("dual", C.c_int),
                ("f_star", C.c_double), ("target_rel_gap", C.c_double),
                ("objective_every", C.c_int), ("resume", C.c_int), ("k0", C.c_longlong),
                ("target_rel_dist", C.c_double)]


class PDParams(C.Structure):
    _fields_ = [("sigma", C.c_double), ("tau", C.c_double), ("p", C.c_double),
                ("seed", C.c_uint64), ("max_iter", C.c_int), ("n_inner", C.c_int),
                ("dual", C.c_int), ("f_star", C.c_double), ("target_rel_gap", C.c_double),
                ("objective_every", C.c_int), ("resume", C.c_int), ("k0", C.c_longlong),
                ("target_rel_dist", C.c_double)]


class PDXParams(C.Structure):
    _fields_ = [("sigma", C.c_double), ("tau", C.c_double), ("max_iter", C.c_int),
                ("f_star", C.c_double), ("target_rel_gap", C.c_double),
                ("objective_every", C.c_int), ("target_rel_dist", C.c_double)]


class RofParams(C.Structure):
    _fields_ = [("alpha", C.c_double), ("eps", C.c_double), ("gamma", C.c_double), ("p", C.c_double),
                ("seed", C.c_uint64), ("max_iter", C.c_int), ("f_star", C.c_double),
                ("target_rel_gap", C.c_double), ("accelerated", C.c_int), ("u_ref", C.c_void_p),
                ("target_rel_dist", C.c_double)]


class Trace(C.Structure):
    _fields_ = [("cap", C.c_int), ("objective", C.POINTER(C.c_double)),
                ("coins", C.POINTER(C.c_ubyte)), ("t_s", C.POINTER(C.c_double)),
                ("iters_run", C.c_int), ("prox_calls", C.c_int), ("reached", C.c_int),
                ("reached_iter", C.c_int), ("time_to_target_s", C.c_double),
                ("solve_ms", C.c_double), ("fgp_ms", C.c_double),
                ("fgp_launches", C.c_longlong), ("fgp_pixel_iters", C.c_longlong),
                ("rel_dist", C.POINTER(C.c_double))]


# (name, restype, argtypes) of every entry point declared in include/tvs.h
SIGNATURES = [
    ("tvs_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    ("tvs_destroy", C.c_int, [C.c_void_p]),
    ("tvs_last_error", C.c_char_p, []),
    ("tvs_device_bytes", C.c_size_t, [C.c_void_p]),
    ("tvs_problem_create", C.c_int, [C.c_void_p, C.POINTER(ProblemDesc), C.c_void_p, C.c_int,
                                     C.POINTER(C.c_void_p)]),
    ("tvs_problem_set_reference", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("tvs_problem_set_data", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("tvs_problem_destroy", C.c_int, [C.c_void_p]),
    ("tvs_op_apply", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    ("tvs_objective", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    ("tv_prox", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_void_p,
                          C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    ("tv_prox_gap", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_double, C.c_int,
                              C.c_void_p, C.POINTER(C.c_double)]),
    ("tvs_fgp_config", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]),
    ("tv_prox_noalloc", C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_double,
                                  C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    ("pgd_solve", C.c_int, [C.c_void_p, C.POINTER(FBParams), C.c_void_p, C.c_int, C.POINTER(Trace)]),
    ("fista_solve", C.c_int, [C.c_void_p, C.POINTER(FBParams), C.c_void_p, C.c_int, C.POINTER(Trace)]),
    ("proxskip_solve", C.c_int, [C.c_void_p, C.POINTER(FBParams), C.c_void_p, C.c_int,
                                 C.POINTER(Trace)]),
    ("pdhg_solve", C.c_int, [C.c_void_p, C.POINTER(PDParams), C.c_void_p, C.c_void_p, C.c_int,
                             C.POINTER(Trace)]),
    ("pdhgskip_solve", C.c_int, [C.c_void_p, C.POINTER(PDParams), C.c_void_p, C.c_void_p, C.c_int,
                                 C.POINTER(Trace)]),
    ("pdhgskip1_solve", C.c_int, [C.c_void_p, C.POINTER(PDParams), C.c_void_p, C.c_void_p, C.c_int,
                                  C.POINTER(Trace)]),
    ("pdhg_explicit_solve", C.c_int, [C.c_void_p, C.POINTER(PDXParams), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_int, C.POINTER(Trace)]),
    ("proxskip_solve_batch", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(FBParams),
                                       C.POINTER(C.c_void_p), C.c_int, C.POINTER(Trace)]),
    ("dual_rof_solve", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_void_p, C.POINTER(RofParams), C.c_void_p,
                                 C.c_void_p, C.c_int, C.POINTER(Trace)]),
    ("tvs_coin", C.c_int, [C.c_uint64, C.c_double, C.c_int64]),
    ("tvs_coin_schedule_device", C.c_int, [C.c_void_p, C.c_uint64, C.c_double, C.c_int64, C.c_int,
                                           C.c_void_p]),
]


class TVSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libtvs.so not found at {path}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def check(status: int):
    if status != TVS_OK:
        raise TVSError(status, lib().tvs_last_error().decode(errors="replace"))
