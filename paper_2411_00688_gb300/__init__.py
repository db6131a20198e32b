"""GB300-native ProxSkip / PDHGSkip-2 for TV-regularised imaging inverse problems.

The compute path is libtvs.so (CUDA for sm_103a behind the C ABI in
include/tvs.h); this package is its Python binding.  Importing the binding
loads the library and fails if it has not been built.
"""

from .api import (  # noqa: F401
    Context,
    Problem,
    dual_rof_solve,
    SolveTrace,
    fista_solve,
    pd_steps,
    pdhg_solve,
    pdhgskip1_solve,
    pdhg_explicit_solve,
    pdhgskip_solve,
    pgd_solve,
    proxskip_solve,
    proxskip_solve_batch,
    tv_prox,
    tv_prox_gap,
    tv_prox_noalloc,
    tvs_coin,
    tvs_coin_schedule_device,
    tvs_fgp_config,
    tvs_objective,
    tvs_op_apply,
)
from ._lib import LIB_PATH, TVSError, lib  # noqa: F401

lib()  # load now: no CPU fallback exists
