"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws random numbers and rasterises shapes; it contains none of the
solvers' arithmetic (no difference operators, no blur, no projector, no prox).
Measurements b = A u + noise are formed by the caller with its own operator A,
so the CUDA path and the oracle each apply their own A to the phantom drawn here.
"""

from .phantoms import (  # noqa: F401
    shapes_phantom_2d,
    ellipses_phantom_2d,
    ellipsoids_phantom_3d,
    gaussian_noise,
    poisson_counts,
    batch_problem_specs,
    rng,
)
from .configs import (  # noqa: F401
    DenoiseConfig,
    DeblurConfig,
    CTConfig,
    Denoise3DConfig,
    BatchConfig,
    CONFIGS,
)
