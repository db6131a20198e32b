"""Power method for ||A||^2 = largest eigenvalue of A^T A (FP64 oracle).

Used to set step sizes: gamma = 1/L with L = ||A||^2 for the smooth data term of
Eq. 5 (Section 3.1) and sigma tau ||K||^2 <= 1 for PDHG (Section 3.3).
"""

from __future__ import annotations

import numpy as np


def power_method(apply_normal, shape, n_iter: int = 500, seed: int = 12345):
    """Rayleigh quotient of ``apply_normal`` (x -> A^T A x) after ``n_iter`` steps."""
    g = np.random.Generator(np.random.PCG64(seed))
    x = g.standard_normal(size=shape)
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(n_iter):
        y = apply_normal(x)
        lam = float(np.vdot(x, y).real)
        nrm = np.linalg.norm(y)
        if nrm == 0.0:
            return 0.0
        x = y / nrm
    return lam
