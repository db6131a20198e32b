"""Helpers shared by the GPU parity tests (inputs, tolerances, comparisons)."""

import numpy as np

# Tolerances for the FP32 CUDA path against the FP64 oracle: final iterate
# <= 1e-4 relative l2, objective <= 1e-6 relative; with a bf16 / f16 dual field
# <= 2e-3 relative l2.
TOL_X_F32 = 1e-4
TOL_OBJ = 1e-6
TOL_X_HALF = 2e-3


# A result also has to meet the bound element by element: max |a - b| <= ELEM *
# tol * max |b|, so that an error confined to a few rows or columns (an image
# edge, a tile seam, a corner), which the l2 norm of a large image dilutes, is
# still caught.
ELEM = 10.0


def max_rel(a, b):
    """max |a - b| / max |b| (elementwise, relative to the largest reference value)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = np.abs(b).max() if b.size else 0.0
    return float(np.abs(a - b).max() / (m if m > 0 else 1.0)) if b.size else 0.0


def assert_close(a, b, tol, msg=None):
    """rel_l2(a, b) <= tol and max |a - b| <= ELEM * tol * max |b|."""
    r, e = rel_l2(a, b), max_rel(a, b)
    assert r <= tol, f"relative l2 {r:.3e} > {tol:.1e} {msg or ''}"
    assert e <= ELEM * tol, f"largest element error {e:.3e} of max |ref| > {ELEM * tol:.1e} {msg or ''}"


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def f32(a):
    """float32 copy of a, and the float64 view of those same values."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a32, a32.astype(np.float64)


def cuda(a32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)
