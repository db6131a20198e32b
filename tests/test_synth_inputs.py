"""The seeded synthetic inputs follow the recipe they state: sizes, value ranges,
the batch's size and parameter distributions, and determinism (CPU only)."""

import numpy as np
import pytest

from synth import configs, phantoms


def test_generators_are_deterministic():
    a = phantoms.shapes_phantom_2d(40, 50, 6, 7)
    b = phantoms.shapes_phantom_2d(40, 50, 6, 7)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, phantoms.shapes_phantom_2d(40, 50, 6, 8))
    np.testing.assert_array_equal(phantoms.gaussian_noise((9, 4), 0.3, 2), phantoms.gaussian_noise((9, 4), 0.3, 2))


@pytest.mark.parametrize("intensity", [(0.0, 1.0), (0.0, 0.5)])
def test_shapes_phantom_values_and_support(intensity):
    img = phantoms.shapes_phantom_2d(64, 96, 12, 3, intensity=intensity)
    assert img.shape == (64, 96) and img.dtype == np.float64
    vals = np.unique(img)
    assert vals.min() >= 0.0 and vals.max() <= intensity[1]
    assert len(vals) >= 2 and np.count_nonzero(img) > 0  # shapes painted over a zero background


def test_ellipses_and_ellipsoids_shapes():
    e2 = phantoms.ellipses_phantom_2d(32, 10, 4, intensity=(0.0, 0.5))
    assert e2.shape == (32, 32) and e2.min() >= 0.0 and e2.max() <= 0.5
    e3 = phantoms.ellipsoids_phantom_3d(16, 5, 5)
    assert e3.shape == (16, 16, 16) and e3.min() >= 0.0 and e3.max() <= 1.0


def test_gaussian_noise_moments():
    n = phantoms.gaussian_noise((400, 500), 0.1, 11)
    assert abs(n.mean()) < 5 * 0.1 / np.sqrt(n.size)
    assert abs(n.std() - 0.1) < 0.002


def test_poisson_counts_mean():
    lam = np.full((300, 300), 1e4)
    c = phantoms.poisson_counts(lam, 12)
    assert np.all(c == np.round(c)) and abs(c.mean() - 1e4) < 5 * np.sqrt(1e4 / c.size)


def test_batch_specs_follow_the_recipe():
    cfg = configs.BatchConfig()
    specs = cfg.specs()
    assert len(specs) == 256
    H = np.array([s["H"] for s in specs])
    W = np.array([s["W"] for s in specs])
    assert H.min() >= 64 and H.max() <= 1024 and W.min() >= 64 and W.max() <= 1024
    # log-uniform: log(side / 64) / log(16) is uniform on [0, 1] (KS test, 1 % level)
    from scipy import stats
    u = np.log(np.concatenate([H, W]) / 64.0) / np.log(16.0)
    assert stats.kstest(u, "uniform").pvalue > 0.01
    assert [s["kind"] for s in specs[:4]] == ["denoise", "deblur", "denoise", "deblur"]
    for s in specs:
        assert 0.01 <= s["alpha"] <= 0.2 and 0.05 <= s["p"] <= 0.5 and 1.0 <= s["blur_sigma"] <= 3.0
        assert s["seed"] == s["index"]
    assert specs == cfg.specs()  # same seed, same batch


def test_workload_configs_match_their_sizes():
    assert configs.DeblurConfig().phantom().shape == (1024, 1024)
    ct = configs.CTConfig()
    assert ct.pixel_size == 1.0 / 512 and (ct.n_angles, ct.n_det) == (720, 725)
    assert configs.DenoiseConfig().noise().shape == (256, 256)
