"""The five synthetic workloads (sizes, parameters and seeds).

Seeds follow 1000 * workload_number + role, role 0 = phantom, 1 = noise,
2 = sizes / per-problem parameters.  These records carry numbers only; the
measurement b is formed by whoever consumes them (see ``phantom_and_noise``).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import phantoms


@dataclass(frozen=True)
class DenoiseConfig:
    """2D TV denoising: 256x256, 12 rectangles/ellipses, noise 0.1, alpha 0.1."""
    name: str = "denoise2d_256"
    H: int = 256
    W: int = 256
    n_shapes: int = 12
    noise_sigma: float = 0.1
    alpha: float = 0.1
    gamma: float = 1.0
    p: float = 0.1
    seed: int = 0
    max_iter: int = 500
    n_inner: int = 100
    number: int = 1

    def phantom(self):
        return phantoms.shapes_phantom_2d(self.H, self.W, self.n_shapes, 1000 * self.number + 0)

    def noise(self):
        return phantoms.gaussian_noise((self.H, self.W), self.noise_sigma, 1000 * self.number + 1)


@dataclass(frozen=True)
class DeblurConfig:
    """2D TV deblurring: 1024x1024, 40 ellipses, 9x9 Gaussian sigma 2, noise 0.01."""
    name: str = "deblur2d_1024"
    H: int = 1024
    W: int = 1024
    n_ellipses: int = 40
    blur_sigma: float = 2.0
    blur_radius: int = 4
    noise_sigma: float = 0.01
    alpha: float = 0.02
    ps: tuple = (0.5, 0.1, 0.05)
    seed: int = 0
    max_iter: int = 1000
    n_inner: int = 50
    number: int = 2

    def phantom(self):
        return phantoms.ellipses_phantom_2d(self.H, self.n_ellipses, 1000 * self.number + 0, W=self.W)

    def noise(self):
        return phantoms.gaussian_noise((self.H, self.W), self.noise_sigma, 1000 * self.number + 1)


@dataclass(frozen=True)
class CTConfig:
    """2D parallel-beam CT: 512x512, 10 ellipses U[0,0.5], 720 angles, 725 bins.

    The image spans unit length (pixel size 1/N) and detector bins have the pixel
    width; 1e4 photons per ray.
    """
    name: str = "ct2d_512"
    N: int = 512
    n_ellipses: int = 10
    n_angles: int = 720
    n_det: int = 725
    photons: float = 1e4
    alpha: float = 0.5
    ps: tuple = (0.2, 0.05)
    seed: int = 0
    max_iter: int = 2000
    n_inner: int = 50
    number: int = 3

    @property
    def pixel_size(self):
        return 1.0 / self.N

    def phantom(self):
        return phantoms.ellipses_phantom_2d(self.N, self.n_ellipses, 1000 * self.number + 0,
                                            intensity=(0.0, 0.5))

    def counts(self, clean_sinogram):
        """Poisson photon counts for line integrals ``clean_sinogram``."""
        return phantoms.poisson_counts(self.photons * np.exp(-np.asarray(clean_sinogram)),
                                       1000 * self.number + 1)


@dataclass(frozen=True)
class Denoise3DConfig:
    """3D TV denoising: 512^3, 60 ellipsoids, noise 0.05, alpha 0.05."""
    name: str = "denoise3d_512"
    N: int = 512
    n_ellipsoids: int = 60
    noise_sigma: float = 0.05
    alpha: float = 0.05
    gamma: float = 1.0
    p: float = 0.1
    seed: int = 0
    max_iter: int = 200
    n_inner: int = 30
    number: int = 4

    def phantom(self):
        return phantoms.ellipsoids_phantom_3d(self.N, self.n_ellipsoids, 1000 * self.number + 0)

    def noise(self):
        return phantoms.gaussian_noise((self.N,) * 3, self.noise_sigma, 1000 * self.number + 1,
                                       dtype=np.float32)


@dataclass(frozen=True)
class BatchConfig:
    """256 independent 2D problems with log-uniform sides in [64, 1024]."""
    name: str = "batch2d_256"
    n_problems: int = 256
    lo: int = 64
    hi: int = 1024
    denoise_sigma: float = 0.1
    deblur_noise: float = 0.01
    max_iter: int = 200
    n_inner: int = 50
    number: int = 5
    specs_seed: int = field(default=5002)

    def specs(self):
        return phantoms.batch_problem_specs(self.n_problems, self.specs_seed, self.lo, self.hi)

    def phantom(self, spec):
        return phantoms.shapes_phantom_2d(spec["H"], spec["W"], 8, 5000 + 10 * spec["index"])

    def noise(self, spec):
        sigma = self.denoise_sigma if spec["kind"] == "denoise" else self.deblur_noise
        return phantoms.gaussian_noise((spec["H"], spec["W"]), sigma, 5001 + 10 * spec["index"])


CONFIGS = {
    "denoise2d_256": DenoiseConfig(),
    "deblur2d_1024": DeblurConfig(),
    "ct2d_512": CTConfig(),
    "denoise3d_512": Denoise3DConfig(),
    "batch2d_256": BatchConfig(),
}
