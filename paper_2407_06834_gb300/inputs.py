"""Seeded synthetic inputs and the workload table.

This module holds no arithmetic of the method (no kernel sums, no NFFT, no
solver).  It only draws the synthetic images that stand in for the paper's
photographs (Sec. 5.1 uses scikit-image samples and private photos, which are
not reproduced here) and lists the workloads.  Both the CUDA path and the CPU
oracle receive its arrays as plain inputs.

Image recipe (seeded NumPy PCG64):
  * pixel coordinates (x, y) in [0, 1]^2, x along columns, y along rows;
  * background ramp a0 + a1 x + a2 y, a0 ~ U[0.2, 0.4], a1, a2 ~ U[-0.2, 0.2];
  * 4 discs, then 4 axis-aligned rectangles, painted in that order; centre
    ~ U[0,1]^2, radius / half-size ~ U[0.05, 0.25], intensity ~ U[0, 1];
  * clean image clipped to [0, 1];
  * noisy f = clean + N(0, 0.1^2), not clipped (Sec. 5 adds the noise h to the
    clean image without clipping).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

NOISE_STD = 0.1


def synthetic_image(n1: int, n2: int, seed: int, noise_std: float = NOISE_STD
                    ) -> Tuple[np.ndarray, np.ndarray]:
    """Return (clean, noisy), both float64 arrays of shape (n1, n2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    y = (np.arange(n1, dtype=np.float64) + 0.5) / n1
    x = (np.arange(n2, dtype=np.float64) + 0.5) / n2
    X, Y = np.meshgrid(x, y)
    a0 = rng.uniform(0.2, 0.4)
    a1, a2 = rng.uniform(-0.2, 0.2, size=2)
    img = a0 + a1 * X + a2 * Y
    for _ in range(4):
        cx, cy = rng.uniform(0.0, 1.0, size=2)
        r = rng.uniform(0.05, 0.25)
        val = rng.uniform(0.0, 1.0)
        img[(X - cx) ** 2 + (Y - cy) ** 2 <= r * r] = val
    for _ in range(4):
        cx, cy = rng.uniform(0.0, 1.0, size=2)
        hx, hy = rng.uniform(0.05, 0.25, size=2)
        val = rng.uniform(0.0, 1.0)
        img[(np.abs(X - cx) <= hx) & (np.abs(Y - cy) <= hy)] = val
    clean = np.clip(img, 0.0, 1.0)
    noisy = clean + rng.normal(0.0, noise_std, size=clean.shape)
    return clean, noisy


def raster_windows(radius: int) -> np.ndarray:
    """Feature windows as consecutive raster-order triples of patch dims.

    A patch of radius rho has D = (2 rho + 1)^2 dims, numbered in raster order
    (row offset major).  Window l holds dims {3l, 3l+1, 3l+2}; the last window
    is completed with -1 entries (a zero-valued dimension).  Returns an int32
    array of shape (L, 3) with L = ceil(D / 3), the window count of Sec. 5.
    """
    D = (2 * radius + 1) ** 2
    L = -(-D // 3)
    w = np.full((L, 3), -1, dtype=np.int32)
    for d in range(D):
        w[d // 3, d % 3] = d
    return w


def random_vector(n: int, seed: int) -> np.ndarray:
    """A seeded standard-normal float64 vector (test right-hand sides)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n)


@dataclass
class Workload:
    """One named workload: image size, features, kernel and NFFT parameters."""
    name: str
    n1: int
    n2: int
    seed: int = 0
    radius: int = 1                 # patch radius rho: 3x3 patches
    pad: str = "reflect"            # "reflect" or "zero"
    sigma: float = 0.2              # kernel width, exp(-||.||^2 / sigma^2)
    alpha: float = 0.5              # lambda / mu with mu = 1
    M: int = 32                     # bandwidth per dim
    n_os: int = 64                  # oversampled FFT grid per dim
    m: int = 4                      # window half-width in grid cells
    torus_fill: float = 0.0         # 0 = automatic choice
    tol: float = 1e-6
    sigmas: Optional[List[float]] = None

    @property
    def N(self) -> int:
        return self.n1 * self.n2

    @property
    def windows(self) -> np.ndarray:
        return raster_windows(self.radius)

    @property
    def L(self) -> int:
        return int(self.windows.shape[0])

    def image(self) -> np.ndarray:
        return synthetic_image(self.n1, self.n2, self.seed)[1]


# The workloads: 64^2 (oracle-sized), 512^2 with 3x3 patches and 3 windows,
# 2048^2 with 5x5 patches and 9 windows (the timed one), and 1024^2 with the
# 2048^2 workload's patches and NFFT parameters (the same kernel
# instantiations on a quarter of the points, for multi-pass profiles).
WORKLOADS = {
    "img64": Workload("img64", 64, 64),
    "img512": Workload("img512", 512, 512),
    "img1024": Workload("img1024", 1024, 1024, radius=2, M=64, n_os=128, m=6),
    "img2048": Workload("img2048", 2048, 2048, radius=2, M=64, n_os=128, m=6,
                        sigmas=[0.1, 0.2, 0.4]),
}

# Uneven image sizes of the batched (sigma, alpha) sweep: 64 solves over a
# log grid of 8 sigmas in [0.05, 1] and 8 alphas in [0.01, 10]; pair (i, j)
# goes to image (i + j) mod 8.
SWEEP_SIZES = [256, 384, 512, 768, 1024, 320, 640, 896]


def sweep_pairs():
    sig = np.geomspace(0.05, 1.0, 8)
    alp = np.geomspace(0.01, 10.0, 8)
    out = []
    for i in range(8):
        for j in range(8):
            out.append(((i + j) % 8, float(sig[i]), float(alp[j])))
    return out


# ---- learned warm start: seeded training / evaluation draws --------------

def net_init(shapes, seed: int) -> np.ndarray:
    """Initial parameters of a convolutional network, flat float32.

    shapes: (cout, k, cin) per layer, in parameter order; each layer's
    weights [cout][k][k][cin] are drawn N(0, 2 / (k k cin)) (He et al. 2015),
    its biases are zero.  The last layer (the linear head) is drawn 100x
    smaller, so that the network starts close to u0 = f, c = 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for i, (cout, k, cin) in enumerate(shapes):
        std = np.sqrt(2.0 / (k * k * cin))
        if i == len(shapes) - 1:
            std *= 0.01
        parts.append(rng.normal(0.0, std, size=cout * k * k * cin))
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)


def learned_draws(count: int, seed: int, sigma_range=(0.05, 1.0), alpha_range=(0.01, 10.0)):
    """(image seed, sigma, alpha) triples, sigma and alpha log-uniform over
    the bilevel search ranges; image seeds start at 1000 * (seed + 1) so the
    training images differ from the workload images (seed 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ls = rng.uniform(np.log(sigma_range[0]), np.log(sigma_range[1]), size=count)
    la = rng.uniform(np.log(alpha_range[0]), np.log(alpha_range[1]), size=count)
    base = 1000 * (seed + 1)
    return [(base + i, float(np.exp(s)), float(np.exp(a))) for i, (s, a) in enumerate(zip(ls, la))]
