"""Seeded synthetic inputs shared by the oracle-side tests, the GPU tests and bench.py.

This module holds no NUFFT arithmetic: it only draws images, trajectories and
noise.  Every generator uses ``numpy.random.default_rng`` with a fixed seed
(image = 1, trajectory = 2, noise = 3) so both sides see the same bytes.
Trajectories are returned as float32 arrays of shape (M, d) in radians, with
column i paired with image axis i (C order); images are complex64 in C order.

Workloads (the paper measures on a 512^2 brain simulation and a 256^2
reconstruction, Section 2.3 / Section 4.2; those data are not available, so
these stand-ins keep the shapes and sampling structure):

* ``radial2d_uniform``: 2D radial, spokes at uniform angles pi*s/S.
* ``radial2d_golden``: 2D radial, golden-angle spoke increments (111.2461 deg).
* ``kooshball3d``: 3D radial, diameters along Fibonacci-lattice directions.
* ``spiral2d``: 2D Archimedean spiral interleaves (used by small tests only).
* ``ellipse_phantom``: piecewise-constant sum of ellipses (Shepp-Logan-like,
  own set of ellipses).
"""
from __future__ import annotations

import math

import numpy as np

SEED_IMAGE = 1
SEED_TRAJ = 2
SEED_NOISE = 3
SEED_COILS = 4

GOLDEN_ANGLE_DEG = 111.2461


def _rho(n_samples: int) -> np.ndarray:
    """Samples along a diameter, rho_i = -pi + 2*pi*i/n, i.e. covering [-pi, pi)."""
    return -math.pi + 2.0 * math.pi * np.arange(n_samples, dtype=np.float64) / n_samples


def radial2d_uniform(n_spokes: int, n_samples: int) -> np.ndarray:
    theta = math.pi * np.arange(n_spokes, dtype=np.float64) / n_spokes
    rho = _rho(n_samples)
    om = np.empty((n_spokes, n_samples, 2), dtype=np.float64)
    om[..., 0] = np.cos(theta)[:, None] * rho[None, :]
    om[..., 1] = np.sin(theta)[:, None] * rho[None, :]
    return om.reshape(-1, 2).astype(np.float32)


def radial2d_golden(n_spokes: int, n_samples: int, first_spoke: int = 0) -> np.ndarray:
    theta = np.deg2rad(GOLDEN_ANGLE_DEG) * (first_spoke + np.arange(n_spokes, dtype=np.float64))
    rho = _rho(n_samples)
    om = np.empty((n_spokes, n_samples, 2), dtype=np.float64)
    om[..., 0] = np.cos(theta)[:, None] * rho[None, :]
    om[..., 1] = np.sin(theta)[:, None] * rho[None, :]
    return om.reshape(-1, 2).astype(np.float32)


def fibonacci_directions(n: int) -> np.ndarray:
    """n unit vectors on the sphere from the Fibonacci lattice (z evenly spaced,
    azimuth advancing by the golden angle pi*(3 - sqrt 5))."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def kooshball3d(n_spokes: int, n_samples: int) -> np.ndarray:
    dirs = fibonacci_directions(n_spokes)
    rho = _rho(n_samples)
    om = dirs[:, None, :] * rho[None, :, None]
    return om.reshape(-1, 3).astype(np.float32)


def spiral2d(n_interleaves: int, n_samples: int, turns: float = 8.0) -> np.ndarray:
    """Archimedean spiral interleaves reaching |omega| = pi at the last sample."""
    tau = np.arange(n_samples, dtype=np.float64) / n_samples
    r = math.pi * tau
    om = np.empty((n_interleaves, n_samples, 2), dtype=np.float64)
    for q in range(n_interleaves):
        ang = 2.0 * math.pi * turns * tau + 2.0 * math.pi * q / n_interleaves
        om[q, :, 0] = r * np.cos(ang)
        om[q, :, 1] = r * np.sin(ang)
    return om.reshape(-1, 2).astype(np.float32)


def uniform_random_om(M: int, d: int, seed: int = SEED_TRAJ) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-math.pi, math.pi, size=(M, d)).astype(np.float32)


def complex_normal_image(shape, seed: int = SEED_IMAGE) -> np.ndarray:
    """Real and imaginary parts i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im).astype(np.complex64)


# (centre_x, centre_y, semi_axis_x, semi_axis_y, rotation_deg, value) in [-1, 1]^2
_ELLIPSES = (
    (0.00, 0.00, 0.72, 0.90, 0.0, 1.00),
    (0.00, -0.02, 0.66, 0.84, 0.0, -0.75),
    (0.24, 0.05, 0.12, 0.32, -15.0, -0.20),
    (-0.22, 0.05, 0.16, 0.40, 15.0, -0.20),
    (0.00, 0.38, 0.22, 0.24, 0.0, 0.15),
    (0.00, -0.55, 0.05, 0.04, 0.0, 0.12),
    (-0.10, -0.55, 0.04, 0.04, 0.0, 0.10),
    (0.08, -0.30, 0.05, 0.08, 30.0, 0.18),
)


def ellipse_phantom(n: int) -> np.ndarray:
    """Piecewise-constant n x n phantom (complex64, zero imaginary part)."""
    c = (np.arange(n, dtype=np.float64) - n / 2) / (n / 2)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    img = np.zeros((n, n), dtype=np.float64)
    for cx, cy, ax, ay, rot, val in _ELLIPSES:
        a = np.deg2rad(rot)
        u = (xx - cx) * np.cos(a) + (yy - cy) * np.sin(a)
        v = -(xx - cx) * np.sin(a) + (yy - cy) * np.cos(a)
        img[(u / ax) ** 2 + (v / ay) ** 2 <= 1.0] += val
    return img.astype(np.complex64)


def complex_noise(M: int, sigma: float, seed: int = SEED_NOISE) -> np.ndarray:
    """i.i.d. N(0, sigma^2) on real and imaginary parts."""
    rng = np.random.default_rng(seed)
    return (sigma * (rng.standard_normal(M) + 1j * rng.standard_normal(M))).astype(np.complex64)


def coil_maps(nc: int, Nd, seed: int = SEED_COILS) -> np.ndarray:
    """nc smooth complex coil sensitivities of image shape Nd (complex64):
    Gaussian windows (sigma = N/3) centred on a circle (2D; on a ring in the
    first two axes in 3D) with a random linear phase per coil."""
    rng = np.random.default_rng(seed)
    Nd = tuple(int(v) for v in Nd)
    grids = np.meshgrid(*[np.arange(N, dtype=np.float64) - N / 2 for N in Nd], indexing="ij")
    maps = np.empty((nc,) + Nd, dtype=np.complex64)
    R = 0.4 * min(Nd[:2])
    for i in range(nc):
        ang = 2 * math.pi * i / nc
        centre = [R * math.cos(ang), R * math.sin(ang)] + [0.0] * (len(Nd) - 2)
        r2 = sum((g - c) ** 2 for g, c in zip(grids, centre))
        sigma = min(Nd[:2]) / 3.0
        slope = rng.uniform(-0.05, 0.05, size=len(Nd))
        phase = sum(sl * g for sl, g in zip(slope, grids)) + rng.uniform(0, 2 * math.pi)
        maps[i] = (np.exp(-r2 / (2 * sigma * sigma)) * np.exp(1j * phase)).astype(np.complex64)
    return maps


def dynamic_radial_frames(n_frames: int = 8, n_samples: int = 512, lo: int = 13, hi: int = 89,
                          seed: int = SEED_TRAJ):
    """Golden-angle radial frames with uneven spoke counts drawn from U{lo..hi};
    the golden-angle sequence continues across frames.  Returns a list of
    float32 (M_f, 2) trajectories."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(lo, hi + 1, size=n_frames)
    frames, first = [], 0
    for c in counts:
        frames.append(radial2d_golden(int(c), n_samples, first_spoke=first))
        first += int(c)
    return frames


# ---- the named workloads -------------------------------------------------------

WORKLOADS = {
    # 2D 64x64 -> 128x128, J=6, 64 uniform spokes x 128 samples (8192 points)
    "radial2d_64": dict(d=2, Nd=(64, 64), Kd=(128, 128), Jd=(6, 6)),
    # 2D 256x256 -> 512x512, J=6, golden-angle 403 spokes x 512 samples (206,336 points)
    "radial2d_256": dict(d=2, Nd=(256, 256), Kd=(512, 512), Jd=(6, 6)),
    # 3D 128^3 -> 256^3, J=6, kooshball 8192 spokes x 256 samples (2,097,152 points)
    "kooshball3d_128": dict(d=3, Nd=(128, 128, 128), Kd=(256, 256, 256), Jd=(6, 6, 6)),
    # the same 2D radial workload on a 1.5x oversampled 384x384 grid (a size with a factor 3)
    "radial2d_256_K384": dict(d=2, Nd=(256, 256), Kd=(384, 384), Jd=(6, 6)),
    # 2D 256x256 -> 512x512, J=6, 16 spiral interleaves x 2048 samples, om + N(0, 1e-3) rad (32,768 points)
    "spiral2d_256": dict(d=2, Nd=(256, 256), Kd=(512, 512), Jd=(6, 6)),
}


def make_workload(name: str):
    """Return (spec dict, om float32 (M,d), x complex64 image, y_noise or None)."""
    spec = dict(WORKLOADS[name])
    if name == "radial2d_64":
        om = radial2d_uniform(64, 128)
        x = complex_normal_image(spec["Nd"])
        noise = None
    elif name in ("radial2d_256", "radial2d_256_K384"):
        om = radial2d_golden(403, 512)
        x = ellipse_phantom(256)
        noise = complex_noise(om.shape[0], 0.1)
    elif name == "kooshball3d_128":
        om = kooshball3d(8192, 256)
        x = complex_normal_image(spec["Nd"])
        noise = None
    elif name == "spiral2d_256":
        rng = np.random.default_rng(SEED_TRAJ)
        om = (spiral2d(16, 2048).astype(np.float64) + 1e-3 * rng.standard_normal((16 * 2048, 2))).astype(np.float32)
        x = ellipse_phantom(256)
        noise = complex_noise(om.shape[0], 0.1)
    else:  # pragma: no cover
        raise KeyError(name)
    spec["M"] = om.shape[0]
    return spec, om, x, noise
