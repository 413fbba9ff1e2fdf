"""Seeded synthetic inputs shared by the FP64 oracle tests, the GPU tests and the benchmark.

This module only draws random numbers and lays out regular grids of input values.  It holds none of the
method's arithmetic (no deposit, FFT, Poisson kernel, time integrals or ray updates), so the oracle and the
CUDA path can both be fed from it without sharing any computation.

Conventions (the same on both sides):
  * white noise is drawn with ``numpy.random.default_rng(seed).standard_normal`` in float64, shaped
    ``(n, n, n)`` with the last axis fastest; the GPU receives it cast to float32;
  * angles are in radians; image-plane arrays are row-major ``(M, M, 2)`` with the first axis the image
    y index and the second the image x index, flattened to ``(M*M, 2)`` as ``(theta_x, theta_y)``.
"""
from __future__ import annotations

import math

import numpy as np

ARCMIN = math.pi / (180.0 * 60.0)
DEGREE = math.pi / 180.0


def white_noise(seed: int, n_side: int) -> np.ndarray:
    """Unit-variance Gaussian white noise on an ``n_side**3`` lattice (float64, C order)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_side, n_side, n_side))


def pixel_grid(m: int, fov_rad: float) -> np.ndarray:
    """Pixel-centre angles of an ``m x m`` image of side ``fov_rad`` centred on the optical axis.

    Returns ``(m*m, 2)`` float64 ``(theta_x, theta_y)``; pixel ``(iy, ix)`` is row ``iy*m + ix``.
    """
    d = fov_rad / m
    c = (np.arange(m, dtype=np.float64) + 0.5 - 0.5 * m) * d
    ty, tx = np.meshgrid(c, c, indexing="ij")
    return np.stack([tx.ravel(), ty.ravel()], axis=1)


def polar_impact_grid(n_radial: int, n_azimuth: int, b_min_cells: float, b_max_cells: float,
                      cell: float, chi_lens: float) -> np.ndarray:
    """Ray angles on a polar grid whose impact parameters at ``chi_lens`` are log-uniform in cells.

    Radius ``i`` has ``b_i = b_min * (b_max/b_min)**(i/(n_radial-1))`` cells; azimuth ``j`` sits at
    ``(j + 1/2) * 2 pi / n_azimuth``.  Row ``i*n_azimuth + j`` holds ``(theta_x, theta_y)`` in radians.
    """
    i = np.arange(n_radial, dtype=np.float64)
    b = b_min_cells * (b_max_cells / b_min_cells) ** (i / (n_radial - 1)) * cell
    phi = (np.arange(n_azimuth, dtype=np.float64) + 0.5) * (2.0 * math.pi / n_azimuth)
    bb, pp = np.meshgrid(b, phi, indexing="ij")
    th = bb / chi_lens
    return np.stack([(th * np.cos(pp)).ravel(), (th * np.sin(pp)).ravel()], axis=1)


def uniform_positions(seed: int, n: int, box: float) -> np.ndarray:
    """``n`` positions uniform in ``[0, box)^3`` (float64, shape ``(n, 3)``)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, box, size=(n, 3))


def small_displacements(seed: int, n_side: int, scale: float) -> np.ndarray:
    """Gaussian displacements of rms ``scale`` for an ``n_side**3`` lattice, SoA ``(3, n_side**3)``."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((3, n_side ** 3))


def gaussian_field(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """A float64 Gaussian random array of the given shape (white, rms ``scale``)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(shape)


def complex_spectrum(seed: int, n_mesh: int, scale: float = 1.0) -> np.ndarray:
    """Random complex half spectrum ``(n, n, n//2+1)`` (complex128), as the input of a k-space kernel."""
    rng = np.random.default_rng(seed)
    shape = (n_mesh, n_mesh, n_mesh // 2 + 1)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def sample_indices(seed: int, n_total: int, n_sample: int) -> np.ndarray:
    """Sorted distinct indices in ``[0, n_total)`` for spot checks of large outputs."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, size=min(n_sample, n_total), replace=False))


def replica_transforms(seed: int, n_replicas: int, n_mesh: int):
    """Random proper axis rotations and whole-cell translations of the box replicas that tile a light cone.

    Returns (perm, sign, shift) int32 arrays of shape (n_replicas, 3): sky axis a of replica k maps to box axis
    perm[k, a] with sign sign[k, a] (det = +1: a rotation by multiples of 90 degrees), and box axis b is
    translated by shift[k, b] cells in [0, n_mesh)."""
    rng = np.random.default_rng(seed)
    perms = [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2)]
    parity = [1, 1, 1, -1, -1, -1]
    perm = np.zeros((n_replicas, 3), np.int32)
    sign = np.zeros((n_replicas, 3), np.int32)
    for k in range(n_replicas):
        i = int(rng.integers(len(perms)))
        s = rng.choice([-1, 1], size=2)
        perm[k] = perms[i]
        sign[k] = (s[0], s[1], parity[i] * s[0] * s[1])
    shift = rng.integers(0, n_mesh, size=(n_replicas, 3)).astype(np.int32)
    return perm, sign, shift
