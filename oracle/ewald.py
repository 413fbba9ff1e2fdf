"""Periodic point-mass fields by Ewald summation (test infrastructure only).

Used to pin the oracle's PM force and its point-mass lensing against sums that involve no mesh and no FFT:

  * 3D: the gradient of the potential of a unit point mass in a periodic cube of side L with a uniform
    neutralising background (what an FFT Poisson solve with the k = 0 mode removed computes),
      grad phi / (G M) = sum_n (r_n / |r_n|^3) [erfc(al |r_n|) + 2 al |r_n| exp(-al^2 |r_n|^2) / sqrt(pi)]
                       + (4 pi / L^3) sum_{k != 0} (k / k^2) exp(-k^2 / (4 al^2)) sin(k . r),   r_n = r - n L;
  * 2D: the lensing sum of the periodic point-mass images of Appendix D (Eq. "pointmass_periodic"),
    sum_m (b - m) / |b - m|^2, for the zero-mean periodic lattice (the projection of the 3D problem above
    over one period along the line of sight),
      D(b) = sum_m (b_m / |b_m|^2) exp(-al^2 |b_m|^2) + (2 pi / L^2) sum_{k != 0} (k / k^2) exp(-k^2/(4 al^2)) sin(k . b).
    ``lattice_sum_2d`` gives the paper's direct nearest-images sum for comparison; for a symmetric square
    of images it differs from D(b) by the background term (pi / L^2) b.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc


def grad_phi_3d(r: np.ndarray, box: float, n_real: int = 3, n_recip: int = 8,
                alpha: float | None = None) -> np.ndarray:
    """Gradient of the periodic potential of a unit mass (G M = 1) at displacements r (n, 3) from it.

    ``alpha`` is the Ewald splitting parameter (default 2 / box); the sum does not depend on it once both
    parts have converged."""
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    r = r - box * np.round(r / box)
    al = 2.0 / box if alpha is None else alpha
    out = np.zeros_like(r)
    rng = range(-n_real, n_real + 1)
    for i in rng:
        for j in rng:
            for k in rng:
                d = r - box * np.array([i, j, k], dtype=np.float64)
                s = np.sqrt((d * d).sum(axis=1))
                f = (erfc(al * s) + 2.0 * al * s / math.sqrt(math.pi) * np.exp(-(al * s) ** 2)) / s ** 3
                out += d * f[:, None]
    kf = 2.0 * math.pi / box
    rng = range(-n_recip, n_recip + 1)
    for i in rng:
        for j in rng:
            for k in rng:
                if i == 0 and j == 0 and k == 0:
                    continue
                kv = kf * np.array([i, j, k], dtype=np.float64)
                k2 = float(kv @ kv)
                amp = 4.0 * math.pi / box ** 3 * math.exp(-k2 / (4.0 * al * al)) / k2
                out += amp * np.sin(r @ kv)[:, None] * kv[None, :]
    return out


def deflection_sum_2d(b: np.ndarray, box: float, n_real: int = 4, n_recip: int = 10,
                      alpha: float | None = None) -> np.ndarray:
    """Zero-mean periodic lensing sum D(b) (n, 2) for transverse offsets b (n, 2) from the lens column
    (``alpha``: the splitting parameter, default 2 / box)."""
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    b = b - box * np.round(b / box)
    al = 2.0 / box if alpha is None else alpha
    out = np.zeros_like(b)
    rng = range(-n_real, n_real + 1)
    for i in rng:
        for j in rng:
            d = b - box * np.array([i, j], dtype=np.float64)
            s2 = (d * d).sum(axis=1)
            out += d * (np.exp(-al * al * s2) / s2)[:, None]
    kf = 2.0 * math.pi / box
    rng = range(-n_recip, n_recip + 1)
    for i in rng:
        for j in rng:
            if i == 0 and j == 0:
                continue
            kv = kf * np.array([i, j], dtype=np.float64)
            k2 = float(kv @ kv)
            amp = 2.0 * math.pi / box ** 2 * math.exp(-k2 / (4.0 * al * al)) / k2
            out += amp * np.sin(b @ kv)[:, None] * kv[None, :]
    return out


def lattice_sum_2d(b: np.ndarray, box: float, n_images: int = 32) -> np.ndarray:
    """The nearest images on a symmetric square, (2 (n_images // 2) + 1)^2 of them, of the paper's sum
    sum_m (b - m) / |b - m|^2 (no background term)."""
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    half = n_images // 2
    out = np.zeros_like(b)
    for i in range(-half, half + 1):
        for j in range(-half, half + 1):
            d = b - box * np.array([i, j], dtype=np.float64)
            out += d / (d * d).sum(axis=1)[:, None]
    return out
