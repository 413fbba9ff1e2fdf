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


def mode_spec(seed: int, n: int, n_modes: int, scale: float) -> dict:
    """A real periodic field on an ``n^3`` mesh made of cosine modes,
    ``f(i, j, k) = sum_m a_m cos(2 pi (m . (i, j, k)) / n + phi_m)``: integer mode vectors whose largest component
    spreads geometrically from 1 to ``n/2 - 1`` (no zero mode, no Nyquist component), amplitudes ``scale N(0, 1)``,
    phases uniform in ``[0, 2 pi)``.  Evaluate with ``mode_field_values`` or ``mode_field_device``."""
    rng = np.random.default_rng(seed)
    top = n // 2 - 1
    modes = []
    for t in np.geomspace(1.0, top, n_modes):
        m = np.round(rng.uniform(-1.0, 1.0, size=3) * t).astype(np.int64)
        m[rng.integers(3)] = int(round(t)) * (1 if rng.random() < 0.5 else -1)
        modes.append(np.clip(m, -top, top))
    return dict(modes=np.array(modes, dtype=np.int64), amp=scale * rng.standard_normal(n_modes),
                phase=rng.uniform(0.0, 2.0 * np.pi, n_modes))


def mode_field_values(spec: dict, n: int, flat_idx: np.ndarray) -> np.ndarray:
    """The mode field (float64) at flat mesh indices ``(i n + j) n + k``; the phase index ``m . (i, j, k) mod n`` is
    formed in integers."""
    idx = np.asarray(flat_idx, dtype=np.int64)
    i, j, k = idx // (n * n), (idx // n) % n, idx % n
    out = np.zeros(idx.shape, dtype=np.float64)
    for m, a, ph in zip(spec["modes"], spec["amp"], spec["phase"]):
        t = (m[0] * i + m[1] * j + m[2] * k) % n
        out += a * np.cos(2.0 * np.pi * t / n + ph)
    return out


def mode_field_device(spec: dict, n: int, device, slab: int = 32):
    """The mode field on the whole mesh as a float32 torch tensor ``(n, n, n)`` on ``device``, built in float64
    ``slab`` x-planes at a time (the same values as ``mode_field_values``, rounded to float32)."""
    import torch
    out = torch.empty(n, n, n, dtype=torch.float32, device=device)
    jj = torch.arange(n, dtype=torch.int64, device=device).view(1, -1, 1)
    kk = torch.arange(n, dtype=torch.int64, device=device).view(1, 1, -1)
    for x0 in range(0, n, slab):
        ii = torch.arange(x0, min(n, x0 + slab), dtype=torch.int64, device=device).view(-1, 1, 1)
        acc = torch.zeros(ii.shape[0], n, n, dtype=torch.float64, device=device)
        for m, a, ph in zip(spec["modes"], spec["amp"], spec["phase"]):
            t = (int(m[0]) * ii + int(m[1]) * jj + int(m[2]) * kk) % n
            acc += float(a) * torch.cos(t.double() * (2.0 * np.pi / n) + float(ph))
        out[x0:x0 + ii.shape[0]] = acc.float()
    return out


def bounded_particle_state(seed: int, n_side: int, disp_max: float, mom_max: float):
    """Displacements and momenta uniform in ``[-disp_max, disp_max]`` and ``[-mom_max, mom_max]`` per component for
    an ``n_side^3`` lattice, float32 SoA ``(3, n_side^3)`` each (bounded, so that a particle's reach is known)."""
    rng = np.random.default_rng(seed)
    n = n_side ** 3
    disp = (2.0 * rng.random((3, n), dtype=np.float32) - 1.0) * np.float32(disp_max)
    mom = (2.0 * rng.random((3, n), dtype=np.float32) - 1.0) * np.float32(mom_max)
    return disp, mom
