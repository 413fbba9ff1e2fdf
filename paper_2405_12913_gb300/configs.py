"""Workloads of the HRT hot path (synthetic stand-ins for the paper's point-mass test and cosmological runs).

Each workload states its sizes, time grids and ray geometry; both the CUDA path and the tests build their
inputs from these numbers and the seeded generators of ``synthetic``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

DEG = math.pi / 180.0


@dataclass(frozen=True)
class PointMassWorkload:
    """Static point-mass lens (Sec. 6.1 geometry scaled to a 64^3 box): one particle at the box centre on a
    mesh node, observer 1 Gpc/h in front of it, 64 KDK steps across the lens box, then a free drift to the
    source plane; rays on a polar grid with impact parameters log-uniform in 0.1..20 mesh cells."""
    name: str = "point_mass_64"
    n_mesh: int = 64
    box: float = 200.0
    mass: float = 1.0e15
    chi_lens: float = 1000.0
    chi_source: float = 2000.0
    n_steps: int = 64
    n_radial: int = 128
    n_azimuth: int = 128
    b_min_cells: float = 0.1
    b_max_cells: float = 20.0
    deconv_p: float = 4.0
    smooth_cells: float = 1.0
    samples_per_cell: float = 1.0

    @property
    def cell(self) -> float:
        return self.box / self.n_mesh

    @property
    def observer(self):
        return (0.5 * self.box, 0.5 * self.box, 0.5 * self.box - self.chi_lens)

    @property
    def lens_position(self):
        return (0.5 * self.box, 0.5 * self.box, 0.5 * self.box)

    @property
    def chi_grid(self):
        a, b = self.chi_lens - 0.5 * self.box, self.chi_lens + 0.5 * self.box
        return [a + (b - a) * i / self.n_steps for i in range(self.n_steps + 1)]


@dataclass(frozen=True)
class CosmoWorkload:
    """Cosmological co-evolution: Zel'dovich ICs from seeded white noise (power law x BBKS, sigma8 = 0.8),
    forward leapfrog to a = 1, then reverse steps of particles and rays with source planes."""
    name: str
    n_side: int
    n_mesh: int
    box: float
    a_init: float
    n_forward: int
    a_min: float
    n_reverse: int
    n_pix: int
    fov_deg: float
    source_steps: tuple
    omega_m: float = 0.3
    h: float = 0.7
    n_s: float = 0.96
    sigma8: float = 0.8
    deconv_p: float = 4.0
    smooth_cells: float = 1.0
    samples_per_cell: float = 1.0
    seed: int = 1000
    nbins: int = 20

    @property
    def observer(self):
        return (0.5 * self.box, 0.5 * self.box, 0.0)

    @property
    def forward_grid(self):
        return [self.a_init + (1.0 - self.a_init) * i / self.n_forward for i in range(self.n_forward + 1)]

    @property
    def reverse_grid(self):
        return [1.0 - (1.0 - self.a_min) * i / self.n_reverse for i in range(self.n_reverse + 1)]

    @property
    def dtheta(self) -> float:
        return self.fov_deg * DEG / self.n_pix

    @property
    def n_rays(self) -> int:
        return self.n_pix * self.n_pix

    @property
    def ell_range(self):
        theta = self.n_pix * self.dtheta
        return 2.0 * math.pi / theta, math.pi / self.dtheta


POINT_MASS = PointMassWorkload()

# 128^3 particles, 256^3 mesh, L = 256 Mpc/h; 32 forward steps a = 0.02 -> 1, 16 reverse steps 1 -> 0.5
# (source at z = 1); 512^2 rays over 3.5 deg.
COSMO_256 = CosmoWorkload(name="cosmo_128p_256m_512r", n_side=128, n_mesh=256, box=256.0, a_init=0.02,
                          n_forward=32, a_min=0.5, n_reverse=16, n_pix=512, fov_deg=3.5, source_steps=(16,))

# 512^3 particles, 1024^3 mesh, L = 1000 Mpc/h; 64 forward steps a = 0.02 -> 1, 64 reverse steps 1 -> 1/3
# with source planes z = 0.5, 1, 2 at reverse steps 32, 48, 64; 2048^2 rays over 10 deg.
COSMO_1024 = CosmoWorkload(name="cosmo_512p_1024m_2048r", n_side=512, n_mesh=1024, box=1000.0, a_init=0.02,
                           n_forward=64, a_min=1.0 / 3.0, n_reverse=64, n_pix=2048, fov_deg=10.0,
                           source_steps=(32, 48, 64))

# The 1024^3 recipe scaled to 128^3 particles / 256^3 mesh / 512^2 rays (same box and geometry).
COSMO_1024_SCALED = CosmoWorkload(name="cosmo_1024_recipe_at_128p_256m_512r", n_side=128, n_mesh=256,
                                  box=1000.0, a_init=0.02, n_forward=64, a_min=1.0 / 3.0, n_reverse=64, n_pix=512,
                                  fov_deg=10.0, source_steps=(32, 48, 64))

# The 1024^3 recipe at half the side, same cell size (256^3 particles, 512^3 mesh, 500 Mpc/h box, 1024^2 rays over
# 10 deg): a case of a few GB on the device for detailed counters of the full-size kernels.
COSMO_512_HALF = CosmoWorkload(name="cosmo_256p_512m_1024r", n_side=256, n_mesh=512, box=500.0, a_init=0.02,
                               n_forward=64, a_min=1.0 / 3.0, n_reverse=64, n_pix=1024, fov_deg=10.0,
                               source_steps=(32, 48, 64))

# Small case the FP64 oracle runs in seconds: mesh 60 (not a power of two), 20^3 particles (a ragged last
# block), 60^2 rays, 8 forward and 8 reverse steps.
COSMO_TINY = CosmoWorkload(name="cosmo_20p_60m_60r", n_side=20, n_mesh=60, box=120.0, a_init=0.05, n_forward=8,
                           a_min=0.6, n_reverse=8, n_pix=60, fov_deg=6.0, source_steps=(4, 8), nbins=8)

# Differentiation: the 256^3 recipe's ingredients at a size where the FP64 oracle's autograd runs in seconds
# (8^3 particles, 16^3 mesh, 16^2 rays, 3 forward and 3 reverse steps, one source plane).
COSMO_GRAD = CosmoWorkload(name="grad_8p_16m_16r", n_side=8, n_mesh=16, box=32.0, a_init=0.1, n_forward=3, a_min=0.7,
                           n_reverse=3, n_pix=16, fov_deg=6.0, source_steps=(3,), nbins=4)

# Differentiation at the 256^3-recipe sizes (128^3 particles, 256^3 mesh, 512^2 rays; checkpoint every 4 steps).
COSMO_GRAD_256 = CosmoWorkload(name="grad_128p_256m_512r", n_side=128, n_mesh=256, box=256.0, a_init=0.02,
                               n_forward=32, a_min=0.5, n_reverse=16, n_pix=512, fov_deg=3.5, source_steps=(16,))

WORKLOADS = {w.name: w for w in (POINT_MASS, COSMO_256, COSMO_1024, COSMO_1024_SCALED, COSMO_512_HALF, COSMO_TINY,
                                         COSMO_GRAD, COSMO_GRAD_256)}
