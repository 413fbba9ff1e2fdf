"""Co-evolution driver of the FP64 oracle (test infrastructure only).

Alg. 1 of arXiv 2405.12913, written out for the whole ray bundle, with the readings of the paper's silent
points that the CUDA path also takes:

  * one PM force per step, computed from the particles at the snapshot a_n at the start of the step; both
    ray half-kicks of the step use it, with the growth time correction referred to tau_c = tau(a_n);
  * the particle leapfrog kicks from the momentum time a_p to the half step a_{n+1/2} = (a_n + a_{n+1})/2,
    then drifts from a_n to a_{n+1}; the same code runs forward (a increasing) and in reverse;
  * forward run: Zel'dovich ICs at a_init, then steps to a = 1 and a final kick to a_p = 1 (synchronised);
  * reverse co-evolution from a = 1: per step the rays are traced through the shell [chi(a_n), chi(a_{n+1})],
    then the particles step back, then the PM force is recomputed at a_{n+1}; observables are read out after
    the steps whose end is a source plane.

The static point-mass problem (flat, non-expanding, a = 1) uses the Poisson prefactor 4 pi G rho_mean and no
time correction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import cosmology as cosmo
from . import pm, rays, raymesh
from .units import C_LIGHT, G_NEWTON


@dataclass
class Cosmo:
    omega_m: float = 0.3
    h: float = 0.7
    n_s: float = 0.96
    sigma8: float = 0.8


@dataclass
class Particles:
    q: torch.Tensor
    disp: torch.Tensor
    mom: torch.Tensor
    a_x: float
    a_p: float


@dataclass
class Filter:
    """k-space filter of the gradient fields: sinc^-p deconvolution and Gaussian smoothing in mesh cells."""
    deconv_p: float = 4.0
    smooth_cells: float = 1.0


def pm_force(part: Particles, box: float, n_mesh: int, pref: float, flt: Filter):
    rho = pm.cic_deposit(part.q + part.disp, box, n_mesh)
    return pm.poisson_gradient(rho, box, pref, flt.deconv_p, flt.smooth_cells * box / n_mesh)


def particle_step(part: Particles, grads, a_next: float, om: float, box: float) -> Particles:
    a_half = 0.5 * (part.a_x + a_next)
    kick = cosmo.kick_integral(part.a_p, a_half, om)
    drift = cosmo.drift_integral(part.a_x, a_next, om)
    disp, mom = pm.particle_kick_drift(part.disp, part.mom, part.q, grads, box, kick, drift)
    return Particles(part.q, disp, mom, a_next, a_half)


def particle_sync(part: Particles, grads, om: float, box: float) -> Particles:
    kick = cosmo.kick_integral(part.a_p, part.a_x, om)
    disp, mom = pm.particle_kick_drift(part.disp, part.mom, part.q, grads, box, kick, 0.0)
    return Particles(part.q, disp, mom, part.a_x, part.a_x)


def initial_particles(noise: np.ndarray, box: float, c: Cosmo, a_init: float) -> Particles:
    n = noise.shape[0]
    disp, mom = pm.zeldovich(noise, box, c.omega_m, c.h, c.n_s, c.sigma8, a_init)
    return Particles(pm.lattice(n, box), disp, mom, a_init, a_init)


def run_forward(part: Particles, a_grid, box: float, n_mesh: int, c: Cosmo, flt: Filter):
    """Leapfrog along ``a_grid`` (a_grid[0] == part.a_x) and synchronise; returns (particles, grads)."""
    om = c.omega_m
    grads = pm_force(part, box, n_mesh, 1.5 * om / part.a_x, flt)
    for a_next in a_grid[1:]:
        part = particle_step(part, grads, a_next, om, box)
        grads = pm_force(part, box, n_mesh, 1.5 * om / a_next, flt)
    part = particle_sync(part, grads, om, box)
    return part, grads


def growth_weight(a_c: float, om: float):
    """Time correction of Eq. "kick": g(chi) = D1(a(chi)) a_c / (D1(a_c) a(chi))."""
    d_c = cosmo.growth_D1(a_c, om)

    def g(chi: float) -> float:
        a = cosmo.a_of_chi(chi, om)
        return cosmo.growth_D1(a, om) / d_c * a_c / a
    return g


@dataclass
class ReverseResult:
    part: Particles
    grads: list
    rays: dict
    maps: dict = field(default_factory=dict)   # source step -> (kappa, g1, g2, omega)
    thetas: dict = field(default_factory=dict)  # source step -> theta
    face_min: dict = field(default_factory=dict)  # source step -> per ray, nearest approach of a node to a face


def run_reverse(part: Particles, grads, a_grid, box: float, n_mesh: int, c: Cosmo, flt: Filter,
                theta0: torch.Tensor, observer, source_steps, samples_per_cell: float = 1.0,
                move_particles: bool = True, replicas=None, ray_mesh=None,
                face_distance: bool = False) -> ReverseResult:
    """Reverse co-evolution along the decreasing ``a_grid`` (a_grid[0] == part.a_x, normally 1); with
    ``replicas`` = (perm, sign, shift) the rays cross a light cone tiled by rotated, translated replicas; with
    ``ray_mesh`` = (mu, m_pix, iota, p_min) the kicks come from the ray mesh of Sec. 5.2 (``raymesh``).  With
    ``face_distance`` (direct kick) the result also holds, per source step and ray, the nearest approach of any
    line-of-sight node so far to a transverse cell face (``rays.face_distance``)."""
    om = c.omega_m
    state = rays.init_state(theta0)
    res = ReverseResult(part, grads, state)
    nearest = torch.full((theta0.shape[0],), math.inf, dtype=torch.float64) if face_distance else None
    for n in range(len(a_grid) - 1):
        a_n, a_n1 = a_grid[n], a_grid[n + 1]
        chi_n, chi_n1 = cosmo.chi_of_a(a_n, om), cosmo.chi_of_a(a_n1, om)
        theta_n = state["theta"]
        if ray_mesh is None:
            state = rays.ray_step(state, grads[0], grads[1], box, observer, chi_n, chi_n1, samples_per_cell,
                                  growth_weight(a_n, om), gz=grads[2], replicas=replicas)
            if nearest is not None:
                nearest = torch.minimum(nearest, rays.step_face_distance(theta_n, state["theta"], box, n_mesh,
                                                                         observer, chi_n, chi_n1, samples_per_cell))
        else:
            state = raymesh.ray_step(state, grads[0], grads[1], box, observer, chi_n, chi_n1,
                                     growth_weight(a_n, om), *ray_mesh, gz=grads[2], replicas=replicas)
        if (n + 1) in source_steps:
            res.maps[n + 1] = rays.observables(state["A"])
            res.thetas[n + 1] = state["theta"].clone()
            if nearest is not None:
                res.face_min[n + 1] = nearest.clone()
        if move_particles:
            part = particle_step(part, grads, a_n1, om, box)
            grads = pm_force(part, box, n_mesh, 1.5 * om / a_n1, flt)
    res.part, res.grads, res.rays = part, grads, state
    return res


# ----------------------------------------------------------------------------------------------------------
# Static point-mass lens (Sec. 6.1): flat space, a = 1, no growth correction.
# ----------------------------------------------------------------------------------------------------------

@dataclass
class PointMass:
    n_mesh: int = 64
    box: float = 200.0
    mass: float = 1.0e15          # Msun/h
    chi_lens: float = 1000.0      # Mpc/h
    chi_source: float = 2000.0
    n_steps: int = 64
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
    def pref(self) -> float:
        return 4.0 * math.pi * G_NEWTON * self.mass / self.box ** 3

    @property
    def chi_grid(self):
        a, b = self.chi_lens - 0.5 * self.box, self.chi_lens + 0.5 * self.box
        return [a + (b - a) * i / self.n_steps for i in range(self.n_steps + 1)]


def point_mass_fields(pmc: PointMass):
    x = torch.tensor([pmc.lens_position], dtype=torch.float64)
    rho = pm.cic_deposit(x, pmc.box, pmc.n_mesh)
    return pm.poisson_gradient(rho, pmc.box, pmc.pref, pmc.deconv_p, pmc.smooth_cells * pmc.cell)


def point_mass_trace(pmc: PointMass, theta0: torch.Tensor, grads=None):
    """Trace rays through the lens box (the 64 steps span one box length around the lens) and drift freely
    to the source; returns the final ray state.  Before the box eta = 0, so the drift there is the identity."""
    if grads is None:
        grads = point_mass_fields(pmc)
    state = rays.init_state(theta0)
    chis = pmc.chi_grid
    one = lambda chi: 1.0  # noqa: E731  (static potential: no growth correction)
    for n in range(pmc.n_steps):
        state = rays.ray_step(state, grads[0], grads[1], pmc.box, pmc.observer, chis[n], chis[n + 1],
                              pmc.samples_per_cell, one)
    return rays.free_drift(state, chis[-1], pmc.chi_source)


def point_mass_born_ewald(pmc: PointMass, theta0: np.ndarray, n_nodes: int = 600) -> np.ndarray:
    """Born deflection theta0 - theta_s of the exact periodic (3D Ewald) point-mass field integrated along the
    unperturbed rays over the lens box:  alpha = (2/c^2) int grad_perp phi(X(theta0, chi)) (chi_s - chi)/chi_s.

    The radial integral uses Gauss-Legendre nodes in t with chi - chi_lens = b sinh(t), which resolves the
    peak of width b at the lens."""
    from . import ewald
    theta0 = np.atleast_2d(theta0)
    a, b_end = pmc.chi_lens - 0.5 * pmc.box, pmc.chi_lens + 0.5 * pmc.box
    xg, wg = np.polynomial.legendre.leggauss(n_nodes)
    out = np.zeros_like(theta0)
    for i, th in enumerate(theta0):
        b = max(pmc.chi_lens * float(np.hypot(*th)), 1e-3)
        t0, t1 = math.asinh((a - pmc.chi_lens) / b), math.asinh((b_end - pmc.chi_lens) / b)
        t = 0.5 * (t1 - t0) * xg + 0.5 * (t1 + t0)
        w = 0.5 * (t1 - t0) * wg
        chi = pmc.chi_lens + b * np.sinh(t)
        jac = b * np.cosh(t)
        X = np.stack([pmc.observer[0] + chi * th[0], pmc.observer[1] + chi * th[1], pmc.observer[2] + chi], 1)
        r = X - np.array(pmc.lens_position)
        g = ewald.grad_phi_3d(r, pmc.box) * (G_NEWTON * pmc.mass)
        weight = w * jac * (pmc.chi_source - chi) / pmc.chi_source
        out[i] = (2.0 / C_LIGHT ** 2) * (g[:, :2] * weight[:, None]).sum(axis=0)
    return out
