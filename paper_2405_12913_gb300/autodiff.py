"""Reverse-mode differentiation of the HRT co-evolution for PyTorch, on the library's native adjoint.

The paper names an adjoint method for HRT as future work (Sec. 7); the library provides it at the context level
(``hrt_set_checkpointing`` records a run from white-noise initial conditions with a checkpoint every k steps,
``hrt_adjoint`` walks it backwards with the hand-written adjoint kernels and chains Omega_m through its FP64
coefficients).  This module wraps that for autograd:

``ContextSim`` runs the whole simulation in a recording context -- Zel'dovich ICs from white noise, the forward
leapfrog to a = 1, the synchronising kick, and the reverse co-evolution of particles and rays of Alg. 1 -- and
returns the convergence maps of the source planes and the final ray angles; its ``backward`` is one
``hrt_adjoint`` call.  ``HRTKappa`` is the ``torch.autograd.Function`` over it and ``KappaPower`` the binned
power spectrum with its adjoint kernel, so that a loss on P(ell) differentiates end to end.

All arithmetic on the particles, meshes, rays and coefficients runs in libhrt; Python only sequences the calls.
"""
from __future__ import annotations

import torch

from . import hrt


class ContextSim:
    """One workload (``configs.CosmoWorkload``) run in a recording context; gradients from ``hrt_adjoint``."""

    def __init__(self, W, theta0: torch.Tensor, checkpoint_every: int = 4, ray_mesh=None):
        """``ray_mesh``: an ``hrt.make_raymesh_config`` to kick the rays on the ray mesh of Sec. 5.2 (the adjoint
        then holds each half shell's mesh geometry fixed), or None for the direct line-of-sight gather."""
        self.W = W
        self.k = max(1, int(checkpoint_every))
        self.theta0 = theta0.to(device="cuda", dtype=torch.float64).contiguous()
        self.n_rays = self.theta0.shape[0]
        self.n_slots = len(W.source_steps)
        self.rm_cfg = ray_mesh
        self.ctx = None

    def forward(self, noise: torch.Tensor, om: float):
        """Returns (kappa maps [n_slots, n_rays], final ray angles [n_rays, 2]) and keeps the recorded run."""
        W = self.W
        self.close()
        cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, float(om), W.h, W.n_s, W.sigma8, W.deconv_p,
                              W.smooth_cells, W.samples_per_cell, W.observer, n_sources=max(self.n_slots, 1))
        ctx = hrt.Context(cfg)
        self.ctx = ctx
        ctx.hrt_set_checkpointing(self.k)
        if self.rm_cfg is not None:
            ctx.hrt_set_ray_mesh(self.rm_cfg)
        ctx.hrt_init_particles_zeldovich(noise.reshape(-1).contiguous(), W.a_init)
        for a in W.forward_grid[1:]:
            ctx.hrt_step(a)
        ctx.hrt_sync_particles()
        ctx.hrt_init_rays(self.theta0)
        slots = {s: i for i, s in enumerate(W.source_steps)}
        for n, a in enumerate(W.reverse_grid[1:], start=1):
            ctx.hrt_step(a, slots.get(n, -1))
        kappa = torch.stack([ctx.hrt_read_maps(i)[0] for i in range(self.n_slots)])
        theta = ctx.hrt_read_rays()[0]
        return kappa, theta

    def backward(self, kappa_bar: torch.Tensor, theta_bar: torch.Tensor | None = None):
        """kappa_bar [n_slots, n_rays], theta_bar [n_rays, 2] or None -> (noise_bar, dL/dOmega_m)."""
        return self.ctx.hrt_adjoint(kappa_bar.to(torch.float32).contiguous(),
                                    None if theta_bar is None else theta_bar.to(torch.float64).contiguous())

    def close(self):
        if self.ctx is not None:
            self.ctx.close()
            self.ctx = None


class HRTKappa(torch.autograd.Function):
    """(kappa maps [n_slots, n_rays], final ray angles [n_rays, 2]) = HRT(noise, Omega_m), with the library's
    adjoint of the recorded run (``hrt_adjoint``) as backward.

    The convergence comes from the distortion matrix, whose recursion uses the transverse derivative of the
    trilinear force interpolant: a piecewise-constant function of the ray positions.  kappa is therefore smooth
    only between the parameter values at which a line-of-sight sample crosses a mesh-cell face; the gradient
    returned here is the derivative within those pieces (what autograd of the same discrete method gives).
    The final angles are continuous in the parameters."""

    @staticmethod
    def forward(ctx, noise, omega_m, sim: ContextSim):
        ctx.sim = sim
        ctx.noise_shape = noise.shape
        kappa, theta = sim.forward(noise.detach().to(torch.float32), float(omega_m))
        return kappa, theta

    @staticmethod
    def backward(ctx, kappa_bar, theta_bar):
        kb = (kappa_bar.contiguous() if kappa_bar is not None
              else torch.zeros(ctx.sim.n_slots, ctx.sim.n_rays, dtype=torch.float32, device="cuda"))
        tb = theta_bar.contiguous().to(torch.float64) if theta_bar is not None else None
        noise_bar, om_bar = ctx.sim.backward(kb, tb)
        return noise_bar.reshape(ctx.noise_shape), torch.tensor(om_bar, dtype=torch.float64), None


class KappaPower(torch.autograd.Function):
    """Binned convergence power spectrum P_b (FP64, host) of an m x m kappa map with its adjoint kernel."""

    @staticmethod
    def forward(ctx, kappa, m, dtheta, nbins, ell_min, ell_max):
        k = kappa.detach().to(torch.float32).contiguous()
        ell, p, cnt = hrt.hrt_kappa_power(k, m, dtheta, nbins, ell_min, ell_max)
        ctx.save_for_backward(k)
        ctx.args = (m, dtheta, nbins, ell_min, ell_max)
        return torch.from_numpy(p)

    @staticmethod
    def backward(ctx, p_bar):
        (k,) = ctx.saved_tensors
        m, dtheta, nbins, ell_min, ell_max = ctx.args
        kb = torch.empty_like(k)
        hrt.hrt_kappa_power_adjoint(k, m, dtheta, nbins, ell_min, ell_max, p_bar.detach().cpu().numpy(), kb)
        return kb, None, None, None, None, None
