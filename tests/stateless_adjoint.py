"""The adjoint of the co-evolution sequenced in Python over the library's stateless adjoint calls: a cross-check
of the library's own context-level adjoint (hrt_set_checkpointing / hrt_adjoint), which runs the same calls
natively.  Test infrastructure: the forward run keeps a checkpoint every k steps, the backward pass recomputes
each segment and walks it in reverse, and dL/dOmega_m is chained on the host with FP64 central differences of
the coefficient builders (IC table, Poisson prefactors, kick and drift integrals, line-of-sight nodes and
weights, drift coefficients, ray-mesh plane weights)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from paper_2405_12913_gb300 import hrt

_EPS_OM = 1e-5


@dataclass
class Step:
    kind: str      # "F" forward leapfrog, "S" synchronising kick, "R" reverse co-evolution
    a_x: float     # position time before the step
    a_next: float  # position time after the step
    a_p: float     # momentum time before the step
    slot: int      # map slot written after a reverse step (-1: none)


class DiffSim:
    """Forward run with checkpoints and its adjoint for one workload (see ``configs.CosmoWorkload``)."""

    def __init__(self, W, theta0: torch.Tensor, checkpoint_every: int = 4, ray_mesh=None):
        """``ray_mesh``: an ``hrt.make_raymesh_config`` to kick the rays on the ray mesh of Sec. 5.2 (the adjoint then
        holds the mesh geometry of each half shell fixed: dL/dOmega_m acts through the plane weights and the
        drift coefficients, not through lambda_lim), or None for the direct line-of-sight gather."""
        self.W = W
        self.k = max(1, int(checkpoint_every))
        n, L = W.n_mesh, W.box
        self.n, self.L, self.ns = n, L, W.n_side
        self.np, self.m = W.n_side ** 3, n ** 3
        self.pm = hrt.PM(n, L)
        self.flt = hrt.make_filter(W.deconv_p, W.smooth_cells * L / n)
        self.geom = hrt.make_geom(n, L, W.observer, W.samples_per_cell, image_width=W.n_pix)
        self.theta0 = theta0.to(device="cuda", dtype=torch.float64).contiguous()
        self.n_rays = self.theta0.shape[0]
        self.n_slots = len(W.source_steps)
        self.rm_cfg = ray_mesh
        self.rm = hrt.RayMesh(ray_mesh) if ray_mesh is not None else None

    # ------------------------------------------------------------------------------------------- plan
    def plan(self):
        W = self.W
        steps = []
        a_p = W.a_init
        fg = W.forward_grid
        for i in range(len(fg) - 1):
            steps.append(Step("F", fg[i], fg[i + 1], a_p, -1))
            a_p = 0.5 * (fg[i] + fg[i + 1])
        steps.append(Step("S", 1.0, 1.0, a_p, -1))
        a_p = 1.0
        slots = {s: i for i, s in enumerate(W.source_steps)}
        rg = W.reverse_grid
        for i in range(len(rg) - 1):
            steps.append(Step("R", rg[i], rg[i + 1], a_p, slots.get(i + 1, -1)))
            a_p = 0.5 * (rg[i] + rg[i + 1])
        return steps

    @staticmethod
    def coefficients(step: Step, om: float):
        """Kick and drift integrals of a particle step (FP64 host)."""
        if step.kind == "S":
            return hrt.hrt_cosmo_time_integrals(om, step.a_p, step.a_x)[0], 0.0
        a_half = 0.5 * (step.a_x + step.a_next)
        return (hrt.hrt_cosmo_time_integrals(om, step.a_p, a_half)[0],
                hrt.hrt_cosmo_time_integrals(om, step.a_x, step.a_next)[1])

    # ------------------------------------------------------------------------------------------- forward
    def _fields(self, d, a, om):
        rho = torch.empty(self.m, device="cuda")
        hrt.hrt_cic_scatter(d, self.ns, self.n, self.L, rho)
        g = torch.empty(3, self.m, device="cuda")
        self.pm.solve(rho, 1.5 * om / a, self.flt, g)
        return g

    def _ensure_rays(self, st, step: Step):
        """Rays start at the observer with the first reverse step."""
        if step.kind == "R" and st["rays"] is None:
            st["rays"] = hrt.RayState(self.n_rays)
            hrt.hrt_rays_init(st["rays"], self.theta0)

    def _step(self, st, step: Step, om: float, maps=None):
        """Advances st = dict(d, m, rays, g) by one step in place (g: fields at st's positions and a_x)."""
        K, D = self.coefficients(step, om)
        self._ensure_rays(st, step)
        if step.kind == "R":
            chi0, chi1 = hrt.hrt_cosmo_eval(om, step.a_x)[1], hrt.hrt_cosmo_eval(om, step.a_next)[1]
            out = maps[step.slot] if (maps is not None and step.slot >= 0) else None
            if self.rm is not None:
                self.rm.hrt_raymesh_ray_step(st["rays"], st["g"][0], st["g"][1], self.geom, chi0, chi1, step.a_x, om,
                                             out)
            else:
                hrt.hrt_ray_step(st["rays"], st["g"][0], st["g"][1], self.geom, chi0, chi1, step.a_x, om, out)
        if step.kind == "S":
            hrt.hrt_particle_kick_drift(st["g"], self.n, self.L, self.ns, st["d"], st["m"], K, 0.0)
            return
        rho = torch.empty(self.m, device="cuda")
        hrt.hrt_particle_kick_drift_deposit(st["g"], self.n, self.L, self.ns, st["d"], st["m"], K, D, rho)
        g = torch.empty(3, self.m, device="cuda")
        self.pm.solve(rho, 1.5 * om / step.a_next, self.flt, g)
        st["g"] = g

    @staticmethod
    def _snapshot(st):
        rays = None
        if st["rays"] is not None:
            rays = hrt.RayState(st["rays"].n_rays)
            for name in ("theta", "eta", "A", "B"):
                getattr(rays, name).copy_(getattr(st["rays"], name))
        return dict(d=st["d"].clone(), m=st["m"].clone(), rays=rays, g=st["g"].clone())

    def initial_state(self, noise: torch.Tensor, om: float):
        W = self.W
        d = torch.empty(3, self.np, device="cuda")
        m = torch.empty(3, self.np, device="cuda")
        hrt.hrt_ic_zeldovich(noise, self.ns, self.L, om, W.h, W.n_s, W.sigma8, W.a_init, d, m)
        return dict(d=d, m=m, rays=None, g=self._fields(d, W.a_init, om))

    def forward(self, noise: torch.Tensor, om: float):
        """Returns the kappa maps [n_slots, n_rays]; keeps the checkpoints for ``backward``."""
        self.noise = noise.contiguous()
        self.om = float(om)
        self.steps = self.plan()
        maps = torch.zeros(max(self.n_slots, 1), 4, self.n_rays, device="cuda")
        st = self.initial_state(self.noise, self.om)
        self.d0 = st["d"].clone()
        self.checkpoints = {}
        for i, step in enumerate(self.steps):
            self._ensure_rays(st, step)
            if i % self.k == 0:
                self.checkpoints[i] = self._snapshot(st)
            self._step(st, step, self.om, maps)
        self.maps = maps
        theta = st["rays"].theta.clone() if st["rays"] is not None else torch.zeros_like(self.theta0)
        return maps[:, 0, :].clone(), theta

    # ------------------------------------------------------------------------------------------- backward
    def backward(self, kappa_bar: torch.Tensor, theta_bar: torch.Tensor | None = None):
        """kappa_bar [n_slots, n_rays] and theta_bar [n_rays, 2] (cotangent of the final ray angles, or None)
        -> (noise_bar tensor, dL/dOmega_m float)."""
        W, om = self.W, self.om
        n_steps = len(self.steps)
        d_bar = torch.zeros(3, self.np, device="cuda")
        m_bar = torch.zeros(3, self.np, device="cuda")
        r_bar = hrt.RayState(self.n_rays)
        for name in ("theta", "eta", "A", "B"):
            getattr(r_bar, name).zero_()
        if theta_bar is not None:
            r_bar.theta.copy_(theta_bar)
        rho_bar = torch.zeros(self.m, device="cuda")
        coef_bar = torch.zeros(n_steps, 2, dtype=torch.float64, device="cuda")
        node_bar = torch.zeros(n_steps, 3, hrt.MAX_RAY_NODES, dtype=torch.float64, device="cuda")
        drift_bar = torch.zeros(n_steps, dtype=torch.float64, device="cuda")
        pref_bar = np.zeros(n_steps)
        plane_bar = np.zeros((n_steps, 2, 512))
        starts = sorted(self.checkpoints)
        for s0 in reversed(starts):
            s1 = min(s0 + self.k, n_steps)
            st = self._snapshot(self.checkpoints[s0])
            pre = []
            for i in range(s0, s1):
                self._ensure_rays(st, self.steps[i])
                pre.append(self._snapshot(st))
                self._step(st, self.steps[i], om)
            for i in reversed(range(s0, s1)):
                step, ps = self.steps[i], pre[i - s0]
                K, D = self.coefficients(step, om)
                if step.kind == "R" and step.slot >= 0:
                    # kappa = 1 - (A11 + A22)/2 read out after the step
                    kb = kappa_bar[step.slot].to(torch.float32)
                    r_bar.A[:, 0] -= 0.5 * kb
                    r_bar.A[:, 3] -= 0.5 * kb
                g_bar = torch.zeros(3, self.m, device="cuda")
                if step.kind == "S":
                    hrt.hrt_cic_scatter_adjoint(rho_bar, ps["d"], self.ns, self.n, self.L, d_bar)
                    hrt.hrt_particle_kick_drift_adjoint(ps["g"], self.n, self.L, self.ns, ps["d"], ps["m"], K, 0.0,
                                                        None, d_bar, m_bar, g_bar, coef_bar[i])
                else:
                    hrt.hrt_particle_kick_drift_adjoint(ps["g"], self.n, self.L, self.ns, ps["d"], ps["m"], K, D,
                                                        rho_bar, d_bar, m_bar, g_bar, coef_bar[i])
                if step.kind == "R":
                    chi0, chi1 = hrt.hrt_cosmo_eval(om, step.a_x)[1], hrt.hrt_cosmo_eval(om, step.a_next)[1]
                    if self.rm is not None:
                        plane_bar[i], db = self.rm.hrt_raymesh_ray_step_adjoint(
                            ps["rays"], ps["g"][0], ps["g"][1], self.geom, chi0, chi1, step.a_x, om, r_bar, g_bar[0],
                            g_bar[1])
                        drift_bar[i] += db
                    else:
                        hrt.hrt_ray_step_adjoint(ps["rays"], ps["g"][0], ps["g"][1], self.geom, chi0, chi1, step.a_x,
                                                 om, r_bar, g_bar[0], g_bar[1], node_bar[i], drift_bar[i:i + 1])
                pref = 1.5 * om / step.a_x
                pref_bar[i] = hrt.hrt_dot(g_bar, ps["g"]) / pref
                rho_bar = torch.empty(self.m, device="cuda")
                self.pm.solve_adjoint(g_bar, pref, self.flt, rho_bar)
        # initial density from the IC positions, then the ICs
        hrt.hrt_cic_scatter_adjoint(rho_bar, self.d0, self.ns, self.n, self.L, d_bar)
        noise_bar = torch.empty_like(self.noise)
        table_bar, ratio_bar = hrt.hrt_ic_zeldovich_adjoint(self.noise, self.ns, self.L, om, W.h, W.n_s, W.sigma8,
                                                            W.a_init, d_bar, m_bar, self.d0, noise_bar)
        om_bar = self._omega_chain(coef_bar.cpu().numpy(), node_bar.cpu().numpy(), drift_bar.cpu().numpy(),
                                   pref_bar, table_bar, ratio_bar, plane_bar)
        return noise_bar, om_bar

    def _omega_chain(self, coef_bar, node_bar, drift_bar, pref_bar, table_bar, ratio_bar, plane_bar) -> float:
        W, om, e = self.W, self.om, _EPS_OM
        total = 0.0
        for i, step in enumerate(self.steps):
            kp, dp = self.coefficients(step, om + e)
            km, dm = self.coefficients(step, om - e)
            total += coef_bar[i, 0] * (kp - km) / (2 * e) + coef_bar[i, 1] * (dp - dm) / (2 * e)
            total += pref_bar[i] * 1.5 / step.a_x
            if step.kind == "R" and self.rm is not None:
                # plane weights at the nominal geometry: w is proportional to g(chi_p) / x2d^2, x2d held fixed
                hi, lo = self._mesh_coefficients(step, om + e), self._mesh_coefficients(step, om - e)
                x2d0 = self._mesh_coefficients(step, om)[2]
                if hi[0] != lo[0] or not np.array_equal(hi[1], lo[1]):
                    raise RuntimeError("a ray-mesh plane changes half shell within the Omega_m difference step")
                for h in range(2):
                    k = hi[0][h]
                    wp = hi[3][h, :k] * (hi[2][h] / x2d0[h]) ** 2
                    wm = lo[3][h, :k] * (lo[2][h] / x2d0[h]) ** 2
                    total += float(plane_bar[i, h, :k] @ ((wp - wm) / (2 * e)))
                total += drift_bar[i] * (hi[4] - lo[4]) / (2 * e)
            elif step.kind == "R":
                hi = self._ray_coefficients(step, om + e)
                lo = self._ray_coefficients(step, om - e)
                if hi[0] != lo[0]:
                    raise RuntimeError("line-of-sight node count changes within the Omega_m difference step")
                k = hi[0]
                for j, (a, b) in enumerate(zip(hi[1:4], lo[1:4])):
                    total += float(node_bar[i, j, :k] @ ((a - b) / (2 * e)))
                total += drift_bar[i] * (hi[4] - lo[4]) / (2 * e)
        tp, rp = hrt.hrt_ic_table(self.ns, self.L, om + e, W.h, W.n_s, W.sigma8, W.a_init)
        tm, rm = hrt.hrt_ic_table(self.ns, self.L, om - e, W.h, W.n_s, W.sigma8, W.a_init)
        # the kernels use the float32 table with D1 folded in and mom = ratio * disp
        total += float(table_bar @ ((tp - tm) / (2 * e))) + ratio_bar * (rp - rm) / (2 * e)
        return total

    def _ray_coefficients(self, step: Step, om: float):
        chi0, chi1 = hrt.hrt_cosmo_eval(om, step.a_x)[1], hrt.hrt_cosmo_eval(om, step.a_next)[1]
        n1, n2, cw, cwr, chi, d = hrt.hrt_ray_step_coefficients(self.geom, chi0, chi1, step.a_x, om)
        return n1 + n2, cw, cwr, chi, d

    def _mesh_coefficients(self, step: Step, om: float):
        """(plane counts, plane chi [2][512], x2d per half shell, FP64 plane weights [2][512], drift)."""
        chi0, chi1 = hrt.hrt_cosmo_eval(om, step.a_x)[1], hrt.hrt_cosmo_eval(om, step.a_next)[1]
        counts, chi, w, d = hrt.hrt_raymesh_step_planes(self.rm_cfg, self.geom, chi0, chi1, step.a_x, om)
        mid = 0.5 * (chi0 + chi1)
        cell = self.L / self.n
        x2d = [hrt.hrt_raymesh_geometry(self.rm_cfg, a, b, cell)[1] for a, b in ((chi0, mid), (mid, chi1))]
        return counts, np.round(chi, 9), x2d, w, d

    def close(self):
        self.pm.close()
        if self.rm is not None:
            self.rm.close()
