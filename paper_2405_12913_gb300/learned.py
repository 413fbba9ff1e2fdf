"""Learned correction of the coarse-mesh ray force, trained on the method's own coarse/fine mesh pairs.

The paper sharpens the PM force with a trained factor g in k/k^2 -> (k/k^2) g (Sec. 6.2).  Here g = 1 + MLP(|k| cell,
a, ln N_mesh) multiplies the Green's function of the ray gradient fields of a coarse mesh (the particles keep the
plain force), and is trained so that the convergence power spectrum of the coarse run matches that of a run with
the same initial conditions on a mesh four times finer.  The plain kernel (g = 1) is the fallback and the
yardstick: ``evaluate``, ``compare`` and ``ladder`` report the P(ell) error of both forms against the fine run on
held-out seeds.

Training uses only libhrt kernels: the tensor-core MLP forward, the ray-step and k-space-table adjoints, the FP32
MLP backward and an Adam kernel.  The particles do not depend on g, so the density spectrum of each reverse step is
computed once per seed (plain coarse run) and every training iteration re-traces only the rays.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass, replace

import numpy as np
import torch

from . import hrt

N_TABLE = 512


class MLP:
    """Parameters (FP32 master + BF16 copy) and Adam state of the correction network on the GPU."""

    def __init__(self, seed: int = 0):
        rng = np.random.default_rng(seed)
        p = np.zeros(hrt.MLP_PARAMS, np.float32)
        H, IN = 64, 16
        w1 = rng.standard_normal((H, 3)) * math.sqrt(2.0 / 3.0)
        W1 = np.zeros((H, IN))
        W1[:, :3] = w1
        o = 0
        p[o:o + H * IN] = W1.ravel()
        o += H * IN + H
        p[o:o + H * H] = (rng.standard_normal((H, H)) * math.sqrt(2.0 / H)).ravel()
        o += H * H + H
        p[o:o + H * H] = (rng.standard_normal((H, H)) * math.sqrt(2.0 / H)).ravel()
        # output layer zero: g = 1 at the start (the plain kernel)
        self.w = torch.tensor(p, device="cuda")
        self.wb = torch.empty(hrt.MLP_PARAMS, dtype=torch.bfloat16, device="cuda")
        hrt.hrt_mlp_to_bf16(self.w, self.wb)
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.step = 0

    @staticmethod
    def inputs(kmax: float, cell: float, a: float, n_mesh: int) -> torch.Tensor:
        k = torch.linspace(0.0, kmax, N_TABLE, dtype=torch.float64)
        x = torch.stack([k * cell, torch.full_like(k, a), torch.full_like(k, math.log(n_mesh))], dim=1)
        return x.to(device="cuda", dtype=torch.float32).contiguous()

    def table(self, x: torch.Tensor) -> torch.Tensor:
        g = torch.empty(x.shape[0], device="cuda")
        hrt.hrt_mlp_forward(x, self.wb, self.w, g)
        return g

    def accumulate(self, x, g_bar, grad):
        hrt.hrt_mlp_backward(x, self.wb, self.w, g_bar, grad)

    def adam(self, grad, lr):
        self.step += 1
        hrt.hrt_mlp_adam(self.w, self.wb, grad, self.m, self.v, lr, 0.9, 0.999, 1e-8, self.step)

    def state(self):
        return self.w.detach().cpu().numpy()


@dataclass
class PairSpec:
    """Coarse/fine mesh pair: shared particles, box, time grids and rays; meshes differ."""
    n_side: int = 256
    n_coarse: int = 256
    n_fine: int = 1024
    box: float = 256.0
    a_init: float = 0.02
    n_forward: int = 32
    a_min: float = 0.5
    n_reverse: int = 16
    n_pix: int = 1024
    fov_deg: float = 3.5
    omega_m: float = 0.3
    h: float = 0.7
    n_s: float = 0.96
    sigma8: float = 0.8
    deconv_p: float = 4.0
    smooth_cells: float = 1.0
    nbins: int = 20
    ell_cut: float = 1.0e4

    @property
    def forward_grid(self):
        return [self.a_init + (1.0 - self.a_init) * i / self.n_forward for i in range(self.n_forward + 1)]

    @property
    def reverse_grid(self):
        return [1.0 - (1.0 - self.a_min) * i / self.n_reverse for i in range(self.n_reverse + 1)]

    @property
    def observer(self):
        return (0.5 * self.box, 0.5 * self.box, 0.0)

    @property
    def dtheta(self):
        return self.fov_deg * math.pi / 180.0 / self.n_pix

    @property
    def ell_range(self):
        return 2.0 * math.pi / (self.n_pix * self.dtheta), math.pi / self.dtheta


def _theta0(S: PairSpec) -> torch.Tensor:
    d = S.fov_deg * math.pi / 180.0 / S.n_pix
    c = (torch.arange(S.n_pix, dtype=torch.float64) + 0.5 - 0.5 * S.n_pix) * d
    ty, tx = torch.meshgrid(c, c, indexing="ij")
    return torch.stack([tx.reshape(-1), ty.reshape(-1)], dim=1).cuda()


def _noise(seed: int, n: int) -> torch.Tensor:
    w = np.random.default_rng(seed).standard_normal((n, n, n))
    return torch.tensor(w, dtype=torch.float32, device="cuda")


def plain_run(S: PairSpec, n_mesh: int, seed: int, record_spectra: bool = False):
    """Plain HRT run on an n_mesh^3 mesh (context API): returns (kappa map, [density spectra per reverse step])."""
    kappa, spectra, _ = run(S, n_mesh, seed, record_spectra=record_spectra)
    return kappa, spectra


def run(S: PairSpec, n_mesh: int, seed: int, params: torch.Tensor | None = None, record_spectra: bool = False,
        timed: bool = False, pparams: torch.Tensor | None = None):
    """HRT run on an n_mesh^3 mesh through the context API, with the learned ray correction ``params`` and the
    learned particle-force correction ``pparams`` (None: plain; without a ray correction the rays read the
    particle fields, corrected or not).  Returns (kappa map, [density spectra per reverse step], milliseconds of
    the reverse co-evolution steps (CUDA events on the context's stream) or None)."""
    cfg = hrt.make_config(n_mesh, S.box, S.n_side, S.omega_m, S.h, S.n_s, S.sigma8, S.deconv_p, S.smooth_cells,
                          1.0, S.observer, n_sources=1, ray_fields=0 if params is None else 2,
                          ray_deconv_p=S.deconv_p, ray_smooth_cells=S.smooth_cells)
    ctx = hrt.Context(cfg)
    if params is not None:
        ctx.hrt_set_ray_correction(params)
    if pparams is not None:
        ctx.hrt_set_particle_correction(pparams)
    ctx.hrt_init_particles_zeldovich(_noise(seed, S.n_side).reshape(-1), S.a_init)
    for a in S.forward_grid[1:]:
        ctx.hrt_step(a)
    ctx.hrt_sync_particles()
    ctx.hrt_init_rays(_theta0(S))
    spectra = []
    rg = S.reverse_grid
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)] if timed else None
    if timed:
        torch.cuda.synchronize()
        ev[0].record()
    for n in range(S.n_reverse):
        if record_spectra:
            spectra.append(_ctx_density_spectrum(ctx, S, n_mesh, rg[n]))
        ctx.hrt_step(rg[n + 1], 0 if n + 1 == S.n_reverse else -1)
    ms = None
    if timed:
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
    kappa = ctx.hrt_read_maps(0)[0].clone()
    ctx.close()
    return kappa, spectra, ms


def _ctx_density_spectrum(ctx, S, n_mesh, a):
    """Density spectrum of the context's current particles (the density behind its current force)."""
    disp, _, _, _ = ctx.hrt_read_particles()
    rho = torch.empty(n_mesh ** 3, device="cuda")
    hrt.hrt_cic_scatter(disp, S.n_side, n_mesh, S.box, rho)
    pm = _pm_cache(n_mesh, S.box)
    spec = torch.empty(n_mesh, n_mesh, n_mesh // 2 + 1, dtype=torch.complex64, device="cuda")
    pm.forward_fft(rho, spec)
    return spec


_PMS: dict = {}


def _pm_cache(n, box):
    key = (n, box)
    if key not in _PMS:
        _PMS[key] = hrt.PM(n, box)
    return _PMS[key]


def power(S: PairSpec, kappa: torch.Tensor):
    lmin, lmax = S.ell_range
    return hrt.hrt_kappa_power(kappa.contiguous(), S.n_pix, S.dtheta, S.nbins, lmin, lmax)


class RayTrainer:
    """Ray-only forward/backward of the coarse run with the learned ray table, on stored density spectra."""

    def __init__(self, S: PairSpec):
        self.S = S
        n = S.n_coarse
        self.cell = S.box / n
        self.kmax = math.sqrt(3.0) * math.pi / self.cell * 1.0001
        self.pm = _pm_cache(n, S.box)
        self.geom = hrt.make_geom(n, S.box, S.observer, 1.0, image_width=S.n_pix)
        self.theta0 = _theta0(S)
        rg = S.reverse_grid
        self.steps = []
        for i in range(S.n_reverse):
            a0, a1 = rg[i], rg[i + 1]
            self.steps.append((a0, a1, hrt.hrt_cosmo_eval(S.omega_m, a0)[1], hrt.hrt_cosmo_eval(S.omega_m, a1)[1]))
        self.x = [MLP.inputs(self.kmax, self.cell, a0, n) for (a0, _, _, _) in self.steps]

    def _filter(self, table):
        return hrt.make_filter(self.S.deconv_p, self.S.smooth_cells * self.cell, table, self.kmax)

    def forward(self, mlp: MLP | None, spectra, keep: bool):
        S, n = self.S, self.S.n_coarse
        rays = hrt.RayState(self.theta0.shape[0])
        hrt.hrt_rays_init(rays, self.theta0)
        maps = torch.empty(4, rays.n_rays, device="cuda")
        saved = []
        for i, (a0, a1, c0, c1) in enumerate(self.steps):
            table = mlp.table(self.x[i]) if mlp is not None else torch.ones(N_TABLE, device="cuda")
            f = self._filter(table)
            fields = torch.empty(2, n ** 3, device="cuda")
            self.pm.gradient_from_spectrum(spectra[i], 1.5 * S.omega_m / a0, f, 2, fields)
            if keep:
                pre = hrt.RayState(rays.n_rays)
                for name in ("theta", "eta", "A", "B"):
                    getattr(pre, name).copy_(getattr(rays, name))
                saved.append((pre, fields, table))
            hrt.hrt_ray_step(rays, fields[0], fields[1], self.geom, c0, c1, a0, S.omega_m,
                             maps if i + 1 == len(self.steps) else None)
        return maps[0].clone(), saved

    def backward(self, mlp: MLP, spectra, saved, kappa_bar, grad):
        S, n = self.S, self.S.n_coarse
        r_bar = hrt.RayState(self.theta0.shape[0])
        for name in ("theta", "eta", "A", "B"):
            getattr(r_bar, name).zero_()
        r_bar.A[:, 0] -= 0.5 * kappa_bar
        r_bar.A[:, 3] -= 0.5 * kappa_bar
        nb = torch.zeros(3, hrt.MAX_RAY_NODES, dtype=torch.float64, device="cuda")
        db = torch.zeros(1, dtype=torch.float64, device="cuda")
        gbar_hat = torch.empty(2, n, n, n // 2 + 1, dtype=torch.complex64, device="cuda")
        for i in reversed(range(len(self.steps))):
            a0, a1, c0, c1 = self.steps[i]
            pre, fields, table = saved[i]
            gb = torch.zeros(2, n ** 3, device="cuda")
            hrt.hrt_ray_step_adjoint(pre, fields[0], fields[1], self.geom, c0, c1, a0, S.omega_m, r_bar, gb[0], gb[1],
                                     nb, db)
            self.pm.forward_fft(gb[0], gbar_hat[0])
            self.pm.forward_fft(gb[1], gbar_hat[1])
            tb = torch.zeros(N_TABLE, device="cuda")
            hrt.hrt_kspace_table_adjoint(gbar_hat, 2, spectra[i], n, S.box, 1.5 * S.omega_m / a0, self._filter(table),
                                         tb)
            mlp.accumulate(self.x[i], tb, grad)


class ForceTrainer:
    """Force matching of the particle correction (the analogue of the trained force sharpening of Sec. 6.2): at
    snapshots of fine-mesh runs, the coarse-mesh PM force with the learned factor g, interpolated at the
    particles, against the fine-mesh force there.  Loss per snapshot: sum_p |F_coarse - F_fine|^2 / sum_p
    |F_fine|^2.  Gradients go through the gather adjoint (``hrt_particle_kick_drift_adjoint``), forward FFTs of
    the field cotangents and ``hrt_kspace_table_adjoint`` into the MLP; all arithmetic in libhrt kernels.

    anchor = (kcell, weight): adds weight * mean over the table rows with |k| cell < kcell of (g - 1)^2, which holds
    the factor at 1 on the large scales that the coarse mesh already resolves (the force error hardly weighs
    them, yet they set the growth of the large-scale power)."""

    def __init__(self, S: PairSpec, n_coarse: int, anchor=None):
        self.S, self.n = S, n_coarse
        self.anchor = anchor
        self.cell = S.box / n_coarse
        self.kmax = math.sqrt(3.0) * math.pi / self.cell * 1.0001
        self.pm = _pm_cache(n_coarse, S.box)
        self.samples = []

    def _filter(self, table):
        return hrt.make_filter(self.S.deconv_p, self.S.smooth_cells * self.cell, table, self.kmax)

    def add_seed(self, seed: int, snapshots):
        """Fine run of the seed (plain force) up to a = 1; at each snapshot a the particles, their fine-mesh force
        and the coarse density spectrum of the same particles."""
        S, n = self.S, self.n
        cfg = hrt.make_config(S.n_fine, S.box, S.n_side, S.omega_m, S.h, S.n_s, S.sigma8, S.deconv_p,
                              S.smooth_cells, 1.0, S.observer)
        ctx = hrt.Context(cfg)
        ctx.hrt_init_particles_zeldovich(_noise(seed, S.n_side).reshape(-1), S.a_init)
        want = sorted(snapshots)
        for a in S.forward_grid[1:]:
            ctx.hrt_step(a)
            while want and abs(a - want[0]) < 1e-9:
                disp, _, _, _ = ctx.hrt_read_particles()
                grad = ctx.hrt_read_grad()
                f_fine = torch.zeros(3, S.n_side ** 3, device="cuda")
                hrt.hrt_particle_kick_drift(grad, S.n_fine, S.box, S.n_side, disp.clone(), f_fine, -1.0, 0.0)
                del grad
                rho = torch.empty(n ** 3, device="cuda")
                hrt.hrt_cic_scatter(disp, S.n_side, n, S.box, rho)
                spec = torch.empty(n, n, n // 2 + 1, dtype=torch.complex64, device="cuda")
                self.pm.forward_fft(rho, spec)
                self.samples.append(dict(a=a, disp=disp, f_fine=f_fine, norm=float((f_fine.double() ** 2).sum()),
                                         spec=spec, x=MLP.inputs(self.kmax, self.cell, a, n)))
                want.pop(0)
        ctx.close()

    def loss_and_grad(self, mlp: MLP | None, sample, grad=None):
        """Relative force error of one snapshot; with grad, adds the MLP parameter gradient."""
        S, n = self.S, self.n
        table = mlp.table(sample["x"]) if mlp is not None else torch.ones(N_TABLE, device="cuda")
        f = self._filter(table)
        pref = 1.5 * S.omega_m / sample["a"]
        fields = torch.empty(3, n ** 3, device="cuda")
        self.pm.gradient_from_spectrum(sample["spec"], pref, f, 3, fields)
        zeros = torch.zeros(3, S.n_side ** 3, device="cuda")
        fc = zeros.clone()
        disp = sample["disp"]
        hrt.hrt_particle_kick_drift(fields, n, S.box, S.n_side, disp.clone(), fc, -1.0, 0.0)
        r = fc - sample["f_fine"]
        loss = float((r.double() ** 2).sum()) / sample["norm"]
        low = None
        if self.anchor is not None and mlp is not None:
            kcell, weight = self.anchor
            low = (sample["x"][:, 0] < kcell).to(torch.float32)
            nlow = max(float(low.sum()), 1.0)
            loss += weight * float((low * (table - 1.0) ** 2).sum()) / nlow
        if grad is not None:
            m_bar = (2.0 / sample["norm"]) * r
            g_bar = torch.zeros(3, n ** 3, device="cuda")
            hrt.hrt_particle_kick_drift_adjoint(fields, n, S.box, S.n_side, disp.clone(), zeros, -1.0, 0.0, None,
                                                torch.zeros_like(zeros), m_bar.contiguous(), g_bar,
                                                torch.zeros(2, dtype=torch.float64, device="cuda"))
            gbar_hat = torch.empty(3, n, n, n // 2 + 1, dtype=torch.complex64, device="cuda")
            for j in range(3):
                self.pm.forward_fft(g_bar[j].contiguous(), gbar_hat[j])
            tb = torch.zeros(N_TABLE, device="cuda")
            hrt.hrt_kspace_table_adjoint(gbar_hat, 3, sample["spec"], n, S.box, pref, f, tb)
            if low is not None:
                tb += (2.0 * self.anchor[1] / nlow) * low * (table - 1.0)
            mlp.accumulate(sample["x"], tb, grad)
        return loss


def train_particle(S: PairSpec, train_seeds, test_seeds, iters: int = 300, lr: float = 2e-3, log=print,
                   snapshots=(0.2, 0.4, 0.6, 0.8, 1.0), meshes=None, anchor=None):
    """Adam on the particle-correction MLP by force matching (ForceTrainer), over the coarse meshes (default
    S.n_coarse; ln N_mesh is an input, so one network serves them all) and the training seeds' snapshots; returns
    the network and the relative force errors of the plain and the learned coarse force on the held-out seeds."""
    meshes = tuple(meshes) if meshes else (S.n_coarse,)
    t0 = time.time()
    fg = S.forward_grid
    snaps = sorted({min(fg[1:], key=lambda a: abs(a - t)) for t in snapshots})
    trainers = {m: ForceTrainer(S, m, anchor) for m in meshes}
    test = {m: ForceTrainer(S, m) for m in meshes}
    for m in meshes:
        for s in train_seeds:
            trainers[m].add_seed(s, snaps)
        for s in test_seeds:
            test[m].add_seed(s, snaps)
    log(f"force snapshots: {len(train_seeds)} + {len(test_seeds)} seeds x {len(snaps)} times x {len(meshes)} meshes "
        f"in {time.time() - t0:.1f} s")
    mlp = MLP(seed=1)
    history = []
    norm = sum(len(t.samples) for t in trainers.values())
    for it in range(iters):
        grad = torch.zeros(hrt.MLP_PARAMS, device="cuda")
        loss = 0.0
        for t in trainers.values():
            for smp in t.samples:
                loss += t.loss_and_grad(mlp, smp, grad) / norm
        grad /= norm
        mlp.adam(grad, lr)
        history.append(loss)
        if it % 25 == 0 or it == iters - 1:
            log(f"iter {it:3d} force loss {loss:.4e} ({time.time() - t0:.1f} s)")
    result = {"snapshots": snaps, "meshes": list(meshes), "train_seconds": time.time() - t0,
              "loss_first_last": [history[0], history[-1]], "held_out": {}}
    for m, t in test.items():
        plain = [t.loss_and_grad(None, smp) for smp in t.samples]
        learned_err = [t.loss_and_grad(mlp, smp) for smp in t.samples]
        result["held_out"][str(m)] = {"plain_rel_force_err2": float(np.mean(plain)),
                                      "learned_rel_force_err2": float(np.mean(learned_err))}
    return mlp, result


def _bins(S: PairSpec, ell, cnt):
    return (cnt > 0) & (ell <= S.ell_cut)


def train(S: PairSpec, train_seeds, test_seeds, iters: int = 60, lr: float = 2e-3, log=print, meshes=None,
          batch_seeds: int = 0):
    """Adam on the MLP parameters: loss = mean over coarse meshes and training seeds of sum over the bins with
    ell <= S.ell_cut of (P_coarse / P_fine - 1)^2, each coarse mesh paired with the S.n_fine run of the same ICs
    (meshes: the coarse sides, default S.n_coarse; ln N_mesh is an input, so one network serves them all).  With
    batch_seeds > 0 each Adam step uses that many training seeds drawn without replacement (a seeded generator),
    which keeps the cost of a step bounded at large ray counts while every seed takes part in the training."""
    meshes = tuple(meshes) if meshes else (S.n_coarse,)
    t0 = time.time()
    fine, spectra, plain_p = {}, {}, {}
    for s in list(train_seeds) + list(test_seeds):
        kf, _ = plain_run(S, S.n_fine, s)
        ell, pf, cnt = power(S, kf)
        fine[s] = pf
        for m in meshes:
            kc, sp = plain_run(S, m, s, record_spectra=True)
            spectra[(m, s)], plain_p[(m, s)] = sp, power(S, kc)[1]
    sel = _bins(S, ell, cnt)
    log(f"paired runs: {len(fine)} seeds x {len(meshes)} meshes in {time.time() - t0:.1f} s")
    trainers = {m: RayTrainer(replace(S, n_coarse=m)) for m in meshes}
    mlp = MLP(seed=0)
    history = []
    train_seeds = list(train_seeds)
    per_step = batch_seeds if 0 < batch_seeds < len(train_seeds) else len(train_seeds)
    pick = np.random.default_rng(12345)
    norm = per_step * len(meshes)
    lmin, lmax = S.ell_range
    for it in range(iters):
        grad = torch.zeros(hrt.MLP_PARAMS, device="cuda")
        loss = 0.0
        batch = (train_seeds if per_step == len(train_seeds)
                 else sorted(pick.choice(train_seeds, size=per_step, replace=False).tolist()))
        for m in meshes:
            for s in batch:
                kappa, saved = trainers[m].forward(mlp, spectra[(m, s)], keep=True)
                _, p, _ = power(S, kappa)
                r = p / fine[s] - 1.0
                loss += float((r[sel] ** 2).sum()) / norm
                p_bar = np.where(sel, 2.0 * r / fine[s], 0.0) / norm
                kb = torch.empty_like(kappa)
                hrt.hrt_kappa_power_adjoint(kappa, S.n_pix, S.dtheta, S.nbins, lmin, lmax, p_bar, kb)
                trainers[m].backward(mlp, spectra[(m, s)], saved, kb, grad)
                del saved
        mlp.adam(grad, lr)
        history.append(loss)
        if it % 10 == 0 or it == iters - 1:
            log(f"iter {it:3d} loss {loss:.4e} ({time.time() - t0:.1f} s)")
    per_mesh = {m: evaluate(S, trainers[m], mlp, test_seeds, fine, {s: spectra[(m, s)] for s in test_seeds},
                            {s: plain_p[(m, s)] for s in test_seeds}, sel) for m in meshes}
    result = dict(per_mesh[meshes[0]]) if len(meshes) == 1 else {
        "per_mesh": per_mesh,
        **{k: float(np.mean([r[k] for r in per_mesh.values()])) for k in
           ("plain_mean_rel_err", "learned_mean_rel_err", "plain_max_rel_err", "learned_max_rel_err")}}
    result["meshes"] = list(meshes)
    result["history"] = history
    result["train_seconds"] = time.time() - t0
    return mlp, result


def evaluate(S, trainer, mlp, seeds, fine, spectra, plain_p, sel):
    err_plain, err_learned = [], []
    for s in seeds:
        kappa, _ = trainer.forward(mlp, spectra[s], keep=False)
        _, p, _ = power(S, kappa)
        err_learned.append(np.abs(p[sel] / fine[s][sel] - 1.0))
        err_plain.append(np.abs(plain_p[s][sel] / fine[s][sel] - 1.0))
    ep, el = np.array(err_plain), np.array(err_learned)
    return {"bins": int(sel.sum()), "plain_mean_rel_err": float(ep.mean()), "plain_max_rel_err": float(ep.max()),
            "learned_mean_rel_err": float(el.mean()), "learned_max_rel_err": float(el.max()),
            "plain_err_per_bin": ep.mean(axis=0).tolist(), "learned_err_per_bin": el.mean(axis=0).tolist()}


def compare(S: PairSpec, params: torch.Tensor, seeds, log=print):
    """The learned form against the plain one at equal cost and against the fine mesh: per held-out seed, the
    coarse plain, coarse learned and fine plain runs; P(ell) relative errors of both coarse forms against the
    fine run (bins with ell <= S.ell_cut), and the reverse co-evolution rate (particles + rays, sim-steps/s)
    of each form, timed with CUDA events (the first seed's runs are an untimed warm-up of plans and memory)."""
    rates = {"coarse_plain": [], "coarse_learned": [], "fine_plain": []}
    err_plain, err_learned = [], []
    for i, s in enumerate([seeds[0]] + list(seeds)):
        kf, _, mf = run(S, S.n_fine, s, timed=True)
        kc, _, mc = run(S, S.n_coarse, s, timed=True)
        kl, _, ml = run(S, S.n_coarse, s, params=params, timed=True)
        if i == 0:
            continue
        ell, pf, cnt = power(S, kf)
        sel = _bins(S, ell, cnt)
        err_plain.append(np.abs(power(S, kc)[1][sel] / pf[sel] - 1.0))
        err_learned.append(np.abs(power(S, kl)[1][sel] / pf[sel] - 1.0))
        for k, ms in (("fine_plain", mf), ("coarse_plain", mc), ("coarse_learned", ml)):
            rates[k].append(S.n_reverse / (ms * 1e-3))
        log(f"seed {s}: plain err {err_plain[-1].mean():.4f} learned err {err_learned[-1].mean():.4f}; "
            f"sim-steps/s fine {rates['fine_plain'][-1]:.1f} coarse {rates['coarse_plain'][-1]:.1f} "
            f"learned {rates['coarse_learned'][-1]:.1f}")
    ep, el = np.array(err_plain), np.array(err_learned)
    return {"seeds": list(seeds), "n_pix": S.n_pix, "bins": int(ep.shape[1]),
            "sim_steps_per_s": {k: float(np.median(v)) for k, v in rates.items()},
            "plain_mean_rel_err": float(ep.mean()), "plain_max_rel_err": float(ep.max()),
            "learned_mean_rel_err": float(el.mean()), "learned_max_rel_err": float(el.max()),
            "plain_err_per_bin": ep.mean(axis=0).tolist(), "learned_err_per_bin": el.mean(axis=0).tolist()}


def ell_within(ell, rel, tol: float = 0.01) -> float:
    """Largest bin ell up to which every bin's relative error is within tol (0 if the first bin is not)."""
    last = 0.0
    for e, r in zip(ell, rel):
        if not r <= tol:
            break
        last = float(e)
    return last


def ladder_seeds(S: PairSpec, seeds, meshes=(256, 512, 768), cuts=None, learned_forms=(), log=print):
    """``ladder`` on several held-out seeds: per form the median sim-steps/s and, per ell cut, the largest and the
    mean P(ell) error over the seeds and bins, the largest error per bin over the seeds, the ell up to which every
    bin is within 1 % on every seed, and whether all bins with ell <= cut are within 1 % on every seed; then, for
    the plain and the learned forms, the coarsest mesh that meets 1 % in every bin up to each cut on all seeds
    (None when none does), per form name."""
    cuts = tuple(cuts) if cuts else (S.ell_cut,)
    per_seed = [ladder(S, None, s, meshes=meshes, cuts=cuts, log=log, learned_forms=list(learned_forms))
                for s in seeds]
    forms = []
    for i, row in enumerate(per_seed[0]):
        rows = [ps[i] for ps in per_seed]
        out = {"mesh": row["mesh"], "form": row["form"],
               "sim_steps_per_s": float(np.median([r["sim_steps_per_s"] for r in rows]))}
        if "errors" in row:
            out["errors"] = {}
            for key in row["errors"]:
                errs = [r["errors"][key] for r in rows]
                per_bin = np.max(np.array([e["per_bin"] for e in errs]), axis=0)
                out["errors"][key] = {
                    "bins": errs[0]["bins"], "max_rel_err": float(max(e["max_rel_err"] for e in errs)),
                    "mean_rel_err": float(np.mean([e["mean_rel_err"] for e in errs])),
                    "ell_within_1pct_all_seeds": float(min(e["ell_within_1pct"] for e in errs)),
                    "meets_1pct_all_seeds": bool(per_bin.max() <= 0.01),
                    "max_rel_err_per_bin": [float(x) for x in per_bin],
                    "bin_ell": errs[0]["ell"]}
        forms.append(out)
    coarsest = {}
    names = sorted({f["form"] for f in forms if "errors" in f})
    for key in [f"ell_le_{c:g}" for c in cuts]:
        for name in names:
            ok = [f["mesh"] for f in forms
                  if f["form"] == name and "errors" in f and f["errors"][key]["meets_1pct_all_seeds"]]
            coarsest[f"{name}, {key}"] = min(ok) if ok else None
    return {"seeds": list(seeds), "forms": forms, "coarsest_mesh_within_1pct": coarsest}


def ladder(S: PairSpec, params: torch.Tensor | None, seed: int, meshes=(256, 512, 768), cuts=None, log=print,
           learned_meshes=None, learned_forms=None):
    """Accuracy against speed on one held-out seed: for each coarse mesh the plain form, and the learned forms
    (learned_forms: (mesh, ray parameters or None, name[, particle parameters]); else params at learned_meshes)
    against the plain S.n_fine run: reverse co-evolution sim-steps/s, and for each ell cut (default S.ell_cut) the
    mean and largest P(ell) error over the bins with ell <= cut and the ell up to which every bin is within 1 %."""
    cuts = tuple(cuts) if cuts else (S.ell_cut,)
    run(S, S.n_fine, seed)  # warm-up of plans and memory
    kf, _, mf = run(S, S.n_fine, seed, timed=True)
    ell, pf, cnt = power(S, kf)
    rows = [{"mesh": S.n_fine, "form": "plain", "sim_steps_per_s": S.n_reverse / (mf * 1e-3)}]
    lm = tuple(learned_meshes) if learned_meshes else (S.n_coarse,)
    forms = [(m, None, "plain") for m in meshes]
    if learned_forms:
        forms += list(learned_forms)
    elif params is not None:
        forms += [(m, params, "learned") for m in lm]
    for form in forms:
        m, w, name = form[:3]
        wp = form[3] if len(form) > 3 else None
        run(S, m, seed, params=w, pparams=wp)
        k, _, ms = run(S, m, seed, params=w, timed=True, pparams=wp)
        p = power(S, k)[1]
        row = {"mesh": m, "form": name,
               "sim_steps_per_s": S.n_reverse / (ms * 1e-3), "errors": {}}
        for cut in cuts:
            sel = (cnt > 0) & (ell <= cut)
            rel = np.abs(p[sel] / pf[sel] - 1.0)
            row["errors"][f"ell_le_{cut:g}"] = {"bins": int(sel.sum()), "mean_rel_err": float(rel.mean()),
                                                "max_rel_err": float(rel.max()),
                                                "ell_within_1pct": ell_within(ell[sel], rel),
                                                "per_bin": [float(x) for x in rel],
                                                "ell": [float(x) for x in ell[sel]]}
        rows.append(row)
        log(str(row))
    return rows


def main():
    ap = argparse.ArgumentParser(description="train and evaluate the learned ray-force correction")
    ap.add_argument("--train-seeds", type=int, default=16)
    ap.add_argument("--test-seeds", type=int, default=4)
    ap.add_argument("--iters", type=int, default=60)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--n-pix", type=int, default=1024)
    ap.add_argument("--out", default=None, help="write the trained FP32 parameters (.npy) here")
    ap.add_argument("--compare-n-pix", type=int, default=4096,
                    help="rays per side of the learned/plain/fine comparison on the held-out seeds (0: skip)")
    ap.add_argument("--params", default=None, help="skip training: compare with these parameters (.npy)")
    ap.add_argument("--ell-cut", type=float, default=PairSpec.ell_cut, help="largest bin ell in the training loss")
    ap.add_argument("--meshes", default=None, help="coarse mesh sides to train on, e.g. 256,512 (default 256)")
    ap.add_argument("--ladder-n-pix", type=int, default=0,
                    help="rays per side of the accuracy-vs-speed ladder on the first held-out seed (0: skip)")
    ap.add_argument("--batch-seeds", type=int, default=0,
                    help="training seeds per Adam step, drawn from the training seeds (0: all)")
    ap.add_argument("--particle", action="store_true",
                    help="train the particle-force correction by force matching instead of the ray correction")
    ap.add_argument("--anchor-kcell", type=float, default=0.0,
                    help="particle training: hold g at 1 for |k| cell below this (0: no anchor)")
    ap.add_argument("--anchor-weight", type=float, default=10.0, help="weight of that penalty")
    a = ap.parse_args()
    S = replace(PairSpec(), n_pix=a.n_pix, ell_cut=a.ell_cut)
    test = list(range(100, 100 + a.test_seeds))
    out = {}
    if a.particle:
        meshes = tuple(int(x) for x in a.meshes.split(",")) if a.meshes else None
        anchor = (a.anchor_kcell, a.anchor_weight) if a.anchor_kcell > 0 else None
        mlp, res = train_particle(S, range(a.train_seeds), test, a.iters, a.lr, log=lambda m: print(m, flush=True),
                                  meshes=meshes, anchor=anchor)
        if a.out:
            np.save(a.out, mlp.state())
        print(json.dumps({"particle_training": res}))
        return
    if a.params:
        w = torch.tensor(np.load(a.params), dtype=torch.float32, device="cuda")
    else:
        meshes = tuple(int(x) for x in a.meshes.split(",")) if a.meshes else None
        mlp, res = train(S, range(a.train_seeds), test, a.iters, a.lr, log=lambda m: print(m, flush=True),
                         meshes=meshes, batch_seeds=a.batch_seeds)
        if a.out:
            np.save(a.out, mlp.state())
        w = mlp.w
        out["training"] = {k: v for k, v in res.items() if k != "history"}
        out["training"]["loss_first_last"] = [res["history"][0], res["history"][-1]]
    if a.compare_n_pix:
        out["comparison"] = compare(replace(S, n_pix=a.compare_n_pix), w, test, log=lambda m: print(m, flush=True))
    if a.ladder_n_pix:
        out["ladder"] = ladder(replace(S, n_pix=a.ladder_n_pix), w, test[0],
                               cuts=sorted({a.ell_cut, PairSpec.ell_cut}), log=lambda m: print(m, flush=True),
                               learned_meshes=tuple(int(x) for x in a.meshes.split(",")) if a.meshes else None)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
