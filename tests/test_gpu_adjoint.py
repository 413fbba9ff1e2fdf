"""Adjoint kernels and the differentiable simulation against the FP64 oracle's autograd and finite differences.

Each adjoint kernel is the vector-Jacobian product of its forward kernel; the oracle's torch-float64 functions
give the same products by autograd.  Float32 kernels against float64 autograd agree to ~1e-5 of the scale of each
cotangent; the end-to-end gradients through a whole run agree to the accumulated float32 rounding (1e-3)."""
import math

import numpy as np
import pytest
import torch

import synthetic
from oracle import pm as opm
from oracle import rays as orays
from oracle import sim as osim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrt():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt as h
    return h


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _close(got, want, rel):
    got, want = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    scale = np.abs(want).max()
    assert scale > 0
    err = np.abs(got - want).max() / scale
    assert err <= rel, err


def test_deposit_adjoint_matches_autograd(hrt):
    n_side, n, box = 16, 32, 48.0
    disp = synthetic.small_displacements(31, n_side, 2.0)
    rho_bar = synthetic.gaussian_field(32, (n ** 3,))
    db = torch.zeros(3, n_side ** 3, device="cuda")
    hrt.hrt_cic_scatter_adjoint(_cuda(rho_bar), _cuda(disp), n_side, n, box, db)
    d = torch.tensor(disp.T.copy(), requires_grad=True)
    rho = opm.cic_deposit(opm.lattice(n_side, box) + d, box, n)
    (rho.reshape(-1) * torch.tensor(rho_bar)).sum().backward()
    _close(db.cpu().numpy(), d.grad.numpy().T, 2e-5)


def test_pm_solve_adjoint_matches_autograd(hrt):
    n, box, pref = 32, 64.0, 0.8
    rho = synthetic.gaussian_field(33, (n, n, n), 0.4) + 1.0
    gbar = synthetic.gaussian_field(34, (3, n, n, n))
    pm = hrt.PM(n, box)
    f = hrt.make_filter(4.0, box / n)
    rb = torch.empty(n ** 3, device="cuda")
    pm.solve_adjoint(_cuda(gbar), pref, f, rb)
    r = torch.tensor(rho, requires_grad=True)
    g = opm.poisson_gradient(r, box, pref, 4.0, box / n)
    sum((gj * torch.tensor(gbar[j])).sum() for j, gj in enumerate(g)).backward()
    _close(rb.cpu().numpy(), r.grad.numpy().reshape(-1), 2e-5)
    pm.close()


@pytest.mark.parametrize("fused", [False, True])
def test_kick_drift_adjoint_matches_autograd(hrt, fused):
    n_side, n, box, kick, drift = 16, 32, 48.0, 0.17, 0.43
    disp = synthetic.small_displacements(35, n_side, 1.5)
    mom = synthetic.small_displacements(36, n_side, 1.0)
    grads = synthetic.gaussian_field(37, (3, n, n, n))
    dbar1 = synthetic.gaussian_field(38, (3, n_side ** 3))
    mbar1 = synthetic.gaussian_field(39, (3, n_side ** 3))
    rho_bar = synthetic.gaussian_field(40, (n ** 3,)) if fused else None
    db, mb = _cuda(dbar1), _cuda(mbar1)
    gb = torch.zeros(3, n ** 3, device="cuda")
    cb = torch.zeros(2, dtype=torch.float64, device="cuda")
    hrt.hrt_particle_kick_drift_adjoint(_cuda(grads), n, box, n_side, _cuda(disp), _cuda(mom), kick, drift,
                                        _cuda(rho_bar) if fused else None, db, mb, gb, cb)
    q = opm.lattice(n_side, box)
    d = torch.tensor(disp.T.copy(), requires_grad=True)
    m = torch.tensor(mom.T.copy(), requires_grad=True)
    g = [torch.tensor(grads[j], requires_grad=True) for j in range(3)]
    K = torch.tensor(kick, dtype=torch.float64, requires_grad=True)
    D = torch.tensor(drift, dtype=torch.float64, requires_grad=True)
    d1, m1 = opm.particle_kick_drift(d, m, q, g, box, K, D)
    loss = (d1 * torch.tensor(dbar1.T)).sum() + (m1 * torch.tensor(mbar1.T)).sum()
    if fused:
        loss = loss + (opm.cic_deposit(q + d1, box, n).reshape(-1) * torch.tensor(rho_bar)).sum()
    loss.backward()
    _close(db.cpu().numpy(), d.grad.numpy().T, 3e-5)
    _close(mb.cpu().numpy(), m.grad.numpy().T, 3e-5)
    for j in range(3):
        _close(gb[j].cpu().numpy(), g[j].grad.numpy().reshape(-1), 2e-5)
    c = cb.cpu().numpy()
    assert c[0] == pytest.approx(float(K.grad), rel=2e-5)
    assert c[1] == pytest.approx(float(D.grad), rel=2e-5)


def _smooth(n, box, seed):
    rng = np.random.default_rng(seed)
    g = np.arange(n) * box / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    gx, gy = np.zeros((n, n, n)), np.zeros((n, n, n))
    for _ in range(6):
        mm = rng.integers(-3, 4, size=3)
        k = 2 * math.pi * mm / box
        a, ph = rng.normal() * 3e3, rng.uniform(0, 2 * math.pi)
        arg = k[0] * X + k[1] * Y + k[2] * Z + ph
        gx += -a * k[0] * np.sin(arg)
        gy += -a * k[1] * np.sin(arg)
    return gx, gy


@pytest.mark.parametrize("a_ref,c0,c1", [(0.0, 210.0, 300.0), (0.75, 650.0, 760.0)])
def test_ray_step_adjoint_matches_autograd(hrt, a_ref, c0, c1):
    n, box, obs, s = 32, 64.0, (20.3, 41.7, 3.0), 1.0
    gx, gy = _smooth(n, box, 41)
    theta0 = synthetic.pixel_grid(19, 0.25)
    wfn = (lambda chi: 1.0) if a_ref == 0.0 else osim.growth_weight(a_ref, 0.3)
    # a non-trivial pre-step state: one oracle step from the observer side
    pre = orays.ray_step(orays.init_state(torch.tensor(theta0)), torch.tensor(gx), torch.tensor(gy), box, obs,
                         0.6 * c0, c0, s, wfn)
    R = theta0.shape[0]
    rays = hrt.RayState(R)
    rays.theta.copy_(pre["theta"])
    rays.eta.copy_(pre["eta"])
    rays.A.copy_(pre["A"].reshape(R, 4))
    rays.B.copy_(pre["B"].reshape(R, 4))
    cot = {k: synthetic.gaussian_field(50 + i, v.shape) for i, (k, v) in enumerate(pre.items())}
    cot["theta"] *= 1e3
    bar = hrt.RayState(R)
    bar.theta.copy_(torch.tensor(cot["theta"]))
    bar.eta.copy_(torch.tensor(cot["eta"]))
    bar.A.copy_(torch.tensor(cot["A"].reshape(R, 4)))
    bar.B.copy_(torch.tensor(cot["B"].reshape(R, 4)))
    gxb = torch.zeros(n ** 3, device="cuda")
    gyb = torch.zeros(n ** 3, device="cuda")
    nb = torch.zeros(3, 1024, dtype=torch.float64, device="cuda")
    drb = torch.zeros(1, dtype=torch.float64, device="cuda")
    geom = hrt.make_geom(n, box, obs, s)
    hrt.hrt_ray_step_adjoint(rays, _cuda(gx), _cuda(gy), geom, c0, c1, a_ref, 0.3, bar, gxb, gyb, nb, drb)
    st = {k: v.clone().requires_grad_(True) for k, v in pre.items()}
    fx = torch.tensor(gx, requires_grad=True)
    fy = torch.tensor(gy, requires_grad=True)
    out = orays.ray_step(st, fx, fy, box, obs, c0, c1, s, wfn)
    sum((out[k] * torch.tensor(cot[k])).sum() for k in out).backward()
    _close(bar.theta.cpu().numpy(), st["theta"].grad.numpy(), 2e-4)
    _close(bar.eta.cpu().numpy(), st["eta"].grad.numpy(), 2e-4)
    _close(bar.A.cpu().numpy(), st["A"].grad.numpy().reshape(R, 4), 2e-4)
    _close(bar.B.cpu().numpy(), st["B"].grad.numpy().reshape(R, 4), 2e-4)
    _close(gxb.cpu().numpy(), fx.grad.numpy().reshape(-1), 2e-4)
    _close(gyb.cpu().numpy(), fy.grad.numpy().reshape(-1), 2e-4)


@pytest.mark.parametrize("seed", [3, 4])
def test_tiled_ray_step_adjoint_matches_autograd(hrt, seed):
    # a step across replica boundaries of a light cone tiled by rotated, translated replicas
    n, box, obs, s = 32, 64.0, (20.3, 41.7, 3.0), 1.0
    reps = synthetic.replica_transforms(seed, 12, n)
    g3 = [synthetic.gaussian_field(90 + seed + c, (n, n, n), 3e3) for c in range(3)]
    theta0 = synthetic.pixel_grid(19, 0.25)
    a_ref, c0, c1 = 0.75, 100.0, 150.0
    wfn = osim.growth_weight(a_ref, 0.3)
    gt = [torch.tensor(g) for g in g3]
    pre = orays.ray_step(orays.init_state(torch.tensor(theta0)), gt[0], gt[1], box, obs, 60.0, c0, s, wfn, gz=gt[2],
                         replicas=reps)
    R = theta0.shape[0]
    rays = hrt.RayState(R)
    rays.theta.copy_(pre["theta"])
    rays.eta.copy_(pre["eta"])
    rays.A.copy_(pre["A"].reshape(R, 4))
    rays.B.copy_(pre["B"].reshape(R, 4))
    cot = {k: synthetic.gaussian_field(70 + i, v.shape) for i, (k, v) in enumerate(pre.items())}
    cot["theta"] *= 1e3
    bar = hrt.RayState(R)
    bar.theta.copy_(torch.tensor(cot["theta"]))
    bar.eta.copy_(torch.tensor(cot["eta"]))
    bar.A.copy_(torch.tensor(cot["A"].reshape(R, 4)))
    bar.B.copy_(torch.tensor(cot["B"].reshape(R, 4)))
    gb = torch.zeros(3, n ** 3, device="cuda")
    nb = torch.zeros(3, 1024, dtype=torch.float64, device="cuda")
    drb = torch.zeros(1, dtype=torch.float64, device="cuda")
    geom = hrt.make_geom(n, box, obs, s, replicas=reps)
    hrt.hrt_ray_step_tiled_adjoint(rays, _cuda(np.stack(g3)), geom, c0, c1, a_ref, 0.3, bar, gb, nb, drb)
    st = {k: v.clone().requires_grad_(True) for k, v in pre.items()}
    f3 = [torch.tensor(g, requires_grad=True) for g in g3]
    out = orays.ray_step(st, f3[0], f3[1], box, obs, c0, c1, s, wfn, gz=f3[2], replicas=reps)
    sum((out[k] * torch.tensor(cot[k])).sum() for k in out).backward()
    _close(bar.theta.cpu().numpy(), st["theta"].grad.numpy(), 2e-4)
    _close(bar.eta.cpu().numpy(), st["eta"].grad.numpy(), 2e-4)
    _close(bar.A.cpu().numpy(), st["A"].grad.numpy().reshape(R, 4), 2e-4)
    _close(bar.B.cpu().numpy(), st["B"].grad.numpy().reshape(R, 4), 2e-4)
    for c in range(3):
        _close(gb[c].cpu().numpy(), f3[c].grad.numpy().reshape(-1), 2e-4)


def test_kappa_power_adjoint_matches_autograd(hrt):
    m, dth, nb = 64, 4e-4, 8
    kap = synthetic.gaussian_field(60, (m, m), 0.02)
    lam = synthetic.gaussian_field(61, (nb,))
    lmin, lmax = 2 * math.pi / (m * dth), math.pi / dth
    kb = torch.empty(m * m, device="cuda")
    hrt.hrt_kappa_power_adjoint(_cuda(kap), m, dth, nb, lmin, lmax, lam, kb)
    # torch restatement of the binned power for autograd (bins as in the oracle)
    k = torch.tensor(kap, requires_grad=True)
    f = torch.fft.fft2(k)
    p = (f.abs() ** 2) * dth ** 4 / (m * dth) ** 2
    n = np.fft.fftfreq(m, 1.0 / m).round()
    ell = 2 * math.pi * np.sqrt(n[:, None] ** 2 + n[None, :] ** 2) / (m * dth)
    with np.errstate(divide="ignore"):
        t = nb * np.log(ell / lmin) / math.log(lmax / lmin) + 1e-9
    b = np.where((ell > 0) & (t >= 0) & (t < nb), np.floor(t), -1)
    loss = 0.0
    for i in range(nb):
        sel = torch.tensor(b == i)
        if sel.any():
            loss = loss + lam[i] * p[sel].mean()
    loss.backward()
    _close(kb.cpu().numpy(), k.grad.numpy().reshape(-1), 2e-5)


def test_ic_adjoint_matches_autograd(hrt):
    n, box, a = 16, 64.0, 0.1
    noise = synthetic.white_noise(62, n)
    dbar = synthetic.gaussian_field(63, (3, n ** 3))
    mbar = synthetic.gaussian_field(64, (3, n ** 3))
    disp = torch.empty(3, n ** 3, device="cuda")
    mom = torch.empty(3, n ** 3, device="cuda")
    hrt.hrt_ic_zeldovich(_cuda(noise), n, box, 0.3, 0.7, 0.96, 0.8, a, disp, mom)
    nb = torch.empty(n ** 3, device="cuda")
    hrt.hrt_ic_zeldovich_adjoint(_cuda(noise), n, box, 0.3, 0.7, 0.96, 0.8, a, _cuda(dbar), _cuda(mbar), disp, nb)
    w = torch.tensor(noise, requires_grad=True)
    d, mm = opm.zeldovich(w, box, 0.3, 0.7, 0.96, 0.8, a)
    ((d * torch.tensor(dbar.T)).sum() + (mm * torch.tensor(mbar.T)).sum()).backward()
    _close(nb.cpu().numpy(), w.grad.numpy().reshape(-1), 3e-5)


def test_2lpt_adjoint_matches_autograd(hrt):
    n, box, a = 16, 64.0, 0.1
    noise = synthetic.white_noise(65, n)
    dbar = synthetic.gaussian_field(66, (3, n ** 3))
    mbar = synthetic.gaussian_field(67, (3, n ** 3))
    nb = torch.empty(n ** 3, device="cuda")
    tb, cb = hrt.hrt_ic_2lpt_adjoint(_cuda(noise), n, box, 0.3, 0.7, 0.96, 0.8, a, _cuda(dbar), _cuda(mbar), nb)
    w = torch.tensor(noise, requires_grad=True)
    d, mm = opm.lpt2(w, box, 0.3, 0.7, 0.96, 0.8, a)
    ((d * torch.tensor(dbar.T)).sum() + (mm * torch.tensor(mbar.T)).sum()).backward()
    _close(nb.cpu().numpy(), w.grad.numpy().reshape(-1), 3e-5)
    # the second-order part is not negligible here: the first-order (Zel'dovich) transpose alone differs
    nz = torch.empty(n ** 3, device="cuda")
    disp = torch.empty(3, n ** 3, device="cuda")
    mom = torch.empty(3, n ** 3, device="cuda")
    hrt.hrt_ic_zeldovich(_cuda(noise), n, box, 0.3, 0.7, 0.96, 0.8, a, disp, mom)
    hrt.hrt_ic_zeldovich_adjoint(_cuda(noise), n, box, 0.3, 0.7, 0.96, 0.8, a, _cuda(dbar), _cuda(mbar), disp, nz)
    assert float((nz - nb).abs().max()) > 1e-3 * float(nb.abs().max())
    # the combine coefficients' cotangents: L is linear in them, so sum_k c_k dL/dc_k = L
    disp2 = torch.empty(3, n ** 3, device="cuda")
    mom2 = torch.empty(3, n ** 3, device="cuda")
    hrt.hrt_ic_2lpt(_cuda(noise), n, box, 0.3, 0.7, 0.96, 0.8, a, disp2, mom2)
    L = float((disp2.double() * _cuda(dbar).double()).sum() + (mom2.double() * _cuda(mbar).double()).sum())
    coefs = hrt.hrt_ic_2lpt_coefficients(0.3, 0.7, 0.96, 0.8, a)
    assert abs(float(coefs @ cb) - L) <= 1e-4 * abs(L)


def _oracle_run(W, noise, theta0, om):
    c = osim.Cosmo(om, W.h, W.n_s, W.sigma8)
    flt = osim.Filter(W.deconv_p, W.smooth_cells)
    part = osim.initial_particles(noise, W.box, c, W.a_init)
    part, grads = osim.run_forward(part, W.forward_grid, W.box, W.n_mesh, c, flt)
    res = osim.run_reverse(part, grads, W.reverse_grid, W.box, W.n_mesh, c, flt, theta0, W.observer,
                           set(W.source_steps), W.samples_per_cell)
    return torch.stack([res.maps[s][0] for s in W.source_steps]), res.rays["theta"]


def _torch_power(kap, m, dth, nb, lmin, lmax):
    """Binned power of a torch map (bins as in the oracle), differentiable for the reference gradient."""
    f = torch.fft.fft2(kap)
    p = (f.abs() ** 2) * dth ** 4 / (m * dth) ** 2
    n = np.fft.fftfreq(m, 1.0 / m).round()
    ell = 2 * math.pi * np.sqrt(n[:, None] ** 2 + n[None, :] ** 2) / (m * dth)
    with np.errstate(divide="ignore"):
        t = nb * np.log(ell / lmin) / math.log(lmax / lmin) + 1e-9
    b = np.where((ell > 0) & (t >= 0) & (t < nb), np.floor(t), -1)
    return torch.stack([p[torch.tensor(b == i)].mean() for i in range(nb)])


def _tiny_fd(fn, x, steps=(3e-8, 1e-7, 3e-7)):
    """Median of FP64 central differences at steps that resolve the pieces between derivative kinks (for a
    function that is continuous in x, like the final ray angles)."""
    vals = sorted((fn(x + e) - fn(x - e)) / (2 * e) for e in steps)
    return vals[len(vals) // 2]


def _piecewise_fd(fn, x, steps=(1e-8, 2e-8, 4e-8, 8e-8, 1.6e-7)):
    """FP64 central differences of a piecewise-smooth function at increasing tiny steps: those below the
    distance to the nearest jump agree with the derivative of the piece; larger ones straddle the jump."""
    return [(fn(x + e) - fn(x - e)) / (2 * e) for e in steps]


def test_end_to_end_gradient_matches_oracle(hrt):
    from paper_2405_12913_gb300 import autodiff
    from paper_2405_12913_gb300.configs import COSMO_GRAD as W
    noise = synthetic.white_noise(W.seed, W.n_side)
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE))
    kbar = synthetic.gaussian_field(70, (len(W.source_steps), W.n_rays))
    om0 = W.omega_m + 1.234e-6  # a generic point (no line-of-sight sample exactly on a cell face)
    # GPU: forward and adjoint through the autograd function (checkpoint every 2 steps)
    sim = autodiff.ContextSim(W, theta0, checkpoint_every=2)
    w_gpu = _cuda(noise).reshape(-1).requires_grad_(True)
    om_gpu = torch.tensor(om0, dtype=torch.float64, requires_grad=True)
    kap, _ = autodiff.HRTKappa.apply(w_gpu, om_gpu, sim)
    (kap.double() * _cuda(kbar, torch.float64)).sum().backward()
    g_gpu = w_gpu.grad.cpu().double().numpy()
    om_bar = float(om_gpu.grad)
    # oracle: autograd for the noise
    w = torch.tensor(noise, requires_grad=True)
    kap_o, _ = _oracle_run(W, w, theta0, om0)
    assert np.abs(kap.detach().cpu().numpy() - kap_o.detach().numpy()).max() <= 1e-3 * kap_o.detach().abs().max()
    (kap_o * torch.tensor(kbar)).sum().backward()
    g_o = w.grad.numpy().reshape(-1)
    rel = np.linalg.norm(g_gpu - g_o) / np.linalg.norm(g_o)
    assert rel < 2e-3, rel
    # Omega_m: kappa jumps where a line-of-sight sample crosses a cell face, and Omega_m moves every node;
    # the derivative of the piece is what the tiny steps below the nearest jump give
    with torch.no_grad():
        fds = _piecewise_fd(lambda om: float((_oracle_run(W, torch.tensor(noise), theta0, om)[0]
                                              * torch.tensor(kbar)).sum()), om0)
    agree = [abs(om_bar - v) <= 1e-3 * abs(v) for v in fds]
    assert sum(agree) >= 2, (om_bar, fds)
    sim.close()


def test_power_loss_gradient_matches_oracle(hrt):
    # the differentiation workload's loss: sum_ell (P(ell) - P_target(ell))^2 over the log ell bins
    from paper_2405_12913_gb300 import autodiff
    from paper_2405_12913_gb300.configs import COSMO_GRAD as W
    noise = synthetic.white_noise(W.seed + 1, W.n_side)
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE))
    lmin, lmax = W.ell_range
    target = torch.tensor(synthetic.gaussian_field(73, (W.nbins,), 1e-9)).abs()
    sim = autodiff.ContextSim(W, theta0, checkpoint_every=3)
    w = _cuda(noise).reshape(-1).requires_grad_(True)
    om = torch.tensor(W.omega_m, dtype=torch.float64, requires_grad=True)
    kap, _ = autodiff.HRTKappa.apply(w, om, sim)
    p = autodiff.KappaPower.apply(kap[0], W.n_pix, W.dtheta, W.nbins, lmin, lmax)
    scale = float((p.detach() ** 2).sum())
    (((p - target) ** 2).sum() / scale).backward()
    direction = synthetic.gaussian_field(74, (W.n_side ** 3,))
    ad = float((w.grad.cpu().double() * torch.tensor(direction)).sum())
    wo = torch.tensor(noise, requires_grad=True)

    def oracle_loss(wn, omv):
        k, _ = _oracle_run(W, wn, theta0, omv)
        po = _torch_power(k[0].reshape(W.n_pix, W.n_pix), W.n_pix, W.dtheta, W.nbins, lmin, lmax)
        return ((po - target) ** 2).sum() / scale

    oracle_loss(wo, W.omega_m).backward()
    ad_o = float((wo.grad.reshape(-1) * torch.tensor(direction)).sum())
    assert ad == pytest.approx(ad_o, rel=5e-3), (ad, ad_o)
    with torch.no_grad():
        fds = _piecewise_fd(lambda x: float(oracle_loss(torch.tensor(noise), x)), W.omega_m)
    assert sum(abs(float(om.grad) - v) <= 5e-3 * abs(v) for v in fds) >= 2, (float(om.grad), fds)
    sim.close()


def test_deflection_loss_gradient_matches_central_differences(hrt):
    # the final angles are continuous in the parameters: GPU adjoint vs GPU central differences, step 1e-3
    from paper_2405_12913_gb300 import autodiff
    from paper_2405_12913_gb300.configs import COSMO_GRAD as W
    noise = synthetic.white_noise(W.seed + 2, W.n_side)
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE))
    tb = _cuda(synthetic.gaussian_field(75, (W.n_rays, 2)), torch.float64)
    sim = autodiff.ContextSim(W, theta0, checkpoint_every=2)

    def loss(wn, omv):
        _, th = autodiff.HRTKappa.apply(wn, omv, sim)
        return ((th - theta0.cuda()) * tb).sum() * 1e4

    w = _cuda(noise).reshape(-1).requires_grad_(True)
    om = torch.tensor(W.omega_m, dtype=torch.float64, requires_grad=True)
    loss(w, om).backward()
    direction = _cuda(synthetic.gaussian_field(76, (W.n_side ** 3,)))
    eps = 1e-3
    with torch.no_grad():
        fd = (float(loss(w.detach() + eps * direction, om.detach()))
              - float(loss(w.detach() - eps * direction, om.detach()))) / (2 * eps)
        ad = float((w.grad * direction).sum())
        assert ad == pytest.approx(fd, rel=1e-2), (ad, fd)
    # Omega_m moves every line-of-sight node, so the derivative of the angles has dense kinks in Omega_m (a step
    # of 3e-4 averages over them); compare with FP64 differences of the oracle at steps that resolve them
    def oracle_loss(om_v):
        with torch.no_grad():
            _, th = _oracle_run(W, torch.tensor(noise), theta0, om_v)
            return float(((th - theta0) * tb.cpu()).sum() * 1e4)

    assert float(om.grad) == pytest.approx(_tiny_fd(oracle_loss, W.omega_m), rel=1e-3)
    sim.close()


@pytest.mark.parametrize("split", [False, True])
def test_pm_solve_adjoint_dot_product_at_256(hrt, split):
    # the PM solve is linear in rho: <PM rho, gbar> = <rho, PM^T gbar> at any size (here 256^3, the
    # differentiation workload's mesh; the forward solve on the split and on the 3D path)
    n, box, pref = 256, 256.0, 0.9
    g = torch.Generator(device="cuda").manual_seed(7)
    rho = torch.randn(n ** 3, device="cuda", generator=g)
    gbar = torch.randn(3, n ** 3, device="cuda", generator=g)
    pm = hrt.PM(n, box)
    pm.set_split(split)
    f = hrt.make_filter(4.0, box / n)
    grad = torch.empty(3, n ** 3, device="cuda")
    pm.solve(rho.clone(), pref, f, grad)
    rb = torch.empty(n ** 3, device="cuda")
    pm.solve_adjoint(gbar.clone(), pref, f, rb)
    lhs = float((grad.double() * gbar.double()).sum())
    rhs = float((rho.double() * rb.double()).sum())
    assert lhs == pytest.approx(rhs, rel=1e-5), (lhs, rhs)
    pm.close()


def test_power_loss_gradient_at_128p_256m_matches_central_differences(hrt):
    # the differentiation workload (128^3 white-noise modes, 256^3 mesh, 512^2 rays, checkpoint every 4 steps):
    # loss = sum over the log ell bins of (P(ell) - P_target(ell))^2; the adjoint's derivative along a random
    # noise direction against central differences with eps = 1e-3.  kappa jumps where line-of-sight samples
    # cross cell faces (measured spread of the differences over eps = 1e-4 .. 3e-3: about 2 %), hence 3 %.
    from paper_2405_12913_gb300 import autodiff
    from paper_2405_12913_gb300.configs import COSMO_GRAD_256 as W
    noise = _cuda(synthetic.white_noise(W.seed, W.n_side)).reshape(-1)
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE))
    lmin, lmax = W.ell_range
    sim = autodiff.ContextSim(W, theta0, checkpoint_every=4)
    om = torch.tensor(W.omega_m, dtype=torch.float64)

    def loss(wn, target, scale):
        kap, _ = autodiff.HRTKappa.apply(wn, om, sim)
        p = autodiff.KappaPower.apply(kap[0], W.n_pix, W.dtheta, W.nbins, lmin, lmax)
        return ((p - target) ** 2).sum() / scale

    with torch.no_grad():
        kap, _ = autodiff.HRTKappa.apply(noise, om, sim)
        target = 0.8 * autodiff.KappaPower.apply(kap[0], W.n_pix, W.dtheta, W.nbins, lmin, lmax)
    scale = float((target ** 2).sum())
    w = noise.clone().requires_grad_(True)
    loss(w, target, scale).backward()
    d = _cuda(synthetic.gaussian_field(74, (W.n_side ** 3,)))
    ad = float((w.grad.double() * d.double()).sum())
    eps = 1e-3
    with torch.no_grad():
        fd = (float(loss(noise + eps * d, target, scale)) - float(loss(noise - eps * d, target, scale))) / (2 * eps)
    assert ad == pytest.approx(fd, rel=3e-2), (ad, fd)
    sim.close()


def _oracle_run_mesh(W, noise, theta0, om, rm_args):
    c = osim.Cosmo(om, W.h, W.n_s, W.sigma8)
    flt = osim.Filter(W.deconv_p, W.smooth_cells)
    part = osim.initial_particles(noise, W.box, c, W.a_init)
    part, grads = osim.run_forward(part, W.forward_grid, W.box, W.n_mesh, c, flt)
    res = osim.run_reverse(part, grads, W.reverse_grid, W.box, W.n_mesh, c, flt, theta0, W.observer,
                           set(W.source_steps), W.samples_per_cell, ray_mesh=rm_args)
    return torch.stack([res.maps[s][0] for s in W.source_steps]), res.rays["theta"]


def test_ray_mesh_end_to_end_gradient_matches_oracle_differences(hrt, monkeypatch):
    """The differentiable simulation with the ray-mesh kick: the noise gradient of a loss on the kappa maps and
    the final angles against FP64 central differences of the oracle run with the ray-mesh kick (tiny steps that
    resolve the pieces of the piecewise-smooth kappa)."""
    from paper_2405_12913_gb300 import autodiff
    from paper_2405_12913_gb300.configs import COSMO_GRAD as W
    rm_args = (W.dtheta, W.n_pix, 0.5, 8.0)
    noise = synthetic.white_noise(W.seed + 3, W.n_side)
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE))
    kbar = synthetic.gaussian_field(77, (len(W.source_steps), W.n_rays))
    tb = synthetic.gaussian_field(78, (W.n_rays, 2))
    om0 = W.omega_m + 1.234e-6
    sim = autodiff.ContextSim(W, theta0, checkpoint_every=2,
                           ray_mesh=hrt.make_raymesh_config(rm_args[2], rm_args[3], rm_args[0], rm_args[1]))
    w = _cuda(noise).reshape(-1).requires_grad_(True)
    om = torch.tensor(om0, dtype=torch.float64, requires_grad=True)
    kap, th = autodiff.HRTKappa.apply(w, om, sim)
    loss = (kap.double() * _cuda(kbar, torch.float64)).sum() + 1e4 * ((th - theta0.cuda()) * _cuda(tb, torch.float64)).sum()
    loss.backward()
    direction = synthetic.gaussian_field(79, (W.n_side ** 3,))
    ad = float((w.grad.cpu().double() * torch.tensor(direction)).sum())

    def oracle_loss(wn, omv):
        with torch.no_grad():
            k, t = _oracle_run_mesh(W, wn, theta0, omv, rm_args)
            return float((k * torch.tensor(kbar)).sum() + 1e4 * ((t - theta0) * torch.tensor(tb)).sum())

    k_o, _ = _oracle_run_mesh(W, torch.tensor(noise), theta0, om0, rm_args)
    assert np.abs(kap.detach().cpu().numpy() - k_o.numpy()).max() <= 1e-3 * k_o.abs().max()
    d = torch.tensor(direction).reshape(noise.shape)
    fds = _piecewise_fd(lambda e: oracle_loss(torch.tensor(noise) + e * d, om0), 0.0)
    assert sum(abs(ad - v) <= 2e-3 * abs(v) for v in fds) >= 2, (ad, fds)
    # Omega_m: the adjoint holds each half shell's ray-mesh geometry (lambda_lim, x2d, N) fixed.  Differences of
    # the oracle with the geometries of the run at om0 replayed agree with it; with the geometry moving with the
    # shell boundaries they differ by about 1 % (the discretisation's own dependence on Omega_m)
    from oracle import raymesh as orm
    real_geometry = orm.geometry
    calls = []

    def recording(*a):
        out = real_geometry(*a)
        calls.append(out)
        return out

    monkeypatch.setattr(orm, "geometry", recording)
    oracle_loss(torch.tensor(noise), om0)
    recorded = list(calls)
    replay = {"i": 0}

    def replaying(*a):
        out = recorded[replay["i"] % len(recorded)]
        replay["i"] += 1
        return out

    monkeypatch.setattr(orm, "geometry", replaying)
    fds_fixed = _piecewise_fd(lambda x: oracle_loss(torch.tensor(noise), x), om0)
    monkeypatch.setattr(orm, "geometry", real_geometry)
    fds_om = _piecewise_fd(lambda x: oracle_loss(torch.tensor(noise), x), om0)
    print("ray-mesh dL/dOmega_m: adjoint %.6g, oracle differences at fixed geometry %s, with moving geometry %s"
          % (float(om.grad), fds_fixed, fds_om))
    assert sum(abs(float(om.grad) - v) <= 2e-3 * abs(v) for v in fds_fixed) >= 2, (float(om.grad), fds_fixed)
    assert sum(abs(float(om.grad) - v) <= 2e-2 * abs(v) for v in fds_om) >= 2, (float(om.grad), fds_om)
    sim.close()


@pytest.mark.parametrize("mesh", [False, True])
def test_context_adjoint_matches_the_differentiable_simulation(hrt, mesh):
    """hrt_adjoint of a recorded context run (checkpoints every 2 steps) against the same adjoint calls sequenced
    in Python over the stateless ABI (tests/stateless_adjoint.py, checkpoints every 3 steps, with its own FP64
    chain for Omega_m): the gradients agree to the rounding of the atomics."""
    from stateless_adjoint import DiffSim
    from paper_2405_12913_gb300 import autodiff
    from paper_2405_12913_gb300.configs import COSMO_GRAD as W
    rm_cfg = hrt.make_raymesh_config(0.5, 8.0, W.dtheta, W.n_pix) if mesh else None
    noise = synthetic.white_noise(W.seed + 4, W.n_side)
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE))
    kbar = _cuda(synthetic.gaussian_field(81, (len(W.source_steps), W.n_rays)))
    tb = _cuda(synthetic.gaussian_field(82, (W.n_rays, 2)), torch.float64) * 1e4
    # the context, recording its run
    cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                          W.samples_per_cell, W.observer, n_sources=len(W.source_steps))
    ctx = hrt.Context(cfg)
    ctx.hrt_set_checkpointing(2)
    if mesh:
        ctx.hrt_set_ray_mesh(rm_cfg)
    ctx.hrt_init_particles_zeldovich(_cuda(noise).reshape(-1), W.a_init)
    for a in W.forward_grid[1:]:
        ctx.hrt_step(a)
    ctx.hrt_sync_particles()
    ctx.hrt_init_rays(theta0.cuda())
    slots = {s: i for i, s in enumerate(W.source_steps)}
    for n, a in enumerate(W.reverse_grid[1:], start=1):
        ctx.hrt_step(a, slots.get(n, -1))
    kap_ctx = torch.stack([ctx.hrt_read_maps(i)[0] for i in range(len(W.source_steps))])
    nb_ctx, om_ctx = ctx.hrt_adjoint(kbar.contiguous(), tb.contiguous())
    torch.cuda.synchronize()
    # the differentiable simulation
    sim = DiffSim(W, theta0, checkpoint_every=3, ray_mesh=rm_cfg)
    w = _cuda(noise).reshape(-1).requires_grad_(True)
    om = torch.tensor(W.omega_m, dtype=torch.float64, requires_grad=True)
    kap, th = autodiff.HRTKappa.apply(w, om, sim)
    ((kap.double() * kbar.double()).sum() + ((th - theta0.cuda()) * tb).sum()).backward()
    assert float((kap_ctx - kap.detach()).abs().max()) <= 1e-4 * float(kap.detach().abs().max())
    g_ctx, g_sim = nb_ctx.double().cpu(), w.grad.double().cpu()
    rel = float((g_ctx - g_sim).norm() / g_sim.norm())
    assert rel < 1e-3, rel
    assert om_ctx == pytest.approx(float(om.grad), rel=1e-3), (om_ctx, float(om.grad))
    # a run that cannot be differentiated is refused with the reason
    ctx.hrt_drift_free(1000.0, 1100.0)
    with pytest.raises(hrt.HRTError):
        ctx.hrt_adjoint(kbar.contiguous())
    sim.close()
    ctx.close()


def test_context_adjoint_from_2lpt_ics_matches_central_differences(hrt):
    """The recorded context run from 2LPT initial conditions: the noise gradient of a loss on the final ray angles
    against central differences of the same context run (on one GB300: adjoint 0.21152, differences 0.21146,
    0.21486, 0.20183 at steps 3e-4, 1e-3, 3e-3)."""
    from paper_2405_12913_gb300.configs import COSMO_GRAD as W
    noise = _cuda(synthetic.white_noise(W.seed + 5, W.n_side)).reshape(-1)
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE)).cuda()
    tb = _cuda(synthetic.gaussian_field(83, (W.n_rays, 2)), torch.float64) * 1e4
    cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                          W.samples_per_cell, W.observer, n_sources=len(W.source_steps))
    ctx = hrt.Context(cfg)
    ctx.hrt_set_checkpointing(2)

    def run(w):
        ctx.hrt_init_particles_2lpt(w, W.a_init)
        for a in W.forward_grid[1:]:
            ctx.hrt_step(a)
        ctx.hrt_sync_particles()
        ctx.hrt_init_rays(theta0)
        for a in W.reverse_grid[1:]:
            ctx.hrt_step(a)
        th = ctx.hrt_read_rays()[0]
        return float(((th - theta0) * tb).sum())

    run(noise)
    nb, om_bar = ctx.hrt_adjoint(None, tb.contiguous())
    direction = _cuda(synthetic.gaussian_field(84, (W.n_side ** 3,)))
    ad = float((nb.double() * direction.double()).sum())
    # the angles' derivative has kinks (piecewise-linear interpolants), so float32 central differences scatter
    # with the step: the adjoint must lie within their spread (the 2LPT transpose itself is checked against
    # autograd above)
    fds = [(run(noise + e * direction) - run(noise - e * direction)) / (2 * e) for e in (3e-4, 1e-3, 3e-3)]
    lo, hi = min(fds), max(fds)
    assert lo - 0.02 * abs(lo) <= ad <= hi + 0.02 * abs(hi), (ad, fds)
    assert np.isfinite(om_bar)
    ctx.close()


@pytest.mark.parametrize("mesh", [False, True])
@pytest.mark.parametrize("tiling", ["identity", "random"])
def test_context_adjoint_through_a_tiled_light_cone(hrt, tiling, mesh):
    """A recorded context run through a light cone tiled by 40 box replicas, with the direct gather or the ray
    mesh.  Replicas that neither rotate nor shift the box tile it like the periodic images, so that run's
    gradients equal the untiled run's; random rotations and shifts are checked against central differences of the
    same context run (their spread, as the angles' derivative has kinks)."""
    from paper_2405_12913_gb300.configs import COSMO_GRAD as W
    k = 40
    if tiling == "identity":
        reps = (np.tile(np.arange(3, dtype=np.int32), (k, 1)), np.ones((k, 3), np.int32), np.zeros((k, 3), np.int32))
    else:
        reps = synthetic.replica_transforms(17, k, W.n_mesh)
    noise = _cuda(synthetic.white_noise(W.seed + 6, W.n_side)).reshape(-1)
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE)).cuda()
    kbar = _cuda(synthetic.gaussian_field(85, (len(W.source_steps), W.n_rays)))
    tb = _cuda(synthetic.gaussian_field(86, (W.n_rays, 2)), torch.float64) * 1e4
    cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                          W.samples_per_cell, W.observer, n_sources=len(W.source_steps))
    slots = {s: i for i, s in enumerate(W.source_steps)}

    def run(ctx, w):
        ctx.hrt_init_particles_zeldovich(w, W.a_init)
        for a in W.forward_grid[1:]:
            ctx.hrt_step(a)
        ctx.hrt_sync_particles()
        ctx.hrt_init_rays(theta0)
        for n, a in enumerate(W.reverse_grid[1:], start=1):
            ctx.hrt_step(a, slots.get(n, -1))
        kap = torch.stack([ctx.hrt_read_maps(i)[0] for i in range(len(W.source_steps))])
        th = ctx.hrt_read_rays()[0]
        return float((kap.double() * kbar.double()).sum() + ((th - theta0) * tb).sum())

    def gradients(replicas):
        ctx = hrt.Context(cfg)
        ctx.hrt_set_checkpointing(2)
        if mesh:
            ctx.hrt_set_ray_mesh(hrt.make_raymesh_config(0.5, 8.0, W.dtheta, W.n_pix))
        if replicas is not None:
            ctx.hrt_set_replicas(replicas)
        loss = run(ctx, noise)
        nb, om_bar = ctx.hrt_adjoint(kbar.contiguous(), tb.contiguous())
        return ctx, loss, nb.double(), om_bar

    ctx, loss, nb, om_bar = gradients(reps)
    assert np.isfinite(om_bar) and bool(torch.isfinite(nb).all())
    if tiling == "identity":
        ctx0, loss0, nb0, om0 = gradients(None)
        ctx0.close()
        assert loss == pytest.approx(loss0, rel=1e-4, abs=1e-6)
        rel = float((nb - nb0).norm() / nb0.norm())
        assert rel < 1e-3, rel
        assert om_bar == pytest.approx(om0, rel=1e-3)
    else:
        direction = _cuda(synthetic.gaussian_field(87, (W.n_side ** 3,)))
        ad = float((nb * direction.double()).sum())
        fds = [(run(ctx, noise + e * direction) - run(ctx, noise - e * direction)) / (2 * e)
               for e in (3e-4, 1e-3, 3e-3)]
        lo, hi = min(fds), max(fds)
        print("tiled context adjoint %.6g, central differences %s" % (ad, fds))
        assert lo - 0.02 * abs(lo) <= ad <= hi + 0.02 * abs(hi), (ad, fds)
    ctx.close()
