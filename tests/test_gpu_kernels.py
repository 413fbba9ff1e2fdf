"""Kernel-level parity of the CUDA path (through the C ABI) against the FP64 oracle on seeded inputs.

Tolerances: float32 arithmetic on O(1) values accumulated over at most a few hundred terms, and float32 FFTs
of length <= 2^30, stay below ~1e-5 of the output scale; every comparison states its scale."""
import math

import numpy as np
import pytest
import torch

import synthetic
from oracle import pm as opm
from oracle import power as opow
from oracle import rays as orays

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrt():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt as h
    return h


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _lattice_disp(seed, n_side, scale):
    return synthetic.small_displacements(seed, n_side, scale)  # (3, n^3)


@pytest.mark.parametrize("n_side,n_mesh,box,scale", [(20, 60, 120.0, 3.0), (16, 64, 64.0, 0.7), (1, 8, 8.0, 0.0),
                                                     (32, 64, 96.0, 4.0), (64, 128, 128.0, 2.0)])
def test_cic_scatter_matches_oracle(hrt, n_side, n_mesh, box, scale):
    disp = _lattice_disp(1, n_side, scale)
    if n_side == 1:
        disp = np.array([[3.3], [4.0], [7.9]])
    rho = torch.empty(n_mesh ** 3, device="cuda")
    hrt.hrt_cic_scatter(_cuda(disp), n_side, n_mesh, box, rho)
    q = opm.lattice(n_side, box)
    want = opm.cic_deposit(q + torch.tensor(disp.T), box, n_mesh).reshape(-1).numpy()
    got = rho.cpu().double().numpy()
    assert np.abs(got - want).max() <= 2e-6 * max(1.0, np.abs(want).max())
    assert got.sum() == pytest.approx(n_mesh ** 3, rel=1e-6)


def test_cic_scatter_large_displacements_wrap(hrt):
    # displacements of several box lengths (both signs) wrap periodically
    n_side, n_mesh, box = 8, 16, 32.0
    disp = _lattice_disp(2, n_side, 40.0)
    rho = torch.empty(n_mesh ** 3, device="cuda")
    hrt.hrt_cic_scatter(_cuda(disp), n_side, n_mesh, box, rho)
    want = opm.cic_deposit(opm.lattice(n_side, box) + torch.tensor(disp.T), box, n_mesh).reshape(-1).numpy()
    assert np.abs(rho.cpu().double().numpy() - want).max() <= 1e-4 * np.abs(want).max()


@pytest.mark.parametrize("n,p,smooth", [(60, 4.0, 1.0), (32, 0.0, 0.0), (32, 2.0, 0.5)])
def test_kspace_gradient_matches_oracle(hrt, n, p, smooth):
    box, pref = 90.0, 2.7
    spec = synthetic.complex_spectrum(3, n)
    out = torch.empty(3, n, n, n // 2 + 1, dtype=torch.complex64, device="cuda")
    cell = box / n
    f = hrt.make_filter(p, smooth * cell)
    hrt.hrt_kspace_gradient(_cuda(spec, torch.complex64), n, box, pref, f, 3, out)
    want = opm.poisson_gradient_hat(torch.tensor(spec), box, pref, p, smooth * cell)
    for j in range(3):
        w = want[j].numpy() / n ** 3
        g = out[j].cpu().numpy().astype(np.complex128)
        assert np.abs(g - w).max() <= 3e-6 * np.abs(w).max()


def test_kspace_second_set_and_learned_table(hrt):
    n, box, pref = 32, 64.0, 1.3
    spec = synthetic.complex_spectrum(4, n)
    kmax = 2 * math.pi / box * n
    table = np.linspace(1.0, 1.6, 33).astype(np.float32)
    out = torch.empty(3, n, n, n // 2 + 1, dtype=torch.complex64, device="cuda")
    out2 = torch.empty(2, n, n, n // 2 + 1, dtype=torch.complex64, device="cuda")
    fa = hrt.make_filter(0.0, 0.0)
    gt = _cuda(table)
    fb = hrt.make_filter(4.0, 2.0, gt, kmax)
    hrt.hrt_kspace_gradient(_cuda(spec, torch.complex64), n, box, pref, fa, 3, out, fb, 2, out2)

    def g_of_k(k):
        t = k / kmax * 32
        i = torch.clamp(t.floor().long(), 0, 31)
        w = t - i
        tab = torch.tensor(table, dtype=torch.float64)
        v = tab[i] * (1 - w) + tab[torch.clamp(i + 1, max=32)] * w
        return torch.where(t >= 32, torch.ones_like(v), v)

    want_a = opm.poisson_gradient_hat(torch.tensor(spec), box, pref, 0.0, 0.0)
    want_b = opm.poisson_gradient_hat(torch.tensor(spec), box, pref, 4.0, 2.0, g_of_k)
    for j in range(3):
        w = want_a[j].numpy() / n ** 3
        assert np.abs(out[j].cpu().numpy() - w).max() <= 3e-6 * np.abs(w).max()
    for j in range(2):
        w = want_b[j].numpy() / n ** 3
        assert np.abs(out2[j].cpu().numpy() - w).max() <= 3e-6 * np.abs(w).max()


@pytest.mark.parametrize("n", [60, 64])
def test_pm_solve_matches_oracle(hrt, n):
    box, pref = 100.0, 0.9
    rho = synthetic.gaussian_field(5, (n, n, n), 0.5) + 1.0
    pm = hrt.PM(n, box)
    grad = torch.empty(3, n, n, n, device="cuda")
    f = hrt.make_filter(4.0, box / n)
    pm.solve(_cuda(rho), pref, f, grad)
    want = opm.poisson_gradient(torch.tensor(rho), box, pref, 4.0, box / n)
    for j in range(3):
        w = want[j].numpy()
        assert np.abs(grad[j].cpu().double().numpy() - w).max() <= 2e-5 * np.abs(w).max()
    pm.close()


@pytest.mark.parametrize("fused", [True, False])
def test_pm_solve_fused_callback_and_ray_fields(hrt, fused):
    # the batched C2R with the k-space load callback (fused) and the separate k-space kernel both match the
    # oracle, for the particle fields and for separately filtered ray fields with a learned table
    n, box, pref = 64, 128.0, 1.1
    rho = synthetic.gaussian_field(15, (n, n, n), 0.5) + 1.0
    pm = hrt.PM(n, box, n_ray_fields=2)
    pm.set_fused(fused)
    kmax = 2 * math.pi / box * n
    table = np.linspace(1.2, 0.7, 65).astype(np.float32)
    gt = _cuda(table)
    grad = torch.empty(3, n, n, n, device="cuda")
    rgrad = torch.empty(2, n, n, n, device="cuda")
    pm.solve(_cuda(rho), pref, hrt.make_filter(0.0, 0.0), grad, hrt.make_filter(4.0, box / n, gt, kmax), rgrad)

    def g_of_k(k):
        t = k / kmax * 64
        i = torch.clamp(t.floor().long(), 0, 63)
        w = t - i
        tab = torch.tensor(table, dtype=torch.float64)
        v = tab[i] * (1 - w) + tab[torch.clamp(i + 1, max=64)] * w
        return torch.where(t >= 64, torch.ones_like(v), v)

    want = opm.poisson_gradient(torch.tensor(rho), box, pref, 0.0, 0.0)
    want_r = opm.poisson_gradient(torch.tensor(rho), box, pref, 4.0, box / n, g_of_k)
    for j in range(3):
        w = want[j].numpy()
        assert np.abs(grad[j].cpu().double().numpy() - w).max() <= 2e-5 * np.abs(w).max()
    for j in range(2):
        w = want_r[j].numpy()
        assert np.abs(rgrad[j].cpu().double().numpy() - w).max() <= 2e-5 * np.abs(w).max()
    pm.close()


@pytest.mark.parametrize("drift,n_side,n,box", [(0.37, 20, 60, 120.0), (0.0, 20, 60, 120.0), (0.37, 64, 128, 160.0)])
def test_particle_kick_drift_matches_oracle(hrt, drift, n_side, n, box):
    disp = _lattice_disp(6, n_side, 2.5)
    mom = _lattice_disp(7, n_side, 1.0)
    grads = [synthetic.gaussian_field(8 + j, (n, n, n)) for j in range(3)]
    gd = _cuda(np.stack(grads))
    d_dev, m_dev = _cuda(disp), _cuda(mom)
    hrt.hrt_particle_kick_drift(gd, n, box, n_side, d_dev, m_dev, 0.21, drift)
    q = opm.lattice(n_side, box)
    d_want, m_want = opm.particle_kick_drift(torch.tensor(disp.T), torch.tensor(mom.T), q,
                                             [torch.tensor(g) for g in grads], box, 0.21, drift)
    assert np.abs(m_dev.cpu().double().numpy() - m_want.numpy().T).max() <= 2e-6
    assert np.abs(d_dev.cpu().double().numpy() - d_want.numpy().T).max() <= 2e-6


@pytest.mark.parametrize("n_side,n,box", [(20, 60, 120.0), (32, 64, 80.0)])
def test_fused_kick_drift_deposit_matches_oracle(hrt, n_side, n, box):
    disp = _lattice_disp(16, n_side, 2.5)
    mom = _lattice_disp(17, n_side, 1.0)
    grads = [synthetic.gaussian_field(18 + j, (n, n, n)) for j in range(3)]
    d_dev, m_dev = _cuda(disp), _cuda(mom)
    rho = torch.full((n ** 3,), 7.0, device="cuda")  # overwritten
    hrt.hrt_particle_kick_drift_deposit(_cuda(np.stack(grads)), n, box, n_side, d_dev, m_dev, -0.13, 0.52, rho)
    q = opm.lattice(n_side, box)
    d_want, m_want = opm.particle_kick_drift(torch.tensor(disp.T), torch.tensor(mom.T), q,
                                             [torch.tensor(g) for g in grads], box, -0.13, 0.52)
    assert np.abs(d_dev.cpu().double().numpy() - d_want.numpy().T).max() <= 2e-6
    assert np.abs(m_dev.cpu().double().numpy() - m_want.numpy().T).max() <= 2e-6
    want = opm.cic_deposit(q + d_want, box, n).reshape(-1).numpy()
    assert np.abs(rho.cpu().double().numpy() - want).max() <= 2e-5 * np.abs(want).max()


def _smooth_grads(n, box, seed):
    # gradient fields of a smooth random potential: a handful of low Fourier modes, amplitude ~1e3
    rng = np.random.default_rng(seed)
    g = np.arange(n) * box / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    gx = np.zeros((n, n, n))
    gy = np.zeros((n, n, n))
    for _ in range(6):
        m = rng.integers(-3, 4, size=3)
        k = 2 * math.pi * m / box
        a, ph = rng.normal() * 3e3, rng.uniform(0, 2 * math.pi)
        arg = k[0] * X + k[1] * Y + k[2] * Z + ph
        gx += -a * k[0] * np.sin(arg)
        gy += -a * k[1] * np.sin(arg)
    return gx, gy


@pytest.mark.parametrize("a_ref,chis,s,npix", [(0.0, [(150.0, 210.0), (210.0, 300.0)], 1.0, 37),
                                               (0.8, [(600.0, 660.0)], 2.0, 37),
                                               (0.0, [(300.0, 210.0)], 1.0, 37),
                                               (0.7, [(900.0, 990.0), (990.0, 1100.0)], 1.0, 48)])
def test_ray_step_matches_oracle(hrt, a_ref, chis, s, npix):
    from oracle import cosmology as oc
    from oracle import sim
    n, box = 48, 96.0
    # observer off the mesh nodes: the transverse derivative of the trilinear interpolant jumps on cell faces,
    # where float32 and float64 positions may pick different (equally valid) one-sided cells
    obs = (30.3, 61.7, 5.0)
    gx, gy = _smooth_grads(n, box, 9)
    # 37^2 = 1369 rays: a ragged last block of 128; 48^2 rays: the 16 x 8 tiled walk of an image
    theta0 = synthetic.pixel_grid(npix, 0.3)
    rays = hrt.RayState(theta0.shape[0])
    hrt.hrt_rays_init(rays, _cuda(theta0, torch.float64))
    geom = hrt.make_geom(n, box, obs, s, image_width=npix if npix % 16 == 0 else 0)
    maps = torch.empty(4, theta0.shape[0], device="cuda")
    st = orays.init_state(torch.tensor(theta0))
    wfn = (lambda chi: 1.0) if a_ref == 0.0 else sim.growth_weight(a_ref, 0.3)
    for (c0, c1) in chis:
        hrt.hrt_ray_step(rays, _cuda(gx), _cuda(gy), geom, c0, c1, a_ref, 0.3, maps)
        st = orays.ray_step(st, torch.tensor(gx), torch.tensor(gy), box, obs, c0, c1, s, wfn)
    th = rays.theta.cpu().numpy()
    eta = rays.eta.cpu().double().numpy()
    A = rays.A.cpu().double().numpy().reshape(-1, 2, 2)
    B = rays.B.cpu().double().numpy().reshape(-1, 2, 2)
    dth = th - theta0
    dth_w = st["theta"].numpy() - theta0
    scale = np.abs(dth_w).max()
    assert scale > 1e-6
    assert np.abs(dth - dth_w).max() <= 1e-4 * scale
    assert np.abs(eta - st["eta"].numpy()).max() <= 1e-4 * np.abs(st["eta"].numpy()).max()
    assert np.abs(A - st["A"].numpy()).max() <= 2e-6
    assert np.abs(B - st["B"].numpy()).max() <= 1e-4 * np.abs(st["B"].numpy()).max()
    k, g1, g2, om = orays.observables(st["A"])
    got = maps.cpu().double().numpy()
    for i, w in enumerate((k, g1, g2)):
        assert np.abs(got[i] - w.numpy()).max() <= 2e-6
    assert np.abs(got[3] - om.numpy()).max() <= 2e-6


def test_ray_drift_free_and_readout(hrt):
    theta0 = synthetic.pixel_grid(9, 0.1)
    rays = hrt.RayState(81)
    hrt.hrt_rays_init(rays, _cuda(theta0, torch.float64))
    rays.eta.copy_(_cuda(synthetic.gaussian_field(3, (81, 2), 5.0)))
    rays.B.copy_(_cuda(synthetic.gaussian_field(4, (81, 4), 0.1)))
    eta = rays.eta.cpu().double().numpy()
    B = rays.B.cpu().double().numpy()
    hrt.hrt_ray_drift_free(rays, 100.0, 900.0)
    d = (1 / 100.0 - 1 / 900.0) / 2997.92458
    assert np.abs(rays.theta.cpu().numpy() - (theta0 + d * eta)).max() <= 1e-15
    assert np.abs(rays.A.cpu().double().numpy() - (np.array([1, 0, 0, 1]) + d * B)).max() <= 1e-7
    maps = torch.empty(4, 81, device="cuda")
    hrt.hrt_ray_readout(rays, maps)
    k, g1, g2, om = orays.observables(torch.tensor(rays.A.cpu().double().numpy().reshape(-1, 2, 2)))
    assert np.abs(maps[0].cpu().numpy() - k.numpy()).max() <= 1e-7


@pytest.mark.parametrize("m,nbins", [(64, 8), (256, 20), (2048, 20)])
def test_kappa_power_matches_oracle(hrt, m, nbins):
    dth = 3e-4
    kap = synthetic.gaussian_field(10 + m, (m, m), 0.02)
    lmin, lmax = 2 * math.pi / (m * dth), math.pi / dth
    ell, p, cnt = hrt.hrt_kappa_power(_cuda(kap), m, dth, nbins, lmin, lmax)
    ell_w, p_w, cnt_w = opow.kappa_power(kap, dth, nbins, lmin, lmax)
    assert np.array_equal(cnt, cnt_w)
    ok = cnt_w > 0
    assert np.allclose(ell[ok], ell_w[ok], rtol=1e-12)
    assert np.allclose(p[ok], p_w[ok], rtol=1e-5)


def test_zeldovich_ics_match_oracle(hrt):
    n, box, a = 32, 128.0, 0.05
    noise = synthetic.white_noise(11, n)
    disp = torch.empty(3, n ** 3, device="cuda")
    mom = torch.empty(3, n ** 3, device="cuda")
    hrt.hrt_ic_zeldovich(_cuda(noise), n, box, 0.3, 0.7, 0.96, 0.8, a, disp, mom)
    d_w, m_w = opm.zeldovich(noise, box, 0.3, 0.7, 0.96, 0.8, a)
    scale = np.abs(d_w.numpy()).max()
    assert np.abs(disp.cpu().double().numpy() - d_w.numpy().T).max() <= 2e-5 * scale
    assert np.abs(mom.cpu().double().numpy() - m_w.numpy().T).max() <= 2e-5 * np.abs(m_w.numpy()).max()


def test_invalid_arguments_enqueue_nothing(hrt):
    rho = torch.zeros(8 ** 3, device="cuda")
    with pytest.raises(hrt.HRTError) as e:
        hrt.hrt_cic_scatter(torch.zeros(3, 27, device="cuda"), 3, 8, 10.0, rho)  # 8 % 3 != 0
    assert e.value.status == 1
    rays = hrt.RayState(4)
    geom = hrt.make_geom(8, 10.0, (0, 0, 0), 1000.0)
    g = torch.zeros(8 ** 3, device="cuda")
    with pytest.raises(hrt.HRTError) as e:  # more than 1024 nodes in one step
        hrt.hrt_ray_step(rays, g, g, geom, 10.0, 50.0)
    assert e.value.status == 1
    with pytest.raises(hrt.HRTError):
        hrt.hrt_ray_drift_free(rays, 0.0, 10.0)
    torch.cuda.synchronize()


@pytest.mark.parametrize("n,rays", [(256, True), (256, False), (512, True), (512, False), (1024, True)])
def test_pm_split_path_matches_3d_path(hrt, n, rays):
    # batched 2D (y, z) plans + the x-pass kernel against 3D plans + the k-space kernel, for the particle fields
    # alone (one filter set) and with separately filtered ray fields with a learned table (two sets); the two
    # paths differ by FP32 FFT rounding only.  Every mesh side of the x-pass: 32 R1 points with R1 = 8, 16, 32
    # (4, 2 and 1 pencils per warp)
    box, pref = 1000.0 * n / 1024, 0.45
    g = torch.Generator(device="cuda").manual_seed(n)
    rho = 1.0 + 0.5 * torch.randn(n, n, n, device="cuda", generator=g)
    kmax = math.sqrt(3.0) * math.pi * n / box * 1.0001
    gt = torch.linspace(1.3, 0.8, 512, device="cuda")
    f = hrt.make_filter(4.0, box / n)
    fr = hrt.make_filter(4.0, box / n, gt, kmax)
    out = {}
    for split in (False, True):
        pm = hrt.PM(n, box, n_ray_fields=2 if rays else 0)
        pm.set_split(split)
        grad = torch.empty(3, n, n, n, device="cuda")
        if rays:
            rgrad = torch.empty(2, n, n, n, device="cuda")
            pm.solve(rho.clone(), pref, f, grad, fr, rgrad)
            out[split] = (grad, rgrad)
        else:
            pm.solve(rho.clone(), pref, f, grad)
            out[split] = (grad,)
        torch.cuda.synchronize()
        if split:
            with pytest.raises(hrt.HRTError):
                pm.density_spectrum(torch.empty(n, n, n // 2 + 1, dtype=torch.complex64, device="cuda"))
        pm.close()
    for k in range(len(out[False])):
        for j in range(out[False][k].shape[0]):
            ref = out[False][k][j]
            err = (out[True][k][j] - ref).abs().max().item()
            assert err <= 2e-5 * ref.abs().max().item(), (k, j, err, ref.abs().max().item())


def test_2lpt_ics_match_oracle(hrt):
    n, box, a = 32, 128.0, 0.1
    noise = synthetic.white_noise(12, n)
    disp = torch.empty(3, n ** 3, device="cuda")
    mom = torch.empty(3, n ** 3, device="cuda")
    hrt.hrt_ic_2lpt(_cuda(noise), n, box, 0.3, 0.7, 0.96, 0.8, a, disp, mom)
    d_w, m_w = opm.lpt2(noise, box, 0.3, 0.7, 0.96, 0.8, a)
    assert np.abs(disp.cpu().double().numpy() - d_w.numpy().T).max() <= 2e-5 * np.abs(d_w.numpy()).max()
    assert np.abs(mom.cpu().double().numpy() - m_w.numpy().T).max() <= 2e-5 * np.abs(m_w.numpy()).max()
    # the second-order part alone (2LPT minus Zel'dovich) to 1e-3 of its size
    dz = torch.empty_like(disp)
    mz = torch.empty_like(mom)
    hrt.hrt_ic_zeldovich(_cuda(noise), n, box, 0.3, 0.7, 0.96, 0.8, a, dz, mz)
    dz_w, _ = opm.zeldovich(noise, box, 0.3, 0.7, 0.96, 0.8, a)
    second = (disp - dz).cpu().double().numpy()
    second_w = (d_w - dz_w).numpy().T
    assert np.abs(second_w).max() > 1e-3 * np.abs(d_w.numpy()).max()
    assert np.abs(second - second_w).max() <= 1e-3 * np.abs(second_w).max()
    # the context entry point gives the same particles
    cfg = hrt.make_config(2 * n, box, n, 0.3, 0.7, 0.96, 0.8, observer=(0.5 * box, 0.5 * box, 0.0))
    ctx = hrt.Context(cfg)
    ctx.hrt_init_particles_2lpt(_cuda(noise).reshape(-1), a)
    cd, cm, a_pos, a_mom = ctx.hrt_read_particles()
    assert a_pos == a_mom == a
    assert torch.equal(cd.reshape(3, -1), disp) and torch.equal(cm.reshape(3, -1), mom)
    ctx.close()


def _smooth_grads3(n, box, seed):
    # the three gradient components of a smooth random potential (a handful of low Fourier modes)
    rng = np.random.default_rng(seed)
    g = np.arange(n) * box / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    out = [np.zeros((n, n, n)) for _ in range(3)]
    for _ in range(6):
        m = rng.integers(-3, 4, size=3)
        k = 2 * math.pi * m / box
        a, ph = rng.normal() * 3e3, rng.uniform(0, 2 * math.pi)
        arg = k[0] * X + k[1] * Y + k[2] * Z + ph
        for c in range(3):
            out[c] += -a * k[c] * np.sin(arg)
    return out


@pytest.mark.parametrize("seed", [21, 22])
def test_tiled_ray_step_matches_oracle(hrt, seed):
    # light cone tiled by six rotated, translated replicas; the shells cross the replica boundaries at
    # observer_z + chi = 192 and 288
    n, box = 48, 96.0
    obs = (30.3, 61.7, 5.0)
    g3 = _smooth_grads3(n, box, seed)
    reps = synthetic.replica_transforms(seed, 6, n)
    theta0 = synthetic.pixel_grid(32, 0.3)
    rays = hrt.RayState(theta0.shape[0])
    hrt.hrt_rays_init(rays, _cuda(theta0, torch.float64))
    geom = hrt.make_geom(n, box, obs, 1.0, image_width=32, replicas=reps)
    grad = _cuda(np.stack(g3))
    maps = torch.empty(4, theta0.shape[0], device="cuda")
    st = orays.init_state(torch.tensor(theta0))
    t3 = [torch.tensor(x) for x in g3]
    for (c0, c1) in [(150.0, 210.0), (210.0, 300.0)]:
        hrt.hrt_ray_step_tiled(rays, grad, geom, c0, c1, 0.0, 0.3, maps)
        st = orays.ray_step(st, t3[0], t3[1], box, obs, c0, c1, 1.0, lambda chi: 1.0, gz=t3[2], replicas=reps)
    th = rays.theta.cpu().numpy()
    dth, dth_w = th - theta0, st["theta"].numpy() - theta0
    scale = np.abs(dth_w).max()
    assert scale > 1e-6
    assert np.abs(dth - dth_w).max() <= 1e-4 * scale
    assert np.abs(rays.eta.cpu().double().numpy() - st["eta"].numpy()).max() <= 1e-4 * np.abs(st["eta"].numpy()).max()
    assert np.abs(rays.A.cpu().double().numpy().reshape(-1, 2, 2) - st["A"].numpy()).max() <= 2e-6
    B_w = st["B"].numpy()
    assert np.abs(rays.B.cpu().double().numpy().reshape(-1, 2, 2) - B_w).max() <= 1e-4 * np.abs(B_w).max()
    k, g1, g2, om = orays.observables(st["A"])
    got = maps.cpu().double().numpy()
    for i, w in enumerate((k, g1, g2, om)):
        assert np.abs(got[i] - w.numpy()).max() <= 2e-6


def test_tiled_ray_step_with_identity_replicas_is_the_plain_step(hrt):
    n, box = 48, 96.0
    obs = (30.3, 61.7, 5.0)
    g3 = _smooth_grads3(n, box, 23)
    ident = (np.tile([0, 1, 2], (6, 1)), np.ones((6, 3), np.int32), np.zeros((6, 3), np.int32))
    theta0 = _cuda(synthetic.pixel_grid(32, 0.3), torch.float64)
    a_rays, b_rays = hrt.RayState(theta0.shape[0]), hrt.RayState(theta0.shape[0])
    hrt.hrt_rays_init(a_rays, theta0)
    hrt.hrt_rays_init(b_rays, theta0)
    grad = _cuda(np.stack(g3))
    plain = hrt.make_geom(n, box, obs, 1.0, image_width=32)
    tiled = hrt.make_geom(n, box, obs, 1.0, image_width=32, replicas=ident)
    hrt.hrt_ray_step(a_rays, grad[0], grad[1], plain, 150.0, 300.0, 0.0, 0.3)
    hrt.hrt_ray_step_tiled(b_rays, grad, tiled, 150.0, 300.0, 0.0, 0.3)
    d = (a_rays.theta - theta0).abs().max().item()
    assert (b_rays.theta - a_rays.theta).abs().max().item() <= 1e-6 * d
    assert (b_rays.A - a_rays.A).abs().max().item() <= 1e-6
    with pytest.raises(hrt.HRTError):  # the plain step refuses a tiled geometry
        hrt.hrt_ray_step(a_rays, grad[0], grad[1], tiled, 150.0, 300.0, 0.0, 0.3)
    short = hrt.make_geom(n, box, obs, 1.0, replicas=tuple(t[:2] for t in ident))
    with pytest.raises(hrt.HRTError):  # nodes beyond the last replica
        hrt.hrt_ray_step_tiled(b_rays, grad, short, 150.0, 300.0, 0.0, 0.3)


def test_warp_aggregated_deposit_matches_the_plain_deposit(hrt):
    # clustered displacements (many particles of a warp in the same cells) and scattered ones
    n_side, n, box = 64, 128, 100.0
    g = torch.Generator(device="cuda").manual_seed(3)
    i = torch.arange(n_side, device="cuda", dtype=torch.float32) * (box / n_side)
    q = torch.stack(torch.meshgrid(i, i, i, indexing="ij")).reshape(3, -1)
    for scale in (0.3, 8.0, -1.0):
        if scale > 0:
            disp = (scale * torch.randn(3, n_side ** 3, generator=g, device="cuda")).contiguous()
        else:
            # collapse onto 8 points: most lanes of a warp share their targets
            c = torch.floor(q / (box / 2)) * (box / 2) + box / 4
            disp = (c - q + 0.01 * torch.randn(3, n_side ** 3, generator=g, device="cuda")).contiguous()
        rho0 = torch.empty(n ** 3, device="cuda")
        rho1 = torch.empty_like(rho0)
        hrt.hrt_cic_scatter(disp, n_side, n, box, rho0)
        hrt.hrt_cic_scatter_warp_aggregated(disp, n_side, n, box, rho1)
        torch.cuda.synchronize()
        assert torch.allclose(rho0, rho1, rtol=1e-5, atol=1e-5 * float(rho0.abs().max()))
        assert abs(float(rho0.double().sum()) - n ** 3) < 1e-3 * n ** 3
    with pytest.raises(hrt.HRTError):
        hrt.hrt_cic_scatter_warp_aggregated(torch.zeros(3, 24 ** 3, device="cuda"), 24, 48, 100.0,
                                            torch.empty(48 ** 3, device="cuda"))


def test_empty_ray_sets_are_no_ops(hrt):
    # zero rays: every ray call (direct and ray-mesh step, free drift, readout and their adjoints) succeeds and
    # leaves the field and node cotangents at zero
    n, box = 16, 32.0
    g = torch.randn(n ** 3, device="cuda")
    geom = hrt.make_geom(n, box, (3.3, 7.7, 1.0))
    rays, bar = hrt.RayState(0), hrt.RayState(0)
    maps = torch.empty(4, 0, device="cuda")
    hrt.hrt_ray_step(rays, g, g, geom, 10.0, 12.0, 0.8, 0.3, maps)
    hrt.hrt_ray_drift_free(rays, 12.0, 14.0)
    hrt.hrt_ray_readout(rays, maps)
    gb = torch.zeros(n ** 3, device="cuda")
    nb = torch.zeros(3, 1024, dtype=torch.float64, device="cuda")
    drb = torch.zeros(1, dtype=torch.float64, device="cuda")
    hrt.hrt_ray_step_adjoint(rays, g, g, geom, 10.0, 12.0, 0.8, 0.3, bar, gb, gb, nb, drb)
    rm = hrt.RayMesh(hrt.make_raymesh_config(0.5, 8, 0.004, 40))
    rm.hrt_raymesh_ray_step(rays, g, g, geom, 10.0, 12.0, 0.8, 0.3)
    pb, db = rm.hrt_raymesh_ray_step_adjoint(rays, g, g, geom, 10.0, 12.0, 0.8, 0.3, bar, gb, gb)
    torch.cuda.synchronize()
    rm.close()
    assert float(gb.abs().max()) == 0.0 and float(nb.abs().max()) == 0.0 and float(drb.abs().max()) == 0.0
    assert not np.any(pb) and db == 0.0
