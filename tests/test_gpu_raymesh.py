"""The ray-mesh kick operator (Sec. 5.2, Sec. 5.3, App. C) on the GPU against the FP64 oracle: the filtered mesh of
one half shell, one KDK ray step with the A/B recursion, and a full co-evolution run of the context; then the
operator on the point-mass lens against the Born integral of the exact periodic field."""
import math

import numpy as np
import pytest
import torch

import synthetic
from oracle import power as opow
from oracle import raymesh, sim
from oracle.units import C_LIGHT, G_NEWTON

pytestmark = pytest.mark.gpu

BOX, N = 64.0, 32
OBS = (0.31 * BOX, 0.58 * BOX, 0.7)


@pytest.fixture(scope="module")
def hrt():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt as h
    return h


def _fields(seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    gx = scale * torch.randn(N, N, N, generator=g, dtype=torch.float64)
    gy = scale * torch.randn(N, N, N, generator=g, dtype=torch.float64)
    return gx.float(), gy.float()


# (chi_a, chi_b, mu, m_pix, iota, p_min, a_ref, window)
KICKS = [
    (150.5, 181.3, 0.004, 40, 0.5, 8, 0.0, None),
    (181.3, 150.5, 0.004, 40, 0.5, 8, 0.0, None),          # towards the observer
    (150.5, 181.3, 0.003, 64, 0.25, 16, 0.0, None),
    (40.2, 71.9, 0.003, 50, 1.0, 4, 0.8, None),            # near the observer, growth correction
    (900.0, 1000.0, 0.0025, 64, 0.5, 8, 0.6, None),        # pixel-limited lambda_lim
    (150.5, 181.3, 0.004, 40, 0.5, 8, 0.0, (160.0, 171.0)),  # static-lens window
    (150.6, 150.65, 0.004, 40, 0.5, 8, 0.0, None),         # no plane: zero mesh
]


@pytest.mark.parametrize("case", range(len(KICKS)))
def test_raymesh_kick_matches_oracle(hrt, case):
    ca, cb, mu, m_pix, iota, p_min, a_ref, window = KICKS[case]
    gx, gy = _fields(10 + case)
    om = 0.3
    wfn = sim.growth_weight(a_ref, om) if a_ref > 0 else (lambda chi: 1.0)
    K, x2d, n2d = raymesh.mesh_kick(gx.double(), gy.double(), BOX, OBS, ca, cb, wfn, mu, m_pix, iota, p_min,
                                    window=window)
    cfg = hrt.make_raymesh_config(iota, p_min, mu, m_pix)
    lam, x2d_g, n2d_g = hrt.hrt_raymesh_geometry(cfg, ca, cb, BOX / N)
    assert n2d_g == n2d and x2d_g == pytest.approx(x2d, rel=1e-15)
    rm = hrt.RayMesh(cfg)
    geom = hrt.make_geom(N, BOX, OBS, window=window if window else (-1e300, 1e300))
    out = rm.hrt_raymesh_kick(gx.cuda().reshape(-1), gy.cuda().reshape(-1), geom, ca, cb, a_ref, om)
    torch.cuda.synchronize()
    got = out.permute(2, 0, 1).double().cpu()
    rm.close()
    scale = float(K.abs().max())
    if scale == 0.0:
        assert float(got.abs().max()) == 0.0
        return
    err = float((got - K).abs().max())
    # float32 deposit (~3e-6 relative) and float32 FFTs of an N^2 mesh
    assert err <= 3e-5 * scale, (err / scale, n2d)


@pytest.mark.parametrize("case", [0, 1, 3, 4])
def test_raymesh_ray_step_matches_oracle(hrt, case):
    ca, cb, mu, m_pix, iota, p_min, a_ref, _ = KICKS[case]
    gx, gy = _fields(30 + case, 3e3)
    om = 0.3
    wfn = sim.growth_weight(a_ref, om) if a_ref > 0 else (lambda chi: 1.0)
    rng = np.random.default_rng(case)
    n = 4096
    half = 0.5 * m_pix * mu
    th0 = torch.tensor(rng.uniform(-1.2 * half, 1.2 * half, size=(n, 2)))   # some rays beyond the image
    eta0 = torch.tensor(rng.normal(0, 2e-5, size=(n, 2))).float().double()
    A0 = torch.tensor(rng.normal(0, 1, size=(n, 2, 2))).float().double()
    B0 = torch.tensor(rng.normal(0, 1e-2, size=(n, 2, 2))).float().double()
    st = dict(theta=th0.clone(), eta=eta0.clone(), A=A0.clone(), B=B0.clone())
    want = raymesh.ray_step(st, gx.double(), gy.double(), BOX, OBS, ca, cb, wfn, mu, m_pix, iota, p_min)

    rays = hrt.RayState(n)
    rays.theta.copy_(th0.cuda())
    rays.eta.copy_(eta0.float().cuda())
    rays.A.copy_(A0.reshape(n, 4).float().cuda())
    rays.B.copy_(B0.reshape(n, 4).float().cuda())
    maps = torch.zeros(4, n, dtype=torch.float32, device="cuda")
    rm = hrt.RayMesh(hrt.make_raymesh_config(iota, p_min, mu, m_pix))
    rm.hrt_raymesh_ray_step(rays, gx.cuda().reshape(-1), gy.cuda().reshape(-1), hrt.make_geom(N, BOX, OBS), ca, cb,
                            a_ref, om, maps)
    torch.cuda.synchronize()
    rm.close()
    th = rays.theta.cpu()
    deta = rays.eta.double().cpu() - eta0
    dB = rays.B.double().cpu().reshape(n, 2, 2) - B0
    d_eta_o = want["eta"] - eta0
    d_B_o = want["B"] - B0
    assert float(d_eta_o.abs().max()) > 1e-6 and float(d_B_o.abs().max()) > 1e-3   # the kicks matter
    # the bilinear derivative jumps on ray-mesh cell faces: allow a rare ray on the other side of one
    bad_eta = ((deta - d_eta_o).abs().max(dim=1).values > 1e-4 * float(d_eta_o.abs().max())).sum()
    bad_B = ((dB - d_B_o).abs().amax(dim=(1, 2)) > 1e-4 * float(d_B_o.abs().max())).sum()
    assert int(bad_eta) == 0 and int(bad_B) <= 2, (int(bad_eta), int(bad_B))
    dth_o = want["theta"] - th0
    assert float((th - want["theta"]).abs().max()) <= 1e-4 * float(dth_o.abs().max()) + 1e-15
    A = rays.A.double().cpu().reshape(n, 2, 2)
    assert float((A - want["A"]).abs().max()) <= 1e-6
    k_o = 1.0 - 0.5 * (want["A"][:, 0, 0] + want["A"][:, 1, 1])
    assert float((maps[0].double().cpu() - k_o).abs().max()) <= 1e-6


@pytest.mark.parametrize("seed", [1, 2])
def test_tiled_raymesh_kick_matches_oracle(hrt, seed):
    """The filtered mesh of half shells that cross replica boundaries of a tiled light cone."""
    g = torch.Generator().manual_seed(60 + seed)
    g3 = [torch.randn(N, N, N, generator=g, dtype=torch.float64).float() for _ in range(3)]
    reps = synthetic.replica_transforms(seed, 12, N)
    cfg = hrt.make_raymesh_config(0.5, 8, 0.004, 40)
    rm = hrt.RayMesh(cfg)
    geom = hrt.make_geom(N, BOX, OBS, replicas=reps)
    for ca, cb in ((120.3, 141.0), (141.0, 120.3), (300.2, 400.9)):
        K, _, _ = raymesh.mesh_kick(g3[0].double(), g3[1].double(), BOX, OBS, ca, cb, lambda chi: 1.0, 0.004, 40,
                                    0.5, 8, gz=g3[2].double(), replicas=reps)
        out = rm.hrt_raymesh_kick(g3[0].cuda().reshape(-1), g3[1].cuda().reshape(-1), geom, ca, cb,
                                  grad_z=g3[2].cuda().reshape(-1))
        torch.cuda.synchronize()
        err = float((out.permute(2, 0, 1).double().cpu() - K).abs().max())
        assert err <= 3e-5 * float(K.abs().max()), (ca, cb, err / float(K.abs().max()))
    # a plane beyond the last replica is refused
    with pytest.raises(hrt.HRTError):
        rm.hrt_raymesh_kick(g3[0].cuda().reshape(-1), g3[1].cuda().reshape(-1), geom, 700.0, 800.0,
                            grad_z=g3[2].cuda().reshape(-1))
    rm.close()


def test_raymesh_rejects_bad_configurations(hrt):
    from paper_2405_12913_gb300.hrt import HRTError
    with pytest.raises(HRTError):
        hrt.RayMesh(hrt.make_raymesh_config(0.0, 8, 0.001, 64))
    with pytest.raises(HRTError):
        hrt.RayMesh(hrt.make_raymesh_config(0.5, -1, 0.001, 64))
    cfg = hrt.make_raymesh_config(0.5, 8, 1e-3, 4096, n2d_max=1024)
    assert hrt.hrt_raymesh_geometry(hrt.make_raymesh_config(0.5, 8, 1e-3, 4096), 1000.0, 1010.0, 2.0)[2] == 8192
    with pytest.raises(HRTError):      # needs an 8192^2 mesh
        hrt.hrt_raymesh_geometry(cfg, 1000.0, 1010.0, 2.0)
    rm = hrt.RayMesh(hrt.make_raymesh_config(0.5, 8, 0.004, 40))
    gx, gy = _fields(1)
    big = hrt.RayMesh(hrt.make_raymesh_config(1.0, 0, 1.0, 1))   # a ray-mesh cell of ~160 mesh cells at chi = 300
    with pytest.raises(HRTError):
        big.hrt_raymesh_kick(gx.cuda().reshape(-1), gy.cuda().reshape(-1), hrt.make_geom(N, BOX, OBS), 300.0, 310.0)
    big.close()
    geom = hrt.make_geom(N, BOX, OBS, replicas=(np.array([[0, 1, 2]]), np.array([[1, 1, 1]]), np.array([[0, 0, 0]])))
    with pytest.raises(HRTError):      # no light-cone tiling
        rm.hrt_raymesh_kick(gx.cuda().reshape(-1), gy.cuda().reshape(-1), geom, 150.5, 181.3)
    rm.close()


@pytest.mark.parametrize("tiled", [False, True])
def test_context_run_with_the_ray_mesh_matches_oracle(hrt, tiled):
    """The small cosmological co-evolution with the context's kick operator switched to the ray mesh, against
    the oracle's reverse run with the ray-mesh kick; also through a light cone tiled by 16 rotated, translated
    replicas."""
    from paper_2405_12913_gb300.configs import COSMO_TINY as W
    rm_args = (W.dtheta, W.n_pix, 0.5, 8.0)
    reps = synthetic.replica_transforms(31, 16, W.n_mesh) if tiled else None
    noise = synthetic.white_noise(W.seed, W.n_side)
    theta0 = synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE)
    cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                          W.samples_per_cell, W.observer, n_sources=len(W.source_steps))
    ctx = hrt.Context(cfg)
    ctx.hrt_set_ray_mesh(hrt.make_raymesh_config(rm_args[2], rm_args[3], rm_args[0], rm_args[1]))
    if tiled:
        ctx.hrt_set_replicas(reps)
    ctx.hrt_init_particles_zeldovich(torch.tensor(noise, dtype=torch.float32, device="cuda"), W.a_init)
    for a in W.forward_grid[1:]:
        ctx.hrt_step(a)
    ctx.hrt_sync_particles()
    ctx.hrt_init_rays(torch.tensor(theta0, device="cuda"))
    slots = {s: i for i, s in enumerate(W.source_steps)}
    for n, a in enumerate(W.reverse_grid[1:], start=1):
        ctx.hrt_step(a, slots.get(n, -1))
    maps = {s: ctx.hrt_read_maps(i).cpu().double().numpy() for s, i in slots.items()}
    th = ctx.hrt_read_rays()[0].cpu().numpy()
    lmin, lmax = W.ell_range
    pk = {s: ctx.hrt_ctx_kappa_power(i, W.n_pix, W.dtheta, W.nbins, lmin, lmax) for s, i in slots.items()}
    ctx.close()

    c = sim.Cosmo(W.omega_m, W.h, W.n_s, W.sigma8)
    flt = sim.Filter(W.deconv_p, W.smooth_cells)
    part = sim.initial_particles(noise, W.box, c, W.a_init)
    part, grads = sim.run_forward(part, W.forward_grid, W.box, W.n_mesh, c, flt)
    res = sim.run_reverse(part, grads, W.reverse_grid, W.box, W.n_mesh, c, flt, torch.tensor(theta0), W.observer,
                          set(W.source_steps), W.samples_per_cell, replicas=reps, ray_mesh=rm_args)
    for s in W.source_steps:
        kap_o = res.maps[s][0].numpy()
        rms = kap_o.std()
        assert rms > 1e-4
        for i in range(4):
            err = np.abs(maps[s][i] - res.maps[s][i].numpy())
            assert (err > 1e-3 * rms).mean() <= 2e-3 and np.median(err) <= 1e-4 * rms, (s, i, err.max() / rms)
        ell_o, p_o, cnt_o = opow.kappa_power(kap_o.reshape(W.n_pix, W.n_pix), W.dtheta, W.nbins, lmin, lmax)
        ell, p, cnt = pk[s]
        assert np.array_equal(cnt, cnt_o)
        ok = cnt_o > 0
        assert np.allclose(p[ok], p_o[ok], rtol=1e-3), np.abs(p[ok] / p_o[ok] - 1).max()
    alpha_o = theta0 - res.rays["theta"].numpy()
    assert np.abs((theta0 - th) - alpha_o).max() <= 1e-4 * np.abs(alpha_o).max()


def test_point_mass_with_the_ray_mesh_against_born_integral(hrt):
    """Sec. 6.1 with the paper's kick operator: the 3D field carries only the CIC deconvolution (the ray mesh does
    the smoothing, at lambda_lim); deflections above 4 cells against the Born integral of the exact periodic
    field, normalised by the single-lens deflection."""
    from paper_2405_12913_gb300.configs import POINT_MASS as W
    theta0 = synthetic.polar_impact_grid(W.n_radial, W.n_azimuth, W.b_min_cells, W.b_max_cells, W.cell, W.chi_lens)
    half = W.b_max_cells * W.cell / W.chi_lens
    mu = 0.1 * W.cell / W.chi_lens
    m_pix = int(math.ceil(2 * half / mu))
    cfg = hrt.make_config(W.n_mesh, W.box, 1, deconv_p=W.deconv_p, smooth_cells=0.0,
                          samples_per_cell=W.samples_per_cell, observer=W.observer, static_mode=True,
                          static_pref=hrt.hrt_static_prefactor(W.mass, W.box), n_sources=1)
    ctx = hrt.Context(cfg)
    ctx.hrt_set_ray_mesh(hrt.make_raymesh_config(0.5, 32.0, mu, m_pix))
    lens = torch.tensor([[W.lens_position[0]], [W.lens_position[1]], [W.lens_position[2]]], dtype=torch.float32,
                        device="cuda")
    ctx.hrt_init_particles(lens, torch.zeros_like(lens), 1.0)
    ctx.hrt_init_rays(torch.tensor(theta0, device="cuda"))
    chis = W.chi_grid
    for i in range(W.n_steps):
        ctx.hrt_step_static(chis[i], chis[i + 1], -1)
    ctx.hrt_drift_free(chis[-1], W.chi_source)
    th = ctx.hrt_read_rays()[0].cpu().numpy()
    ctx.close()
    alpha = theta0 - th
    b = W.chi_lens * np.hypot(theta0[:, 0], theta0[:, 1]) / W.cell
    pmc = sim.PointMass(W.n_mesh, W.box, W.mass, W.chi_lens, W.chi_source, W.n_steps, W.deconv_p, 0.0,
                        W.samples_per_cell)
    sel = np.flatnonzero(b > 4.0)[::53]
    born = sim.point_mass_born_ewald(pmc, theta0[sel], 300)
    lever = (W.chi_source - W.chi_lens) / W.chi_source * 4 * G_NEWTON * W.mass / C_LIGHT ** 2
    err = np.linalg.norm(alpha[sel] - born, axis=1) / (lever / (b[sel] * W.cell))
    far = b[sel] > 10.0
    print("ray mesh point mass: median %.4f max %.4f; beyond 10 cells median %.4f max %.4f"
          % (np.median(err), err.max(), np.median(err[far]), err[far].max()))
    # the largest errors lie along the mesh axes at 4-12 cells, where the unsmoothed 3D force is anisotropic
    assert np.median(err) < 0.002 and err.max() < 0.04
    assert np.median(err[far]) < 0.001


class _Planes:
    """An n^3 field that is zero except on the listed z planes; the oracle reads only planes [:, :, iz]."""

    def __init__(self, n, planes):
        self.shape = (n, n, n)
        self.planes = planes
        self.zero = np.zeros((n, n), dtype=np.float32)

    def __getitem__(self, key):
        return self.planes.get(key[2], self.zero)


def test_raymesh_ray_step_at_the_bench_size(hrt):
    """The last reverse step of the 1024^3 workload in the bench's ray-mesh configuration (2048^2 rays over 10 deg,
    iota 0.5, p_min 256: two 2048^2 ray meshes over 1024^3 gradient fields), random fields on the shell's planes:
    4096 sampled rays against the oracle step."""
    from paper_2405_12913_gb300.configs import COSMO_1024 as W
    om = W.omega_m
    n, box = W.n_mesh, W.box
    a0, a1 = W.reverse_grid[-2], W.reverse_grid[-1]
    chi0, chi1 = hrt.hrt_cosmo_eval(om, a0)[1], hrt.hrt_cosmo_eval(om, a1)[1]
    cell = box / n
    kzs = sorted({k % n for k, _ in raymesh.shell_planes(chi0, chi1, cell, W.observer[2])})
    rng = np.random.default_rng(7)
    px = {k: rng.normal(0, 3e3, size=(n, n)).astype(np.float32) for k in kzs}
    py = {k: rng.normal(0, 3e3, size=(n, n)).astype(np.float32) for k in kzs}
    gx = torch.zeros(n, n, n, dtype=torch.float32, device="cuda")
    gy = torch.zeros_like(gx)
    for k in kzs:
        gx[:, :, k] = torch.from_numpy(px[k]).cuda()
        gy[:, :, k] = torch.from_numpy(py[k]).cuda()
    theta0 = synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE)
    nr = theta0.shape[0]
    g = torch.Generator().manual_seed(3)
    eta0 = (2e-5 * torch.randn(nr, 2, generator=g)).float()
    A0 = (torch.eye(2).reshape(1, 4) + 0.05 * torch.randn(nr, 4, generator=g)).float()
    B0 = (1e-2 * torch.randn(nr, 4, generator=g)).float()
    rays = hrt.RayState(nr)
    rays.theta.copy_(torch.from_numpy(theta0).cuda())
    rays.eta.copy_(eta0.cuda())
    rays.A.copy_(A0.cuda())
    rays.B.copy_(B0.cuda())
    rm = hrt.RayMesh(hrt.make_raymesh_config(0.5, 256.0, W.dtheta, W.n_pix))
    rm.hrt_raymesh_ray_step(rays, gx.reshape(-1), gy.reshape(-1), hrt.make_geom(n, box, W.observer), chi0, chi1,
                            a0, om)
    torch.cuda.synchronize()
    rm.close()
    del gx, gy
    idx = synthetic.sample_indices(11, nr, 4096)
    st = dict(theta=torch.from_numpy(theta0[idx]), eta=eta0[idx].double(), A=A0[idx].double().reshape(-1, 2, 2),
              B=B0[idx].double().reshape(-1, 2, 2))
    e0, b0 = st["eta"].clone(), st["B"].clone()
    want = raymesh.ray_step(st, _Planes(n, px), _Planes(n, py), box, W.observer, chi0, chi1,
                            sim.growth_weight(a0, om), W.dtheta, W.n_pix, 0.5, 256.0)
    deta = rays.eta[idx].double().cpu() - e0
    dB = rays.B[idx].double().cpu().reshape(-1, 2, 2) - b0
    d_eta_o, d_B_o = want["eta"] - e0, want["B"] - b0
    assert float(d_eta_o.abs().max()) > 1e-7 and float(d_B_o.abs().max()) > 1e-4
    bad_eta = ((deta - d_eta_o).abs().max(dim=1).values > 1e-4 * float(d_eta_o.abs().max())).sum()
    bad_B = ((dB - d_B_o).abs().amax(dim=(1, 2)) > 1e-4 * float(d_B_o.abs().max())).sum()
    assert int(bad_eta) == 0 and int(bad_B) <= 2, (int(bad_eta), int(bad_B))
    dth = rays.theta[idx].cpu() - want["theta"]
    assert float(dth.abs().max()) <= 1e-4 * float((want["theta"] - torch.from_numpy(theta0[idx])).abs().max()) + 1e-15


def test_raymesh_kick_adjoint_is_the_transpose(hrt):
    """<kick(g), K_bar> = <g, kick^T(K_bar)> for the linear map from the gradient fields to the filtered mesh of a
    half shell, and sum_p w_p dL/dw_p = L (L is linear in the plane weights)."""
    gx, gy = _fields(70)
    om, a_ref = 0.3, 0.8
    for ca, cb, mu, m_pix, iota, p_min in ((150.5, 181.3, 0.004, 40, 0.5, 8), (181.3, 150.5, 0.003, 64, 0.25, 16),
                                           (40.2, 71.9, 0.003, 50, 1.0, 4)):
        cfg = hrt.make_raymesh_config(iota, p_min, mu, m_pix)
        rm = hrt.RayMesh(cfg)
        geom = hrt.make_geom(N, BOX, OBS)
        gxd, gyd = gx.cuda().reshape(-1), gy.cuda().reshape(-1)
        K = rm.hrt_raymesh_kick(gxd, gyd, geom, ca, cb, a_ref, om)
        g = torch.Generator(device="cuda").manual_seed(5)
        Kb = torch.randn(K.shape, generator=g, device="cuda")
        gxb = torch.zeros_like(gxd)
        gyb = torch.zeros_like(gyd)
        pb = rm.hrt_raymesh_kick_adjoint(gxd, gyd, Kb, geom, ca, cb, a_ref, om, gxb, gyb)
        torch.cuda.synchronize()
        lhs = float((K.double() * Kb.double()).sum())
        rhs = float((gxd.double() * gxb.double()).sum() + (gyd.double() * gyb.double()).sum())
        assert abs(lhs - rhs) <= 1e-4 * abs(lhs), (lhs, rhs)
        n, chi, w, _ = hrt.hrt_raymesh_step_planes(cfg, geom, ca, cb, a_ref, om)
        # the step's first half shell [ca, (ca + cb) / 2) is not this kick's shell: list this shell's planes
        planes = raymesh.shell_planes(ca, cb, BOX / N, OBS[2])
        wq = np.array([-(2.0 / C_LIGHT) * c * sim.growth_weight(a_ref, om)(c) * (1 if cb >= ca else -1) * (BOX / N) ** 3
                       / (c * c * hrt.hrt_raymesh_geometry(cfg, ca, cb, BOX / N)[1] ** 2) for _, c in planes])
        assert abs(float((wq * pb[:len(planes)]).sum()) - lhs) <= 1e-4 * abs(lhs)
        rm.close()


@pytest.mark.parametrize("case", [0, 3])
def test_raymesh_ray_step_adjoint_matches_oracle_derivative(hrt, case):
    """<bar_after, J v> from central differences of the FP64 oracle step along a direction v of the state and the
    fields, against <J^T bar_after, v> from the GPU adjoint; and per plane, w_p dL/dw_p equals the plane's share
    of <g, g_bar>."""
    ca, cb, mu, m_pix, iota, p_min, a_ref, _ = KICKS[case]
    om = 0.3
    wfn = sim.growth_weight(a_ref, om) if a_ref > 0 else (lambda chi: 1.0)
    gx, gy = _fields(80 + case, 3e3)
    rng = np.random.default_rng(90 + case)
    n = 2048
    half = 0.5 * m_pix * mu
    th0 = torch.tensor(rng.uniform(-half, half, size=(n, 2)))
    eta0 = torch.tensor(rng.normal(0, 2e-5, size=(n, 2))).float().double()
    A0 = torch.tensor(rng.normal(0, 1, size=(n, 2, 2))).float().double()
    B0 = torch.tensor(rng.normal(0, 1e-2, size=(n, 2, 2))).float().double()
    # cotangent of the state after the step and a direction for the state before it and the fields
    wb = {k: torch.tensor(rng.normal(0, 1, size=s)) for k, s in (("theta", (n, 2)), ("eta", (n, 2)), ("A", (n, 2, 2)),
                                                                 ("B", (n, 2, 2)))}
    wb["theta"] *= 1e3
    v = {k: torch.tensor(rng.normal(0, 1, size=s)) for k, s in (("theta", (n, 2)), ("eta", (n, 2)), ("A", (n, 2, 2)),
                                                                ("B", (n, 2, 2)))}
    v["theta"] *= 1e-6
    v["eta"] *= 1e-3
    vgx = torch.tensor(rng.normal(0, 1, size=(N, N, N))) * 30.0
    vgy = torch.tensor(rng.normal(0, 1, size=(N, N, N))) * 30.0

    def L(eps, part):
        st = dict(theta=th0.clone(), eta=eta0.clone(), A=A0.clone(), B=B0.clone())
        gxe, gye = gx.double(), gy.double()
        if part == "g":
            gxe, gye = gxe + eps * vgx, gye + eps * vgy
        else:
            st[part] = st[part] + eps * v[part]
        out = raymesh.ray_step(st, gxe, gye, BOX, OBS, ca, cb, wfn, mu, m_pix, iota, p_min)
        return sum(float((wb[k] * out[k]).sum()) for k in wb)

    eps = 1e-4
    jvp = {part: (L(eps, part) - L(-eps, part)) / (2 * eps) for part in ("theta", "eta", "A", "B", "g")}

    rays = hrt.RayState(n)
    rays.theta.copy_(th0.cuda())
    rays.eta.copy_(eta0.float().cuda())
    rays.A.copy_(A0.reshape(n, 4).float().cuda())
    rays.B.copy_(B0.reshape(n, 4).float().cuda())
    bar = hrt.RayState(n)
    bar.theta.copy_(wb["theta"].cuda())
    bar.eta.copy_(wb["eta"].float().cuda())
    bar.A.copy_(wb["A"].reshape(n, 4).float().cuda())
    bar.B.copy_(wb["B"].reshape(n, 4).float().cuda())
    gxd, gyd = gx.cuda().reshape(-1), gy.cuda().reshape(-1)
    gxb, gyb = torch.zeros_like(gxd), torch.zeros_like(gyd)
    cfg = hrt.make_raymesh_config(iota, p_min, mu, m_pix)
    rm = hrt.RayMesh(cfg)
    geom = hrt.make_geom(N, BOX, OBS)
    pb, _ = rm.hrt_raymesh_ray_step_adjoint(rays, gxd, gyd, geom, ca, cb, a_ref, om, bar, gxb, gyb)
    torch.cuda.synchronize()
    rm.close()
    vjp = {"theta": float((bar.theta.cpu() * v["theta"]).sum()), "eta": float((bar.eta.double().cpu() * v["eta"]).sum()),
           "A": float((bar.A.double().cpu().reshape(n, 2, 2) * v["A"]).sum()),
           "B": float((bar.B.double().cpu().reshape(n, 2, 2) * v["B"]).sum()),
           "g": float((gxb.double().cpu() * vgx.reshape(-1)).sum()) + float((gyb.double().cpu() * vgy.reshape(-1)).sum())}
    for part in jvp:
        assert abs(vjp[part] - jvp[part]) <= 2e-3 * abs(jvp[part]), (part, vjp[part], jvp[part])
    # plane weights: w_p dL/dw_p = sum over the plane's nodes of g . g_bar
    counts, chi, w, _ = hrt.hrt_raymesh_step_planes(cfg, geom, ca, cb, a_ref, om)
    gbx, gby = gxb.double().cpu().reshape(N, N, N), gyb.double().cpu().reshape(N, N, N)
    g64x, g64y = gx.double().reshape(N, N, N), gy.double().reshape(N, N, N)
    for h in range(2):
        for q in range(counts[h]):
            kz = int(round((chi[h, q] + OBS[2]) / (BOX / N))) % N
            share = float((g64x[:, :, kz] * gbx[:, :, kz]).sum() + (g64y[:, :, kz] * gby[:, :, kz]).sum())
            assert abs(w[h, q] * pb[h, q] - share) <= 1e-4 * (abs(share) + 1e-30) + 1e-9 * float(np.abs(pb).max() * np.abs(w).max())


@pytest.mark.parametrize("seed", [1, 2])
def test_tiled_raymesh_kick_adjoint_is_the_transpose(hrt, seed):
    """Through a tiled light cone: <kick(g), K_bar> = <g, kick^T(K_bar)> over the three box fields for half shells
    that cross replica boundaries, sum_p w_p dL/dw_p = L, and with replicas that neither rotate nor shift the box
    the transpose equals the untiled one (no cotangent on the z field)."""
    g = torch.Generator().manual_seed(70 + seed)
    g3 = [torch.randn(N, N, N, generator=g, dtype=torch.float64).float().cuda().reshape(-1) for _ in range(3)]
    reps = synthetic.replica_transforms(seed, 12, N)
    ident = (np.tile(np.arange(3, dtype=np.int32), (12, 1)), np.ones((12, 3), np.int32), np.zeros((12, 3), np.int32))
    om, a_ref = 0.3, 0.8
    cfg = hrt.make_raymesh_config(0.5, 8, 0.004, 40)
    rm = hrt.RayMesh(cfg)
    for ca, cb in ((110.3, 141.0), (141.0, 110.3), (250.2, 300.9)):
        geom = hrt.make_geom(N, BOX, OBS, replicas=reps)
        K = rm.hrt_raymesh_kick(g3[0], g3[1], geom, ca, cb, a_ref, om, grad_z=g3[2])
        gen = torch.Generator(device="cuda").manual_seed(seed)
        Kb = torch.randn(K.shape, generator=gen, device="cuda")
        gb = [torch.zeros_like(g3[0]) for _ in range(3)]
        pb = rm.hrt_raymesh_kick_adjoint(g3[0], g3[1], Kb, geom, ca, cb, a_ref, om, gb[0], gb[1], grad_z=g3[2],
                                         gz_bar=gb[2])
        torch.cuda.synchronize()
        lhs = float((K.double() * Kb.double()).sum())
        rhs = sum(float((g3[c].double() * gb[c].double()).sum()) for c in range(3))
        assert abs(lhs - rhs) <= 1e-4 * abs(lhs), (ca, cb, lhs, rhs)
        assert float(gb[2].abs().max()) > 0.0
        planes = raymesh.shell_planes(ca, cb, BOX / N, OBS[2])
        x2d = hrt.hrt_raymesh_geometry(cfg, ca, cb, BOX / N)[1]
        wq = np.array([-(2.0 / C_LIGHT) * c * sim.growth_weight(a_ref, om)(c) * (1 if cb >= ca else -1) * (BOX / N) ** 3
                       / (c * c * x2d ** 2) for _, c in planes])
        assert abs(float((wq * pb[:len(planes)]).sum()) - lhs) <= 1e-4 * abs(lhs)
        # identity replicas against the untiled transpose
        gi = [torch.zeros_like(g3[0]) for _ in range(3)]
        pbi = rm.hrt_raymesh_kick_adjoint(g3[0], g3[1], Kb, hrt.make_geom(N, BOX, OBS, replicas=ident), ca, cb, a_ref,
                                          om, gi[0], gi[1], grad_z=g3[2], gz_bar=gi[2])
        gu = [torch.zeros_like(g3[0]) for _ in range(2)]
        pbu = rm.hrt_raymesh_kick_adjoint(g3[0], g3[1], Kb, hrt.make_geom(N, BOX, OBS), ca, cb, a_ref, om, gu[0], gu[1])
        torch.cuda.synchronize()
        for c in range(2):
            assert float((gi[c] - gu[c]).abs().max()) <= 1e-5 * float(gu[c].abs().max())
        assert float(gi[2].abs().max()) == 0.0
        assert np.allclose(pbi, pbu, rtol=1e-5, atol=1e-12 * np.abs(pbu).max())
    rm.close()


@pytest.mark.parametrize("case", [0, 1])
def test_tiled_raymesh_ray_step_adjoint_matches_oracle_derivative(hrt, case):
    """The ray-mesh KDK step through a tiled light cone (a shell across a replica boundary): <bar_after, J v> from
    central differences of the FP64 oracle step along a direction v of the state and the three fields, against
    <J^T bar_after, v> from the GPU adjoint."""
    ca, cb = ((110.3, 141.0), (141.0, 110.3))[case]
    mu, m_pix, iota, p_min, a_ref, om = 0.004, 40, 0.5, 8, 0.8, 0.3
    wfn = sim.growth_weight(a_ref, om)
    reps = synthetic.replica_transforms(5 + case, 12, N)
    g = torch.Generator().manual_seed(95 + case)
    g3 = [3e3 * torch.randn(N, N, N, generator=g, dtype=torch.float64).float() for _ in range(3)]
    rng = np.random.default_rng(96 + case)
    n = 2048
    half = 0.5 * m_pix * mu
    th0 = torch.tensor(rng.uniform(-half, half, size=(n, 2)))
    eta0 = torch.tensor(rng.normal(0, 2e-5, size=(n, 2))).float().double()
    A0 = torch.tensor(rng.normal(0, 1, size=(n, 2, 2))).float().double()
    B0 = torch.tensor(rng.normal(0, 1e-2, size=(n, 2, 2))).float().double()
    shapes = (("theta", (n, 2)), ("eta", (n, 2)), ("A", (n, 2, 2)), ("B", (n, 2, 2)))
    wb = {k: torch.tensor(rng.normal(0, 1, size=s)) for k, s in shapes}
    wb["theta"] *= 1e3
    v = {k: torch.tensor(rng.normal(0, 1, size=s)) for k, s in shapes}
    v["theta"] *= 1e-6
    v["eta"] *= 1e-3
    vg = [torch.tensor(rng.normal(0, 1, size=(N, N, N))) * 30.0 for _ in range(3)]

    def L(eps, part):
        st = dict(theta=th0.clone(), eta=eta0.clone(), A=A0.clone(), B=B0.clone())
        ge = [x.double() for x in g3]
        if part == "g":
            ge = [ge[c] + eps * vg[c] for c in range(3)]
        else:
            st[part] = st[part] + eps * v[part]
        out = raymesh.ray_step(st, ge[0], ge[1], BOX, OBS, ca, cb, wfn, mu, m_pix, iota, p_min, gz=ge[2],
                               replicas=reps)
        return sum(float((wb[k] * out[k]).sum()) for k in wb)

    eps = 1e-4
    jvp = {part: (L(eps, part) - L(-eps, part)) / (2 * eps) for part in ("theta", "eta", "A", "B", "g")}

    rays = hrt.RayState(n)
    rays.theta.copy_(th0.cuda())
    rays.eta.copy_(eta0.float().cuda())
    rays.A.copy_(A0.reshape(n, 4).float().cuda())
    rays.B.copy_(B0.reshape(n, 4).float().cuda())
    bar = hrt.RayState(n)
    bar.theta.copy_(wb["theta"].cuda())
    bar.eta.copy_(wb["eta"].float().cuda())
    bar.A.copy_(wb["A"].reshape(n, 4).float().cuda())
    bar.B.copy_(wb["B"].reshape(n, 4).float().cuda())
    gd = [x.cuda().reshape(-1) for x in g3]
    gb = [torch.zeros_like(gd[0]) for _ in range(3)]
    rm = hrt.RayMesh(hrt.make_raymesh_config(iota, p_min, mu, m_pix))
    geom = hrt.make_geom(N, BOX, OBS, replicas=reps)
    rm.hrt_raymesh_ray_step_adjoint(rays, gd[0], gd[1], geom, ca, cb, a_ref, om, bar, gb[0], gb[1], grad_z=gd[2],
                                    gz_bar=gb[2])
    torch.cuda.synchronize()
    rm.close()
    vjp = {"theta": float((bar.theta.cpu() * v["theta"]).sum()), "eta": float((bar.eta.double().cpu() * v["eta"]).sum()),
           "A": float((bar.A.double().cpu().reshape(n, 2, 2) * v["A"]).sum()),
           "B": float((bar.B.double().cpu().reshape(n, 2, 2) * v["B"]).sum()),
           "g": sum(float((gb[c].double().cpu() * vg[c].reshape(-1)).sum()) for c in range(3))}
    for part in jvp:
        assert abs(vjp[part] - jvp[part]) <= 2e-3 * abs(jvp[part]), (part, vjp[part], jvp[part])
