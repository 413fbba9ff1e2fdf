"""The direct path at the full size of the 1024^3 workload (1024^3 mesh, 512^3 particles, 2048^2 rays over 10 deg),
in the launch configuration of the timed step, against the FP64 oracle on sampled outputs that the oracle computes
one by one: the Poisson solve of a density made of cosine modes (Sec. 2), the kick-drift-deposit of every
particle, and the last reverse ray step (Alg. 1).  Inputs are seeded cosine-mode fields and bounded particle
states from `synthetic`; the oracle reads the fields through a view that evaluates them at the nodes it asks for."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import pm as opm
from oracle import rays as orays
from oracle import sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrt():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt as h
    return h


@pytest.fixture(scope="module")
def W():
    from paper_2405_12913_gb300.configs import COSMO_1024
    return COSMO_1024


class _ModeField:
    """The oracle's view of a cosine-mode field on an n^3 mesh: ``reshape(-1)[idx]`` evaluates it at flat node
    indices, rounded to float32 like the device copy."""

    def __init__(self, spec, n):
        self.spec, self.n, self.shape = spec, n, (n, n, n)

    def reshape(self, *shape):
        return self

    def __getitem__(self, idx):
        v = synthetic.mode_field_values(self.spec, self.n, np.asarray(idx))
        return torch.from_numpy(v.astype(np.float32).astype(np.float64))


def test_pm_solve_at_the_full_size(hrt, W):
    # the split solve (batched 2D plans around the x-pass kernel) at 1024^3: 4096 sampled nodes of the three
    # gradient fields against the oracle's gradient of each cosine mode
    n, box = W.n_mesh, W.box
    spec = synthetic.mode_spec(31, n, 12, 0.3)
    rho = 1.0 + synthetic.mode_field_device(spec, n, "cuda")
    pref = 1.5 * W.omega_m
    smooth = W.smooth_cells * box / n
    pm = hrt.PM(n, box)
    grad = torch.empty(3, n, n, n, device="cuda")
    pm.solve(rho, pref, hrt.make_filter(W.deconv_p, smooth), grad)
    torch.cuda.synchronize()
    pm.close()
    del rho
    idx = synthetic.sample_indices(32, n ** 3, 4096)
    want = opm.mode_gradient(spec["modes"], spec["amp"], spec["phase"], idx, n, box, pref, W.deconv_p, smooth)
    got = grad.reshape(3, -1)[:, torch.from_numpy(idx).cuda()].double().cpu().numpy()
    del grad
    for j in range(3):
        scale = np.abs(want[j]).max()
        assert scale > 0.0
        err = np.abs(got[j] - want[j])
        assert err.max() <= 1e-4 * scale and np.median(err) <= 1e-5 * scale, (j, err.max() / scale)


def test_kick_drift_deposit_at_the_full_size(hrt, W):
    # every particle kicked, drifted and deposited; 4096 sampled particles against the oracle step, the density
    # at 48 sampled cells against the oracle deposit of every particle that can reach them, and the total mass
    n, ns, box = W.n_mesh, W.n_side, W.box
    cell, spacing = box / n, box / ns
    specs = [synthetic.mode_spec(41 + c, n, 6, 200.0) for c in range(3)]
    disp_max, mom_max, kick, drift = 2.0 * cell, 20.0, 1e-3, 0.05
    # bound on the distance a particle ends from its lattice site, so that a cell's contributors are known
    g_max = max(float(np.abs(s["amp"]).sum()) for s in specs)
    reach = disp_max + (mom_max + g_max * kick) * drift
    assert reach < 3.5 * cell
    disp, mom = synthetic.bounded_particle_state(43, ns, disp_max, mom_max)
    grad = torch.stack([synthetic.mode_field_device(s, n, "cuda") for s in specs])
    d_dev, m_dev = torch.from_numpy(disp).cuda(), torch.from_numpy(mom).cuda()
    rho = torch.empty(n ** 3, device="cuda")
    hrt.hrt_particle_kick_drift_deposit(grad, n, box, ns, d_dev, m_dev, kick, drift, rho)
    torch.cuda.synchronize()
    del grad
    fields = [_ModeField(s, n) for s in specs]

    def lattice_q(p):
        return torch.from_numpy(np.stack([p // (ns * ns), (p // ns) % ns, p % ns], axis=1) * spacing)

    def oracle_step(p):
        return opm.particle_kick_drift(torch.from_numpy(disp[:, p].T).double(), torch.from_numpy(mom[:, p].T).double(),
                                       lattice_q(p), fields, box, kick, drift)

    idx = synthetic.sample_indices(44, ns ** 3, 4096)
    d_want, m_want = oracle_step(idx)
    sel = torch.from_numpy(idx).cuda()
    d_got = d_dev[:, sel].double().cpu().numpy().T
    m_got = m_dev[:, sel].double().cpu().numpy().T
    assert np.abs(d_got - d_want.numpy()).max() <= 2e-6 * box / ns
    assert np.abs(m_got - m_want.numpy()).max() <= 2e-6 * mom_max
    # density: sampled cells and every lattice site within reach of them (periodic)
    total = float(rho.sum(dtype=torch.float64))
    assert abs(total - n ** 3) <= 1e-6 * n ** 3
    cells = synthetic.sample_indices(45, n ** 3, 48)
    ci = np.stack([cells // (n * n), (cells // n) % n, cells % n], axis=1)
    r = int(np.ceil((reach + cell) / spacing)) + 1
    off = np.arange(-r, r + 1)
    sites = set()
    for c in ci:
        base = (c * cell // spacing).astype(np.int64)
        sx, sy, sz = [(base[a] + off) % ns for a in range(3)]
        grid = (sx[:, None, None] * ns + sy[None, :, None]) * ns + sz[None, None, :]
        sites.update(grid.reshape(-1).tolist())
    near = np.array(sorted(sites), dtype=np.int64)
    d_near, _ = oracle_step(near)
    want = opm.cic_deposit(lattice_q(near) + d_near, box, n, mass=n ** 3 / ns ** 3).reshape(-1)[torch.from_numpy(cells)]
    got = rho[torch.from_numpy(cells).cuda()].double().cpu()
    assert float(want.abs().max()) > 0.0
    assert float((got - want).abs().max()) <= 2e-5 * float(want.abs().max()) + 1e-6


def test_ray_step_at_the_full_size(hrt, W):
    # the last reverse step of the workload (2048^2 rays, the context's 16 x 8 image walk) over 1024^3 cosine-mode
    # fields: 4096 sampled rays against the oracle step
    n, box, om = W.n_mesh, W.box, W.omega_m
    a0, a1 = W.reverse_grid[-2], W.reverse_grid[-1]
    chi0, chi1 = hrt.hrt_cosmo_eval(om, a0)[1], hrt.hrt_cosmo_eval(om, a1)[1]
    specs = [synthetic.mode_spec(51 + c, n, 8, 3e3) for c in range(2)]
    gx, gy = (synthetic.mode_field_device(s, n, "cuda") for s in specs)
    theta0 = synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE)
    nr = theta0.shape[0]
    g = torch.Generator().manual_seed(53)
    eta0 = (2e-5 * torch.randn(nr, 2, generator=g)).float()
    A0 = (torch.eye(2).reshape(1, 4) + 0.05 * torch.randn(nr, 4, generator=g)).float()
    B0 = (1e-2 * torch.randn(nr, 4, generator=g)).float()
    rays = hrt.RayState(nr)
    rays.theta.copy_(torch.from_numpy(theta0).cuda())
    rays.eta.copy_(eta0.cuda())
    rays.A.copy_(A0.cuda())
    rays.B.copy_(B0.cuda())
    geom = hrt.make_geom(n, box, W.observer, W.samples_per_cell, image_width=W.n_pix)
    hrt.hrt_ray_step(rays, gx.reshape(-1), gy.reshape(-1), geom, chi0, chi1, a0, om)
    torch.cuda.synchronize()
    del gx, gy
    idx = synthetic.sample_indices(54, nr, 4096)
    st = dict(theta=torch.from_numpy(theta0[idx]), eta=eta0[idx].double(), A=A0[idx].double().reshape(-1, 2, 2),
              B=B0[idx].double().reshape(-1, 2, 2))
    e0, b0 = st["eta"].clone(), st["B"].clone()
    want = orays.ray_step(st, _ModeField(specs[0], n), _ModeField(specs[1], n), box, W.observer, chi0, chi1,
                          W.samples_per_cell, sim.growth_weight(a0, om))
    deta = rays.eta[idx].double().cpu() - e0
    dB = rays.B[idx].double().cpu().reshape(-1, 2, 2) - b0
    d_eta_o, d_B_o = want["eta"] - e0, want["B"] - b0
    assert float(d_eta_o.abs().max()) > 1e-7 and float(d_B_o.abs().max()) > 1e-4
    # the transverse derivative of the trilinear interpolant jumps on cell faces, where float32 and float64
    # positions may take different (equally valid) cells: every ray whose B (or A, below) differs must have a
    # line-of-sight node, in the oracle's own step, within 1e-5 cell of a transverse face (the float32 position
    # fraction of the kernel is good to about 1e-6 cell); eta is continuous there and must agree everywhere
    near = orays.step_face_distance(torch.from_numpy(theta0[idx]), want["theta"], box, n, W.observer, chi0, chi1,
                                    W.samples_per_cell) < 1e-5
    bad_eta = ((deta - d_eta_o).abs().max(dim=1).values > 1e-4 * float(d_eta_o.abs().max())).sum()
    err_B = (dB - d_B_o).abs().amax(dim=(1, 2)) / float(d_B_o.abs().max())
    off_face_B = (err_B > 1e-4) & ~near
    assert int(bad_eta) == 0 and not bool(off_face_B.any()), (int(bad_eta), int((err_B > 1e-4).sum()),
                                                                sorted(err_B[off_face_B].tolist()))
    assert float(err_B.median()) <= 1e-6
    dth = rays.theta[idx].cpu() - want["theta"]
    assert float(dth.abs().max()) <= 1e-4 * float((want["theta"] - torch.from_numpy(theta0[idx])).abs().max()) + 1e-15
    # A takes d B after the first half kick, so a ray whose B took the other cell carries it into A
    a0_ = A0[idx].double().reshape(-1, 2, 2)
    dA_o = want["A"] - a0_
    err_A = (rays.A[idx].double().cpu().reshape(-1, 2, 2) - a0_ - dA_o).abs().amax(dim=(1, 2)) / float(dA_o.abs().max())
    assert float(dA_o.abs().max()) > 0.0
    off_face_A = (err_A > 1e-4) & ~near
    assert not bool(off_face_A.any()) and float(err_A.median()) <= 1e-5, sorted(err_A[off_face_A].tolist())
