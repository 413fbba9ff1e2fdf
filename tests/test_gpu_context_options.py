"""Context calls that no other test covers: the FP32-angle precision ablation of the direct kick (the ray angles
of Alg. 1 kept in FP32 instead of FP64) and the accessor of the context's ray state."""
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrt():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt as h
    return h


def _context(hrt, W):
    cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                          W.samples_per_cell, W.observer, n_sources=len(W.source_steps))
    ctx = hrt.Context(cfg)
    ctx.hrt_init_particles_zeldovich(torch.tensor(synthetic.white_noise(W.seed, W.n_side), dtype=torch.float32,
                                                  device="cuda"), W.a_init)
    for a in W.forward_grid[1:]:
        ctx.hrt_step(a)
    ctx.hrt_sync_particles()
    return ctx


def _theta0(W):
    return torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE), device="cuda")


def _reverse(ctx, W):
    slots = {s: i for i, s in enumerate(W.source_steps)}
    grid = W.reverse_grid
    for n in range(1, W.n_reverse + 1):
        ctx.hrt_step(grid[n], slots.get(n, -1))
    r = W.n_pix ** 2
    theta = torch.empty(r, 2, dtype=torch.float64, device="cuda")
    kappa = torch.empty(r, dtype=torch.float32, device="cuda")
    ctx.hrt_read_rays_into(theta)
    ctx.hrt_read_maps_into(len(W.source_steps) - 1, kappa)
    torch.cuda.synchronize()
    return theta, kappa


def test_fp32_angle_ablation_changes_the_rays_by_more_than_run_to_run_noise(hrt):
    # two FP64 runs differ only by the order of the deposit's float reductions; the FP32 run also rounds the
    # angles after every drift and forms the positions in FP32: a change well above that noise, yet a small
    # fraction of the deflections
    from paper_2405_12913_gb300.configs import COSMO_TINY as W
    runs = {}
    for name, bits in (("a", 64), ("b", 64), ("fp32", 32)):
        ctx = _context(hrt, W)
        ctx.hrt_set_ray_theta_bits(bits)
        ctx.hrt_init_rays(_theta0(W))
        runs[name] = _reverse(ctx, W)
        ctx.close()
    deflection = (runs["a"][0] - _theta0(W)).abs()
    scale = float(deflection.max())
    assert scale > 0.0
    noise = (runs["a"][0] - runs["b"][0]).abs()
    ablation = (runs["a"][0] - runs["fp32"][0]).abs()
    assert float(ablation.median()) > 0.0
    assert float(ablation.median()) > 10.0 * float(noise.median())
    assert float(ablation.median()) < 1e-3 * scale
    assert float(ablation.max()) < 1e-2 * scale
    # and the maps move with the angles
    assert not torch.equal(runs["a"][1], runs["fp32"][1])


def test_ray_bits_other_than_32_or_64_are_refused(hrt):
    from paper_2405_12913_gb300.configs import COSMO_TINY as W
    ctx = _context(hrt, W)
    for bits in (0, 16, 128):
        with pytest.raises(hrt.HRTError):
            ctx.hrt_set_ray_theta_bits(bits)
    ctx.hrt_set_ray_theta_bits(64)
    ctx.close()


def test_the_ray_state_accessor_follows_the_rays(hrt):
    from paper_2405_12913_gb300.configs import COSMO_TINY as W
    ctx = _context(hrt, W)
    r = ctx.hrt_ctx_rays()
    assert r.n_rays == 0 and not r.theta and not r.eta and not r.A and not r.B
    ctx.hrt_init_rays(_theta0(W))
    r = ctx.hrt_ctx_rays()
    assert r.n_rays == W.n_pix ** 2
    ptrs = [r.theta, r.eta, r.A, r.B]
    assert all(ptrs) and len(set(ptrs)) == 4 and all(p % 16 == 0 for p in ptrs)
    ctx.hrt_init_rays(torch.tensor(synthetic.pixel_grid(8, 0.01), device="cuda"))
    assert ctx.hrt_ctx_rays().n_rays == 64
    ctx.close()
