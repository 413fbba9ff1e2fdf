"""Asynchronous read-outs of the ray angles and convergence maps (the per-step results of Algorithm 1): each
copy, made on the context's copy stream beside the next steps, must hold exactly what the stream-ordered read of
the same state holds, whatever the later steps do to the state."""
import numpy as np
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
    ctx.hrt_init_rays(torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE), device="cuda"))
    return ctx


def test_async_readouts_equal_the_stream_ordered_ones(hrt):
    from paper_2405_12913_gb300.configs import COSMO_TINY as W
    ctx = _context(hrt, W)
    r = W.n_pix ** 2
    slots = {s: i for i, s in enumerate(W.source_steps)}
    got_theta, want_theta, got_kappa, want_kappa = [], [], [], []
    grid = W.reverse_grid
    for n in range(1, W.n_reverse + 1):
        ctx.hrt_step(grid[n], slots.get(n, -1))
        h = torch.empty(r, 2, dtype=torch.float64, pin_memory=True)
        ctx.hrt_read_rays_async(h)
        d = torch.empty(r, 2, dtype=torch.float64, device="cuda")
        ctx.hrt_read_rays_into(d)
        got_theta.append(h)
        want_theta.append(d)
        if n in slots:
            k = torch.empty(r, dtype=torch.float32, pin_memory=True)
            ctx.hrt_read_kappa_async(slots[n], k)
            kd = torch.empty(r, dtype=torch.float32, device="cuda")
            ctx.hrt_read_maps_into(slots[n], kd)
            got_kappa.append(k)
            want_kappa.append(kd)
    ctx.hrt_read_wait()
    torch.cuda.synchronize()
    assert len(got_kappa) == len(W.source_steps)
    for h, d in zip(got_theta, want_theta):
        assert torch.equal(h, d.cpu())
    for k, kd in zip(got_kappa, want_kappa):
        assert torch.equal(k, kd.cpu())
    # the angles moved from step to step, so the copies were not all taken from one state
    assert not torch.equal(got_theta[0], got_theta[-1])
    ctx.close()


def test_one_reused_host_buffer_ends_with_the_last_step(hrt):
    from paper_2405_12913_gb300.configs import COSMO_TINY as W
    ctx = _context(hrt, W)
    r = W.n_pix ** 2
    h = torch.empty(r, 2, dtype=torch.float64, pin_memory=True)
    grid = W.reverse_grid
    for n in range(1, 4):
        ctx.hrt_step(grid[n])
        ctx.hrt_read_rays_async(h)
    ctx.hrt_read_wait()
    ctx.hrt_read_wait()  # a second wait with nothing in flight
    d = torch.empty(r, 2, dtype=torch.float64, device="cuda")
    ctx.hrt_read_rays_into(d)
    torch.cuda.synchronize()
    assert torch.equal(h, d.cpu())
    ctx.close()


def test_rays_initialised_again_with_fewer_rays_keep_the_pending_copy(hrt):
    # the staging regions follow the ray count: a read of the old rays still in flight must not be overwritten
    # by the staging of a read made after the rays were initialised again with fewer rays
    from paper_2405_12913_gb300.configs import COSMO_TINY as W
    ctx = _context(hrt, W)
    r = W.n_pix ** 2
    grid = W.reverse_grid
    ctx.hrt_step(grid[1])
    h = torch.empty(r, 2, dtype=torch.float64, pin_memory=True)
    ctx.hrt_read_rays_async(h)
    d = torch.empty(r, 2, dtype=torch.float64, device="cuda")
    ctx.hrt_read_rays_into(d)
    n2 = W.n_pix // 2
    ctx.hrt_init_rays(torch.tensor(synthetic.pixel_grid(n2, W.fov_deg * synthetic.DEGREE / 2), device="cuda"))
    ctx.hrt_step(grid[2], 0)
    k = torch.empty(n2 * n2, dtype=torch.float32, pin_memory=True)
    ctx.hrt_read_kappa_async(0, k)
    kd = torch.empty(n2 * n2, dtype=torch.float32, device="cuda")
    ctx.hrt_read_maps_into(0, kd)
    ctx.hrt_read_wait()
    torch.cuda.synchronize()
    assert torch.equal(h, d.cpu())
    assert torch.equal(k, kd.cpu())
    assert torch.count_nonzero(k) > 0
    ctx.close()


def test_async_readouts_reject_bad_arguments(hrt):
    from paper_2405_12913_gb300.configs import COSMO_TINY as W
    cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                          W.samples_per_cell, W.observer, n_sources=1)
    ctx = hrt.Context(cfg)
    ctx.hrt_read_wait()  # nothing asked for yet
    with pytest.raises(hrt.HRTError):  # no rays
        ctx.hrt_read_rays_async(torch.empty(4, 2, dtype=torch.float64))
    ctx.hrt_init_particles_zeldovich(torch.tensor(synthetic.white_noise(W.seed, W.n_side), dtype=torch.float32,
                                                  device="cuda"), W.a_init)
    ctx.hrt_init_rays(torch.tensor(synthetic.pixel_grid(8, 0.01), device="cuda"))
    r = 64
    with pytest.raises(ValueError):  # too small
        ctx.hrt_read_rays_async(torch.empty(r - 1, 2, dtype=torch.float64))
    with pytest.raises(ValueError):  # device memory
        ctx.hrt_read_rays_async(torch.empty(r, 2, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):  # wrong type
        ctx.hrt_read_kappa_async(0, torch.empty(r, dtype=torch.float64))
    with pytest.raises(hrt.HRTError):  # source out of range
        ctx.hrt_read_kappa_async(1, torch.empty(r, dtype=torch.float32))
    assert hrt._lib.hrt_read_rays_async(ctx._h, None) != 0  # NULL destination
    ctx.close()
