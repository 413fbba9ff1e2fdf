"""Failure handling of the C ABI, made on the host only (no GPU fault, trap or hang is caused): every device
allocation of a whole run failing in turn (an injected out-of-memory), the bounded host wait for a stream, and the
opt-in checks for NaN and infinity.  Bad values are placed in host-prepared inputs and are caught by the scan
before any kernel computes with them."""
import math

import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

OOM, STATE, NONFINITE, TIMEOUT = 2, 4, 5, 6


@pytest.fixture(scope="module")
def hrt():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt as h
    yield h
    h.hrt_inject_alloc_failure(0)
    h.hrt_set_host_wait_limit(0.0)


@pytest.fixture(scope="module")
def W():
    from paper_2405_12913_gb300.configs import COSMO_TINY
    return COSMO_TINY


def _config(hrt, W):
    return hrt.make_config(W.n_mesh, W.box, W.n_side, deconv_p=W.deconv_p, smooth_cells=W.smooth_cells,
                           observer=W.observer, n_sources=len(W.source_steps))


def _inputs(W):
    noise = torch.tensor(synthetic.white_noise(W.seed, W.n_side), dtype=torch.float32, device="cuda")
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE))
    return noise, theta0


def _run(hrt, W, noise, theta0, retry_steps):
    """ICs, forward steps to a = 1, rays, reverse steps with maps, the power spectrum of the last map.  With
    retry_steps an injected failure of a step or of the power spectrum is answered by repeating the call once.
    Returns (events, kappa, p) where events lists the calls that failed."""
    events = []
    ctx = hrt.Context(_config(hrt, W))
    try:
        ctx.hrt_init_particles_zeldovich(noise, W.a_init)

        def call(name, fn):
            try:
                return fn()
            except hrt.HRTError as e:
                assert e.status == OOM and "injected" in str(e), (name, e)
                events.append(name)
                if not retry_steps:
                    raise
                return fn()

        for a in W.forward_grid[1:]:
            call("forward step", lambda: ctx.hrt_step(a))
        ctx.hrt_init_rays(theta0.cuda())
        slots = {s: i for i, s in enumerate(W.source_steps)}
        grid = W.reverse_grid
        for n in range(1, len(grid)):
            call("reverse step", lambda: ctx.hrt_step(grid[n], slots.get(n, -1)))
        kappa = ctx.hrt_read_maps(len(slots) - 1)[0].cpu().numpy()
        lo, hi = W.ell_range
        _, p, _ = call("kappa power", lambda: ctx.hrt_ctx_kappa_power(len(slots) - 1, W.n_pix, W.dtheta, W.nbins,
                                                                     lo, hi))
        torch.cuda.synchronize()
        return events, kappa, p
    finally:
        ctx.close()


def test_every_injected_allocation_failure_is_reported_and_recoverable(hrt, W):
    # The k-th device allocation of a whole run reports out-of-memory, for every k until the run has no more
    # allocations.  A failure in hrt_create, the ICs or the rays surfaces as HRT_ERR_OOM and the context is
    # destroyed cleanly; a failure inside a step (the particle sort's buffers) or inside the power spectrum
    # leaves the state as it was, so repeating the call gives the same run as one without any failure.
    noise, theta0 = _inputs(W)
    hrt.hrt_inject_alloc_failure(0)
    _, kappa_ref, p_ref = _run(hrt, W, noise, theta0, retry_steps=False)
    scale = np.abs(kappa_ref).max()
    where = []
    for k in range(1, 400):
        hrt.hrt_inject_alloc_failure(k)
        try:
            events, kappa, p = _run(hrt, W, noise, theta0, retry_steps=True)
        except hrt.HRTError as e:
            assert e.status == OOM and "injected" in str(e), (k, e)
            where.append("setup")
            continue
        if not events:
            break  # k is beyond the run's allocations
        where += events
        # the recovered run equals the undisturbed one up to the rounding order of the deposit's atomics
        assert np.abs(kappa - kappa_ref).max() <= 1e-4 * scale, (k, events)
        assert np.allclose(p, p_ref, rtol=1e-3, atol=0.0), (k, events)
    else:
        pytest.fail("the run kept allocating")
    hrt.hrt_inject_alloc_failure(0)
    assert "setup" in where and "kappa power" in where and any(w.endswith("step") for w in where), where


def test_the_injected_failure_of_the_first_force_leaves_no_step(hrt, W):
    # the particle ICs succeed but their force fails to allocate its filter tables: the context refuses to
    # step on the missing force (HRT_ERR_STATE) until new particles bring one
    noise, _ = _inputs(W)
    for k in range(1, 60):
        hrt.hrt_inject_alloc_failure(0)
        ctx = hrt.Context(_config(hrt, W))
        try:
            hrt.hrt_inject_alloc_failure(k)
            try:
                ctx.hrt_init_particles_zeldovich(noise, W.a_init)
            except hrt.HRTError as e:
                assert e.status == OOM
                hrt.hrt_inject_alloc_failure(0)
                with pytest.raises(hrt.HRTError) as e2:
                    ctx.hrt_step(W.forward_grid[1])
                assert e2.value.status == STATE
                ctx.hrt_init_particles_zeldovich(noise, W.a_init)
                ctx.hrt_step(W.forward_grid[1])
                torch.cuda.synchronize()
                continue
            hrt.hrt_inject_alloc_failure(0)
            break
        finally:
            hrt.hrt_inject_alloc_failure(0)
            ctx.close()
    else:
        pytest.fail("the ICs kept allocating")


def test_bounded_host_wait_returns_timeout_then_recovers(hrt):
    # a power spectrum requested behind a hundred queued steps of a 256^3 mesh, with a one-microsecond
    # limit on the host wait, returns HRT_ERR_TIMEOUT having enqueued nothing; without the limit the same call
    # returns the spectrum
    from paper_2405_12913_gb300.configs import COSMO_256 as W
    noise = torch.tensor(synthetic.white_noise(W.seed, W.n_side), dtype=torch.float32, device="cuda")
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE), device="cuda")
    ctx = hrt.Context(hrt.make_config(W.n_mesh, W.box, W.n_side, observer=W.observer, n_sources=1))
    try:
        ctx.hrt_init_particles_zeldovich(noise, W.a_init)
        ctx.hrt_init_rays(theta0)
        grid = W.reverse_grid
        ctx.hrt_step(grid[1], 0)
        torch.cuda.synchronize()
        lo, hi = W.ell_range
        want = ctx.hrt_ctx_kappa_power(0, W.n_pix, W.dtheta, 8, lo, hi)
        for i in range(1, 101):  # forward steps move the particles only: the map stays the same
            ctx.hrt_step(grid[1] + (1.0 - grid[1]) * i / 100)
        hrt.hrt_set_host_wait_limit(1e-6)
        with pytest.raises(hrt.HRTError) as e:
            ctx.hrt_ctx_kappa_power(0, W.n_pix, W.dtheta, 8, lo, hi)
        assert e.value.status == TIMEOUT and "wait limit" in str(e.value)
        hrt.hrt_set_host_wait_limit(0.0)
        got = ctx.hrt_ctx_kappa_power(0, W.n_pix, W.dtheta, 8, lo, hi)
        # the same map: bins equal up to the summation order of the binning's FP64 atomics
        assert np.array_equal(got[2], want[2])
        for g, w in zip(got[:2], want[:2]):
            assert np.allclose(g, w, rtol=1e-12, atol=0.0)
    finally:
        hrt.hrt_set_host_wait_limit(0.0)
        ctx.close()
    with pytest.raises(hrt.HRTError):
        hrt.hrt_set_host_wait_limit(math.nan)


def test_nonfinite_checks_refuse_bad_inputs_and_pass_a_clean_run(hrt, W):
    noise, theta0 = _inputs(W)
    ctx = hrt.Context(_config(hrt, W))
    try:
        ctx.hrt_set_nonfinite_check(True)
        ctx.hrt_init_particles_zeldovich(noise, W.a_init)
        disp, mom, _, _ = ctx.hrt_read_particles()
        # a NaN in a host-prepared displacement, an infinity in a momentum: refused before the force
        for which, val in ((0, math.nan), (1, math.inf)):
            state = [disp.cpu().clone(), mom.cpu().clone()]
            state[which][2, 17] = val
            with pytest.raises(hrt.HRTError) as e:
                ctx.hrt_init_particles(state[0], state[1], W.a_init)
            assert e.value.status == NONFINITE
            with pytest.raises(hrt.HRTError) as e:
                ctx.hrt_step(W.forward_grid[1])
            assert e.value.status == STATE  # no particles
        ctx.hrt_init_particles(disp, mom, W.a_init)
        for a in W.forward_grid[1:]:
            ctx.hrt_step(a)
        # a NaN in a host-prepared ray angle: refused, and the context has no rays
        bad = theta0.clone()
        bad[5, 1] = math.nan
        with pytest.raises(hrt.HRTError) as e:
            ctx.hrt_init_rays(bad)
        assert e.value.status == NONFINITE
        with pytest.raises(hrt.HRTError):
            ctx.hrt_read_maps(0)
        # a clean run with the checks on gives the run without them
        ctx.hrt_init_rays(theta0)
        slots = {s: i for i, s in enumerate(W.source_steps)}
        grid = W.reverse_grid
        for n in range(1, len(grid)):
            ctx.hrt_step(grid[n], slots.get(n, -1))
        got = ctx.hrt_read_maps(len(slots) - 1).cpu().numpy()
    finally:
        ctx.close()
    ctx = hrt.Context(_config(hrt, W))
    try:
        ctx.hrt_init_particles_zeldovich(noise, W.a_init)
        for a in W.forward_grid[1:]:
            ctx.hrt_step(a)
        ctx.hrt_init_rays(theta0)
        for n in range(1, len(grid)):
            ctx.hrt_step(grid[n], slots.get(n, -1))
        want = ctx.hrt_read_maps(len(slots) - 1).cpu().numpy()
    finally:
        ctx.close()
    assert np.isfinite(got).all()
    assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()
