"""The kick-drift-deposit of brick-sorted particles (shared-memory field and density tiles) against the
per-particle kernel: the particle update of Algorithm 1 with the CIC assignment of Sec. 2.2.

The tiled kernel does each particle's arithmetic exactly as the per-particle kernel does, so momenta and
displacements must agree bit for bit, whatever slot ranges the blocks get; the density may differ only in the
order of its float additions.  The cases cover a proper brick sort, a stale sort (particles that left their
brick's tile), a dense brick (several 256-particle chunks in one block), sparse and empty bricks (the global
path), ranges that ignore the bricks altogether, and the periodic wrap of tiles on the last bricks of each axis.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

BXY, BZ = 8, 32


@pytest.fixture(scope="module")
def hrt():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt as h
    return h


def brick_keys(pos_cells, n):
    """Sort key of every particle from its position in cells (float32, as the device computes it)."""
    c = np.floor(pos_cells).astype(np.int64) % n
    ix, iy, iz = c
    nb = n // BXY
    brick = ((iz // BZ) * nb + ix // BXY) * nb + iy // BXY
    return brick * (BXY * BXY) + (ix % BXY) * BXY + iy % BXY


def make_particles(rng, n, n_side, box, dense=0, jitter=0.0):
    """Displacements (box units, [3][np]) of particles spread over the mesh with clumps, voids and, if asked,
    `dense` particles packed into one brick; positions in cells for the sort key; jitter moves particles after
    the key was taken (a stale sort)."""
    ratio = n // n_side
    np_ = n_side ** 3
    q = np.stack(np.meshgrid(*(np.arange(n_side),) * 3, indexing="ij")).reshape(3, -1).astype(np.float64) * ratio
    # clumps: a third of the particles pulled towards 20 centres, the rest displaced by a few cells
    x = q + rng.normal(0.0, 2.0, size=q.shape)
    pull = rng.random(np_) < 0.33
    centres = rng.uniform(0, n, size=(3, 20))
    which = rng.integers(0, 20, size=np_)
    x[:, pull] = centres[:, which[pull]] + rng.normal(0.0, 1.5, size=(3, int(pull.sum())))
    if dense:
        # one brick (not the first or last) gets `dense` particles
        x[:, :dense] = (np.array([[2 * BXY], [3 * BXY], [BZ]]) + rng.uniform(0, 1, size=(3, dense))
                        * np.array([[BXY], [BXY], [BZ]]))
    x %= n
    # a sparse brick (10 particles left) and an empty one: the others move half a box along x
    for (bx, by, bz), keep in (((1, 1, 0), 10), ((3, 0, n // BZ - 1), 0)):
        lo = np.array([[bx * BXY], [by * BXY], [bz * BZ]])
        inside = np.nonzero(((x >= lo) & (x < lo + np.array([[BXY], [BXY], [BZ]]))).all(axis=0))[0]
        x[0, inside[keep:]] = (x[0, inside[keep:]] + n / 2) % n
    key_pos = x.astype(np.float32)
    x = x + rng.normal(0.0, jitter, size=x.shape) if jitter else x
    d = (x - q + n / 2) % n - n / 2  # displacement in cells, wrapped into [-n/2, n/2)
    cell = box / n
    disp = (d * cell).astype(np.float32)
    mom = rng.normal(0.0, 1.0, size=(3, np_)).astype(np.float32)
    return disp, mom, key_pos


def sorted_inputs(disp, mom, key_pos, n):
    keys = brick_keys(key_pos, n)
    perm = np.argsort(keys, kind="stable").astype(np.int32)
    counts = np.bincount(keys, minlength=n ** 3 // 32)
    key_start = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int32)
    return perm, key_start


def run_both(hrt, n, n_side, box, disp, mom, perm, key_start, kick=0.7, drift=0.9, seed=5):
    rng = np.random.default_rng(seed)
    grad = torch.tensor(rng.normal(0.0, 1.0, size=3 * n ** 3).astype(np.float32), device="cuda")
    d_ref = torch.tensor(disp, device="cuda").contiguous()
    m_ref = torch.tensor(mom, device="cuda").contiguous()
    rho_ref = torch.empty(n ** 3, dtype=torch.float32, device="cuda")
    hrt.hrt_particle_kick_drift_deposit(grad, n, box, n_side, d_ref.view(-1), m_ref.view(-1), kick, drift, rho_ref)
    d_s = torch.tensor(disp[:, perm], device="cuda").contiguous()
    m_s = torch.tensor(mom[:, perm], device="cuda").contiguous()
    order = torch.tensor(perm, device="cuda")
    ks = torch.tensor(key_start, device="cuda")
    rho = torch.full((n ** 3,), 7.0, dtype=torch.float32, device="cuda")  # overwritten, not added to
    hrt.hrt_particle_kick_drift_deposit_bricks(grad, n, box, n_side, d_s.view(-1), m_s.view(-1), order, ks, kick,
                                               drift, rho)
    torch.cuda.synchronize()
    inv = torch.empty_like(order)
    inv[order.long()] = torch.arange(order.numel(), dtype=torch.int32, device="cuda")
    d_back = d_s[:, inv.long()]
    m_back = m_s[:, inv.long()]
    return (d_ref, m_ref, rho_ref), (d_back, m_back, rho)


def check(ref, got, n_side):
    d_ref, m_ref, rho_ref = ref
    d, m, rho = got
    assert torch.equal(m, m_ref)
    assert torch.equal(d, d_ref)
    # density: same sums in another order (FP32 atomics on both sides)
    scale = float(rho_ref.abs().max())
    assert float((rho - rho_ref).abs().max()) <= 2e-6 * scale
    assert abs(float(rho.double().sum()) - float(rho_ref.double().sum())) <= 1e-6 * float(rho_ref.double().sum())


@pytest.mark.parametrize("n,n_side,jitter,dense", [(64, 32, 0.0, 0), (64, 32, 0.8, 0), (64, 32, 0.3, 3000),
                                                   (96, 48, 0.5, 700), (32, 16, 0.5, 0)])
def test_brick_kernel_matches_per_particle_kernel(hrt, n, n_side, jitter, dense):
    box = 2.0 * n
    rng = np.random.default_rng(100 + n + dense)
    disp, mom, key_pos = make_particles(rng, n, n_side, box, dense=dense, jitter=jitter)
    perm, key_start = sorted_inputs(disp, mom, key_pos, n)
    counts = np.diff(np.concatenate([key_start[::64], [n_side ** 3]]))
    # the cases reach all three block kinds: tiled, sparse (global path) and empty
    assert (counts >= 32).any() and ((counts > 0) & (counts < 32)).any()
    if dense:
        assert counts.max() > 256
    ref, got = run_both(hrt, n, n_side, box, disp, mom, perm, key_start)
    check(ref, got, n_side)


def test_brick_kernel_with_ranges_that_ignore_the_bricks(hrt):
    # lattice order and random monotone ranges: most particles lie outside their block's tile
    n, n_side, box = 64, 32, 100.0
    rng = np.random.default_rng(7)
    disp, mom, _ = make_particles(rng, n, n_side, box)
    np_ = n_side ** 3
    nbricks = n ** 3 // (BXY * BXY * BZ)
    cuts = np.sort(rng.integers(0, np_ + 1, size=nbricks - 1))
    key_start = np.zeros(n ** 3 // 32, dtype=np.int32)
    key_start[64::64] = cuts
    for k in range(1, 64):  # keys inside a brick: any monotone values
        key_start[k::64] = key_start[::64]
    perm = np.arange(np_, dtype=np.int32)
    ref, got = run_both(hrt, n, n_side, box, disp, mom, perm, key_start)
    check(ref, got, n_side)


def test_brick_kernel_rejects_bad_arguments(hrt):
    g = torch.zeros(3 * 60 ** 3, device="cuda")
    d = torch.zeros(3 * 30 ** 3, device="cuda")
    o = torch.zeros(30 ** 3, dtype=torch.int32, device="cuda")
    r = torch.zeros(60 ** 3, device="cuda")
    with pytest.raises(hrt.HRTError):  # 60 is not a multiple of 32
        hrt.hrt_particle_kick_drift_deposit_bricks(g, 60, 60.0, 30, d, d.clone(), o, o, 1.0, 1.0, r)


def test_context_tiled_and_per_particle_runs_agree(hrt):
    # the same run with TMA tiles, row-copied tiles and the per-particle path: equal up to the rounding order of
    # the deposits
    from paper_2405_12913_gb300.configs import COSMO_256 as W
    import synthetic
    noise = torch.tensor(synthetic.white_noise(W.seed, W.n_side), dtype=torch.float32, device="cuda")
    out = []
    for tiled in (2, 1, 0):
        cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                              W.samples_per_cell, W.observer, n_sources=0)
        ctx = hrt.Context(cfg)
        ctx.hrt_set_tiled_deposit(tiled)
        ctx.hrt_set_particle_sort(2)
        ctx.hrt_init_particles_zeldovich(noise, W.a_init)
        for a in W.forward_grid[1:]:
            ctx.hrt_step(a)
        d, m, _, _ = ctx.hrt_read_particles()
        out.append((d.double().cpu(), m.double().cpu()))
        ctx.close()
    cell = W.box / W.n_mesh
    for d, m in out[:2]:  # TMA tiles, row-copied tiles against per-particle
        assert float((d - out[2][0]).abs().max()) < 1e-3 * cell
        assert float((m - out[2][1]).abs().max()) < 1e-3 * float(out[2][1].abs().max())


def test_caller_particles_are_sorted_before_their_first_force(hrt):
    # particles from the caller (possibly clustered) are sorted inside hrt_init_particles, before the deposit of
    # their first force; initial conditions keep lattice order until the regular interval
    from paper_2405_12913_gb300.configs import COSMO_TINY as W
    import synthetic
    cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                          W.samples_per_cell, W.observer, n_sources=0)
    ctx = hrt.Context(cfg)
    ctx.hrt_set_particle_sort(4)
    ctx.hrt_ctx_set_profiling(True)
    ctx.hrt_init_particles_zeldovich(torch.tensor(synthetic.white_noise(W.seed, W.n_side), dtype=torch.float32,
                                                  device="cuda"), W.a_init)
    grid = W.forward_grid
    sorts = []
    for a in grid[1:5]:
        ctx.hrt_step(a)
        sorts.append(ctx.hrt_ctx_phase_times()["particle_sort"][1])
    assert sorts == [0, 0, 0, 1]
    d, m, _, _ = ctx.hrt_read_particles()
    ctx.hrt_init_particles(d, m, grid[4])
    assert ctx.hrt_ctx_phase_times()["particle_sort"][1] == 1
    sorts = []
    for a in grid[5:9]:
        ctx.hrt_step(a)
        sorts.append(ctx.hrt_ctx_phase_times()["particle_sort"][1])
    assert sorts == [0, 0, 0, 1]
    # the run from the re-sorted particles equals the stored ones read back in lattice order
    d2, m2, _, _ = ctx.hrt_read_particles()
    assert torch.isfinite(d2).all() and torch.isfinite(m2).all()
    ctx.close()
