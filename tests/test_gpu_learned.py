"""The learned ray-force correction: tensor-core MLP, its backward, the table adjoint, and a training run whose
trained network must beat the plain kernel against the fine-mesh run on held-out seeds."""
import math

import numpy as np
import pytest
import torch

import synthetic
from oracle import mlp as omlp
from oracle import pm as opm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrt():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt as h
    return h


def _params(seed):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(omlp.N_PARAMS) * 0.25).astype(np.float32)
    p.reshape(-1)[:64 * 16].reshape(64, 16)[:, 3:] = 0.0
    return p


def _x(rows, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0, 5.4, rows), rng.uniform(0.3, 1.0, rows), np.full(rows, math.log(256.0))], 1)


@pytest.mark.parametrize("rows", [512, 77])
def test_mlp_forward_matches_oracle(hrt, rows):
    p = _params(1)
    x = _x(rows, 2)
    w = torch.tensor(p, device="cuda")
    wb = torch.empty(hrt.MLP_PARAMS, dtype=torch.bfloat16, device="cuda")
    hrt.hrt_mlp_to_bf16(w, wb)
    g = torch.empty(rows, device="cuda")
    hrt.hrt_mlp_forward(torch.tensor(x, dtype=torch.float32, device="cuda"), wb, w, g)
    want = omlp.forward(torch.tensor(x.astype(np.float32), dtype=torch.float64), torch.tensor(p, dtype=torch.float64))
    y = want.numpy() - 1.0
    assert np.abs(g.cpu().double().numpy() - 1.0 - y).max() <= 2e-3 * np.abs(y).max()


def test_mlp_backward_matches_oracle_autograd(hrt):
    rows = 300
    p = _params(3)
    x = _x(rows, 4)
    gbar = np.random.default_rng(5).standard_normal(rows)
    w = torch.tensor(p, device="cuda")
    wb = torch.empty(hrt.MLP_PARAMS, dtype=torch.bfloat16, device="cuda")
    hrt.hrt_mlp_to_bf16(w, wb)
    grad = torch.zeros(hrt.MLP_PARAMS, device="cuda")
    hrt.hrt_mlp_backward(torch.tensor(x, dtype=torch.float32, device="cuda"), wb, w,
                         torch.tensor(gbar, dtype=torch.float32, device="cuda"), grad)
    pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    (omlp.forward(torch.tensor(x.astype(np.float32), dtype=torch.float64), pt, True, False)
     * torch.tensor(gbar)).sum().backward()
    want = pt.grad.numpy().copy()
    want[:64 * 16].reshape(64, 16)[:, 3:] = 0.0
    got = grad.cpu().double().numpy()
    assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()


def test_table_adjoint_matches_oracle_autograd(hrt):
    n, box, pref = 32, 64.0, 1.2
    cell = box / n
    kmax = math.sqrt(3) * math.pi / cell * 1.0001
    nk = 40
    table = 1.0 + 0.3 * np.sin(np.linspace(0, 3, nk)).astype(np.float32)
    rho = synthetic.gaussian_field(80, (n, n, n), 0.5) + 1.0
    gbar = synthetic.gaussian_field(81, (2, n, n, n))
    pm = hrt.PM(n, box)
    rho_hat = torch.empty(n, n, n // 2 + 1, dtype=torch.complex64, device="cuda")
    pm.forward_fft(torch.tensor(rho, dtype=torch.float32, device="cuda").reshape(-1), rho_hat)
    gh = torch.empty(2, n, n, n // 2 + 1, dtype=torch.complex64, device="cuda")
    gb = torch.tensor(gbar, dtype=torch.float32, device="cuda").reshape(2, -1)
    pm.forward_fft(gb[0], gh[0])
    pm.forward_fft(gb[1], gh[1])
    tt = torch.tensor(table, device="cuda")
    f = hrt.make_filter(4.0, cell, tt, kmax)
    tb = torch.zeros(nk, device="cuda")
    hrt.hrt_kspace_table_adjoint(gh, 2, rho_hat, n, box, pref, f, tb)
    tab = torch.tensor(table, dtype=torch.float64, requires_grad=True)

    def g_of_k(k):
        t = k / kmax * (nk - 1)
        i = torch.clamp(t.floor().long(), 0, nk - 2)
        w = t - i
        v = tab[i] * (1 - w) + tab[i + 1] * w
        return torch.where(t >= nk - 1, torch.ones_like(v), v)

    grads = opm.poisson_gradient(torch.tensor(rho), box, pref, 4.0, cell, g_of_k)
    sum((grads[j] * torch.tensor(gbar[j])).sum() for j in range(2)).backward()
    want = tab.grad.numpy()
    assert np.abs(tb.cpu().double().numpy() - want).max() <= 1e-4 * np.abs(want).max()
    pm.close()


def test_trained_correction_beats_plain_kernel_on_held_out_seeds(hrt):
    from dataclasses import replace

    from paper_2405_12913_gb300 import learned
    S = replace(learned.PairSpec(), n_side=64, n_coarse=64, n_fine=256, box=128.0, n_forward=12, n_reverse=6,
                a_min=0.6, n_pix=256, fov_deg=4.0, nbins=12, ell_cut=6.0e3)
    mlp, res = learned.train(S, train_seeds=range(4), test_seeds=range(100, 102), iters=40, lr=3e-3, log=lambda s: None)
    assert res["history"][-1] < 0.5 * res["history"][0]
    assert res["learned_mean_rel_err"] < 0.7 * res["plain_mean_rel_err"], res


def test_context_correction_matches_ray_trainer(hrt):
    """hrt_step with a correction set evaluates g at each step's a inside the context; its kappa equals the
    trainer's ray-only re-trace on the stored density spectra with the same network, and differs from the
    plain kernel's."""
    from dataclasses import replace

    from paper_2405_12913_gb300 import learned
    S = replace(learned.PairSpec(), n_side=32, n_coarse=32, n_fine=64, box=64.0, n_forward=6, n_reverse=4,
                a_min=0.7, n_pix=64, fov_deg=4.0, nbins=6)
    mlp = learned.MLP(seed=3)
    rng = np.random.default_rng(9)
    w = mlp.w.cpu().numpy()
    w[-65:] = rng.standard_normal(65) * 0.05          # output layer: g != 1
    mlp.w.copy_(torch.tensor(w))
    hrt.hrt_mlp_to_bf16(mlp.w, mlp.wb)
    k_plain, spectra = learned.plain_run(S, S.n_coarse, 7, record_spectra=True)
    k_ref, _ = learned.RayTrainer(S).forward(mlp, spectra, keep=False)
    k_ctx, _, _ = learned.run(S, S.n_coarse, 7, params=mlp.w)
    scale = k_ref.abs().max().item()
    # the two paths build the ray fields with different rounding (deposit order, FFT path); kappa jumps where a
    # line-of-sight sample crosses a cell face, so a rare pixel may differ by such a jump
    diff = (k_ctx - k_ref).abs()
    assert (diff > 1e-4 * scale).float().mean().item() <= 2e-3
    assert diff.median().item() <= 1e-6 * scale
    assert (k_ctx - k_plain).abs().max().item() > 1e-3 * scale


def test_context_correction_needs_ray_fields_and_resets(hrt):
    from dataclasses import replace

    from paper_2405_12913_gb300 import learned
    S = replace(learned.PairSpec(), n_side=16, n_coarse=32, box=64.0, n_forward=4, n_reverse=3, a_min=0.7,
                n_pix=32, fov_deg=4.0)
    w = torch.zeros(hrt.MLP_PARAMS, device="cuda")
    cfg = hrt.make_config(32, S.box, S.n_side, observer=S.observer, ray_fields=0)
    ctx = hrt.Context(cfg)
    with pytest.raises(hrt.HRTError):
        ctx.hrt_set_ray_correction(w)
    ctx.close()
    # g = 1 exactly (zero output layer) on the separately filtered ray fields reproduces the plain run
    k_plain, _, _ = learned.run(S, 32, 5)
    k_one, _, _ = learned.run(S, 32, 5, params=w)
    diff = (k_one - k_plain).abs()
    scale = k_plain.abs().max().item()
    assert (diff > 1e-5 * scale).float().mean().item() <= 2e-3  # rare cell-face crossings, as above
    assert diff.median().item() <= 1e-6 * scale


def test_context_fixed_ray_table_matches_ray_trainer(hrt):
    # hrt_set_ray_kernel_table: a fixed g(|k|) on the ray fields, against the trainer's re-trace with the same
    # table at every step
    from dataclasses import replace

    from paper_2405_12913_gb300 import learned
    S = replace(learned.PairSpec(), n_side=32, n_coarse=32, n_fine=64, box=64.0, n_forward=6, n_reverse=4,
                a_min=0.7, n_pix=64, fov_deg=4.0, nbins=6)
    table = torch.linspace(1.4, 0.9, learned.N_TABLE, device="cuda")

    class Fixed:
        def table(self, x):
            return table

    k_plain, spectra = learned.plain_run(S, S.n_coarse, 11, record_spectra=True)
    tr = learned.RayTrainer(S)
    k_ref, _ = tr.forward(Fixed(), spectra, keep=False)
    cfg = hrt.make_config(S.n_coarse, S.box, S.n_side, S.omega_m, S.h, S.n_s, S.sigma8, S.deconv_p,
                          S.smooth_cells, 1.0, S.observer, n_sources=1, ray_fields=2, ray_deconv_p=S.deconv_p,
                          ray_smooth_cells=S.smooth_cells)
    ctx = hrt.Context(cfg)
    ctx.hrt_set_ray_kernel_table(table, tr.kmax)
    ctx.hrt_init_particles_zeldovich(learned._noise(11, S.n_side).reshape(-1), S.a_init)
    for a in S.forward_grid[1:]:
        ctx.hrt_step(a)
    ctx.hrt_sync_particles()
    ctx.hrt_init_rays(learned._theta0(S))
    rg = S.reverse_grid
    for n in range(S.n_reverse):
        ctx.hrt_step(rg[n + 1], 0 if n + 1 == S.n_reverse else -1)
    k_ctx = ctx.hrt_read_maps(0)[0].clone()
    ctx.hrt_set_ray_kernel_table(None)
    ctx.close()
    scale = k_ref.abs().max().item()
    diff = (k_ctx - k_ref).abs()
    assert (diff > 1e-4 * scale).float().mean().item() <= 2e-3  # rare cell-face crossings
    assert diff.median().item() <= 1e-6 * scale
    assert (k_ctx - k_plain).abs().max().item() > 1e-3 * scale


def test_context_particle_correction_is_the_stateless_solve_with_its_table(hrt):
    # the particle-force correction of a context: its force fields after the ICs equal the stateless PM solve of
    # the same density with the network's table at the ICs' scale factor (the same |k| grid as the context's); a
    # network with a zero output layer is the plain force; a recorded run refuses it
    from paper_2405_12913_gb300.configs import COSMO_TINY as W
    from paper_2405_12913_gb300 import learned
    n, box = W.n_mesh, W.box
    noise = torch.tensor(synthetic.white_noise(W.seed, W.n_side), dtype=torch.float32, device="cuda").reshape(-1)
    cfg = hrt.make_config(n, box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                          W.samples_per_cell, W.observer)
    plain = hrt.Context(cfg)
    plain.hrt_init_particles_zeldovich(noise, W.a_init)
    g_plain = plain.hrt_read_grad().clone()
    disp, _, _, _ = plain.hrt_read_particles()
    plain.close()
    cell = box / n
    kmax = math.sqrt(3.0) * math.pi / cell * 1.0001
    for which, p in (("zero output layer", learned.MLP(seed=0).w), ("random", torch.tensor(_params(9), device="cuda"))):
        ctx = hrt.Context(cfg)
        ctx.hrt_set_particle_correction(p)
        ctx.hrt_init_particles_zeldovich(noise, W.a_init)
        got = ctx.hrt_read_grad()
        ctx.close()
        wb = torch.empty(hrt.MLP_PARAMS, dtype=torch.bfloat16, device="cuda")
        hrt.hrt_mlp_to_bf16(p, wb)
        table = torch.empty(learned.N_TABLE, device="cuda")
        hrt.hrt_mlp_forward(learned.MLP.inputs(kmax, cell, W.a_init, n), wb, p, table)
        rho = torch.empty(n ** 3, device="cuda")
        hrt.hrt_cic_scatter(disp, W.n_side, n, box, rho)
        pm = hrt.PM(n, box)
        want = torch.empty(3, n ** 3, device="cuda")
        pm.solve(rho, 1.5 * W.omega_m / W.a_init, hrt.make_filter(W.deconv_p, W.smooth_cells * cell, table, kmax), want)
        pm.close()
        scale = float(want.abs().max())
        assert float((got.reshape(3, -1) - want).abs().max()) <= 1e-5 * scale, which
        if which == "zero output layer":
            assert float((got - g_plain).abs().max()) <= 1e-5 * scale
        else:
            assert float((got - g_plain).abs().max()) > 1e-3 * scale
    ctx = hrt.Context(cfg)
    ctx.hrt_set_checkpointing(2)
    ctx.hrt_set_particle_correction(torch.tensor(_params(9), device="cuda"))
    ctx.hrt_init_particles_zeldovich(noise, W.a_init)
    ctx.hrt_step(W.forward_grid[1])
    with pytest.raises(hrt.HRTError) as e:
        ctx.hrt_adjoint(None)
    assert "particle force" in str(e.value)
    ctx.hrt_set_particle_correction(None)
    ctx.close()


def test_adam_step_matches_the_textbook_update(hrt):
    # Adam with bias correction (Kingma and Ba) in FP32 on the master weights, three steps against a plain FP32
    # PyTorch restatement; the padding columns 3..15 of W1 stay as they were and are zero in the BF16 copy
    n = hrt.MLP_PARAMS
    gen = torch.Generator(device="cuda").manual_seed(5)
    w = torch.randn(n, device="cuda", generator=gen) * 0.2
    w0 = w.clone()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    pad = torch.zeros(n, dtype=torch.bool, device="cuda")
    pad[:64 * 16] = (torch.arange(64 * 16, device="cuda") % 16) >= 3
    w_ref, m_ref, v_ref = w.clone(), m.clone(), v.clone()
    lr, b1, b2, eps = 3e-3, 0.9, 0.999, 1e-8
    # the FP32 constants of the update: beta and 1 - beta in single precision, the bias corrections formed in
    # double and rounded once
    f32 = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")  # noqa: E731
    b1f, b2f = f32(b1), f32(b2)
    for step in range(1, 4):
        g = torch.randn(n, device="cuda", generator=gen)
        hrt.hrt_mlp_adam(w, wb, g, m, v, lr, b1, b2, eps, step)
        mr = b1f * m_ref + (1 - b1f) * g
        vr = b2f * v_ref + (1 - b2f) * g * g
        c1, c2 = f32(1 - b1 ** step), f32(1 - b2 ** step)
        upd = w_ref - f32(lr) * (mr / c1) / (torch.sqrt(vr / c2) + f32(eps))
        w_ref = torch.where(pad, w_ref, upd)
        m_ref = torch.where(pad, m_ref, mr)
        v_ref = torch.where(pad, v_ref, vr)
    torch.cuda.synchronize()
    assert torch.allclose(w, w_ref, rtol=1e-6, atol=1e-7)
    # the kernel may contract b m + (1 - b) g into one FMA: where the terms cancel, the moments differ by a few
    # ulps of the terms ((1 - b1) |g| < 0.5, (1 - b2) g^2 < 0.02), not of the result
    assert torch.allclose(m, m_ref, rtol=1e-6, atol=1e-7) and torch.allclose(v, v_ref, rtol=1e-6, atol=1e-8)
    assert torch.equal(wb[~pad], w[~pad].to(torch.bfloat16))
    assert float(wb[pad].float().abs().max()) == 0.0
    # Adam moves a weight by at most about lr per step (|m_hat| / sqrt(v_hat) <= 1.0012 here)
    moved = (w - w0)[~pad].abs()
    assert 0.5 * lr < float(moved.max()) <= 3.1 * lr
