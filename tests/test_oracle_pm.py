"""Pins of the oracle's particle-mesh force: deposit, FFT Poisson gradient, gather, leapfrog, ICs."""
import itertools
import math

import numpy as np
import pytest
import torch

import synthetic
from oracle import cosmology as cosmo
from oracle import ewald, pm, sim
from oracle.units import G_NEWTON


def test_cic_mass_conservation_and_mean():
    x = torch.tensor(synthetic.uniform_positions(1, 5000, 50.0))
    rho = pm.cic_deposit(x, 50.0, 16)
    assert float(rho.sum()) == pytest.approx(16 ** 3, rel=1e-13)
    assert float(rho.min()) >= 0.0


def test_cic_single_particle_on_node_and_at_cell_centre():
    n, L = 8, 8.0
    rho = pm.cic_deposit(torch.tensor([[3.0, 5.0, 7.0]], dtype=torch.float64), L, n)
    assert float(rho[3, 5, 7]) == n ** 3 and int((rho != 0).sum()) == 1
    rho = pm.cic_deposit(torch.tensor([[3.5, 5.5, 7.5]], dtype=torch.float64), L, n)
    for a, b, c in itertools.product((3, 4), (5, 6), (7, 0)):
        assert float(rho[a, b, c]) == pytest.approx(n ** 3 / 8)
    assert int((rho != 0).sum()) == 8


def test_cic_integer_translation_commutes_with_roll():
    L, n = 32.0, 16
    x = torch.tensor(synthetic.uniform_positions(2, 300, L))
    shift = torch.tensor([2 * L / n, -3 * L / n, 5 * L / n], dtype=torch.float64)
    a = pm.cic_deposit(x + shift, L, n)
    b = torch.roll(pm.cic_deposit(x, L, n), shifts=(2, -3, 5), dims=(0, 1, 2))
    assert torch.allclose(a, b, atol=1e-12)


def _brute_gradient(rho, L, pref, p, sigma):
    """Full-grid DFT sum, O(N^6): grad_j(x) = N^-3 sum_k i k_j G(k) F(k) rho_k e^{ikx}, k_j = 0 at n_j = -N/2."""
    n = rho.shape[0]
    f = np.array([i if i < n // 2 else i - n for i in range(n)])
    idx = np.arange(n)
    ph = np.exp(-2j * math.pi * np.outer(f, idx) / n)  # [freq, pos]
    rho_k = np.einsum("ai,bj,ck,ijk->abc", ph, ph, ph, rho)
    kf = 2 * math.pi / L
    K = [kf * f.reshape(-1, 1, 1), kf * f.reshape(1, -1, 1), kf * f.reshape(1, 1, -1)]
    k2 = K[0] ** 2 + K[1] ** 2 + K[2] ** 2
    cell = L / n
    win = np.ones_like(k2)
    for kk in K:
        win = win * np.sinc(kk * cell / 2 / math.pi) ** (-p)
    win = win * np.exp(-0.5 * k2 * sigma ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        phik = np.where(k2 > 0, -pref * rho_k * win / k2, 0.0)
    out = []
    for j, nf in enumerate((f.reshape(-1, 1, 1), f.reshape(1, -1, 1), f.reshape(1, 1, -1))):
        d = np.where(nf == -n // 2, 0.0, K[j])
        g = 1j * d * phik
        ip = np.conj(ph)  # e^{+ikx}
        out.append(np.einsum("ai,bj,ck,abc->ijk", ip, ip, ip, g).real / n ** 3)
    return out


@pytest.mark.parametrize("p,sigma", [(0.0, 0.0), (4.0, 1.0)])
def test_fft_gradient_matches_brute_force_dft(p, sigma):
    n, L = 8, 16.0
    rho = synthetic.gaussian_field(3, (n, n, n)) + 1.0
    got = pm.poisson_gradient(torch.tensor(rho), L, 0.7, p, sigma)
    want = _brute_gradient(rho, L, 0.7, p, sigma)
    for g, w in zip(got, want):
        assert np.allclose(g.numpy(), w, atol=1e-12 * np.abs(w).max() + 1e-14)


@pytest.mark.parametrize("axis,m", [(0, 3), (1, 5), (2, 2), (2, 7)])
def test_single_mode_poisson_gradient(axis, m):
    # delta = A cos(k x_axis), lap phi = pref delta  =>  d_axis phi = pref A sin(k x) / k, other components 0,
    # times the filter sinc(k cell / 2)^-p exp(-k^2 sigma^2 / 2).
    n, L, A, pref, p, sig = 16, 40.0, 0.3, 2.5, 4.0, 1.7
    x = torch.arange(n, dtype=torch.float64) * (L / n)
    k = 2 * math.pi * m / L
    shape = [1, 1, 1]
    shape[axis] = n
    rho = (1.0 + A * torch.cos(k * x)).view(shape).expand(n, n, n).contiguous()
    grads = pm.poisson_gradient(rho, L, pref, p, sig)
    filt = (math.sin(k * L / n / 2) / (k * L / n / 2)) ** (-p) * math.exp(-0.5 * k * k * sig * sig)
    want = (pref * A / k * filt * torch.sin(k * x)).view(shape).expand(n, n, n)
    for j in range(3):
        if j == axis:
            assert torch.allclose(grads[j], want, atol=1e-12)
        else:
            assert float(grads[j].abs().max()) < 1e-12


def test_ewald_field_of_a_periodic_point_mass():
    # The periodic sum, split into real- and reciprocal-space parts, is exact for any splitting parameter, so a
    # wrong factor in either part shows as a dependence on it; near the mass the field is Newton's r / |r|^3 (the
    # images and the background add O(|r| / L^3)); it vanishes at the half-period points and is odd in r.
    L = 10.0
    r = np.random.default_rng(3).uniform(-0.5, 0.5, (20, 3)) * L
    g0 = ewald.grad_phi_3d(r, L)
    scale = np.abs(g0).max()
    for alpha, n_real, n_recip in ((1.5 / L, 4, 8), (3.0 / L, 3, 12)):
        g = ewald.grad_phi_3d(r, L, n_real=n_real, n_recip=n_recip, alpha=alpha)
        assert np.abs(g - g0).max() < 1e-12 * scale
    near = np.array([[1e-3, 0.5e-3, -0.7e-3]]) * L
    newton = near / np.linalg.norm(near) ** 3
    assert np.abs(ewald.grad_phi_3d(near, L) - newton).max() < 1e-6 * np.abs(newton).max()
    half = np.array([[L / 2, 0, 0], [0, L / 2, 0], [L / 2, L / 2, L / 2]])
    assert np.abs(ewald.grad_phi_3d(half, L)).max() < 1e-12 * scale
    assert np.abs(ewald.grad_phi_3d(-r, L) + g0).max() < 1e-12 * scale


def test_pm_force_matches_periodic_direct_sum():
    # One mass in a periodic box; the PM gradient interpolated at test points 5..12 cells away agrees with the
    # 3D Ewald sum to the PM force accuracy with the 1-cell smoothing and sinc^-4 deconvolution.
    n, L, M = 32, 64.0, 1e14
    cell = L / n
    src = np.array([20.3, 31.7, 11.2])
    rho = pm.cic_deposit(torch.tensor(src[None, :]), L, n)
    pref = 4 * math.pi * G_NEWTON * M / L ** 3
    grads = pm.poisson_gradient(rho, L, pref, 4.0, cell)
    rng = np.random.default_rng(7)
    dirs = rng.standard_normal((40, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = cell * rng.uniform(5.0, 12.0, 40)[:, None] * dirs
    got = pm.cic_gather(grads, torch.tensor(src + r), L).numpy()
    want = ewald.grad_phi_3d(r, L) * G_NEWTON * M
    err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
    assert np.median(err) < 0.01
    assert err.max() < 0.03


def test_gather_of_linear_field_is_exact():
    n, L = 16, 32.0
    cell = L / n
    g = torch.arange(n, dtype=torch.float64) * cell
    X, Y, Z = torch.meshgrid(g, g, g, indexing="ij")
    field = 0.3 + 1.1 * X - 0.7 * Y + 2.3 * Z
    pts = torch.tensor(synthetic.uniform_positions(4, 200, L - 2 * cell))
    got = pm.cic_gather([field], pts, L)[:, 0]
    want = 0.3 + 1.1 * pts[:, 0] - 0.7 * pts[:, 1] + 2.3 * pts[:, 2]
    assert torch.allclose(got, want, atol=1e-12)


def test_kick_drift_with_zero_field():
    n = 4
    q = pm.lattice(n, 8.0)
    d = torch.tensor(synthetic.small_displacements(5, n, 0.3).T.copy())
    p = torch.tensor(synthetic.small_displacements(6, n, 0.3).T.copy())
    zero = [torch.zeros(8, 8, 8, dtype=torch.float64)] * 3
    d2, p2 = pm.particle_kick_drift(d, p, q, zero, 8.0, kick=0.4, drift=0.25)
    assert torch.equal(p2, p)
    assert torch.allclose(d2, d + 0.25 * p, atol=0)


def test_kick_drift_with_a_uniform_field():
    # a uniform gradient is gathered exactly (the CIC weights sum to one); the drift moves the particles with the
    # momentum after the kick
    n, L = 4, 8.0
    q = pm.lattice(n, L)
    d = torch.tensor(synthetic.small_displacements(5, n, 0.3).T.copy())
    p = torch.tensor(synthetic.small_displacements(6, n, 0.3).T.copy())
    g0 = (0.7, -1.3, 0.2)
    fields = [torch.full((8, 8, 8), v, dtype=torch.float64) for v in g0]
    d2, p2 = pm.particle_kick_drift(d, p, q, fields, L, kick=0.4, drift=0.25)
    want_p = p - 0.4 * torch.tensor(g0, dtype=torch.float64)
    assert torch.allclose(p2, want_p, rtol=0, atol=1e-14)
    assert torch.allclose(d2, d + 0.25 * want_p, rtol=0, atol=1e-14)


def test_zeldovich_density_has_the_sign_of_the_linear_field():
    # delta_k = w_k sqrt(P / V_cell) with delta = -div Psi: at a small growth factor the particles deposit
    # 1 + D1 delta on a mesh equal to the lattice, so the deposited density at the lowest wavenumbers is the white
    # noise times a positive factor (and a displacement of the wrong sign would give the opposite density)
    n, L, a = 32, 512.0, 0.01
    noise = synthetic.white_noise(21, n)
    disp, _ = pm.zeldovich(noise, L, 0.3, 0.7, 0.96, 0.8, a)
    assert float(disp.abs().max()) < 0.05 * L / n
    rho = pm.cic_deposit(pm.lattice(n, L) + disp, L, n)
    r_hat, w_hat = torch.fft.fftn(rho - 1.0), torch.fft.fftn(torch.tensor(noise))
    f = pm.signed_freq(n).double()
    nn = torch.sqrt(f.view(-1, 1, 1) ** 2 + f.view(1, -1, 1) ** 2 + f.view(1, 1, -1) ** 2)
    low = (nn > 0) & (nn <= 3)
    c = float((r_hat[low] * w_hat[low].conj()).real.sum()) / math.sqrt(
        float((r_hat[low].abs() ** 2).sum()) * float((w_hat[low].abs() ** 2).sum()))
    assert c > 0.9


def test_zeldovich_momentum_ratio_and_power():
    om, h, ns, s8, a = 0.3, 0.7, 0.96, 0.8, 0.05
    n, L = 32, 256.0
    amp = cosmo.power_amplitude(om, h, ns, s8)
    ratio = a ** 2 * cosmo.E(a, om) * cosmo.growth_f(a, om)
    pk_sum = 0.0
    seeds = range(8)
    for seed in seeds:
        disp, mom = pm.zeldovich(synthetic.white_noise(seed, n), L, om, h, ns, s8, a)
        assert torch.allclose(mom, ratio * disp, rtol=1e-12, atol=0)
        # linear density of the Zel'dovich field: delta = -div Psi, measured spectrally on the lattice
        psi = (disp / cosmo.growth_D1(a, om)).T.reshape(3, n, n, n)
        f = pm.signed_freq(n).double() * (2 * math.pi / L)
        kk = [f.view(-1, 1, 1), f.view(1, -1, 1), f.view(1, 1, -1)]
        div_hat = sum(1j * kk[j] * torch.fft.fftn(psi[j]) for j in range(3))
        pk_sum = pk_sum + (div_hat.abs() ** 2) * (L ** 3) / n ** 6
    pk = pk_sum / len(seeds)
    nn = torch.sqrt(sum((pm.signed_freq(n).double().view(*s)) ** 2 for s in ((-1, 1, 1), (1, -1, 1), (1, 1, -1))))
    for lo in (3, 5, 8):
        sel = (nn >= lo) & (nn < lo + 1)
        kmean = float(nn[sel].mean()) * 2 * math.pi / L
        want = float(cosmo.linear_power(kmean, om, h, ns, amp))
        got = float(pk[sel].mean())
        nmodes = int(sel.sum()) * len(seeds) / 2
        assert got == pytest.approx(want, rel=4.0 / math.sqrt(nmodes) + 0.05)


def test_forward_then_reverse_returns_to_initial_conditions():
    # Time reversibility of the symplectic leapfrog (footnote of Sec. 2, [LiEtAl2024] Table 2).
    c, flt = sim.Cosmo(), sim.Filter()
    n, nm, L = 16, 32, 64.0
    part0 = sim.initial_particles(synthetic.white_noise(11, n), L, c, 0.1)
    grid = [0.1 + 0.9 * i / 6 for i in range(7)]
    part1, grads = sim.run_forward(part0, grid, L, nm, c, flt)
    assert float((part1.disp - part0.disp).abs().max()) > 1.0
    back = list(reversed(grid))
    part = part1
    for a_next in back[1:]:
        part = sim.particle_step(part, grads, a_next, c.omega_m, L)
        grads = sim.pm_force(part, L, nm, 1.5 * c.omega_m / a_next, flt)
    part = sim.particle_sync(part, grads, c.omega_m, L)
    assert float((part.disp - part0.disp).abs().max()) < 1e-9
    assert float((part.mom - part0.mom).abs().max()) < 1e-9 * float(part0.mom.abs().max())


def test_low_k_power_grows_as_growth_factor_squared():
    # Linear theory: delta(k) grows as D1(a).  With the mesh equal to the particle lattice (no lattice alias)
    # and no filter, the lowest-k shell follows D1^2 and the CIC windows only ever slow the growth down.
    c, flt = sim.Cosmo(), sim.Filter(0.0, 0.0)
    n, L = 32, 512.0
    part = sim.initial_particles(synthetic.white_noise(12, n), L, c, 0.02)
    rho0 = pm.cic_deposit(part.q + part.disp, L, n)
    grid = list(np.exp(np.linspace(math.log(0.02), math.log(0.1), 17)))
    part1, _ = sim.run_forward(part, grid, L, n, c, flt)
    rho1 = pm.cic_deposit(part1.q + part1.disp, L, n)
    _, p0 = pm.matter_power(rho0, L, 4)
    _, p1 = pm.matter_power(rho1, L, 4)
    ratio = p1 / p0 / (cosmo.growth_D1(0.1, c.omega_m) / cosmo.growth_D1(0.02, c.omega_m)) ** 2
    assert ratio[0] == pytest.approx(1.0, rel=0.02)
    assert np.all(np.diff(ratio) < 0.0) and ratio.max() < 1.02


def _waves(n, box, amps):
    """delta = sum_axis A_axis cos(k q_axis) on the particle lattice, k = 2 pi 2 / box."""
    k = 2.0 * math.pi * 2 / box
    q = pm.lattice(n, box).numpy()
    delta = sum(a * np.cos(k * q[:, ax]) for ax, a in amps.items())
    return delta.reshape(n, n, n), q, k


def test_lpt_single_plane_wave_has_no_second_order_term():
    # one-dimensional motion: Zel'dovich is exact, the 2LPT source vanishes
    n, box = 16, 32.0
    delta, q, k = _waves(n, box, {1: 0.3})
    psi1, psi2 = pm.lpt_fields(torch.tensor(delta), box)
    assert np.abs(psi2.numpy()).max() < 1e-14
    # Psi1 = -grad phi1 with phi1 = -(A / k^2) cos(k y): Psi1_y = -(A / k) sin(k y), div Psi1 = -delta
    assert np.allclose(psi1[:, 1].numpy(), -(0.3 / k) * np.sin(k * q[:, 1]), atol=1e-13)
    assert np.abs(psi1[:, [0, 2]].numpy()).max() < 1e-14


@pytest.mark.parametrize("direction", [(1, 1, 0), (1, 0, -1), (1, -1, 1)])
def test_lpt_plane_wave_along_a_diagonal_has_no_second_order_term(direction):
    # a plane wave in any direction is one-dimensional motion: its 2LPT source sum_{i<j} phi_ii phi_jj - phi_ij^2
    # vanishes only with the mixed derivatives subtracted; Psi1 = -(A / k^2) k sin(k . q)
    n, box, amp = 16, 32.0, 0.25
    kvec = 2.0 * math.pi / box * np.array(direction, dtype=np.float64)
    q = pm.lattice(n, box).numpy()
    delta = amp * np.cos(q @ kvec)
    psi1, psi2 = pm.lpt_fields(torch.tensor(delta.reshape(n, n, n)), box)
    assert np.abs(psi2.numpy()).max() < 1e-14
    want = -(amp / float(kvec @ kvec)) * np.sin(q @ kvec)[:, None] * kvec[None, :]
    assert np.allclose(psi1.numpy(), want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("axes", [(0, 1), (0, 2)])
def test_lpt_two_orthogonal_waves_closed_form(axes):
    # phi1 = -(A cos kx + B cos ky) / k^2: the source is A B cos kx cos ky, phi2 = -A B cos kx cos ky / (2 k^2),
    # Psi2 = grad phi2 = (A B / (2 k)) (sin kx cos ky, cos kx sin ky); the (0, 2) case runs through the rfft axis
    n, box = 16, 32.0
    a, b = 0.2, 0.35
    delta, q, k = _waves(n, box, {axes[0]: a, axes[1]: b})
    _, psi2 = pm.lpt_fields(torch.tensor(delta), box)
    u, v = k * q[:, axes[0]], k * q[:, axes[1]]
    want = np.zeros((n ** 3, 3))
    want[:, axes[0]] = a * b / (2 * k) * np.sin(u) * np.cos(v)
    want[:, axes[1]] = a * b / (2 * k) * np.cos(u) * np.sin(v)
    assert np.allclose(psi2.numpy(), want, atol=1e-13)


def test_lpt_second_order_mode_follows_the_n_body():
    # Two orthogonal plane waves at the fundamental mode, Einstein-de Sitter (D1 = a, D2 = -(3/7) a^2).  The
    # Zel'dovich displacement has no (1, +-1, 0) modes; the 2LPT one, D2 (A B / 2k) (sin kx cos ky, cos kx sin ky),
    # lives only there.  Particles started from Zel'dovich ICs at a = 0.01 and evolved by the PM leapfrog (mesh =
    # lattice, no filter) build up that mode by a = 1.  The PM force is a little weak at the mesh scale, so the
    # first-order modes grow by a factor r1 slightly below linear theory; the second-order mode, quadratic in them,
    # must then reach r1^2 of the 2LPT amplitude (a wrong sign or coefficient of D2 misses by far more).
    n, box, amp, om = 32, 100.0, 0.3, 1.0
    c = sim.Cosmo(omega_m=om)
    k = 2.0 * math.pi / box
    q = pm.lattice(n, box).numpy()
    delta = amp * np.cos(k * q[:, 0]) + amp * np.cos(k * q[:, 1])
    # the white noise whose linear density (delta_k = w_k sqrt(P(k) / V_cell)) is these waves at a = 1
    p_kf = float(cosmo.linear_power(k, om, c.h, c.n_s, cosmo.power_amplitude(om, c.h, c.n_s, c.sigma8)))
    noise = (delta / math.sqrt(p_kf / (box / n) ** 3)).reshape(n, n, n)
    part = sim.initial_particles(noise, box, c, 0.01)
    grid = list(np.exp(np.linspace(math.log(0.01), 0.0, 41)))
    part1, _ = sim.run_forward(part, grid, box, n, c, sim.Filter(0.0, 0.0))
    disp2, _ = pm.lpt2(noise, box, om, c.h, c.n_s, c.sigma8, 1.0)
    disp1, _ = pm.zeldovich(noise, box, om, c.h, c.n_s, c.sigma8, 1.0)

    def mode(d, comp, m):
        return complex(torch.fft.fftn(d[:, comp].reshape(n, n, n))[m])

    for comp, first in ((0, (1, 0, 0)), (1, (0, 1, 0))):
        r1 = mode(part1.disp, comp, first) / mode(disp1, comp, first)
        assert abs(r1 - 1.0) < 0.03
        for m in ((1, 1, 0), (1, n - 1, 0)):
            assert abs(mode(disp1, comp, m)) < 1e-9 * abs(mode(disp2, comp, m))
            r2 = mode(part1.disp, comp, m) / mode(disp2, comp, m)
            assert abs(r2 / r1 ** 2 - 1.0) < 0.02


def test_lpt_second_order_is_quadratic_and_eds_assembly():
    n, box = 16, 64.0
    noise = synthetic.white_noise(41, n)
    d = synthetic.gaussian_field(42, (n, n, n), 0.05)
    p1, p2 = pm.lpt_fields(torch.tensor(d), box)
    q1, q2 = pm.lpt_fields(torch.tensor(2.0 * d), box)
    assert np.allclose(q1.numpy(), 2.0 * p1.numpy(), rtol=0, atol=1e-14)
    assert np.allclose(q2.numpy(), 4.0 * p2.numpy(), rtol=0, atol=1e-14)
    # Einstein-de Sitter: D1 = a, f1 = 1, D2 = -(3/7) a^2, f2 = 2, E = a^-3/2
    a = 0.05
    disp, mom = pm.lpt2(noise, box, 1.0, 0.7, 0.96, 0.8, a)
    dz, mz = pm.zeldovich(noise, box, 1.0, 0.7, 0.96, 0.8, a)
    psi1 = dz / a
    psi2 = (disp - dz) / (-3.0 / 7.0 * a * a)
    e = a ** -1.5
    assert np.allclose(mom.numpy(), (a * a * e * (a * psi1 + 2.0 * (-3.0 / 7.0) * a * a * psi2)).numpy(), rtol=1e-10,
                       atol=1e-14)
    assert np.abs(psi2.numpy()).max() > 0


def test_mode_gradient_matches_the_grid_solve():
    # the gradient of a cosine-mode density at single nodes (used for spot checks of full-size meshes) against the
    # FFT solve of the same density on the whole mesh, with deconvolution, smoothing and a mode that reaches the
    # largest non-Nyquist frequency on one axis
    n, box, pref = 16, 40.0, 0.7
    spec = synthetic.mode_spec(3, n, 6, 1.0)
    assert int(np.abs(spec["modes"]).max()) == n // 2 - 1
    rho = 1.0 + synthetic.mode_field_values(spec, n, np.arange(n ** 3)).reshape(n, n, n)
    grid = pm.poisson_gradient(torch.tensor(rho), box, pref, 4.0, 0.8 * box / n)
    idx = np.arange(n ** 3)
    want = pm.mode_gradient(spec["modes"], spec["amp"], spec["phase"], idx, n, box, pref, 4.0, 0.8 * box / n)
    for j in range(3):
        g = grid[j].reshape(-1).numpy()
        assert np.abs(g - want[j]).max() <= 1e-12 * np.abs(g).max()
        assert np.abs(g).max() > 0.0
