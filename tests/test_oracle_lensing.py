"""Pins of the oracle's lensing end to end: point-mass lens (Sec. 6.1) and the convergence power spectrum."""
import math
import os

import numpy as np
import pytest
import torch

import synthetic
from oracle import cosmology as cosmo
from oracle import ewald, power, rays, sim
from oracle.units import C_LIGHT, G_NEWTON

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_einstein_radius_worked_example():
    # Sec. 6.1: M = 1.3e15 Msun at chi_l = 350 Mpc/h, chi_s = 850 Mpc/h gives theta_E = 1.8'.
    row = np.loadtxt(os.path.join(GOLDEN, "point_mass_einstein_radius.txt"))
    m_sun, chi_l, chi_s, h, theta_e_arcmin = row
    m = m_sun * h  # Msun -> Msun/h
    theta_e = math.sqrt(4 * G_NEWTON * m / C_LIGHT ** 2 * (chi_s - chi_l) / (chi_l * chi_s))
    assert theta_e / synthetic.ARCMIN == pytest.approx(theta_e_arcmin, abs=0.05)


def point_mass_run_data(stride=1):
    """The oracle's deflections of the point-mass rays and their Born deflections in the exact 3D Ewald field;
    ``stride`` keeps every stride-th ray (impact parameters from 0.1 to 20 cells either way)."""
    pmc = sim.PointMass()
    th = synthetic.polar_impact_grid(128, 128, 0.1, 20.0, pmc.cell, pmc.chi_lens)
    # every second radius at two azimuths (the first and the 38th of 128)
    sel = np.concatenate([np.arange(0, 128 * 128, 256) + 5, np.arange(128, 128 * 128, 256) + 37])
    th = th[sel][::stride]
    st = sim.point_mass_trace(pmc, torch.tensor(th))
    alpha = th - st["theta"].numpy()
    born = sim.point_mass_born_ewald(pmc, th, 400)
    b_cells = pmc.chi_lens * np.hypot(th[:, 0], th[:, 1]) / pmc.cell
    return pmc, th, alpha, born, b_cells


@pytest.fixture(scope="module")
def point_mass_run():
    return point_mass_run_data()


def test_point_mass_deflection_matches_born_ewald_above_threshold(point_mass_run):
    # Above theta_thresh = 4 cells / chi_l the mesh resolves the lens; the paper quotes < 0.5 % there.
    pmc, th, alpha, born, b = point_mass_run
    err = np.linalg.norm(alpha - born, axis=1) / np.linalg.norm(born, axis=1)
    above = b > 4.0
    assert np.median(err[above]) < 0.005
    assert err[above].max() < 0.01
    assert err[b > 9.0].max() < 0.003
    # deflection points away from the lens direction on the sky: alpha parallel to +theta0 / |theta0|
    cosang = (alpha * th).sum(axis=1) / (np.linalg.norm(alpha, axis=1) * np.linalg.norm(th, axis=1))
    assert cosang[above].min() > 0.999
    # inside the threshold the mesh suppresses the deflection (Sec. 6.1)
    assert np.all(np.linalg.norm(alpha[b < 1.0], axis=1) < np.linalg.norm(born[b < 1.0], axis=1))


def test_born_ewald_matches_closed_form_with_periodic_images(point_mass_run):
    # Eq. "pointmass_analytic" with the periodic image sum of Appendix D (and the uniform background of the
    # zero-mean FFT potential): alpha = (chi_s - chi_l)/chi_s 4GM/c^2 sum_m (b - m)/|b - m|^2 - (pi/L^2) b.
    pmc, th, alpha, born, b = point_mass_run
    bvec = th * pmc.chi_lens
    lever = (pmc.chi_source - pmc.chi_lens) / pmc.chi_source * 4 * G_NEWTON * pmc.mass / C_LIGHT ** 2
    direct = lever * (ewald.lattice_sum_2d(bvec, pmc.box, 33) - math.pi / pmc.box ** 2 * bvec)
    ew2 = lever * ewald.deflection_sum_2d(bvec, pmc.box)
    assert np.allclose(direct, ew2, rtol=2e-3, atol=1e-3 * np.abs(ew2).max())
    # the rays form a cone (x = chi theta varies by L / chi_l = 20 % across the box) rather than parallel
    # columns, so the two agree to O(1e-3) at the largest impact parameters and far better inside
    err = np.linalg.norm(born - ew2, axis=1) / np.linalg.norm(ew2, axis=1)
    assert err.max() < 2e-3 and err[b < 5.0].max() < 3e-4
    # and the single-lens term alone is the textbook 4GM/(c^2 b) at small b
    small = b < 0.5
    hat = lever * bvec[small] / (bvec[small] ** 2).sum(axis=1, keepdims=True)
    assert np.allclose(born[small], hat, rtol=2e-3)


def test_periodic_lensing_sum_is_independent_of_the_splitting():
    # the 2D Ewald form of the image sum is exact for any splitting parameter, odd in b, and zero at the
    # half-period points
    L = 10.0
    b = np.random.default_rng(4).uniform(-0.5, 0.5, (20, 2)) * L
    d0 = ewald.deflection_sum_2d(b, L)
    scale = np.abs(d0).max()
    for alpha, n_real, n_recip in ((1.5 / L, 5, 10), (3.0 / L, 4, 14)):
        d = ewald.deflection_sum_2d(b, L, n_real=n_real, n_recip=n_recip, alpha=alpha)
        assert np.abs(d - d0).max() < 1e-12 * scale
    assert np.abs(ewald.deflection_sum_2d(-b, L) + d0).max() < 1e-12 * scale
    assert np.abs(ewald.deflection_sum_2d(np.array([[L / 2, 0.0], [L / 2, L / 2]]), L)).max() < 1e-12 * scale


def test_reverse_run_refers_the_ray_kick_to_the_force_snapshot():
    # Each step's rays see the force of the particles at the start of the step, corrected in time by
    # g(chi) = D1(a) a_c / (D1(a_c) a) with a_c that snapshot's scale factor (Sec. 3.2, Eq. "kick"; reading R8).
    # In the linear regime the snapshot fields scale as D1 / a, so the co-evolution's deflections equal those
    # through the a = 1 fields with the correction referred to a = 1.  A correction referred to the end of the
    # step misses by the change of D1 / a over a step, about 10 % here; the backward N-body's own departure from
    # linear growth stays below 1 %.
    c = sim.Cosmo(sigma8=1e-3)
    om, n, box = c.omega_m, 16, 200.0
    part = sim.initial_particles(synthetic.white_noise(8, n), box, c, 1.0)
    flt = sim.Filter()
    g1 = sim.pm_force(part, box, n, 1.5 * om, flt)
    grid = [1.0, 0.75, 0.5]
    th0 = torch.tensor(synthetic.pixel_grid(16, 2.0 * synthetic.DEGREE))
    obs = (0.37 * box, 0.61 * box, 0.23 * box)
    res = sim.run_reverse(part, g1, grid, box, n, c, flt, th0, obs, {2})
    st = rays.init_state(th0)
    w1 = sim.growth_weight(1.0, om)
    for a, b in zip(grid[:-1], grid[1:]):
        st = rays.ray_step(st, g1[0], g1[1], box, obs, cosmo.chi_of_a(a, om), cosmo.chi_of_a(b, om), 1.0, w1,
                           gz=g1[2])
    d_run, d_ref = res.thetas[2] - th0, st["theta"] - th0
    assert float((d_run - d_ref).norm() / d_ref.norm()) < 0.02


def test_power_of_single_cosine_mode():
    m, dth, amp, mx = 64, 1e-3, 0.02, 5
    x = np.arange(m)
    kappa = amp * np.cos(2 * math.pi * mx * x / m)[None, :] * np.ones((m, 1))
    ell, p, cnt = power.kappa_power(kappa, dth, 8)
    ell_mode = 2 * math.pi * mx / (m * dth)
    b = int(np.floor(8 * math.log(mx) / math.log(m / 2) + 1e-9))
    # two modes (+-mx) of |FFT| = amp M^2 / 2 among cnt[b]: P = 2 (amp M^2 dth^2 / 2)^2 / Theta^2 / cnt
    want = 2 * (amp * m * m * dth * dth / 2) ** 2 / (m * dth) ** 2 / cnt[b]
    assert p[b] == pytest.approx(want, rel=1e-12)
    assert ell[b] > 0 and abs(np.log(ell[b] / ell_mode)) < np.log(m / 2) / 8
    assert np.all(np.delete(p, b) < 1e-30)


def test_power_of_white_noise_is_flat():
    m, dth, sig = 128, 2e-4, 0.1
    acc = 0.0
    for seed in range(6):
        kap = synthetic.gaussian_field(seed, (m, m), sig)
        _, p, cnt = power.kappa_power(kap, dth, 10)
        acc = acc + p
    p = acc / 6
    # E|FFT|^2 = M^2 sigma^2  =>  P = sigma^2 dtheta^2
    ok = cnt > 50
    assert np.allclose(p[ok], sig ** 2 * dth ** 2, rtol=0.15)


def test_bin_edges_put_exact_edge_modes_in_upper_bin():
    # with M/2 = 2^10 and 20 bins the edges fall on |n|^2 = 2^b; those modes open bin b (in double precision the
    # logarithm of the edges of bins 7, 13 and 14 rounds below b)
    m = 2048
    ell, p, cnt = power.kappa_power(np.zeros((m, m)), 1e-4, 20)
    n = np.fft.fftfreq(m, 1.0 / m)
    n2 = (n[:, None] ** 2 + n[None, :] ** 2)
    for b in range(20):
        assert cnt[b] == int(((n2 >= 2 ** b) & (n2 < 2 ** (b + 1))).sum())
