"""Pins of the oracle's background cosmology against closed forms and independent integrators."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import cosmology as cosmo
from oracle import sim
from oracle.units import C_LIGHT


@pytest.mark.parametrize("a", [0.02, 0.3, 0.5, 0.9])
def test_einstein_de_sitter_closed_forms(a):
    # Omega_m = 1: E = a^-3/2, chi = 2c(1 - sqrt a), D1 = a, f = 1,
    # K(a->b) = (2/3)(b^3/2 - a^3/2), Dr(a->b) = 2(a^-1/2 - b^-1/2).
    om = 1.0
    assert cosmo.E(a, om) == pytest.approx(a ** -1.5, rel=1e-14)
    assert cosmo.chi_of_a(a, om) == pytest.approx(2 * C_LIGHT * (1 - math.sqrt(a)), rel=1e-12)
    assert cosmo.growth_D1(a, om) == pytest.approx(a, rel=1e-12)
    assert cosmo.growth_f(a, om) == pytest.approx(1.0, rel=1e-11)
    b = 0.5 * (a + 1.0)
    assert cosmo.kick_integral(a, b, om) == pytest.approx(2 / 3 * (b ** 1.5 - a ** 1.5), rel=1e-12)
    assert cosmo.drift_integral(a, b, om) == pytest.approx(2 * (a ** -0.5 - b ** -0.5), rel=1e-12)
    # signed: reversing the limits flips the sign
    assert cosmo.kick_integral(b, a, om) == pytest.approx(-cosmo.kick_integral(a, b, om), rel=1e-13)


def _growth_ode(om):
    """D(a) / D(1) of the linear growth ODE in a: D'' + (3/a + E'/E) D' - 1.5 Om / (a^5 E^2) D = 0, growing mode
    D ~ a early."""
    def E(a):
        return math.sqrt(om / a ** 3 + 1 - om)

    def rhs(a, y):
        d, dp = y
        e = E(a)
        de = -1.5 * om / (a ** 4 * e)
        return [dp, -(3.0 / a + de / e) * dp + 1.5 * om / (a ** 5 * e * e) * d]

    a0 = 1e-3
    sol = integrate.solve_ivp(rhs, (a0, 1.0), [a0, 1.0], rtol=1e-12, atol=1e-15, dense_output=True)
    d1 = sol.sol(1.0)[0]
    return lambda a: sol.sol(a)[0] / d1


def test_growth_against_ode():
    om = 0.3
    d_ode = _growth_ode(om)
    for a in (0.05, 0.3, 0.6):
        assert cosmo.growth_D1(a, om) == pytest.approx(d_ode(a), rel=2e-6)


def test_growth_weight_of_the_ray_kick():
    # the time correction of the ray kick follows the linear potential, phi ∝ D1 / a (Sec. 3.2): constant in
    # Einstein-de Sitter (D1 = a), 1 at the reference time, and in LCDM the ratio of D1 / a from the growth ODE
    # (the potential decays, so it exceeds 1 at earlier times, farther out)
    g = sim.growth_weight(0.4, 1.0)
    for chi in (50.0, 800.0, 2500.0):
        assert g(chi) == pytest.approx(1.0, rel=1e-10)
    om, a_c = 0.3, 0.6
    g = sim.growth_weight(a_c, om)
    assert g(cosmo.chi_of_a(a_c, om)) == pytest.approx(1.0, rel=1e-12)
    d_ode = _growth_ode(om)
    for a in (0.2, 0.45, 0.8, 0.95):
        want = (d_ode(a) / a) / (d_ode(a_c) / a_c)
        assert g(cosmo.chi_of_a(a, om)) == pytest.approx(want, rel=1e-5)
        assert (want > 1.0) == (a < a_c)


def test_growth_rate_matches_finite_difference():
    om = 0.3
    for a in (0.1, 0.5, 1.0):
        h = 1e-5
        fd = (math.log(cosmo.growth_D1(a * math.exp(h), om)) - math.log(cosmo.growth_D1(a * math.exp(-h), om))) / (2 * h)
        assert cosmo.growth_f(a, om) == pytest.approx(fd, rel=1e-7)


def test_a_of_chi_inverts_chi():
    om = 0.3
    for chi in (10.0, 1000.0, 3600.0):
        assert cosmo.chi_of_a(cosmo.a_of_chi(chi, om), om) == pytest.approx(chi, rel=1e-12)


def test_sigma8_normalisation_independent_quadrature():
    om, h, ns, s8 = 0.3, 0.7, 0.96, 0.8
    amp = cosmo.power_amplitude(om, h, ns, s8)
    lnk = np.linspace(math.log(1e-5), math.log(2e2), 400001)
    k = np.exp(lnk)
    x = 8.0 * k
    w = 3 * (np.sin(x) - x * np.cos(x)) / x ** 3
    pk = cosmo.linear_power(k, om, h, ns, amp)
    s2 = np.trapezoid(k ** 3 * pk * w * w / (2 * math.pi ** 2), lnk)
    assert math.sqrt(s2) == pytest.approx(s8, rel=1e-6)


def test_bbks_limits():
    assert float(cosmo.bbks_transfer(0.0)) == 1.0
    assert float(cosmo.bbks_transfer(1e-6)) == pytest.approx(1.0, abs=1e-5)
    # large-q tail falls as ln(q)/q^2
    t1, t2 = float(cosmo.bbks_transfer(1e3)), float(cosmo.bbks_transfer(2e3))
    assert t2 / t1 == pytest.approx(0.25 * math.log1p(4680) / math.log1p(2340), rel=2e-3)
