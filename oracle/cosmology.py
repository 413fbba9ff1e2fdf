"""Flat LCDM background, linear growth and time integrals in FP64 (test infrastructure only).

Follows Sec. 2 of arXiv 2405.12913 (Poisson equation with the (3/2) Omega_m H0^2 / a prefactor, r = chi in a
flat universe) and the growth-based time correction of Sec. 3.2 (Eq. "kick": phi(tau) = phi(tau_c)
D1(tau)/D1(tau_c) a(tau_c)/a(tau)).  Radiation is neglected and Omega_Lambda = 1 - Omega_m.

Every quantity is a direct quadrature with ``scipy.integrate.quad``:
  E(a)      = sqrt(Omega_m a^-3 + Omega_Lambda)
  chi(a)    = c * int_a^1 da' / (a'^2 E(a'))
  D1(a)     ∝ E(a) * int_0^a da' / (a' E(a'))^3,  normalised to D1(1) = 1
  f(a)      = dln D1 / dln a  (analytic derivative of the line above)
  K(a->b)   = int_a^b da / (a E)      particle kick time integral (p = a^2 dx/dt, dp/dt = -grad phi)
  Dr(a->b)  = int_a^b da / (a^3 E)    particle drift time integral
  P(k)      = A k^n_s T_BBKS(k / (Omega_m h))^2 with A set by sigma8 (top hat of radius 8 Mpc/h)
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

from .units import C_LIGHT

_QUAD = dict(epsabs=0.0, epsrel=1e-13, limit=400)


def E(a: float, om: float) -> float:
    """Dimensionless Hubble rate H(a)/H0 of flat LCDM."""
    return math.sqrt(om / a ** 3 + (1.0 - om))


def chi_of_a(a: float, om: float) -> float:
    """Comoving radial distance from the observer (a = 1) to the light front at scale factor a, Mpc/h."""
    if a == 1.0:
        return 0.0
    val, _ = integrate.quad(lambda x: 1.0 / (x * x * E(x, om)), a, 1.0, **_QUAD)
    return C_LIGHT * val


def a_of_chi(chi: float, om: float) -> float:
    """Inverse of ``chi_of_a`` by Brent's method on the FP64 quadrature."""
    if chi == 0.0:
        return 1.0
    return optimize.brentq(lambda a: chi_of_a(a, om) - chi, 1e-4, 1.0, xtol=1e-15, rtol=1e-15, maxiter=200)


def _growth_integral(a: float, om: float) -> float:
    val, _ = integrate.quad(lambda x: 1.0 / (x * E(x, om)) ** 3, 0.0, a, **_QUAD)
    return val


def growth_D1(a: float, om: float) -> float:
    """Linear growth factor normalised to 1 at a = 1."""
    return (E(a, om) * _growth_integral(a, om)) / (E(1.0, om) * _growth_integral(1.0, om))


def growth_f(a: float, om: float) -> float:
    """Growth rate f = dln D1/dln a = a E'/E + 1 / (a^2 E^3 I(a)), I the growth integral."""
    e = E(a, om)
    return -1.5 * om / (a ** 3 * e * e) + 1.0 / (a * a * e ** 3 * _growth_integral(a, om))


def kick_integral(a: float, b: float, om: float) -> float:
    """Signed particle kick factor int_a^b da / (a E(a))."""
    if a == b:
        return 0.0
    val, _ = integrate.quad(lambda x: 1.0 / (x * E(x, om)), a, b, **_QUAD)
    return val


def drift_integral(a: float, b: float, om: float) -> float:
    """Signed particle drift factor int_a^b da / (a^3 E(a))."""
    if a == b:
        return 0.0
    val, _ = integrate.quad(lambda x: 1.0 / (x ** 3 * E(x, om)), a, b, **_QUAD)
    return val


def bbks_transfer(q):
    """BBKS transfer function of the shape variable q = k / (Omega_m h) (k in h/Mpc); scalar or array."""
    q = np.asarray(q, dtype=np.float64)
    x = 2.34 * np.where(q > 0.0, q, 1.0)
    t = np.log1p(x) / x * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25
    return np.where(q > 0.0, t, 1.0)


def tophat_window(x: float) -> float:
    """Fourier transform of a unit-volume spherical top hat, 3 (sin x - x cos x) / x^3."""
    if x < 1e-4:
        return 1.0 - x * x / 10.0
    return 3.0 * (math.sin(x) - x * math.cos(x)) / x ** 3


def power_shape(k, om: float, h: float, ns: float):
    """Unnormalised linear power k^n_s T(k)^2; scalar or array."""
    k = np.asarray(k, dtype=np.float64)
    return k ** ns * bbks_transfer(k / (om * h)) ** 2


def power_amplitude(om: float, h: float, ns: float, sigma8: float) -> float:
    """Amplitude A with sigma(R = 8 Mpc/h) = sigma8 at a = 1: sigma^2 = int dk k^2 P W^2 / (2 pi^2)."""
    def integrand(lnk):
        k = math.exp(lnk)
        return k ** 3 * float(power_shape(k, om, h, ns)) * tophat_window(8.0 * k) ** 2 / (2.0 * math.pi ** 2)
    s2, _ = integrate.quad(integrand, math.log(1e-6), math.log(1e3), epsabs=0.0, epsrel=1e-12, limit=2000)
    return sigma8 ** 2 / s2


def linear_power(k, om: float, h: float, ns: float, amp: float):
    """Linear matter power spectrum at a = 1, (Mpc/h)^3; scalar or array, 0 at k = 0."""
    k = np.asarray(k, dtype=np.float64)
    return np.where(k > 0.0, amp * power_shape(np.where(k > 0.0, k, 1.0), om, h, ns), 0.0)
