// FP64 host cosmology, see cosmo.h.  Every integral is a composite Gauss-Legendre rule after the substitution
// a = u^2, which turns the integrands of flat LCDM (no radiation) into smooth functions of u:
//   chi(a)   = c int_{sqrt a}^1 2 du / S(u)
//   I(a)     = int_0^a da/(a E)^3 = int_0^{sqrt a} 2 u^4 du / S(u)^3
//   K(a->b)  = int da/(a E)       = int 2 u^2 du / S(u)
//   Dr(a->b) = int da/(a^3 E)     = int 2 du / (u^2 S(u))
// with S(u) = sqrt(Om + (1 - Om) u^6) = u^3 E(u^2).
#include "cosmo.h"

#include <cmath>
#include <mutex>

namespace hrt {
namespace {

constexpr int kGL = 24;  // nodes per panel

struct GaussLegendre {
  double x[kGL], w[kGL];
  GaussLegendre() {
    // Newton iteration on P_n(x) from the asymptotic guess cos(pi (i + 3/4) / (n + 1/2)).
    const int n = kGL;
    for (int i = 0; i < n; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
      double dp = 0.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

const GaussLegendre& gl() {
  static const GaussLegendre rule;
  return rule;
}

// Composite rule on [lo, hi] with panels no wider than max_panel.
template <class F>
double integrate(F&& fn, double lo, double hi, double max_panel) {
  if (lo == hi) return 0.0;
  const GaussLegendre& r = gl();
  double span = hi - lo;
  int panels = static_cast<int>(std::ceil(std::fabs(span) / max_panel));
  if (panels < 1) panels = 1;
  double hp = span / panels, sum = 0.0;
  for (int p = 0; p < panels; ++p) {
    double c = lo + (p + 0.5) * hp, s = 0.0;
    for (int i = 0; i < kGL; ++i) s += r.w[i] * fn(c + 0.5 * hp * r.x[i]);
    sum += 0.5 * hp * s;
  }
  return sum;
}

}  // namespace

double Cosmo::E(double a) const { return std::sqrt(om / (a * a * a) + (1.0 - om)); }

static inline double S(double om, double u) {
  double u3 = u * u * u;
  return std::sqrt(om + (1.0 - om) * u3 * u3);
}

double Cosmo::chi(double a) const {
  const double o = om;
  return kCLight * integrate([o](double u) { return 2.0 / S(o, u); }, std::sqrt(a), 1.0, 0.02);
}

double Cosmo::a_of_chi(double chi_target) const {
  if (chi_target <= 0.0) return 1.0;
  // Newton on chi(a) - chi_target with dchi/da = -c / (a^2 E), started from the Einstein-de Sitter guess.
  double a = 1.0 - chi_target / (2.0 * kCLight);
  a = a > 0.05 ? a * a : 0.05;
  for (int it = 0; it < 60; ++it) {
    double g = chi(a) - chi_target;
    double d = -kCLight / (a * a * E(a));
    double step = g / d;
    double an = a - step;
    if (an <= 0.0) an = 0.5 * a;
    if (an > 1.0) an = 0.5 * (a + 1.0);
    if (std::fabs(an - a) < 1e-16 * a) {
      a = an;
      break;
    }
    a = an;
  }
  return a;
}

double Cosmo::growth_integral(double a) const {
  const double o = om;
  return integrate([o](double u) { double s = S(o, u); return 2.0 * u * u * u * u / (s * s * s); }, 0.0,
                   std::sqrt(a), 0.02);
}

double Cosmo::D1(double a) const { return E(a) * growth_integral(a) / (E(1.0) * growth_integral(1.0)); }

double Cosmo::f(double a) const {
  double e = E(a);
  return -1.5 * om / (a * a * a * e * e) + 1.0 / (a * a * e * e * e * growth_integral(a));
}

double Cosmo::kick(double a, double b) const {
  const double o = om;
  return integrate([o](double u) { return 2.0 * u * u / S(o, u); }, std::sqrt(a), std::sqrt(b), 0.02);
}

double Cosmo::drift(double a, double b) const {
  const double o = om;
  return integrate([o](double u) { return 2.0 / (u * u * S(o, u)); }, std::sqrt(a), std::sqrt(b), 0.005);
}

double bbks_transfer(double q) {
  if (q <= 0.0) return 1.0;
  double x = 2.34 * q;
  double poly = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) + std::pow(6.71 * q, 4);
  return std::log1p(x) / x * std::pow(poly, -0.25);
}

double power_amplitude(double om, double h, double ns, double sigma8) {
  // sigma^2(R) = int dlnk k^3 P(k) W(kR)^2 / (2 pi^2), top hat W(x) = 3 (sin x - x cos x) / x^3, R = 8.
  auto integrand = [&](double lnk) {
    double k = std::exp(lnk);
    double x = 8.0 * k;
    double w = x < 1e-3 ? 1.0 - x * x / 10.0 : 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
    double t = bbks_transfer(k / (om * h));
    return k * k * k * std::pow(k, ns) * t * t * w * w / (2.0 * M_PI * M_PI);
  };
  double s2 = integrate(integrand, std::log(1e-6), std::log(1e3), 0.01);
  return sigma8 * sigma8 / s2;
}

int half_shell_count(double chi_a, double chi_b, double samples_per_cell, double cell) {
  double n = std::ceil(samples_per_cell * std::fabs(chi_b - chi_a) / cell);
  return n < 1.0 ? 1 : static_cast<int>(n);
}

}  // namespace hrt
