// FP64 host cosmology of the HRT library: flat LCDM background, linear growth, particle time integrals and
// the per-step ray node tables.  Sec. 2 (Poisson equation, r = chi) and Sec. 3.2 (growth time correction,
// Eq. "kick") of arXiv 2405.12913.  Host only.
#pragma once

#include <cstdint>
#include <vector>

namespace hrt {

constexpr double kCLight = 2997.92458;       // 100 km/s
constexpr double kGNewton = 4.30091727e-13;  // (Mpc/h) (100 km/s)^2 / (Msun/h)

struct Cosmo {
  double om;
  explicit Cosmo(double omega_m) : om(omega_m) {}
  double E(double a) const;
  double chi(double a) const;        // comoving distance of the light front at a
  double a_of_chi(double chi) const;
  double D1(double a) const;         // normalised to 1 at a = 1
  double f(double a) const;          // dln D1 / dln a
  double kick(double a, double b) const;   // int_a^b da / (a E)
  double drift(double a, double b) const;  // int_a^b da / (a^3 E)
 private:
  double growth_integral(double a) const;  // int_0^a da / (a E)^3
};

double power_amplitude(double om, double h, double ns, double sigma8);
double bbks_transfer(double q);

// Midpoint nodes of one half shell: n = max(1, ceil(s |b - a| / cell)), node j at a + (j + 1/2) h.
int half_shell_count(double chi_a, double chi_b, double samples_per_cell, double cell);

}  // namespace hrt
