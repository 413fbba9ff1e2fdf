"""Code units of the oracle (test infrastructure only).

Lengths are in Mpc/h and time is measured with H0 = 1, so a velocity unit is H0 * 1 Mpc/h = 100 km/s.
The Poisson equation of Sec. 2 then reads  lap(phi) = (3/2) Omega_m delta / a  with phi in (100 km/s)^2.
"""

C_LIGHT = 299792.458 / 100.0           # speed of light, 100 km/s
G_NEWTON = 4.30091727e-9 / 1.0e4       # (Mpc/h) (100 km/s)^2 / (Msun/h)
