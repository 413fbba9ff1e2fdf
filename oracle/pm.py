"""Particle-mesh gravity in FP64 on the CPU (test infrastructure only).

Restates, step by step and without blocking or fusion, the PM force of Sec. 5.1 of arXiv 2405.12913 ("the
most computationally expensive operation ... calculate grad phi via the FFT") and the particle leapfrog that
``nbody_reverse_step`` of Alg. 1 stands for:

  * mesh nodes sit at j * cell, j = 0..N-1, periodic; arrays are indexed [ix, iy, iz] with iz fastest;
  * CIC (cloud-in-cell, trilinear) deposit: a particle at u = x / cell gives weight (1 - f) to node
    floor(u) and f to node floor(u) + 1 along each axis; each particle carries N_mesh^3 / N_particles, so
    the mesh holds rho / rho_mean = 1 + delta;
  * Poisson (Sec. 2):  lap phi = pref * delta, so phi_k = -pref * delta_k / k^2 with phi_0 = 0;
    pref = (3/2) Omega_m / a in the expanding case and 4 pi G rho_mean in the static point-mass case;
  * gradient: (d_j phi)_k = i k_j phi_k * prod_i sinc(k_i cell / 2)^-p * exp(-k^2 sigma^2 / 2), the CIC
    deconvolution and the Gaussian smoothing of the kick operator of Sec. 5.2 taken on the 3D mesh (power
    p per axis, smoothing length sigma in comoving units, the decaying sign of the Gaussian); the signed
    frequency n_i lies in [-N/2, N/2), k_i = 2 pi n_i / L, and the derivative factor i k_j is set to 0 on
    the j-Nyquist plane so that the gradient is real;
  * the same CIC weights interpolate the three gradient fields back to the particles;
  * leapfrog with one force per step: p <- p - grad phi(x) * K, then x <- x + p * D, with K and D the signed
    time integrals of ``cosmology``; positions are kept as displacements from the Lagrangian lattice;
  * Zel'dovich initial conditions: delta_k = w_k sqrt(P(k) / V_cell), Psi_k = i k delta_k / k^2 (0 on the
    Nyquist planes), x = q + D1 Psi, p = a^2 E f D1 Psi.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import torch

from . import cosmology as cosmo

_CORNERS = list(itertools.product((0, 1), repeat=3))


def lattice(n_side: int, box: float) -> torch.Tensor:
    """Lagrangian lattice q = (i, j, k) * box / n_side, particle index (i*n + j)*n + k; shape (n^3, 3)."""
    g = torch.arange(n_side, dtype=torch.float64) * (box / n_side)
    qx, qy, qz = torch.meshgrid(g, g, g, indexing="ij")
    return torch.stack([qx.reshape(-1), qy.reshape(-1), qz.reshape(-1)], dim=1)


def _cic_parts(x: torch.Tensor, box: float, n_mesh: int):
    """Lower-node indices and fractional offsets of positions x (n, 3), wrapped into the periodic box."""
    cell = box / n_mesh
    u = torch.remainder(x, box) / cell
    i0 = torch.floor(u)
    f = u - i0
    i0 = i0.to(torch.int64) % n_mesh
    return i0, f


def cic_deposit(x: torch.Tensor, box: float, n_mesh: int, mass: float | None = None) -> torch.Tensor:
    """Mesh of rho / rho_mean from particle positions x (n, 3); each particle carries ``mass`` (default
    n_mesh^3 / n so that the mean is 1)."""
    n = x.shape[0]
    if mass is None:
        mass = n_mesh ** 3 / n
    x = x.to(torch.float64)
    i0, f = _cic_parts(x, box, n_mesh)
    rho = torch.zeros(n_mesh ** 3, dtype=torch.float64)
    for a, b, c in _CORNERS:
        w = (f[:, 0] if a else 1 - f[:, 0]) * (f[:, 1] if b else 1 - f[:, 1]) * (f[:, 2] if c else 1 - f[:, 2])
        idx = (((i0[:, 0] + a) % n_mesh) * n_mesh + (i0[:, 1] + b) % n_mesh) * n_mesh + (i0[:, 2] + c) % n_mesh
        rho.index_add_(0, idx, w * mass)
    return rho.reshape(n_mesh, n_mesh, n_mesh)


def signed_freq(n: int) -> torch.Tensor:
    """Signed integer frequencies of a length-n FFT axis, in [-n/2, n/2)."""
    return torch.fft.fftfreq(n, d=1.0 / n).round().to(torch.int64)


def _wavevectors(n_mesh: int, box: float):
    """Integer frequencies (nx, ny, nz) of the rfftn half spectrum, broadcastable, z axis non-negative.

    The z axis of rfftn keeps n_z = 0..N/2; n_z = N/2 is the Nyquist frequency and counts as -N/2 (its
    sinc factor is the same and its derivative factor is zero)."""
    nx = signed_freq(n_mesh).view(-1, 1, 1)
    ny = signed_freq(n_mesh).view(1, -1, 1)
    nz = torch.arange(n_mesh // 2 + 1, dtype=torch.int64).view(1, 1, -1)
    return nx, ny, nz


def sinc(x: torch.Tensor) -> torch.Tensor:
    """sin(x) / x with sinc(0) = 1."""
    safe = torch.where(x == 0, torch.ones_like(x), x)
    return torch.where(x == 0, torch.ones_like(x), torch.sin(safe) / safe)


def gradient_multipliers(nx: torch.Tensor, ny: torch.Tensor, nz: torch.Tensor, n_mesh: int, box: float, pref: float,
                         deconv_p: float, smooth: float = 0.0, g_of_k=None) -> list[torch.Tensor]:
    """The factors that map the density spectrum to the spectra of (d_x phi, d_y phi, d_z phi) at integer
    wavevectors (nx, ny, nz) (signed tensors, broadcastable; Sec. 2 Poisson equation):
    i d_j(k) G(k) W(k) [g(|k|)], with G = -pref / k^2 (0 at k = 0), the per-axis deconvolution
    W = prod_i sinc(k_i cell / 2)^(-p) times exp(-k^2 smooth^2 / 2), and d_j = k_j except 0 on a Nyquist plane
    |n_j| = n_mesh / 2 (a real output)."""
    cell = box / n_mesh
    kf = 2.0 * math.pi / box
    kx, ky, kz = kf * nx.double(), kf * ny.double(), kf * nz.double()
    k2 = kx * kx + ky * ky + kz * kz
    green = torch.where(k2 > 0, -pref / torch.where(k2 > 0, k2, torch.ones_like(k2)), torch.zeros_like(k2))
    window = (sinc(kx * cell / 2) * sinc(ky * cell / 2) * sinc(kz * cell / 2)) ** (-deconv_p)
    if smooth > 0.0:
        window = window * torch.exp(-0.5 * k2 * smooth * smooth)
    phi = green * window
    if g_of_k is not None:
        phi = phi * g_of_k(torch.sqrt(k2))
    half = n_mesh // 2
    out = []
    for kj, nj in ((kx, nx), (ky, ny), (kz, nz)):
        d = torch.where(nj.abs() == half, torch.zeros_like(kj), kj)
        out.append(phi * (1j * d))
    return out


def poisson_gradient_hat(rho_hat: torch.Tensor, box: float, pref: float, deconv_p: float,
                         smooth: float = 0.0, g_of_k=None) -> list[torch.Tensor]:
    """Three gradient spectra (d_x phi, d_y phi, d_z phi) from the half spectrum of rho (any k = 0 value).

    ``smooth`` is the Gaussian smoothing length in Mpc/h (0 = none).  ``g_of_k``, if given, is a callable
    on |k| (tensor) returning a multiplicative correction of the Green's function (the learned force
    correction of the ray fields)."""
    n_mesh = rho_hat.shape[0]
    nx, ny, nz = _wavevectors(n_mesh, box)
    return [rho_hat * m for m in gradient_multipliers(nx, ny, nz, n_mesh, box, pref, deconv_p, smooth, g_of_k)]


def mode_gradient(modes: np.ndarray, amp: np.ndarray, phase: np.ndarray, flat_idx: np.ndarray, n_mesh: int,
                  box: float, pref: float, deconv_p: float, smooth: float = 0.0) -> list[np.ndarray]:
    """The gradient fields of poisson_gradient at single mesh nodes, for a density made of cosine modes
    rho = const + sum_m a_m cos(2 pi (m . x) / n + phi_m) with no Nyquist component: each mode's spectrum sits
    at +m and -m, where the multipliers are complex conjugates, so its gradient at node x is
    Re(a_m M_j(m) exp(i (2 pi (m . x) / n + phi_m))).  Nodes are flat indices (i n + j) n + k; returns
    [d_x phi, d_y phi, d_z phi] at them (float64)."""
    m = torch.as_tensor(np.asarray(modes, dtype=np.int64))
    mult = gradient_multipliers(m[:, 0], m[:, 1], m[:, 2], n_mesh, box, pref, deconv_p, smooth)
    idx = np.asarray(flat_idx, dtype=np.int64)
    i, j, k = idx // (n_mesh * n_mesh), (idx // n_mesh) % n_mesh, idx % n_mesh
    t = (np.outer(i, m[:, 0].numpy()) + np.outer(j, m[:, 1].numpy()) + np.outer(k, m[:, 2].numpy())) % n_mesh
    e = np.exp(1j * (2.0 * math.pi * t / n_mesh + np.asarray(phase)[None, :]))
    return [np.real(e @ (np.asarray(amp) * mj.numpy())) for mj in mult]


def poisson_gradient(rho: torch.Tensor, box: float, pref: float, deconv_p: float, smooth: float = 0.0,
                     g_of_k=None):
    """Real gradient fields [d_x phi, d_y phi, d_z phi] on the mesh from rho / rho_mean."""
    n_mesh = rho.shape[0]
    rho_hat = torch.fft.rfftn(rho)
    spectra = poisson_gradient_hat(rho_hat, box, pref, deconv_p, smooth, g_of_k)
    return [torch.fft.irfftn(s, s=(n_mesh,) * 3) for s in spectra]


def cic_gather(fields, x: torch.Tensor, box: float) -> torch.Tensor:
    """CIC (trilinear) interpolation of each field at positions x (n, 3); returns (n, n_fields)."""
    n_mesh = fields[0].shape[0]
    i0, f = _cic_parts(x, box, n_mesh)
    out = torch.zeros(x.shape[0], len(fields), dtype=torch.float64)
    flat = [fl.reshape(-1) for fl in fields]
    for a, b, c in _CORNERS:
        w = (f[:, 0] if a else 1 - f[:, 0]) * (f[:, 1] if b else 1 - f[:, 1]) * (f[:, 2] if c else 1 - f[:, 2])
        idx = (((i0[:, 0] + a) % n_mesh) * n_mesh + (i0[:, 1] + b) % n_mesh) * n_mesh + (i0[:, 2] + c) % n_mesh
        for j, fl in enumerate(flat):
            out[:, j] += w * fl[idx]
    return out


def particle_kick_drift(disp: torch.Tensor, mom: torch.Tensor, q: torch.Tensor, grads, box: float,
                        kick: float, drift: float):
    """One fused leapfrog update: p <- p - grad phi(q + disp) * kick; disp <- disp + p * drift."""
    g = cic_gather(grads, q + disp, box)
    mom = mom - g * kick
    disp = disp + mom * drift
    return disp, mom


def zeldovich(noise: np.ndarray, box: float, om: float, h: float, ns: float, sigma8: float, a_init: float):
    """Zel'dovich displacement and momentum of the lattice particles at a_init from white noise (n,n,n).

    Returns (disp, mom) as (n^3, 3) float64 tensors."""
    n = noise.shape[0]
    amp = cosmo.power_amplitude(om, h, ns, sigma8)
    v_cell = (box / n) ** 3
    w_hat = torch.fft.rfftn(torch.as_tensor(noise, dtype=torch.float64))
    kf = 2.0 * math.pi / box
    nx, ny, nz = _wavevectors(n, box)
    kx, ky, kz = kf * nx.double(), kf * ny.double(), kf * nz.double()
    k2 = kx * kx + ky * ky + kz * kz
    kmag = torch.sqrt(k2)
    pk = torch.as_tensor(cosmo.linear_power(kmag.numpy(), om, h, ns, amp))
    delta_hat = w_hat * torch.sqrt(pk / v_cell)
    delta_hat = torch.where(k2 > 0, delta_hat, torch.zeros_like(delta_hat))
    inv_k2 = torch.where(k2 > 0, 1.0 / torch.where(k2 > 0, k2, torch.ones_like(k2)), torch.zeros_like(k2))
    half = n // 2
    psi = []
    for kj, nj, last in ((kx, nx, False), (ky, ny, False), (kz, nz, True)):
        nyq = (nj == half) if last else (nj == -half)
        d = torch.where(nyq, torch.zeros_like(kj), kj)
        psi.append(torch.fft.irfftn(1j * d * inv_k2 * delta_hat, s=(n, n, n)).reshape(-1))
    psi = torch.stack(psi, dim=1)
    d1 = cosmo.growth_D1(a_init, om)
    f1 = cosmo.growth_f(a_init, om)
    e1 = cosmo.E(a_init, om)
    return d1 * psi, (a_init ** 2 * e1 * f1 * d1) * psi


def _derivative_factors(n: int, box: float):
    """k_j with the derivative of the j-Nyquist plane set to zero (as for the first-order displacement), and k^2."""
    kf = 2.0 * math.pi / box
    nx, ny, nz = _wavevectors(n, box)
    half = n // 2
    d = []
    for nj, last in ((nx, False), (ny, False), (nz, True)):
        nyq = (nj == half) if last else (nj == -half)
        d.append(torch.where(nyq, torch.zeros_like(nj), nj).double() * kf)
    k2 = (kf * nx.double()) ** 2 + (kf * ny.double()) ** 2 + (kf * nz.double()) ** 2
    return d, k2


def lpt_fields(delta: torch.Tensor, box: float):
    """First- and second-order Lagrangian displacement fields at unit growth from a real density contrast
    delta (n, n, n) on the particle lattice (2LPT):

      Psi1 = -grad phi1,  lap phi1 = delta;
      Psi2 = grad phi2,   lap phi2 = sum_{i<j} (phi1_ii phi1_jj - phi1_ij^2),

    so that x = q + D1 Psi1 + D2 Psi2 with D2 < 0.  Derivatives are spectral; the derivative factor of a
    Nyquist plane is zero (second derivatives are products of two first-derivative factors).

    Returns (psi1, psi2) as (n^3, 3) float64 tensors."""
    n = delta.shape[0]
    d, k2 = _derivative_factors(n, box)
    inv_k2 = torch.where(k2 > 0, 1.0 / torch.where(k2 > 0, k2, torch.ones_like(k2)), torch.zeros_like(k2))
    delta_hat = torch.fft.rfftn(torch.as_tensor(delta, dtype=torch.float64))
    phi1_hat = -delta_hat * inv_k2
    psi1 = torch.stack([torch.fft.irfftn(-1j * d[j] * phi1_hat, s=(n, n, n)).reshape(-1) for j in range(3)], 1)
    # phi1_ij = F^-1[(i d_i)(i d_j) phi1_hat]
    hess = {(i, j): torch.fft.irfftn(-d[i] * d[j] * phi1_hat, s=(n, n, n)) for i in range(3) for j in range(i, 3)}
    src = torch.zeros((n, n, n), dtype=torch.float64)
    for i in range(3):
        for j in range(i + 1, 3):
            src = src + hess[(i, i)] * hess[(j, j)] - hess[(i, j)] ** 2
    phi2_hat = -torch.fft.rfftn(src) * inv_k2
    psi2 = torch.stack([torch.fft.irfftn(1j * d[j] * phi2_hat, s=(n, n, n)).reshape(-1) for j in range(3)], 1)
    return psi1, psi2


def lpt2(noise: np.ndarray, box: float, om: float, h: float, ns: float, sigma8: float, a_init: float):
    """Second-order Lagrangian (2LPT) displacement and momentum of the lattice particles at a_init from white noise
    (n,n,n): x = q + D1 Psi1 + D2 Psi2, p = a^2 E (f1 D1 Psi1 + f2 D2 Psi2), with the linear density of
    ``zeldovich`` and D2 = -(3/7) D1^2 Omega_m(a)^(-1/143), f2 = 2 Omega_m(a)^(6/11).

    Returns (disp, mom) as (n^3, 3) float64 tensors."""
    n = noise.shape[0]
    amp = cosmo.power_amplitude(om, h, ns, sigma8)
    v_cell = (box / n) ** 3
    w_hat = torch.fft.rfftn(torch.as_tensor(noise, dtype=torch.float64))
    _, k2 = _derivative_factors(n, box)
    pk = torch.as_tensor(cosmo.linear_power(torch.sqrt(k2).numpy(), om, h, ns, amp))
    delta_hat = torch.where(k2 > 0, w_hat * torch.sqrt(pk / v_cell), torch.zeros_like(w_hat))
    psi1, psi2 = lpt_fields(torch.fft.irfftn(delta_hat, s=(n, n, n)), box)
    d1 = cosmo.growth_D1(a_init, om)
    f1 = cosmo.growth_f(a_init, om)
    e = cosmo.E(a_init, om)
    om_a = om / (a_init ** 3 * e * e)
    d2 = -3.0 / 7.0 * d1 * d1 * om_a ** (-1.0 / 143.0)
    f2 = 2.0 * om_a ** (6.0 / 11.0)
    disp = d1 * psi1 + d2 * psi2
    mom = a_init ** 2 * e * (f1 * d1 * psi1 + f2 * d2 * psi2)
    return disp, mom


def matter_power(rho: torch.Tensor, box: float, nbins: int):
    """Spherically averaged power of delta = rho - 1 in linear k bins of width k_f (test utility).

    Returns (k_mean, P) over bins 1..nbins of |n| (integer shells [b, b+1))."""
    n = rho.shape[0]
    d_hat = torch.fft.fftn(rho - rho.mean())
    p = (d_hat.abs() ** 2) * (box ** 3) / n ** 6
    f = signed_freq(n).double()
    nn = torch.sqrt(f.view(-1, 1, 1) ** 2 + f.view(1, -1, 1) ** 2 + f.view(1, 1, -1) ** 2)
    b = torch.floor(nn).to(torch.int64)
    kf = 2.0 * math.pi / box
    ks, ps = [], []
    for i in range(1, nbins + 1):
        m = b == i
        ks.append(float(nn[m].mean()) * kf)
        ps.append(float(p[m].mean()))
    return np.array(ks), np.array(ps)
