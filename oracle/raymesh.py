"""The paper's kick operator on a 2D ray mesh (Sec. 5.2, Sec. 5.3, App. C) in FP64 on the CPU (test
infrastructure only): an alternative to the direct line-of-sight gather of ``rays.half_kick``.

For a half shell [chi_a, chi_b) (either orientation):

  * the angular resolution limit lam = max(2 cell / (r_a + r_b), mu) (Eq. "reslim"), the ray-mesh spacing
    x2d = iota lam and its size N, the smallest power of two >= ceil(M mu / x2d + p_min / iota) (App. C); the ray
    mesh is N x N nodes at angles (i - N/2) x2d, centred on the field;
  * every 3D mesh node X with chi_a <= X_z - O_z < chi_b (and its transverse periodic images that land on the ray
    mesh) is projected to the angle theta = (X_xy - O_xy) / chi and carries the kick integrand of Eq. "kick",
    -(2/c) r g(chi) grad_perp phi(X), times its line-of-sight extent (cell, signed with the orientation of the
    shell) and its solid angle cell^2 / r^2 over the ray-mesh cell's x2d^2; the values are deposited with 2D CIC
    weights (nodes outside the mesh are dropped);
  * 2D FFT, deconvolution sinc(k_x x2d / 2)^-4 sinc(k_y x2d / 2)^-4 and Gaussian smoothing exp(-k^2 lam^2 / 2),
    inverse FFT;
  * the kick at a ray is the bilinear interpolation of the mesh at its angle, and dK/dtheta the derivative of
    that interpolant (on a cell face the lower cell is used).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .units import C_LIGHT


def geometry(chi_a: float, chi_b: float, cell: float, mu: float, m_pix: int, iota: float, p_min: float):
    """(lam, x2d, N) of the ray mesh of the half shell [chi_a, chi_b)."""
    lam = max(2.0 * cell / (abs(chi_a) + abs(chi_b)), mu)
    x2d = iota * lam
    need = math.ceil(m_pix * mu / x2d + p_min / iota)
    n2d = 1
    while n2d < need:
        n2d *= 2
    return lam, x2d, n2d


def shell_planes(chi_a: float, chi_b: float, cell: float, observer_z: float):
    """(kz, chi) of the node planes z = kz cell with min <= chi = z - O_z < max of the half shell, chi > 0."""
    lo, hi = min(chi_a, chi_b), max(chi_a, chi_b)
    out = []
    for kz in range(math.ceil((observer_z + lo) / cell) - 1, math.ceil((observer_z + hi) / cell) + 1):
        chi = kz * cell - observer_z
        if lo <= chi < hi and chi > 0:
            out.append((kz, chi))
    return out


def plane_fields(g3, kz: int, replicas):
    """Sky-frame transverse gradient (g_x, g_y) on the node plane of sky index kz (>= 0) of a light cone tiled by
    replicas (perm, sign, shift): the plane lies in replica k = kz // n, whose sky axis a maps to box axis
    perm[k, a] at node (sign[k, a] i_a + shift[k, perm[k, a]]) mod n; the sky components are
    sign[k, a] g_{perm[k, a]} there (the tiling of ``rays.replica_frame`` restricted to mesh nodes)."""
    n = g3[0].shape[0]
    perm, sign, shift = (np.asarray(t) for t in replicas)
    k = kz // n
    if kz < 0 or k >= perm.shape[0]:
        raise ValueError("a node plane lies outside the replicas")
    p, sg, sh = perm[k], sign[k], shift[k]
    ii = np.arange(n)
    b = [None, None, None]
    b[p[0]] = ((sg[0] * ii + sh[p[0]]) % n)[:, None]
    b[p[1]] = ((sg[1] * ii + sh[p[1]]) % n)[None, :]
    b[p[2]] = (sg[2] * (kz % n) + sh[p[2]]) % n
    g = [x.numpy() if torch.is_tensor(x) else x for x in g3]
    return sg[0] * g[p[0]][b[0], b[1], b[2]], sg[1] * g[p[1]][b[0], b[1], b[2]]


def mesh_kick(gx: torch.Tensor, gy: torch.Tensor, box: float, observer, chi_a: float, chi_b: float, weight_fn,
              mu: float, m_pix: int, iota: float, p_min: float, filtered: bool = True, window=None, gz=None,
              replicas=None):
    """The filtered kick of the half shell on its ray mesh: returns (K (2, N, N) float64 tensor, x2d, N), with
    K[c, i, j] the component c at the angle ((i - N/2) x2d, (j - N/2) x2d).  ``filtered=False`` returns the CIC
    deposit before the deconvolution and smoothing; planes outside ``window = (chi_lo, chi_hi)`` do not
    contribute.  With ``replicas`` = (perm, sign, shift) the light cone is tiled by rotated, translated box
    replicas (``plane_fields``, which needs the third field gz)."""
    n = gx.shape[0]
    cell = box / n
    lam, x2d, n2d = geometry(chi_a, chi_b, cell, mu, m_pix, iota, p_min)
    sgn = 1.0 if chi_b >= chi_a else -1.0
    mesh = np.zeros((2, n2d, n2d))
    half_extent = 0.5 * n2d * x2d
    # any n^3 array-like whose z planes [:, :, iz] can be read serves (only the shell's planes are read)
    gxn = gx.numpy() if torch.is_tensor(gx) else gx
    gyn = gy.numpy() if torch.is_tensor(gy) else gy
    idx = np.arange(n) * cell
    for kz, chi in shell_planes(chi_a, chi_b, cell, observer[2]):
        if window is not None and not (window[0] <= chi < window[1]):
            continue
        r = chi
        w = -(2.0 / C_LIGHT) * r * weight_fn(chi) * sgn * cell * cell * cell / (r * r * x2d * x2d)
        if replicas is None:
            iz = kz % n
            vx = gxn[:, :, iz] * w
            vy = gyn[:, :, iz] * w
        else:
            px, py = plane_fields((gx, gy, gz), kz, replicas)
            vx, vy = px * w, py * w
        # transverse images that can land on the mesh
        reach = (half_extent + x2d) * r + cell
        a0 = math.floor((observer[0] - reach) / box)
        a1 = math.floor((observer[0] + reach) / box)
        b0 = math.floor((observer[1] - reach) / box)
        b1 = math.floor((observer[1] + reach) / box)
        flat, wx_all, wy_all = [], [], []
        for ia in range(a0, a1 + 1):
            ux = ((idx + ia * box - observer[0]) / r) / x2d + n2d / 2
            selx = np.flatnonzero((ux > -1) & (ux < n2d))     # node columns whose CIC weights reach the mesh
            for ib in range(b0, b1 + 1):
                uy = ((idx + ib * box - observer[1]) / r) / x2d + n2d / 2
                sely = np.flatnonzero((uy > -1) & (uy < n2d))
                if selx.size == 0 or sely.size == 0:
                    continue
                ix = np.floor(ux[selx]).astype(np.int64)
                iy = np.floor(uy[sely]).astype(np.int64)
                fx = ux[selx] - ix
                fy = uy[sely] - iy
                vxs = vx[np.ix_(selx, sely)]
                vys = vy[np.ix_(selx, sely)]
                for dx in (0, 1):
                    wxv = fx if dx else 1 - fx
                    jx = ix + dx
                    okx = (jx >= 0) & (jx < n2d)
                    for dy in (0, 1):
                        wyv = fy if dy else 1 - fy
                        jy = iy + dy
                        oky = (jy >= 0) & (jy < n2d)
                        ww = np.outer(wxv * okx, wyv * oky)
                        flat.append((np.clip(jx, 0, n2d - 1)[:, None] * n2d + np.clip(jy, 0, n2d - 1)[None, :]).ravel())
                        wx_all.append((ww * vxs).ravel())
                        wy_all.append((ww * vys).ravel())
        if flat:
            f = np.concatenate(flat)
            mesh[0] += np.bincount(f, np.concatenate(wx_all), minlength=n2d * n2d).reshape(n2d, n2d)
            mesh[1] += np.bincount(f, np.concatenate(wy_all), minlength=n2d * n2d).reshape(n2d, n2d)
    if not filtered:
        return torch.tensor(mesh), x2d, n2d
    # deconvolution and smoothing on the ray mesh
    k = 2.0 * math.pi * np.fft.fftfreq(n2d, d=x2d)
    kx, ky = np.meshgrid(k, k, indexing="ij")
    filt = (np.sinc(kx * x2d / (2 * math.pi)) ** -4) * (np.sinc(ky * x2d / (2 * math.pi)) ** -4)
    filt = filt * np.exp(-0.5 * (kx ** 2 + ky ** 2) * lam * lam)
    out = np.stack([np.real(np.fft.ifft2(np.fft.fft2(mesh[c]) * filt)) for c in range(2)])
    return torch.tensor(out), x2d, n2d


def gather(K: torch.Tensor, x2d: float, theta: torch.Tensor):
    """Bilinear values of the mesh K (2, N, N) at the angles theta (n, 2) and their derivatives.

    Returns (val (n, 2), T (n, 2, 2)) with T[:, a, b] = dK_a / dtheta_b."""
    n2d = K.shape[1]
    u = theta / x2d + n2d / 2
    i0 = torch.floor(u).to(torch.int64)
    f = u - i0
    val = torch.zeros(theta.shape[0], 2, dtype=torch.float64)
    T = torch.zeros(theta.shape[0], 2, 2, dtype=torch.float64)
    for dx in (0, 1):
        for dy in (0, 1):
            jx, jy = i0[:, 0] + dx, i0[:, 1] + dy
            ok = (jx >= 0) & (jx < n2d) & (jy >= 0) & (jy < n2d)
            jx, jy = jx.clamp(0, n2d - 1), jy.clamp(0, n2d - 1)
            wx = f[:, 0] if dx else 1 - f[:, 0]
            wy = f[:, 1] if dy else 1 - f[:, 1]
            sx, sy = (1.0 if dx else -1.0) / x2d, (1.0 if dy else -1.0) / x2d
            for c in range(2):
                v = torch.where(ok, K[c][jx, jy], torch.zeros_like(wx))
                val[:, c] += wx * wy * v
                T[:, c, 0] += sx * wy * v
                T[:, c, 1] += wx * sy * v
    return val, T


def ray_step(state: dict, gx, gy, box: float, observer, chi_n: float, chi_n1: float, weight_fn, mu: float,
             m_pix: int, iota: float, p_min: float, window=None, gz=None, replicas=None) -> dict:
    """One KDK step with the A/B recursion (Alg. 1 order) whose two half kicks come from ray meshes."""
    theta, eta, A, B = state["theta"], state["eta"], state["A"], state["B"]
    chi_h = 0.5 * (chi_n + chi_n1)
    K1, x1, _ = mesh_kick(gx, gy, box, observer, chi_n, chi_h, weight_fn, mu, m_pix, iota, p_min, window=window,
                          gz=gz, replicas=replicas)
    val, T = gather(K1, x1, theta)
    eta = eta + val
    B = B + T @ A
    d = (chi_n1 - chi_n) / (C_LIGHT * chi_h * chi_h)
    theta = theta + d * eta
    A = A + d * B
    K2, x2, _ = mesh_kick(gx, gy, box, observer, chi_h, chi_n1, weight_fn, mu, m_pix, iota, p_min, window=window,
                          gz=gz, replicas=replicas)
    val, T = gather(K2, x2, theta)
    eta = eta + val
    B = B + T @ A
    return dict(theta=theta, eta=eta, A=A, B=B)
