"""Hamiltonian ray tracing of light rays in FP64 on the CPU (test infrastructure only).

Restates Sec. 3 and Sec. 4 of arXiv 2405.12913 for a bundle of independent rays:

  * state per ray: angle theta (2), conjugate momentum eta (2), distortion matrix A = d theta / d theta_0 and
    the helper B = d eta / d theta_0 (2x2 each); initially theta = theta_0, eta = 0, A = I, B = 0 (Sec. 2 and
    Sec. 4, Eq. "B");
  * flat sky, line of sight along +z from the observer O: the 3D point at radial distance chi is
    X(theta, chi) = O + (r theta_x, r theta_y, chi), r = chi, wrapped into the periodic box;
  * one step over the shell [chi_n, chi_{n+1}] with midpoint chi_{n+1/2} is the KDK of Eqs. "symp_1..3"
    together with the A/B recursion of Eqs. "obsv_recurse1..3", in the order of Alg. 1:
      eta += K_n^{n+1/2}(theta_n);          B += (dK/dtheta) A
      theta += D(eta);                      A += (dD/deta) B
      eta += K_{n+1/2}^{n+1}(theta_{n+1});  B += (dK/dtheta) A
  * the kick of Eq. "kick", K = -(2/c) int r grad_perp phi(X(theta_c, chi)) g(chi) dchi with the time
    correction g = D1(a(chi)) a_c / (D1(a_c) a(chi)), is evaluated at fixed theta_c by the midpoint rule on
    n_sub = max(1, ceil(s |half-shell| / cell)) equal sub-intervals (s samples per mesh cell); the transverse
    gradient grad_perp phi = (d_x phi, d_y phi) comes from the CIC interpolation of the 3D gradient mesh;
  * dK/dtheta = sum_j c_j r_j T(X_j), T the 2x2 derivative of the trilinear interpolant of (d_x phi, d_y phi)
    with respect to the transverse coordinates (x, y) (on a cell face the lower cell is used);
  * the drift of Eq. "drift" with the midpoint radius: D = eta (chi_{n+1} - chi_n) / (c r_{n+1/2}^2), so
    dD/deta = (chi_{n+1} - chi_n) / (c r_{n+1/2}^2) times the identity;
  * readout of Eqs. "obs_first_set" / "obs_second_set" (kappa, gamma_1, gamma_2, omega from A).
"""
from __future__ import annotations

import itertools
import math

import torch

from .units import C_LIGHT

_CORNERS = list(itertools.product((0, 1), repeat=3))


def half_shell_nodes(chi_a: float, chi_b: float, samples_per_cell: float, cell: float):
    """Midpoint-rule nodes of [chi_a, chi_b] (either orientation): returns (chi_j list, signed width h)."""
    n_sub = max(1, math.ceil(samples_per_cell * abs(chi_b - chi_a) / cell))
    h = (chi_b - chi_a) / n_sub
    return [chi_a + (j + 0.5) * h for j in range(n_sub)], h


def interp_xy(gx: torch.Tensor, gy: torch.Tensor, X: torch.Tensor, box: float):
    """Trilinear values of (gx, gy) at X (n, 3) and their transverse derivatives.

    Returns (val (n, 2), T (n, 2, 2)) with T[:, a, b] = d g_a / d x_b for b in (x, y)."""
    n_mesh = gx.shape[0]
    cell = box / n_mesh
    u = torch.remainder(X, box) / cell
    i0 = torch.floor(u)
    f = u - i0
    i0 = i0.to(torch.int64) % n_mesh
    fx, fy, fz = f[:, 0], f[:, 1], f[:, 2]
    val = torch.zeros(X.shape[0], 2, dtype=torch.float64)
    T = torch.zeros(X.shape[0], 2, 2, dtype=torch.float64)
    flat = (gx.reshape(-1), gy.reshape(-1))
    for a, b, c in _CORNERS:
        wx = fx if a else 1 - fx
        wy = fy if b else 1 - fy
        wz = fz if c else 1 - fz
        dwx = (1.0 if a else -1.0) / cell
        dwy = (1.0 if b else -1.0) / cell
        idx = (((i0[:, 0] + a) % n_mesh) * n_mesh + (i0[:, 1] + b) % n_mesh) * n_mesh + (i0[:, 2] + c) % n_mesh
        for comp in range(2):
            v = flat[comp][idx]
            val[:, comp] += wx * wy * wz * v
            T[:, comp, 0] += dwx * wy * wz * v
            T[:, comp, 1] += wx * dwy * wz * v
    return val, T


def interp_grad3(g3, X: torch.Tensor, box: float):
    """Trilinear values of the three gradient fields g3 = (gx, gy, gz) at box points X (n, 3) and their
    derivatives along the three box axes.

    Returns (val (n, 3), D (n, 3, 3)) with D[:, c, b] = d g_c / d x_b (on a cell face the lower cell is used)."""
    n_mesh = g3[0].shape[0]
    cell = box / n_mesh
    u = torch.remainder(X, box) / cell
    i0 = torch.floor(u)
    f = u - i0
    i0 = i0.to(torch.int64) % n_mesh
    val = torch.zeros(X.shape[0], 3, dtype=torch.float64)
    D = torch.zeros(X.shape[0], 3, 3, dtype=torch.float64)
    flat = [g.reshape(-1) for g in g3]
    for corner in _CORNERS:
        w = [f[:, ax] if corner[ax] else 1 - f[:, ax] for ax in range(3)]
        dw = [(1.0 if corner[ax] else -1.0) / cell for ax in range(3)]
        idx = (((i0[:, 0] + corner[0]) % n_mesh) * n_mesh + (i0[:, 1] + corner[1]) % n_mesh) * n_mesh \
            + (i0[:, 2] + corner[2]) % n_mesh
        for comp in range(3):
            v = flat[comp][idx]
            val[:, comp] += w[0] * w[1] * w[2] * v
            D[:, comp, 0] += dw[0] * w[1] * w[2] * v
            D[:, comp, 1] += w[0] * dw[1] * w[2] * v
            D[:, comp, 2] += w[0] * w[1] * dw[2] * v
    return val, D


def replica_frame(X: torch.Tensor, replicas, box: float, n_mesh: int):
    """Light-cone tiling: the unwrapped sky point X (n, 3) lies in replica k = floor(X_z / box); with
    u = X mod box, sky axis a maps to box axis perm[k, a] at sign[k, a] u_a + shift[k, perm[k, a]] cell (mod box).

    Returns (box points (n, 3), perm (n, 3), sign (n, 3) float64)."""
    perm_t, sign_t, shift_t = (torch.as_tensor(x, dtype=torch.int64) for x in replicas)
    k = torch.floor(X[:, 2] / box).to(torch.int64)
    if (k < 0).any() or (k >= perm_t.shape[0]).any():
        raise ValueError("a point lies outside the replicas")
    perm, sign, shift = perm_t[k], sign_t[k].double(), shift_t[k].double()
    cell = box / n_mesh
    u = torch.remainder(X, box)
    Xb = torch.zeros_like(X)
    for a in range(3):
        dst = perm[:, a]
        vals = torch.remainder(sign[:, a] * u[:, a] + torch.gather(shift, 1, dst[:, None])[:, 0] * cell, box)
        Xb.scatter_(1, dst[:, None], vals[:, None])
    return Xb, perm, sign


def tiled_gradient(g3, X: torch.Tensor, replicas, box: float):
    """Transverse gradient of the tiled potential phi(M_k X) seen along the sky directions x, y, and its
    derivative: val_a = sign_a g_{perm a}, T_ab = sign_a sign_b d g_{perm a} / d x_{perm b} at the box point."""
    Xb, perm, sign = replica_frame(X, replicas, box, g3[0].shape[0])
    v3, D3 = interp_grad3(g3, Xb, box)
    n = X.shape[0]
    val = torch.zeros(n, 2, dtype=torch.float64)
    T = torch.zeros(n, 2, 2, dtype=torch.float64)
    rows = torch.arange(n)
    for a in range(2):
        val[:, a] = sign[:, a] * v3[rows, perm[:, a]]
        for b in range(2):
            T[:, a, b] = sign[:, a] * sign[:, b] * D3[rows, perm[:, a], perm[:, b]]
    return val, T


def ray_points(theta: torch.Tensor, chi: float, observer) -> torch.Tensor:
    """3D comoving points X(theta, chi) = O + (chi theta_x, chi theta_y, chi) (unwrapped), shape (n, 3)."""
    r = chi
    X = torch.empty(theta.shape[0], 3, dtype=torch.float64)
    X[:, 0] = observer[0] + r * theta[:, 0]
    X[:, 1] = observer[1] + r * theta[:, 1]
    X[:, 2] = observer[2] + chi
    return X


def half_kick(theta, gx, gy, box, observer, chis, h, weight_fn, window=None, gz=None, replicas=None):
    """Kick K = sum_j c_j grad_perp phi(X(theta, chi_j)) and its Jacobian J = sum_j c_j r_j T_j.

    ``weight_fn(chi)`` is the time-correction factor g(chi); c_j = -(2/c) h r_j g(chi_j).  Nodes outside
    ``window = (chi_lo, chi_hi)`` do not contribute.  With ``replicas`` = (perm, sign, shift) the light cone is
    tiled by rotated and translated replicas (``replica_frame``), which needs the third field gz."""
    K = torch.zeros(theta.shape[0], 2, dtype=torch.float64)
    J = torch.zeros(theta.shape[0], 2, 2, dtype=torch.float64)
    for chi in chis:
        if window is not None and not (window[0] <= chi < window[1]):
            continue
        r = chi
        c = -(2.0 / C_LIGHT) * h * r * weight_fn(chi)
        X = ray_points(theta, chi, observer)
        if replicas is None:
            val, T = interp_xy(gx, gy, X, box)
        else:
            val, T = tiled_gradient((gx, gy, gz), X, replicas, box)
        K += c * val
        J += (c * r) * T
    return K, J


def ray_step(state: dict, gx, gy, box: float, observer, chi_n: float, chi_n1: float,
             samples_per_cell: float, weight_fn, window=None, gz=None, replicas=None) -> dict:
    """One KDK step with the A/B recursion over the shell [chi_n, chi_n1] (Alg. 1 order)."""
    cell = box / gx.shape[0]
    theta, eta, A, B = state["theta"], state["eta"], state["A"], state["B"]
    chi_h = 0.5 * (chi_n + chi_n1)
    chis, h = half_shell_nodes(chi_n, chi_h, samples_per_cell, cell)
    K, J = half_kick(theta, gx, gy, box, observer, chis, h, weight_fn, window, gz, replicas)
    eta = eta + K
    B = B + J @ A
    d = (chi_n1 - chi_n) / (C_LIGHT * chi_h * chi_h)
    theta = theta + d * eta
    A = A + d * B
    chis, h = half_shell_nodes(chi_h, chi_n1, samples_per_cell, cell)
    K, J = half_kick(theta, gx, gy, box, observer, chis, h, weight_fn, window, gz, replicas)
    eta = eta + K
    B = B + J @ A
    return dict(theta=theta, eta=eta, A=A, B=B)


def face_distance(theta: torch.Tensor, box: float, n_mesh: int, observer, chis) -> torch.Tensor:
    """Smallest distance, in cells, of the transverse coordinates of the line-of-sight nodes X(theta, chi_j) to a
    cell face, per ray.  The transverse derivative of the trilinear interpolant (the T of dK/dtheta) is piecewise
    constant and jumps on those faces (reading C12 of the interpolant's derivative, Sec. 4), so a node this close
    to a face may take either cell in any finite precision.  Distances are invariant under the whole-cell shifts
    and sign flips of a tiled light cone."""
    cell = box / n_mesh
    d = torch.full((theta.shape[0],), math.inf, dtype=torch.float64)
    for chi in chis:
        u = torch.remainder(ray_points(theta, chi, observer)[:, :2], box) / cell
        f = u - torch.floor(u)
        d = torch.minimum(d, torch.minimum(f, 1.0 - f).amin(dim=1))
    return d


def step_face_distance(theta_n: torch.Tensor, theta_n1: torch.Tensor, box: float, n_mesh: int, observer,
                       chi_n: float, chi_n1: float, samples_per_cell: float) -> torch.Tensor:
    """``face_distance`` over the nodes of one ``ray_step``: the first half shell at theta_n, the second at
    theta_{n+1} (Alg. 1 order)."""
    cell = box / n_mesh
    chi_h = 0.5 * (chi_n + chi_n1)
    first, _ = half_shell_nodes(chi_n, chi_h, samples_per_cell, cell)
    second, _ = half_shell_nodes(chi_h, chi_n1, samples_per_cell, cell)
    return torch.minimum(face_distance(theta_n, box, n_mesh, observer, first),
                         face_distance(theta_n1, box, n_mesh, observer, second))


def free_drift(state: dict, chi_a: float, chi_b: float) -> dict:
    """Exact solution of the drift equation d theta / d chi = -eta_EOM / r^2 for constant eta over
    [chi_a, chi_b] (chi_a > 0): theta += eta (1/chi_a - 1/chi_b) / c, A += B (1/chi_a - 1/chi_b) / c."""
    d = (1.0 / chi_a - 1.0 / chi_b) / C_LIGHT
    return dict(theta=state["theta"] + d * state["eta"], eta=state["eta"], A=state["A"] + d * state["B"],
                B=state["B"])


def init_state(theta0: torch.Tensor) -> dict:
    n = theta0.shape[0]
    eye = torch.eye(2, dtype=torch.float64).expand(n, 2, 2).clone()
    return dict(theta=theta0.clone().to(torch.float64), eta=torch.zeros(n, 2, dtype=torch.float64), A=eye,
                B=torch.zeros(n, 2, 2, dtype=torch.float64))


def observables(A: torch.Tensor):
    """(kappa, gamma1, gamma2, omega) from the distortion matrix, first order in omega."""
    c1 = 0.5 * (A[:, 0, 0] + A[:, 1, 1])
    c2 = 0.5 * (A[:, 0, 1] - A[:, 1, 0])
    c3 = 0.5 * (A[:, 1, 1] - A[:, 0, 0])
    c4 = 0.5 * (A[:, 0, 1] + A[:, 1, 0])
    kappa = 1.0 - c1
    omega = c2 / (1.0 - kappa)
    g1 = c3 + c4 * omega
    g2 = -c4 + c3 * omega
    return kappa, g1, g2, omega
