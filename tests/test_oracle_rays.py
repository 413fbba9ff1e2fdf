"""Pins of the oracle's ray integrator (Sec. 3), A/B recursion (Sec. 4) and readout."""
import math

import numpy as np
import pytest
import torch

import synthetic
from oracle import pm, rays
from oracle.units import C_LIGHT

BOX, N = 64.0, 32
CELL = BOX / N


def _smooth_fields(amp=3.0e3):
    # gradient fields of a smooth periodic potential phi = A [sin(kx x + 0.3) cos(ky y) + 0.5 cos(kz z - ky y)]
    g = torch.arange(N, dtype=torch.float64) * CELL
    X, Y, Z = torch.meshgrid(g, g, g, indexing="ij")
    k = 2 * math.pi / BOX
    gx = amp * k * torch.cos(k * X + 0.3) * torch.cos(k * Y)
    gy = -amp * k * torch.sin(k * X + 0.3) * torch.sin(k * Y) + 0.5 * amp * k * torch.sin(k * Z - k * Y)
    return gx, gy


OBS = (0.3 * BOX, 0.6 * BOX, 0.0)
ONE = lambda chi: 1.0  # noqa: E731


def _trace(theta0, gx, gy, chis, s=1.0):
    st = rays.init_state(theta0)
    for a, b in zip(chis[:-1], chis[1:]):
        st = rays.ray_step(st, gx, gy, BOX, OBS, a, b, s, ONE)
    return st


def test_half_shell_nodes():
    chis, h = rays.half_shell_nodes(10.0, 17.0, 1.0, 2.0)
    assert len(chis) == 4 and h == pytest.approx(1.75)
    assert chis[0] == pytest.approx(10.875) and chis[-1] == pytest.approx(16.125)
    chis, h = rays.half_shell_nodes(17.0, 10.0, 2.0, 2.0)
    assert len(chis) == 7 and h == pytest.approx(-1.0)
    chis, h = rays.half_shell_nodes(5.0, 5.1, 1.0, 2.0)
    assert len(chis) == 1


def test_zero_potential_leaves_rays_straight():
    th0 = torch.tensor(synthetic.pixel_grid(8, 0.05))
    zero = torch.zeros(N, N, N, dtype=torch.float64)
    st = _trace(th0, zero, zero, [0.0, 40.0, 90.0, 200.0])
    assert torch.equal(st["theta"], th0) and float(st["eta"].abs().max()) == 0.0
    kap, g1, g2, om = rays.observables(st["A"])
    assert float(kap.abs().max()) == 0.0 and float(g1.abs().max()) == 0.0
    assert float(g2.abs().max()) == 0.0 and float(om.abs().max()) == 0.0


def test_interpolant_of_linear_fields_and_its_derivative():
    g = torch.arange(N, dtype=torch.float64) * CELL
    X, Y, Z = torch.meshgrid(g, g, g, indexing="ij")
    gx = 1.0 + 0.5 * X - 0.25 * Y + 0.1 * Z
    gy = -2.0 + 0.3 * X + 0.7 * Y - 0.2 * Z
    pts = torch.tensor(synthetic.uniform_positions(3, 100, BOX - 2 * CELL))
    val, T = rays.interp_xy(gx, gy, pts, BOX)
    assert torch.allclose(val[:, 0], 1.0 + 0.5 * pts[:, 0] - 0.25 * pts[:, 1] + 0.1 * pts[:, 2], atol=1e-12)
    assert torch.allclose(val[:, 1], -2.0 + 0.3 * pts[:, 0] + 0.7 * pts[:, 1] - 0.2 * pts[:, 2], atol=1e-12)
    want = torch.tensor([[0.5, -0.25], [0.3, 0.7]], dtype=torch.float64)
    assert torch.allclose(T, want.expand_as(T), atol=1e-12)


def test_interpolant_derivative_matches_finite_difference():
    gx, gy = _smooth_fields()
    pts = torch.tensor(synthetic.uniform_positions(4, 64, BOX))
    _, T = rays.interp_xy(gx, gy, pts, BOX)
    # inside a cell the interpolant is linear in x and y: a small central difference is exact up to rounding,
    # unless the stencil crosses a cell face; keep points whose stencil stays in the cell.
    eps = 1e-4
    frac = torch.remainder(pts[:, :2], CELL) / CELL
    keep = ((frac > 1e-3) & (frac < 1 - 1e-3)).all(dim=1)
    for b in range(2):
        d = torch.zeros(3, dtype=torch.float64)
        d[b] = eps
        vp, _ = rays.interp_xy(gx, gy, pts + d, BOX)
        vm, _ = rays.interp_xy(gx, gy, pts - d, BOX)
        fd = (vp - vm) / (2 * eps)
        assert torch.allclose(T[keep, :, b], fd[keep], rtol=1e-7, atol=1e-9)


def test_static_step_is_time_reversible():
    gx, gy = _smooth_fields()
    th0 = torch.tensor(synthetic.pixel_grid(6, 0.2))
    st = rays.init_state(th0)
    st = rays.ray_step(st, gx, gy, BOX, OBS, 100.0, 160.0, 1.0, ONE)
    st = rays.ray_step(st, gx, gy, BOX, OBS, 160.0, 230.0, 1.0, ONE)
    mid = {k: v.clone() for k, v in st.items()}
    back = rays.ray_step(st, gx, gy, BOX, OBS, 230.0, 160.0, 1.0, ONE)
    back = rays.ray_step(back, gx, gy, BOX, OBS, 160.0, 100.0, 1.0, ONE)
    st1 = rays.ray_step(back, gx, gy, BOX, OBS, 100.0, 160.0, 1.0, ONE)
    st1 = rays.ray_step(st1, gx, gy, BOX, OBS, 160.0, 230.0, 1.0, ONE)
    assert float((mid["eta"]).abs().max()) > 1e-3
    assert torch.allclose(back["theta"], th0, rtol=0, atol=1e-15)
    for key in ("theta", "eta", "A", "B"):
        assert torch.allclose(st1[key], mid[key], rtol=1e-12, atol=1e-15)


def _step_map(z, gx, gy, a, b):
    st = dict(theta=z[None, :2], eta=z[None, 2:], A=torch.eye(2, dtype=torch.float64)[None],
              B=torch.zeros(1, 2, 2, dtype=torch.float64))
    out = rays.ray_step(st, gx, gy, BOX, OBS, a, b, 1.0, ONE)
    return torch.cat([out["theta"][0], out["eta"][0]])


def test_one_step_phase_space_jacobian_has_unit_determinant():
    # KDK = kick . drift . kick, each a shear of (theta, eta): det M = 1 (symplectic structure, Appendix B).
    gx, gy = _smooth_fields()
    for i, th in enumerate(synthetic.pixel_grid(3, 0.2)):
        z = torch.tensor([th[0], th[1], 0.01 * (i - 4), -0.02], dtype=torch.float64)
        M = torch.autograd.functional.jacobian(lambda v: _step_map(v, gx, gy, 120.0, 190.0), z)
        assert float(torch.det(M)) == pytest.approx(1.0, abs=1e-12)


def check_ab_against_autograd(pixels):
    # A = d theta / d theta_0 and B = d eta / d theta_0 (Eqs. "A", "B") through several steps.
    gx, gy = _smooth_fields()
    chis = [0.0, 30.0, 75.0, 110.0, 170.0, 260.0]
    for th in pixels:
        t0 = torch.tensor(th, dtype=torch.float64)

        def final(t):
            st = _trace(t[None], gx, gy, chis)
            return torch.cat([st["theta"][0], st["eta"][0]])

        jac = torch.autograd.functional.jacobian(final, t0)
        st = _trace(t0[None], gx, gy, chis)
        assert torch.allclose(st["A"][0], jac[:2], rtol=1e-10, atol=1e-14)
        assert torch.allclose(st["B"][0], jac[2:], rtol=1e-10, atol=1e-12)


def test_A_B_recursion_equals_autograd_derivative_of_trajectory():
    check_ab_against_autograd(synthetic.pixel_grid(2, 0.3))


def test_second_order_convergence_in_step_size():
    # KDK error ~ dchi^2 (BCH, Appendix B): halving the step quarters the error of the final angle.
    gx, gy = _smooth_fields(3.0e4)
    th0 = torch.tensor(synthetic.pixel_grid(4, 0.2))

    def run(n):
        chis = list(np.linspace(40.0, 300.0, n + 1))
        return _trace(th0, gx, gy, chis, s=16.0)["theta"]

    ref = run(128)
    e = [float((run(n) - ref).abs().max()) for n in (8, 16, 32)]
    assert 3.0 < e[0] / e[1] < 5.0 and 3.0 < e[1] / e[2] < 5.0


def test_readout_of_rotation_times_shear():
    # A = R(omega) S(kappa, gamma) as in Sec. 4; the readout is exact for kappa to O(omega^2) and for the
    # rest to first order in omega.
    kap, g1, g2, om = 0.05, 0.02, -0.03, 2e-4
    R = torch.tensor([[math.cos(om), math.sin(om)], [-math.sin(om), math.cos(om)]], dtype=torch.float64)
    S = torch.tensor([[1 - kap - g1, -g2], [-g2, 1 - kap + g1]], dtype=torch.float64)
    k, a, b, w = rays.observables((R @ S)[None])
    assert float(k) == pytest.approx(kap, abs=1e-7)
    assert float(a) == pytest.approx(g1, abs=1e-7)
    assert float(b) == pytest.approx(g2, abs=1e-7)
    assert float(w) == pytest.approx(om, rel=1e-3)


def test_free_drift_is_exact_for_constant_momentum():
    st = rays.init_state(torch.tensor([[0.01, -0.02]], dtype=torch.float64))
    st["eta"] = torch.tensor([[3.0, -1.0]], dtype=torch.float64)
    a, b = 100.0, 900.0
    out = rays.free_drift(st, a, b)
    # d theta / d chi = eta_disc / (c chi^2) integrated in closed form
    want = st["theta"] + st["eta"] * (1 / a - 1 / b) / C_LIGHT
    assert torch.allclose(out["theta"], want, rtol=1e-15)
    # the midpoint drift of many small steps converges to it
    chis = np.linspace(a, b, 2001)
    th = st["theta"].clone()
    for x0, x1 in zip(chis[:-1], chis[1:]):
        xm = 0.5 * (x0 + x1)
        th = th + st["eta"] * (x1 - x0) / (C_LIGHT * xm * xm)
    assert torch.allclose(th, want, rtol=1e-7)


def _tiling_fields(n, seed):
    return [torch.tensor(synthetic.gaussian_field(seed + c, (n, n, n))) for c in range(3)]


def test_tiling_with_identity_replicas_is_the_plain_gather():
    n, box = 16, 32.0
    g = _tiling_fields(n, 300)
    rng = np.random.default_rng(301)
    X = torch.tensor(rng.uniform(0, 1, (500, 3)) * [box, box, 3 * box])
    ident = (np.tile([0, 1, 2], (3, 1)), np.ones((3, 3), np.int32), np.zeros((3, 3), np.int32))
    val, T = rays.tiled_gradient(g, X, ident, box)
    val0, T0 = rays.interp_xy(g[0], g[1], X, box)
    assert torch.allclose(val, val0, rtol=0, atol=1e-14) and torch.allclose(T, T0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_tiling_equals_the_gather_of_explicitly_rotated_fields(seed):
    # phi_k(X) = phi(M X): its sky-frame gradient on the mesh is g'_a[i] = sign_a g_{perm a}[M(i)], with
    # M(i)[perm a] = sign_a i_a + shift[perm a] (mod n); the plain gather of g' must equal the tiled gather of g
    n, box = 16, 32.0
    g = _tiling_fields(n, 310 + seed)
    perm, sign, shift = synthetic.replica_transforms(seed, 1, n)
    p, s, sh = perm[0], sign[0], shift[0]
    idx = np.indices((n, n, n)).reshape(3, -1)
    b = np.zeros_like(idx)
    for a in range(3):
        b[p[a]] = (s[a] * idx[a] + sh[p[a]]) % n
    flat = (b[0] * n + b[1]) * n + b[2]
    gp = [torch.tensor(s[a] * g[p[a]].reshape(-1).numpy()[flat].reshape(n, n, n)) for a in range(3)]
    rng = np.random.default_rng(320 + seed)
    X = torch.tensor(rng.uniform(0, 1, (800, 3)) * box)  # replica 0 (0 <= z < box)
    val, T = rays.tiled_gradient(g, X, (perm, sign, shift), box)
    val_p, T_p = rays.interp_xy(gp[0], gp[1], X, box)
    assert torch.allclose(val, val_p, rtol=0, atol=1e-12)
    assert torch.allclose(T, T_p, rtol=0, atol=1e-11)


def test_face_distance_bounds_the_cells_the_nodes_occupy():
    # face_distance is the largest observer shift (in cells) that leaves every node of every ray in its cell:
    # shifts of 0.99 of it along +-x and +-y keep all cells, and one of the four shifts by 1.01 of it moves a node
    # into the next cell.  Checked ray by ray on random angles, with nodes from a real half shell.
    from oracle import rays as orays
    g = torch.Generator().manual_seed(91)
    box, n_mesh, cell = 100.0, 50, 2.0
    chis, _ = orays.half_shell_nodes(300.0, 340.0, 1.0, cell)
    theta = 0.05 * (torch.rand(64, 2, generator=g, dtype=torch.float64) - 0.5)
    obs = (3.7, 41.2, 0.0)
    d = orays.face_distance(theta, box, n_mesh, obs, chis)
    assert float(d.min()) >= 0.0 and float(d.max()) <= 0.5

    def cells(t, o):
        return torch.stack([torch.floor(torch.remainder(orays.ray_points(t, c, o)[:, :2], box) / cell)
                            for c in chis])

    for r in range(theta.shape[0]):
        t = theta[r:r + 1]
        base = cells(t, obs)
        moved_past = False
        for ax in (0, 1):
            for sgn in (1.0, -1.0):
                o_in, o_out = list(obs), list(obs)
                o_in[ax] += sgn * 0.99 * float(d[r]) * cell
                o_out[ax] += sgn * 1.01 * float(d[r]) * cell
                assert torch.equal(cells(t, tuple(o_in)), base)
                moved_past |= not torch.equal(cells(t, tuple(o_out)), base)
        assert moved_past, r
    # a node exactly on a face has distance 0, one at a cell centre 0.5
    on_face = torch.tensor([[0.0, 0.0]], dtype=torch.float64)
    assert float(orays.face_distance(on_face, box, n_mesh, (4.0, 4.0 + 0.5 * cell, 0.0), [10.0])) == 0.0
    assert float(orays.face_distance(on_face, box, n_mesh, (3.0, 5.0, 0.0), [10.0])) == pytest.approx(0.5)
