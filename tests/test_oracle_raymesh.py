"""Pins of the oracle's ray-mesh kick operator (Sec. 5.2, Sec. 5.3, App. C): mesh geometry by hand, the CIC
deposit against a brute-force sum, closed forms for a uniform and a single-mode gradient field, the exactness of
the bilinear gather on a bilinear function, and the A/B recursion of a ray-mesh step against finite differences."""
import math

import numpy as np
import pytest
import torch

from oracle import raymesh
from oracle.units import C_LIGHT

BOX, N = 32.0, 16
CELL = BOX / N
OBS = (0.3 * BOX, 0.6 * BOX, 0.7)
CHI_A, CHI_B = 150.5, 181.3
G = lambda chi: 1.0 + 0.002 * chi  # noqa: E731


def _planes():
    return raymesh.shell_planes(CHI_A, CHI_B, CELL, OBS[2])


def test_geometry_by_hand():
    # lambda = 2 cell / (r_a + r_b) = 4 / 331.8, x2d = lambda / 2, N >= 100 mu / x2d + 8 / 0.5 = 32.59 -> 64
    lam, x2d, n2d = raymesh.geometry(150.5, 181.3, 2.0, 0.001, 100, 0.5, 8)
    assert lam == pytest.approx(4.0 / 331.8, rel=1e-15) and x2d == pytest.approx(2.0 / 331.8, rel=1e-15)
    assert n2d == 64
    # the pixel limit dominates far away: lambda = mu = 0.003, x2d = mu, N >= 100 + 4 -> 128
    lam, x2d, n2d = raymesh.geometry(1000.0, 1010.0, 2.0, 0.003, 100, 1.0, 4)
    assert lam == 0.003 and x2d == 0.003 and n2d == 128
    # either orientation of the shell
    assert raymesh.geometry(181.3, 150.5, 2.0, 0.001, 100, 0.5, 8) == raymesh.geometry(150.5, 181.3, 2.0, 0.001,
                                                                                           100, 0.5, 8)


def test_shell_planes():
    pl = _planes()
    # z = 2 k with 150.5 <= z - 0.7 < 181.3: k = 76 .. 90
    assert [k for k, _ in pl] == list(range(76, 91))
    assert pl[0][1] == pytest.approx(151.3) and pl[-1][1] == pytest.approx(179.3)
    # consecutive half shells share no plane and miss none
    a = raymesh.shell_planes(150.5, 165.9, CELL, OBS[2])
    b = raymesh.shell_planes(165.9, 181.3, CELL, OBS[2])
    assert a + b == pl
    assert raymesh.shell_planes(150.6, 150.65, CELL, OBS[2]) == []


def _rand_fields(seed):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(N, N, N, generator=g, dtype=torch.float64),
            torch.randn(N, N, N, generator=g, dtype=torch.float64))


def test_deposit_matches_brute_force_sum():
    """Every mesh node m collects, from every plane of the shell and every periodic image, the node values times
    the CIC weight (1 - |u - m|)_+ per axis; written here as a gather over mesh nodes (the oracle scatters)."""
    gx, gy = _rand_fields(3)
    mu, m_pix, iota, p_min = 0.002, 40, 0.5, 4
    K, x2d, n2d = raymesh.mesh_kick(gx, gy, BOX, OBS, CHI_A, CHI_B, G, mu, m_pix, iota, p_min, filtered=False)
    want = np.zeros((2, n2d, n2d))
    node = (np.arange(n2d) - n2d / 2) * x2d
    for kz, chi in _planes():
        w = -(2.0 / C_LIGHT) * chi * G(chi) * CELL * (CELL / chi) ** 2 / x2d ** 2
        # all images within reach of the mesh, brute force
        R = int(np.ceil((n2d * x2d * chi) / BOX)) + 2
        coords = np.arange(-R * N, (R + 1) * N) * CELL
        th_x = (coords - OBS[0]) / chi
        th_y = (coords - OBS[1]) / chi
        wx = np.clip(1 - np.abs(th_x[None, :] - node[:, None]) / x2d, 0, None)    # [mesh i][node a]
        wy = np.clip(1 - np.abs(th_y[None, :] - node[:, None]) / x2d, 0, None)
        vals_x = gx.numpy()[np.arange(-R * N, (R + 1) * N) % N][:, np.arange(-R * N, (R + 1) * N) % N, kz % N]
        vals_y = gy.numpy()[np.arange(-R * N, (R + 1) * N) % N][:, np.arange(-R * N, (R + 1) * N) % N, kz % N]
        want[0] += w * wx @ vals_x @ wy.T
        want[1] += w * wx @ vals_y @ wy.T
    np.testing.assert_allclose(K.numpy(), want, rtol=1e-11, atol=1e-13 * np.abs(want).max())


# one node plane at r = 165.3 in the middle of its shell, so that lambda = cell / r: the projected node lattice is
# commensurate with the ray mesh (1 / iota mesh cells) and its pattern lies where the smoothing removes it
ONE_A, ONE_B = 164.3, 166.3


def test_uniform_field_closed_form():
    """A uniform transverse gradient gives K = -(2/c) sum_planes cell r g(r) grad on the whole mesh (the CIC
    deposit of the projected node lattice averages to the field; the smoothing removes the lattice pattern)."""
    gx = torch.full((N, N, N), 3.0, dtype=torch.float64)
    gy = torch.full((N, N, N), -1.5, dtype=torch.float64)
    for iota in (1.0, 0.5, 0.25):
        K, _, _ = raymesh.mesh_kick(gx, gy, BOX, OBS, ONE_A, ONE_B, G, 0.002, 40, iota, 8)
        s = -(2.0 / C_LIGHT) * CELL * 165.3 * G(165.3)
        assert torch.allclose(K[0], torch.full_like(K[0], 3.0 * s), rtol=1e-7)
        assert torch.allclose(K[1], torch.full_like(K[1], -1.5 * s), rtol=1e-7)
    # many planes at incommensurate spacings: the lattice beats with the mesh at the 1 % level (the discretisation
    # features of Sec. 5.3 / App. C), the mean stays at the closed form
    K, _, _ = raymesh.mesh_kick(gx, gy, BOX, OBS, CHI_A, CHI_B, G, 0.002, 40, 0.5, 32)
    s = sum(-(2.0 / C_LIGHT) * CELL * chi * G(chi) for _, chi in _planes())
    assert float((K[0] / (3.0 * s) - 1).abs().max()) < 0.015
    assert abs(float((K[0] / (3.0 * s)).mean()) - 1) < 1e-3
    # the opposite orientation of the same shell negates the kick; a shell without planes gives none
    K2, _, _ = raymesh.mesh_kick(gx, gy, BOX, OBS, CHI_B, CHI_A, G, 0.002, 40, 0.5, 32)
    assert torch.equal(K2, -K)
    K3, _, _ = raymesh.mesh_kick(gx, gy, BOX, OBS, 150.6, 150.65, G, 0.002, 40, 0.5, 8)
    assert float(K3.abs().max()) == 0.0


@pytest.mark.parametrize("shell,tol", [((ONE_A, ONE_B), 1.5e-3), ((CHI_A, CHI_B), 3e-3)])
def test_single_mode_closed_form_with_gaussian_smoothing(shell, tol):
    """grad_x = A cos(k x + a) and grad_y = B sin(k y + b): at a ray angle theta inside the field,
    K_x = sum_planes w_p A cos(k (O_x + r_p theta_x) + a) exp(-(k r_p lambda)^2 / 2) and likewise K_y, with
    w_p = -(2/c) cell r_p g(r_p): the deconvolution undoes both CIC windows up to O((k r x2d)^2)."""
    k = 2 * math.pi / BOX
    g = torch.arange(N, dtype=torch.float64) * CELL
    X, Y, _ = torch.meshgrid(g, g, g, indexing="ij")
    A, a, B, b = 2.0, 0.3, 0.7, -1.1
    gx = A * torch.cos(k * X + a)
    gy = B * torch.sin(k * Y + b)
    mu, m_pix, iota, p_min = 0.0015, 64, 0.25, 32
    ca, cb = shell
    lam, _, _ = raymesh.geometry(ca, cb, CELL, mu, m_pix, iota, p_min)
    K, x2d, n2d = raymesh.mesh_kick(gx, gy, BOX, OBS, ca, cb, G, mu, m_pix, iota, p_min)
    assert n2d * x2d * ca > 3 * BOX   # the mesh spans several periodic images
    rng = np.random.default_rng(5)
    theta = torch.tensor(rng.uniform(-0.5 * m_pix * mu, 0.5 * m_pix * mu, size=(400, 2)))
    val, _ = raymesh.gather(K, x2d, theta)
    want = torch.zeros_like(val)
    for _, r in raymesh.shell_planes(ca, cb, CELL, OBS[2]):
        w = -(2.0 / C_LIGHT) * CELL * r * G(r)
        damp = math.exp(-0.5 * (k * r * lam) ** 2)
        want[:, 0] += w * A * damp * torch.cos(k * (OBS[0] + r * theta[:, 0]) + a)
        want[:, 1] += w * B * damp * torch.sin(k * (OBS[1] + r * theta[:, 1]) + b)
    scale = want.abs().max(dim=0).values
    err = ((val - want).abs() / scale).max(dim=0).values
    assert float(err.max()) < tol, err
    # the smoothing is a 7 % effect here, well above the tolerance
    assert math.exp(-0.5 * (k * ca * lam) ** 2) < 0.94


def test_gather_is_exact_on_bilinear_functions():
    n2d, x2d = 32, 0.01
    t = (torch.arange(n2d, dtype=torch.float64) - n2d / 2) * x2d
    TX, TY = torch.meshgrid(t, t, indexing="ij")
    f = lambda x, y, c: c[0] + c[1] * x + c[2] * y + c[3] * x * y  # noqa: E731
    c0, c1 = (0.3, -2.0, 1.5, 40.0), (-1.0, 0.5, 3.0, -25.0)
    K = torch.stack([f(TX, TY, c0), f(TX, TY, c1)])
    rng = np.random.default_rng(1)
    th = torch.tensor(rng.uniform(-0.15, 0.14, size=(300, 2)))
    val, T = raymesh.gather(K, x2d, th)
    for comp, c in enumerate((c0, c1)):
        assert torch.allclose(val[:, comp], f(th[:, 0], th[:, 1], c), atol=1e-13)
        assert torch.allclose(T[:, comp, 0], c[1] + c[3] * th[:, 1], atol=1e-11)
        assert torch.allclose(T[:, comp, 1], c[2] + c[3] * th[:, 0], atol=1e-11)
    # outside the mesh the kick vanishes
    v, T = raymesh.gather(K, x2d, torch.tensor([[0.5, 0.0], [0.0, -0.3]], dtype=torch.float64))
    assert float(v.abs().max()) == 0.0 and float(T.abs().max()) == 0.0


def test_ray_step_recursion_matches_finite_differences():
    """One ray-mesh KDK step: A = d theta / d u and B = d eta / d u from the recursion equal central differences of
    theta and eta over a parameter u of the initial state theta = t + M u, eta = e + N u (A = M, B = N at the
    start; the interpolant is piecewise bilinear)."""
    gx, gy = _rand_fields(9)
    gx, gy = 2e3 * gx, 2e3 * gy
    args = (BOX, OBS, CHI_A, CHI_B, G, 0.002, 40, 0.5, 8)
    rng = np.random.default_rng(2)
    n = 64
    t0 = torch.tensor(rng.uniform(-0.03, 0.03, size=(n, 2)))
    e0 = torch.tensor(rng.normal(0, 3e-5, size=(n, 2)))
    M = torch.tensor(rng.normal(0, 1, size=(n, 2, 2)))
    Nm = torch.tensor(rng.normal(0, 1e-2, size=(n, 2, 2)))

    def step(u):
        st = dict(theta=t0 + M @ u, eta=e0 + Nm @ u, A=M.clone(), B=Nm.clone())
        return raymesh.ray_step(st, gx, gy, *args)

    out = step(torch.zeros(2, dtype=torch.float64))
    assert float(out["B"].abs().max()) > 1e-2   # the force is not negligible
    h = 1e-9
    for b in range(2):
        e = torch.zeros(2, dtype=torch.float64)
        e[b] = h
        p, m = step(e), step(-e)
        dth = (p["theta"] - m["theta"]) / (2 * h)
        deta = (p["eta"] - m["eta"]) / (2 * h)
        ok_a = (dth - out["A"][:, :, b]).abs().max(dim=1).values < 1e-5
        ok_b = (deta - out["B"][:, :, b]).abs().max(dim=1).values < 1e-5 * float(out["B"].abs().max())
        # a ray whose perturbed path crosses a ray-mesh cell face may differ
        assert int(ok_a.sum()) >= n - 2 and int(ok_b.sum()) >= n - 2


def test_filter_on_a_mesh_periodic_mode_at_mesh_nodes():
    """With r x2d = cell and the observer on a node column, the projected nodes fall on ray-mesh nodes, so the
    deposit samples the field there; a field periodic over the mesh then leaves the filter as the whole answer:
    K = f sinc(w_x / 2)^-4 sinc(w_y / 2)^-4 exp(-(w_x^2 + w_y^2) / (2 iota^2)) at mesh nodes, w the mode's phase
    step per ray-mesh cell (Sec. 5.2)."""
    obs = (10.0, 20.0, 0.7)
    iota, mu, m_pix, p_min = 1.0, 0.002, 40, 48
    lam, x2d, n2d = raymesh.geometry(ONE_A, ONE_B, CELL, mu, m_pix, iota, p_min)
    assert n2d == 64 and abs(165.3 * x2d - CELL) < 1e-12
    g = torch.arange(N, dtype=torch.float64) * CELL
    X, Y, _ = torch.meshgrid(g, g, g, indexing="ij")
    kb = 2 * math.pi / BOX
    # box modes (3, 1) and (2, 1): over the 64-cell ray mesh (4 boxes) they are the mesh modes (12, 4) and (8, 4)
    gx = torch.cos(3 * kb * (X - obs[0]) + 0.4) * torch.cos(kb * (Y - obs[1]))
    gy = 0.5 * torch.sin(2 * kb * (X - obs[0])) * torch.cos(kb * (Y - obs[1]) - 0.9)
    K, _, _ = raymesh.mesh_kick(gx, gy, BOX, obs, ONE_A, ONE_B, G, mu, m_pix, iota, p_min)
    w = -(2.0 / C_LIGHT) * CELL * 165.3 * G(165.3)
    m = torch.arange(n2d, dtype=torch.float64) - n2d / 2
    MX, MY = torch.meshgrid(m, m, indexing="ij")      # node offsets in cells of the 3D mesh

    def resp(qx, qy):
        wx, wy = 2 * math.pi * qx / n2d, 2 * math.pi * qy / n2d
        sinc = lambda v: math.sin(v / 2) / (v / 2)  # noqa: E731
        return sinc(wx) ** -4 * sinc(wy) ** -4 * math.exp(-(wx * wx + wy * wy) / (2 * iota * iota))

    want_x = w * resp(12, 4) * torch.cos(3 * kb * CELL * MX + 0.4) * torch.cos(kb * CELL * MY)
    want_y = w * 0.5 * (0.5 * (resp(8, 4) * (torch.sin(2 * kb * CELL * MX + kb * CELL * MY - 0.9)
                                            + torch.sin(2 * kb * CELL * MX - kb * CELL * MY + 0.9))))
    assert torch.allclose(K[0], want_x, atol=1e-9 * abs(w))
    assert torch.allclose(K[1], want_y, atol=1e-9 * abs(w))


def _g3(seed):
    g = torch.Generator().manual_seed(seed)
    return [torch.randn(N, N, N, generator=g, dtype=torch.float64) for _ in range(3)]


def _rotated(g3, perm, sign, shift):
    """Sky-frame mesh arrays g'_a[i] = sign_a g_{perm a}[M(i)], M(i)[perm a] = sign_a i_a + shift[perm a] (mod n),
    built on the whole mesh at once (independently of the oracle's per-plane map)."""
    n = g3[0].shape[0]
    idx = np.indices((n, n, n)).reshape(3, -1)
    b = np.zeros_like(idx)
    for a in range(3):
        b[perm[a]] = (sign[a] * idx[a] + shift[perm[a]]) % n
    flat = (b[0] * n + b[1]) * n + b[2]
    return [torch.tensor(sign[a] * g3[perm[a]].reshape(-1).numpy()[flat].reshape(n, n, n)) for a in range(3)]


def test_tiled_mesh_with_identity_replicas_is_the_plain_mesh():
    g3 = _g3(40)
    ident = (np.tile([0, 1, 2], (12, 1)), np.ones((12, 3), np.int32), np.zeros((12, 3), np.int32))
    args = (BOX, OBS, CHI_A, CHI_B, G, 0.002, 40, 0.5, 8)
    K, _, _ = raymesh.mesh_kick(g3[0], g3[1], *args)
    Kt, _, _ = raymesh.mesh_kick(g3[0], g3[1], *args, gz=g3[2], replicas=ident)
    assert torch.equal(K, Kt)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiled_mesh_is_the_sum_of_plain_meshes_of_rotated_fields(seed):
    """A shell that spans two replicas: its mesh equals the plain meshes of the two sub-shells, each over the
    explicitly rotated and translated arrays of its replica (the kick is linear in the field)."""
    import synthetic
    g3 = _g3(50 + seed)
    perm, sign, shift = synthetic.replica_transforms(seed, 12, N)
    # replica k holds the sky planes kz with kz // N == k; the shell [150.5, 181.3) with O_z = 0.7 spans planes
    # 76..90, i.e. replicas 4 (kz < 80) and 5
    edge = 80 * CELL - OBS[2]
    args = (BOX, OBS)
    tail = (G, 0.002, 40, 0.5, 8)
    Kt, x2d, n2d = raymesh.mesh_kick(g3[0], g3[1], *args, CHI_A, CHI_B, *tail, gz=g3[2], replicas=(perm, sign, shift))
    parts = []
    for k, (lo, hi) in ((4, (CHI_A, edge)), (5, (edge, CHI_B))):
        r = _rotated(g3, perm[k], sign[k], shift[k])
        parts.append(raymesh.mesh_kick(r[0], r[1], *args, CHI_A, CHI_B, *tail, window=(lo, hi))[0])
    assert torch.allclose(Kt, parts[0] + parts[1], rtol=0, atol=1e-12 * float(Kt.abs().max()))
    # and the tiling matters
    assert float((Kt - raymesh.mesh_kick(g3[0], g3[1], *args, CHI_A, CHI_B, *tail)[0]).abs().max()) > 0.1 * float(Kt.abs().max())
