"""Planted mistakes in the oracle: its pins hold it to the paper, not just to itself.

Each case edits the source of one oracle module in one place, the way a slip would (a dropped term, a wrong sign,
index or operand order), loads the edited copy in place of the module (in memory, on the CPU: the files are not
touched), and runs pins from the oracle's own test files; at least one of them must fail.  The pins are first run
on the oracle as it stands, where all pass, so a failure is the planted mistake's doing."""
import sys
import types

import pytest

import synthetic
import test_oracle_cosmology as cosmo_pins
import test_oracle_lensing as lens_pins
import test_oracle_mlp as mlp_pins
import test_oracle_pm as pm_pins
import test_oracle_raymesh as rm_pins
import test_oracle_rays as ray_pins
from oracle import cosmology, ewald, mlp, pm, power, raymesh, rays, sim


def _point_mass_pins():
    # the point-mass pins on every eighth of their rays (16 rays from 0.1 to 20 cells)
    run = lens_pins.point_mass_run_data(stride=8)
    lens_pins.test_point_mass_deflection_matches_born_ewald_above_threshold(run)


# the pins by name; a pin that takes arguments is called with the listed ones
PINS = {
    "cic_mass": pm_pins.test_cic_mass_conservation_and_mean,
    "cic_node": pm_pins.test_cic_single_particle_on_node_and_at_cell_centre,
    "cic_roll": pm_pins.test_cic_integer_translation_commutes_with_roll,
    "brute_plain": lambda: pm_pins.test_fft_gradient_matches_brute_force_dft(0.0, 0.0),
    "brute_filtered": lambda: pm_pins.test_fft_gradient_matches_brute_force_dft(4.0, 1.0),
    "mode_x": lambda: pm_pins.test_single_mode_poisson_gradient(0, 3),
    "mode_z": lambda: pm_pins.test_single_mode_poisson_gradient(2, 2),
    "ewald_force": pm_pins.test_pm_force_matches_periodic_direct_sum,
    "ewald_3d": pm_pins.test_ewald_field_of_a_periodic_point_mass,
    "ewald_2d": lens_pins.test_periodic_lensing_sum_is_independent_of_the_splitting,
    "gather_linear": pm_pins.test_gather_of_linear_field_is_exact,
    "kd_uniform": pm_pins.test_kick_drift_with_a_uniform_field,
    "growth_d2": pm_pins.test_low_k_power_grows_as_growth_factor_squared,
    "fwd_rev": pm_pins.test_forward_then_reverse_returns_to_initial_conditions,
    "zeldovich": pm_pins.test_zeldovich_momentum_ratio_and_power,
    "zeldovich_sign": pm_pins.test_zeldovich_density_has_the_sign_of_the_linear_field,
    "lpt_diagonal": lambda: pm_pins.test_lpt_plane_wave_along_a_diagonal_has_no_second_order_term((1, -1, 1)),
    "lpt_orthogonal": lambda: pm_pins.test_lpt_two_orthogonal_waves_closed_form((0, 2)),
    "lpt_eds": pm_pins.test_lpt_second_order_is_quadratic_and_eds_assembly,
    "lpt_dynamics": pm_pins.test_lpt_second_order_mode_follows_the_n_body,
    "eds": lambda: cosmo_pins.test_einstein_de_sitter_closed_forms(0.3),
    "growth_ode": cosmo_pins.test_growth_against_ode,
    "growth_fd": cosmo_pins.test_growth_rate_matches_finite_difference,
    "growth_weight": cosmo_pins.test_growth_weight_of_the_ray_kick,
    "nodes": ray_pins.test_half_shell_nodes,
    "interp_linear": ray_pins.test_interpolant_of_linear_fields_and_its_derivative,
    "reversible": ray_pins.test_static_step_is_time_reversible,
    "ab_autograd": lambda: ray_pins.check_ab_against_autograd(synthetic.pixel_grid(2, 0.3)[:1]),
    "readout": ray_pins.test_readout_of_rotation_times_shear,
    "free_drift": ray_pins.test_free_drift_is_exact_for_constant_momentum,
    "point_mass": _point_mass_pins,
    "power_mode": lens_pins.test_power_of_single_cosine_mode,
    "kick_snapshot": lens_pins.test_reverse_run_refers_the_ray_kick_to_the_force_snapshot,
    "power_edges": lens_pins.test_bin_edges_put_exact_edge_modes_in_upper_bin,
    "mlp_chain": mlp_pins.test_a_chain_network_is_silu_three_times,
    "mlp_silu": mlp_pins.test_silu_values,
    "rm_geometry": rm_pins.test_geometry_by_hand,
    "rm_deposit": rm_pins.test_deposit_matches_brute_force_sum,
    "rm_mode": lambda: rm_pins.test_single_mode_closed_form_with_gaussian_smoothing((rm_pins.CHI_A, rm_pins.CHI_B),
                                                                                    3e-3),
    "rm_filter": rm_pins.test_filter_on_a_mesh_periodic_mode_at_mesh_nodes,
    "rm_gather": rm_pins.test_gather_is_exact_on_bilinear_functions,
    "rm_step": rm_pins.test_ray_step_recursion_matches_finite_differences,
    "rm_tiled": lambda: [rm_pins.test_tiled_mesh_is_the_sum_of_plain_meshes_of_rotated_fields(s) for s in (1, 2, 3)],
    "tiled_gather": lambda: [ray_pins.test_tiling_equals_the_gather_of_explicitly_rotated_fields(s) for s in (5, 6, 7)],
}

# (what the slip is, module, text as written, text with the slip, pins of which one must fail)
CASES = [
    # particle-mesh force (Sec. 5.1)
    ("CIC offset taken from the upper node", pm,
     "    f = u - i0\n", "    f = i0 + 1.0 - u\n", ["cic_node", "gather_linear"]),
    ("particle mass not normalised to the mean density", pm,
     "mass = n_mesh ** 3 / n\n", "mass = 1.0\n", ["cic_mass"]),
    ("deposit mesh axes reversed", pm,
     "return rho.reshape(n_mesh, n_mesh, n_mesh)", "return rho.reshape(n_mesh, n_mesh, n_mesh).transpose(0, 2)",
     ["cic_node"]),
    ("Green's function sign", pm,
     "torch.where(k2 > 0, -pref / torch.where", "torch.where(k2 > 0, pref / torch.where", ["mode_x", "brute_plain"]),
    ("k_z^2 dropped from k^2", pm,
     "k2 = kx * kx + ky * ky + kz * kz\n    green", "k2 = kx * kx + ky * ky\n    green", ["mode_z", "brute_plain"]),
    ("sinc argument k cell instead of k cell / 2", pm,
     "sinc(kz * cell / 2)) ** (-deconv_p)", "sinc(kz * cell)) ** (-deconv_p)", ["mode_z", "brute_filtered"]),
    ("CIC window applied instead of divided out", pm,
     ") ** (-deconv_p)", ") ** deconv_p", ["mode_x", "brute_filtered"]),
    ("Gaussian smoothing without the 1/2", pm,
     "torch.exp(-0.5 * k2 * smooth * smooth)", "torch.exp(-k2 * smooth * smooth)", ["mode_x", "brute_filtered"]),
    ("derivative kept on the Nyquist planes", pm,
     "d = torch.where(nj.abs() == half, torch.zeros_like(kj), kj)", "d = kj", ["brute_plain", "brute_filtered"]),
    ("derivative axes swapped", pm,
     "for kj, nj in ((kx, nx), (ky, ny), (kz, nz)):", "for kj, nj in ((ky, ny), (kx, nx), (kz, nz)):",
     ["mode_x", "brute_plain"]),
    ("every gathered component read from the first field", pm,
     "out[:, j] += w * fl[idx]", "out[:, j] += w * flat[0][idx]", ["ewald_force"]),
    ("kick sign", pm,
     "mom = mom - g * kick", "mom = mom + g * kick", ["kd_uniform", "growth_d2"]),
    ("drift with the momentum before the kick", pm,
     "    mom = mom - g * kick\n    disp = disp + mom * drift\n",
     "    disp = disp + mom * drift\n    mom = mom - g * kick\n", ["kd_uniform"]),
    ("Zel'dovich momentum with a instead of a^2", pm,
     "(a_init ** 2 * e1 * f1 * d1) * psi", "(a_init * e1 * f1 * d1) * psi", ["zeldovich"]),
    ("Zel'dovich amplitude without the cell volume", pm,
     "delta_hat = w_hat * torch.sqrt(pk / v_cell)\n", "delta_hat = w_hat * torch.sqrt(pk)\n", ["zeldovich"]),
    ("Zel'dovich displacement sign", pm,
     "psi.append(torch.fft.irfftn(1j * d", "psi.append(torch.fft.irfftn(-1j * d", ["zeldovich_sign"]),
    ("2LPT source with the mixed derivatives added", pm,
     "hess[(i, i)] * hess[(j, j)] - hess[(i, j)] ** 2", "hess[(i, i)] * hess[(j, j)] + hess[(i, j)] ** 2",
     ["lpt_diagonal"]),
    ("2LPT displacement sign", pm,
     "psi2 = torch.stack([torch.fft.irfftn(1j * d[j]", "psi2 = torch.stack([torch.fft.irfftn(-1j * d[j]",
     ["lpt_orthogonal"]),
    ("2LPT growth D2 with the wrong sign", pm,
     "d2 = -3.0 / 7.0 * d1 * d1", "d2 = 3.0 / 7.0 * d1 * d1", ["lpt_eds", "lpt_dynamics"]),
    ("2LPT growth D2 with 1/7 for 3/7", pm,
     "d2 = -3.0 / 7.0 * d1 * d1", "d2 = -1.0 / 7.0 * d1 * d1", ["lpt_eds", "lpt_dynamics"]),
    # the particle leapfrog of the N-body driver (one force per step, Alg. 1)
    ("kick to the end of the step instead of its middle", sim,
     "kick = cosmo.kick_integral(part.a_p, a_half, om)", "kick = cosmo.kick_integral(part.a_p, a_next, om)",
     ["growth_d2", "fwd_rev"]),
    ("drift from the momentum time", sim,
     "drift = cosmo.drift_integral(part.a_x, a_next, om)", "drift = cosmo.drift_integral(part.a_p, a_next, om)",
     ["growth_d2", "fwd_rev"]),
    ("Poisson prefactor times a instead of over a", sim,
     "grads = pm_force(part, box, n_mesh, 1.5 * om / a_next, flt)\n    part = particle_sync",
     "grads = pm_force(part, box, n_mesh, 1.5 * om * a_next, flt)\n    part = particle_sync", ["growth_d2"]),
    ("synchronising kick stopped at the half step", sim,
     "kick = cosmo.kick_integral(part.a_p, part.a_x, om)",
     "kick = cosmo.kick_integral(part.a_p, 0.5 * (part.a_p + part.a_x), om)", ["fwd_rev"]),
    ("ray kick's growth correction referred to the end of the step", sim,
     "samples_per_cell,\n                                  growth_weight(a_n, om), gz=grads[2]",
     "samples_per_cell,\n                                  growth_weight(a_n1, om), gz=grads[2]", ["kick_snapshot"]),
    ("momentum time not advanced", sim,
     "return Particles(part.q, disp, mom, a_next, a_half)", "return Particles(part.q, disp, mom, a_next, part.a_p)",
     ["growth_d2", "fwd_rev"]),
    # the periodic point-mass sums that pin the PM force and the point-mass deflections (App. D)
    ("Ewald: reciprocal part with 2 pi for 4 pi", ewald,
     "amp = 4.0 * math.pi / box ** 3", "amp = 2.0 * math.pi / box ** 3", ["ewald_3d"]),
    ("Ewald: real-space Gaussian term dropped", ewald,
     "(erfc(al * s) + 2.0 * al * s / math.sqrt(math.pi) * np.exp(-(al * s) ** 2)) / s ** 3",
     "erfc(al * s) / s ** 3", ["ewald_3d"]),
    ("Ewald: reciprocal damping with 2 alpha^2", ewald,
     "math.exp(-k2 / (4.0 * al * al)) / k2\n                out", "math.exp(-k2 / (2.0 * al * al)) / k2\n                out",
     ["ewald_3d"]),
    ("Ewald 2D: reciprocal part with 4 pi for 2 pi", ewald,
     "amp = 2.0 * math.pi / box ** 2", "amp = 4.0 * math.pi / box ** 2", ["ewald_2d"]),
    ("Ewald 2D: real-space damping exp(-al |b|^2)", ewald,
     "np.exp(-al * al * s2) / s2", "np.exp(-al * s2) / s2", ["ewald_2d"]),
    # background and time integrals (Sec. 2, Sec. 3.2)
    ("Omega_m a^-2 in E(a)", cosmology,
     "om / a ** 3 + (1.0 - om)", "om / a ** 2 + (1.0 - om)", ["eds"]),
    ("comoving distance without c", cosmology,
     "    return C_LIGHT * val\n", "    return val\n", ["eds"]),
    ("drift integral with a^2", cosmology,
     "1.0 / (x ** 3 * E(x, om)), a, b", "1.0 / (x ** 2 * E(x, om)), a, b", ["eds"]),
    ("growth rate with the sign of its first term flipped", cosmology,
     "return -1.5 * om / (a ** 3 * e * e)", "return 1.5 * om / (a ** 3 * e * e)", ["eds", "growth_fd"]),
    ("growth integral with (a E)^2", cosmology,
     "1.0 / (x * E(x, om)) ** 3, 0.0, a", "1.0 / (x * E(x, om)) ** 2, 0.0, a", ["eds", "growth_ode"]),
    ("kick growth weight with a / a_c", sim,
     "/ d_c * a_c / a\n", "/ d_c * a / a_c\n", ["growth_weight"]),
    ("kick growth weight without the scale factors", sim,
     "/ d_c * a_c / a\n", "/ d_c\n", ["growth_weight"]),
    # rays (Sec. 3, Sec. 4, Alg. 1)
    ("midpoint nodes moved to the left ends", rays,
     "chi_a + (j + 0.5) * h", "chi_a + j * h", ["nodes"]),
    ("kick sign", rays,
     "c = -(2.0 / C_LIGHT) * h * r * weight_fn(chi)", "c = (2.0 / C_LIGHT) * h * r * weight_fn(chi)", ["point_mass"]),
    ("r dropped from the kick", rays,
     "c = -(2.0 / C_LIGHT) * h * r * weight_fn(chi)", "c = -(2.0 / C_LIGHT) * h * weight_fn(chi)", ["point_mass"]),
    ("ray point x from theta_y", rays,
     "X[:, 0] = observer[0] + r * theta[:, 0]", "X[:, 0] = observer[0] + r * theta[:, 1]", ["point_mass"]),
    ("interpolant derivative sign", rays,
     "dwx = (1.0 if a else -1.0) / cell", "dwx = (-1.0 if a else 1.0) / cell", ["interp_linear"]),
    ("interpolant derivative columns swapped", rays,
     "T[:, comp, 0] += dwx * wy * wz * v\n            T[:, comp, 1] += wx * dwy * wz * v",
     "T[:, comp, 1] += dwx * wy * wz * v\n            T[:, comp, 0] += wx * dwy * wz * v", ["interp_linear"]),
    ("r dropped from dK/dtheta", rays,
     "J += (c * r) * T", "J += c * T", ["ab_autograd"]),
    ("B updated with A (dK/dtheta) instead of (dK/dtheta) A", rays,
     "    eta = eta + K\n    B = B + J @ A\n    d = ", "    eta = eta + K\n    B = B + A @ J\n    d = ",
     ["ab_autograd"]),
    ("A drifted with B transposed", rays,
     "    A = A + d * B\n    chis", "    A = A + d * B.transpose(1, 2)\n    chis", ["ab_autograd"]),
    ("second half kick at the angle before the drift", rays,
     "    K, J = half_kick(theta, gx, gy, box, observer, chis, h, weight_fn, window, gz, replicas)\n    eta = eta + K\n"
     "    B = B + J @ A\n    return",
     "    K, J = half_kick(state[\"theta\"], gx, gy, box, observer, chis, h, weight_fn, window, gz, replicas)\n"
     "    eta = eta + K\n    B = B + J @ A\n    return", ["ab_autograd", "reversible"]),
    ("drift radius at the start of the step", rays,
     "d = (chi_n1 - chi_n) / (C_LIGHT * chi_h * chi_h)", "d = (chi_n1 - chi_n) / (C_LIGHT * chi_n * chi_n)",
     ["reversible"]),
    ("free drift reversed", rays,
     "d = (1.0 / chi_a - 1.0 / chi_b) / C_LIGHT", "d = (1.0 / chi_b - 1.0 / chi_a) / C_LIGHT", ["free_drift"]),
    ("convergence sign", rays,
     "kappa = 1.0 - c1", "kappa = c1 - 1.0", ["readout"]),
    ("gamma_2 sign", rays,
     "g2 = -c4 + c3 * omega", "g2 = c4 + c3 * omega", ["readout"]),
    ("rotation not divided by 1 - kappa", rays,
     "omega = c2 / (1.0 - kappa)", "omega = c2", ["readout"]),
    # convergence power spectrum (Sec. 6.2)
    ("map FFT without dtheta^2", power,
     ") * dtheta ** 2\n", ")\n", ["power_mode"]),
    ("power divided by Theta instead of Theta^2", power,
     "p = np.abs(kt) ** 2 / theta ** 2", "p = np.abs(kt) ** 2 / theta", ["power_mode"]),
    ("bin edge offset dropped", power,
     " + 1e-9\n", "\n", ["power_edges"]),
    # learned correction
    ("third hidden layer skipped", mlp,
     "h3 = silu(ra(h2) @ rw(W3).T + b3)", "h3 = h2", ["mlp_chain"]),
    ("a weight matrix transposed", mlp,
     "silu(ra(h1) @ rw(W2).T + b2)", "silu(ra(h1) @ rw(W2) + b2)", ["mlp_chain"]),
    ("bias unpacked before its weights", mlp,
     "    W1 = take(H * IN, (H, IN))[:, :3]\n    b1 = take(H, (H,))\n",
     "    b1 = take(H, (H,))\n    W1 = take(H * IN, (H, IN))[:, :3]\n", ["mlp_chain"]),
    ("sigmoid for SiLU", mlp,
     "return z / (1.0 + torch.exp(-z))", "return 1.0 / (1.0 + torch.exp(-z))", ["mlp_silu", "mlp_chain"]),
    # the ray-mesh kick (Sec. 5.2, App. C)
    ("no Gaussian smoothing", raymesh,
     "filt = filt * np.exp(-0.5 * (kx ** 2 + ky ** 2) * lam * lam)", "filt = filt", ["rm_mode", "rm_filter"]),
    ("sinc^-2 deconvolution", raymesh,
     "(np.sinc(kx * x2d / (2 * math.pi)) ** -4) * (np.sinc(ky * x2d / (2 * math.pi)) ** -4)",
     "(np.sinc(kx * x2d / (2 * math.pi)) ** -2) * (np.sinc(ky * x2d / (2 * math.pi)) ** -2)", ["rm_filter"]),
    ("smoothing length x2d instead of lambda", raymesh,
     "(kx ** 2 + ky ** 2) * lam * lam)", "(kx ** 2 + ky ** 2) * x2d * x2d)", ["rm_mode"]),
    ("lambda off by 2", raymesh,
     "lam = max(2.0 * cell / (abs(chi_a) + abs(chi_b)), mu)", "lam = max(cell / (abs(chi_a) + abs(chi_b)), mu)",
     ["rm_geometry"]),
    ("r dropped from the kick", raymesh,
     "w = -(2.0 / C_LIGHT) * r * weight_fn(chi) * sgn", "w = -(2.0 / C_LIGHT) * weight_fn(chi) * sgn",
     ["rm_deposit"]),
    ("half-cell offset of the projected nodes", raymesh,
     "ux = ((idx + ia * box - observer[0]) / r) / x2d + n2d / 2\n",
     "ux = ((idx + ia * box - observer[0]) / r) / x2d + n2d / 2 + 0.5\n", ["rm_deposit"]),
    ("gather derivative columns swapped", raymesh,
     "T[:, c, 0] += sx * wy * v\n                T[:, c, 1] += wx * sy * v",
     "T[:, c, 1] += sx * wy * v\n                T[:, c, 0] += wx * sy * v", ["rm_gather"]),
    ("replica: sky component without its sign", raymesh,
     "return sg[0] * g[p[0]][b[0], b[1], b[2]], sg[1]", "return g[p[0]][b[0], b[1], b[2]], sg[1]", ["rm_tiled"]),
    ("replica: shift taken on the sky axis", raymesh,
     "b[p[0]] = ((sg[0] * ii + sh[p[0]]) % n)[:, None]", "b[p[0]] = ((sg[0] * ii + sh[0]) % n)[:, None]",
     ["rm_tiled"]),
    ("replica: z sign dropped", raymesh,
     "b[p[2]] = (sg[2] * (kz % n) + sh[p[2]]) % n", "b[p[2]] = ((kz % n) + sh[p[2]]) % n", ["rm_tiled"]),
    ("replica: index off by one", raymesh,
     "    k = kz // n\n", "    k = kz // n + 1\n", ["rm_tiled"]),
    ("replica frame: coordinate without its sign", rays,
     "vals = torch.remainder(sign[:, a] * u[:, a] + torch.gather", "vals = torch.remainder(u[:, a] + torch.gather",
     ["tiled_gather"]),
    ("replica frame: shift taken on the sky axis", rays,
     "torch.gather(shift, 1, dst[:, None])[:, 0] * cell", "shift[:, a] * cell", ["tiled_gather"]),
    ("replica frame: derivative with one sign", rays,
     "T[:, a, b] = sign[:, a] * sign[:, b] * D3", "T[:, a, b] = sign[:, a] * D3", ["tiled_gather"]),
    ("replica frame: derivative indices transposed", rays,
     "D3[rows, perm[:, a], perm[:, b]]", "D3[rows, perm[:, b], perm[:, a]]", ["tiled_gather"]),
    ("B updated with A T instead of T A", raymesh,
     "    eta = eta + val\n    B = B + T @ A\n    d = ", "    eta = eta + val\n    B = B + A @ T\n    d = ", ["rm_step"]),
]


def _plant(monkeypatch, mod, old, new):
    """Load a copy of ``mod`` with ``old`` replaced by ``new`` and put it wherever the oracle's modules and the
    pin files refer to ``mod``."""
    with open(mod.__file__) as f:
        src = f.read()
    assert src.count(old) == 1, f"{mod.__name__}: the text to edit must occur once: {old!r}"
    bad = types.ModuleType(mod.__name__)
    bad.__file__ = mod.__file__
    bad.__package__ = mod.__package__
    exec(compile(src.replace(old, new), f"{mod.__file__} (planted)", "exec"), bad.__dict__)
    monkeypatch.setitem(sys.modules, mod.__name__, bad)
    for m in list(sys.modules.values()):
        name = getattr(m, "__name__", "") or ""
        if m is mod or not (name.startswith("oracle") or name.startswith("test_oracle")):
            continue
        for attr, val in list(vars(m).items()):
            if val is mod:
                monkeypatch.setattr(m, attr, bad)


def test_the_pins_pass_on_the_oracle_as_it_stands():
    for name in sorted({p for case in CASES for p in case[4]}):
        PINS[name]()


@pytest.mark.parametrize("case", CASES, ids=[f"{c[1].__name__.split('.')[-1]}: {c[0]}" for c in CASES])
def test_a_planted_mistake_fails_a_pin(case, monkeypatch):
    what, mod, old, new, pins = case
    _plant(monkeypatch, mod, old, new)
    for name in pins:
        try:
            PINS[name]()
        except AssertionError:
            return
    pytest.fail(f"no pin fails with the mistake planted: {what}")
