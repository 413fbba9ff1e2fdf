"""Writes cosmo_1024_recipe_128p.npz: FP64 oracle outputs of the 1024^3 workload's recipe scaled to 128^3 particles,
256^3 mesh and 512^2 rays (same box, field of view, time grids and source planes), for the GPU parity test of the
full recipe.  Only ``oracle/`` computes the values; ``synthetic`` supplies the seeded inputs and ``configs`` the
sizes.  Runs about six minutes on eight cores:

    python tests/golden/make_cosmo_1024_recipe_128p.py

Stored: particles at a = 1 at 4096 sampled indices; per source plane the binned kappa power spectrum (all bins),
the kappa, gamma1, gamma2, omega maps at 4096 sampled pixels, the rms of the full kappa map and, per sampled pixel,
the nearest approach of any of its line-of-sight nodes so far to a transverse cell face (in cells: where the
interpolant's derivative jumps); the final ray angles at 4096 sampled rays and the largest deflection over all
rays.
"""
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synthetic  # noqa: E402
from oracle import power as opow  # noqa: E402
from oracle import sim  # noqa: E402
from paper_2405_12913_gb300.configs import COSMO_1024_SCALED as W  # noqa: E402

N_SAMPLE = 4096
SAMPLE_SEED = 4242


def main():
    torch.set_num_threads(os.cpu_count())
    noise = synthetic.white_noise(W.seed, W.n_side)
    theta0 = synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE)
    c = sim.Cosmo(W.omega_m, W.h, W.n_s, W.sigma8)
    flt = sim.Filter(W.deconv_p, W.smooth_cells)
    part = sim.initial_particles(noise, W.box, c, W.a_init)
    part, grads = sim.run_forward(part, W.forward_grid, W.box, W.n_mesh, c, flt)
    ip = synthetic.sample_indices(SAMPLE_SEED, W.n_side ** 3, N_SAMPLE)
    out = {"particle_index": ip, "disp": part.disp.numpy()[ip], "mom": part.mom.numpy()[ip],
           "mom_absmax": np.abs(part.mom.numpy()).max()}
    res = sim.run_reverse(part, grads, W.reverse_grid, W.box, W.n_mesh, c, flt, torch.tensor(theta0), W.observer,
                          set(W.source_steps), W.samples_per_cell, face_distance=True)
    ir = synthetic.sample_indices(SAMPLE_SEED + 1, W.n_rays, N_SAMPLE)
    out["ray_index"] = ir
    lmin, lmax = W.ell_range
    for s in W.source_steps:
        maps = np.stack([res.maps[s][i].numpy() for i in range(4)])
        out[f"maps_{s}"] = maps[:, ir]
        out[f"kappa_rms_{s}"] = maps[0].std()
        out[f"face_min_{s}"] = res.face_min[s].numpy()[ir]
        ell, p, cnt = opow.kappa_power(maps[0].reshape(W.n_pix, W.n_pix), W.dtheta, W.nbins, lmin, lmax)
        out[f"ell_{s}"], out[f"power_{s}"], out[f"count_{s}"] = ell, p, cnt
    th = res.rays["theta"].numpy()
    out["theta"] = th[ir]
    out["alpha_absmax"] = np.abs(theta0 - th).max()
    np.savez_compressed(os.path.join(HERE, "cosmo_1024_recipe_128p.npz"), **out)


if __name__ == "__main__":
    main()
