"""Pins of the oracle's gradients (the reference for the adjoint kernels) against FP64 finite differences.

The convergence map of the discrete method is piecewise smooth in the parameters: the A/B recursion uses the
transverse derivative of the trilinear force interpolant, which jumps when a line-of-sight sample crosses a mesh
cell face.  Finite differences therefore match autograd at steps below the spacing of those crossings; the final
ray angles are continuous and match at ordinary steps."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import sim as osim

W_ARGS = dict(n_side=8, n_mesh=16, box=32.0, a_init=0.1, n_forward=3, a_min=0.7, n_reverse=3, n_pix=16, fov=6.0)


def _run(noise, om, theta0):
    a = W_ARGS
    c = osim.Cosmo(om)
    flt = osim.Filter()
    part = osim.initial_particles(noise, a["box"], c, a["a_init"])
    fg = [a["a_init"] + (1 - a["a_init"]) * i / a["n_forward"] for i in range(a["n_forward"] + 1)]
    rg = [1 - (1 - a["a_min"]) * i / a["n_reverse"] for i in range(a["n_reverse"] + 1)]
    part, grads = osim.run_forward(part, fg, a["box"], a["n_mesh"], c, flt)
    obs = (0.5 * a["box"], 0.5 * a["box"], 0.0)
    res = osim.run_reverse(part, grads, rg, a["box"], a["n_mesh"], c, flt, theta0, obs, {a["n_reverse"]})
    return res.maps[a["n_reverse"]][0], res.rays["theta"]


def test_oracle_gradient_matches_small_step_differences():
    noise = synthetic.white_noise(5, W_ARGS["n_side"])
    theta0 = torch.tensor(synthetic.pixel_grid(W_ARGS["n_pix"], W_ARGS["fov"] * synthetic.DEGREE))
    kbar = torch.tensor(synthetic.gaussian_field(6, (W_ARGS["n_pix"] ** 2,)))
    tbar = torch.tensor(synthetic.gaussian_field(7, (W_ARGS["n_pix"] ** 2, 2)))
    direction = torch.tensor(synthetic.gaussian_field(8, (W_ARGS["n_side"],) * 3))
    w = torch.tensor(noise, requires_grad=True)
    k, th = _run(w, 0.3, theta0)
    ((k * kbar).sum() + 1e4 * (th * tbar).sum()).backward()
    ad = float((w.grad * direction).sum())
    with torch.no_grad():
        def loss(eps, smooth_only=False):
            kk, tt = _run(torch.tensor(noise) + eps * direction, 0.3, theta0)
            return float(1e4 * (tt * tbar).sum()) if smooth_only else float((kk * kbar).sum() + 1e4 * (tt * tbar).sum())
        vals = sorted((loss(e) - loss(-e)) / (2 * e) for e in (1e-6, 1.4e-6, 2e-6))
        assert ad == pytest.approx(vals[1], rel=1e-6)
    # the deflection part alone is smooth: an ordinary step agrees too
    w2 = torch.tensor(noise, requires_grad=True)
    _, th2 = _run(w2, 0.3, theta0)
    (1e4 * (th2 * tbar).sum()).backward()
    ad2 = float((w2.grad * direction).sum())
    with torch.no_grad():
        fd2 = (loss(1e-3, True) - loss(-1e-3, True)) / 2e-3
    # theta is continuous but its derivative has kinks at the cell faces: agreement to the kink density
    assert ad2 == pytest.approx(fd2, rel=5e-3)
