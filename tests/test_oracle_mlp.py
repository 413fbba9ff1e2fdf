"""Pins of the oracle's learned-correction network (the reference for the tensor-core MLP kernels)."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp


def _params(seed, last=True):
    rng = np.random.default_rng(seed)
    p = torch.tensor(rng.standard_normal(mlp.N_PARAMS) * 0.2)
    if not last:
        p[-65:] = 0.0
    return p


def test_zero_output_layer_is_the_plain_kernel():
    x = torch.rand(50, 3, dtype=torch.float64) * torch.tensor([5.0, 1.0, 6.0])
    g = mlp.forward(x, _params(1, last=False))
    assert torch.equal(g, torch.ones(50, dtype=torch.float64))


def test_a_chain_network_is_silu_three_times():
    # parameters packed in the stated order (W1 [64][16], b1, W2 [64][64], b2, W3, b3, W4, b4) that route input
    # column 1 through hidden units 0 -> 1 -> 2 with unit weights: g = 1 + silu(silu(silu(x_1))) + b4
    H, IN = 64, 16
    p = torch.zeros(mlp.N_PARAMS, dtype=torch.float64)
    o = 0
    p[o + 0 * IN + 1] = 1.0          # W1[0][1]
    o += H * IN + H
    p[o + 1 * H + 0] = 1.0           # W2[1][0]
    o += H * H + H
    p[o + 2 * H + 1] = 1.0           # W3[2][1]
    o += H * H + H
    p[o + 2] = 1.0                   # W4[2]
    o += H
    p[o] = 0.25                      # b4
    assert o + 1 == mlp.N_PARAMS
    x = torch.rand(10, 3, dtype=torch.float64) * 4 - 2
    silu = torch.nn.functional.silu
    want = 1.0 + silu(silu(silu(x[:, 1]))) + 0.25
    assert torch.allclose(mlp.forward(x, p, False, False), want, rtol=1e-14, atol=1e-15)


def test_silu_values():
    assert float(mlp.silu(torch.tensor(0.0))) == 0.0
    z = torch.tensor([-3.0, 0.5, 4.0], dtype=torch.float64)
    assert torch.allclose(mlp.silu(z), z * torch.sigmoid(z), rtol=1e-15)


def test_output_is_affine_in_the_last_layer():
    x = torch.rand(20, 3, dtype=torch.float64)
    p = _params(2)
    q = p.clone()
    q[-65:] *= 3.0
    g1, g3 = mlp.forward(x, p, False, False), mlp.forward(x, q, False, False)
    assert torch.allclose(g3 - 1.0, 3.0 * (g1 - 1.0), rtol=1e-12)


def test_autograd_matches_central_differences():
    x = torch.rand(8, 3, dtype=torch.float64) * 3
    p = _params(3).requires_grad_(True)
    w = torch.tensor(np.random.default_rng(4).standard_normal(8))
    (mlp.forward(x, p, False, False) * w).sum().backward()
    idx = [0, 5, 1100, 5200, 9400, 9472]
    for i in idx:
        e = 1e-6
        pp, pm = p.detach().clone(), p.detach().clone()
        pp[i] += e
        pm[i] -= e
        fd = float(((mlp.forward(x, pp, False, False) - mlp.forward(x, pm, False, False)) * w).sum()) / (2 * e)
        assert float(p.grad[i]) == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_bfloat16_rounding_stays_small():
    x = torch.rand(64, 3, dtype=torch.float64) * torch.tensor([5.0, 1.0, 5.5])
    p = _params(5)
    g_exact = mlp.forward(x, p, False, False)
    g_bf16 = mlp.forward(x, p, True, True)
    assert float((g_bf16 - g_exact).abs().max()) < 0.05 * float((g_exact - 1).abs().max())
