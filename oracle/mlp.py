"""FP64 restatement of the learned force correction g = 1 + MLP(x) (test infrastructure only).

x = (|k| cell, a, ln N_mesh); three hidden layers of 64 SiLU units (SiLU(z) = z / (1 + e^-z)) and a linear
output y; g = 1 + y multiplies the Green's function of the ray fields, the analogue of the force-sharpening
factor of Sec. 6.2.  Parameters are packed as W1 [64][16] (input columns 3..15 unused), b1 [64], W2 [64][64],
b2 [64], W3 [64][64], b3 [64], W4 [64], b4.  ``round_weights`` / ``round_acts`` reproduce the arithmetic of the
tensor-core forward: weights W1..W4 and the inputs of layers 1-3 rounded to bfloat16, everything else exact.
"""
from __future__ import annotations

import torch

H, IN = 64, 16
N_PARAMS = H * IN + H + H * H + H + H * H + H + H + 1


def unpack(p: torch.Tensor):
    p = p.to(torch.float64)
    i = 0

    def take(n, shape):
        nonlocal i
        t = p[i:i + n].reshape(shape)
        i += n
        return t
    W1 = take(H * IN, (H, IN))[:, :3]
    b1 = take(H, (H,))
    W2 = take(H * H, (H, H))
    b2 = take(H, (H,))
    W3 = take(H * H, (H, H))
    b3 = take(H, (H,))
    W4 = take(H, (H,))
    b4 = take(1, (1,))
    return W1, b1, W2, b2, W3, b3, W4, b4


def _bf16(t: torch.Tensor) -> torch.Tensor:
    """Value rounded to bfloat16 (round to nearest even), derivative 1 kept in float64 (a cast to bfloat16 under
    autograd would also round the gradient)."""
    r = t.detach().to(torch.bfloat16).to(torch.float64)
    return t + (r - t.detach())


def silu(z):
    return z / (1.0 + torch.exp(-z))


def forward(x: torch.Tensor, p: torch.Tensor, round_weights: bool = True, round_acts: bool = True) -> torch.Tensor:
    """g = 1 + MLP(x) for x of shape (rows, 3)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    rw = _bf16 if round_weights else (lambda t: t)
    ra = _bf16 if round_acts else (lambda t: t)
    x = x.to(torch.float64)
    h1 = silu(ra(x) @ rw(W1).T + b1)
    h2 = silu(ra(h1) @ rw(W2).T + b2)
    h3 = silu(ra(h2) @ rw(W3).T + b3)
    return 1.0 + h3 @ rw(W4) + b4
