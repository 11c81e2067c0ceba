"""FP64 CPU reference of the warm-start network (test infrastructure only).

The learned warm start of the Poisson solve maps three node fields of the RZ
grid -- charge density, radius, electrode potential -- to a guess of phi.  The
network is a small U-Net on the node grid (sizes 2^k m + 1 nest by taking
every other node):

  level l = 0..3 with channels C = (16, 32, 64, 64):
    encoder:  x -> relu(conv3(x)) -> relu(conv3(.)) = skip_l ; next level gets
              the even nodes of skip_l
    decoder:  up(level l+1 output) (bilinear node interpolation), concatenated
              with skip_l -> relu(conv3(.)) -> relu(conv3(.))
    head:     conv1x1 (16 -> 1) on the level-0 decoder output
  conv3 = 3x3 convolution with zero padding and a bias.

Inputs (channels): rho / rho_ref, r / R, boundary potential / V_ref; output
phi / V_ref.  This module defines the parameter layout shared by name with
the CUDA implementation's tests and computes the forward pass, the MSE loss
and its gradients in FP64 with torch CPU primitives (conv2d, autograd).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CHANNELS = (16, 32, 64, 64)
IN_CHANNELS = 3


def layer_shapes(channels=CHANNELS, cin=IN_CHANNELS):
    """Ordered (name, weight shape (cout, cin, kh, kw)) of every convolution."""
    c = channels
    out = [("enc0a", (c[0], cin, 3, 3)), ("enc0b", (c[0], c[0], 3, 3))]
    for l in range(1, len(c)):
        out += [(f"enc{l}a", (c[l], c[l - 1], 3, 3)), (f"enc{l}b", (c[l], c[l], 3, 3))]
    for l in range(len(c) - 2, -1, -1):
        out += [(f"dec{l}a", (c[l], c[l + 1] + c[l], 3, 3)), (f"dec{l}b", (c[l], c[l], 3, 3))]
    out.append(("head", (1, c[0], 1, 1)))
    return out


def init_params(seed: int = 0, channels=CHANNELS, cin=IN_CHANNELS) -> dict:
    """He-normal weights, zero biases (numpy FP64)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in layer_shapes(channels, cin):
        fan_in = shp[1] * shp[2] * shp[3]
        p[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=shp)
        p[name + ".b"] = np.zeros(shp[0])
    return p


def n_params(p: dict) -> int:
    return int(sum(v.size for v in p.values()))


def _down(x):
    return x[:, :, ::2, ::2]


def _up(x, shape):
    """Bilinear interpolation from a coarse node grid to the fine one
    (coarse node k sits on fine node 2k)."""
    H, W = shape
    out = torch.zeros(x.shape[0], x.shape[1], H, W, dtype=x.dtype)
    out[:, :, ::2, ::2] = x
    out[:, :, 1::2, ::2] = 0.5 * (x[:, :, :-1, :] + x[:, :, 1:, :])
    out[:, :, ::2, 1::2] = 0.5 * (x[:, :, :, :-1] + x[:, :, :, 1:])
    out[:, :, 1::2, 1::2] = 0.25 * (x[:, :, :-1, :-1] + x[:, :, 1:, :-1] + x[:, :, :-1, 1:] +
                                    x[:, :, 1:, 1:])
    return out


def forward(params: dict, x, channels=CHANNELS):
    """x: (batch, 3, H, W) tensor (FP64); returns (batch, 1, H, W)."""
    t = {k: (v if torch.is_tensor(v) else torch.as_tensor(v)) for k, v in params.items()}
    L = len(channels)

    def conv(name, h, pad=1):
        return F.conv2d(h, t[name + ".w"], t[name + ".b"], padding=pad)

    skips = []
    h = x
    for l in range(L):
        if l > 0:
            h = _down(skips[-1])
        h = F.relu(conv(f"enc{l}a", h))
        h = F.relu(conv(f"enc{l}b", h))
        skips.append(h)
    h = skips[-1]
    for l in range(L - 2, -1, -1):
        u = _up(h, skips[l].shape[2:])
        h = F.relu(conv(f"dec{l}a", torch.cat([u, skips[l]], dim=1)))
        h = F.relu(conv(f"dec{l}b", h))
    return conv("head", h, pad=0)


def loss_and_grads(params: dict, x: np.ndarray, y: np.ndarray):
    """Mean squared error over nodes and its gradient for every parameter."""
    t = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in params.items()}
    out = forward(t, torch.as_tensor(x, dtype=torch.float64))
    loss = ((out - torch.as_tensor(y, dtype=torch.float64)) ** 2).mean()
    loss.backward()
    return float(loss), {k: v.grad.numpy() for k, v in t.items()}
