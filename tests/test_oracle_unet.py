"""Pins of the FP64 reference U-Net (oracle/unet.py) against facts that do not
come from its own code: finite differences of the loss, the exact action of
shift and identity kernels (orientation and zero padding of the 3x3
convolution), exactness of the bilinear node interpolation on bilinear
functions, and a closed-form loss/gradient for a network whose convolutions
are all zero.
"""
import numpy as np
import pytest
import torch

from oracle import unet

pytestmark = pytest.mark.filterwarnings("ignore::UserWarning")

TINY = (2, 3, 4, 4)


def _tiny_params(seed=0):
    p = unet.init_params(seed, channels=TINY)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * rng.normal(size=p[k].shape)
    return p


def _loss(p, x, y):
    with torch.no_grad():
        out = unet.forward(p, torch.as_tensor(x), channels=TINY)
    return float(((out.numpy() - y) ** 2).mean())


def test_gradients_match_central_differences():
    # 17 x 17 nodes: levels 17, 9, 5, 3
    rng = np.random.default_rng(5)
    p = _tiny_params(3)
    x = rng.normal(size=(2, 3, 17, 17))
    y = rng.normal(size=(2, 1, 17, 17))
    t = {k: torch.tensor(v, requires_grad=True) for k, v in p.items()}
    out = unet.forward(t, torch.as_tensor(x), channels=TINY)
    loss = ((out - torch.as_tensor(y)) ** 2).mean()
    loss.backward()
    grads = {k: v.grad.numpy() for k, v in t.items()}
    h = 1e-6
    checked = 0
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            q = {k: v.copy() for k, v in p.items()}
            q[name].reshape(-1)[idx] += h
            lp = _loss(q, x, y)
            q[name].reshape(-1)[idx] -= 2 * h
            lm = _loss(q, x, y)
            fd = (lp - lm) / (2 * h)
            g = grads[name].reshape(-1)[idx]
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (name, idx, fd, g)
            checked += 1
    assert checked > 40


def test_loss_and_grads_agree_with_forward():
    rng = np.random.default_rng(2)
    p = _tiny_params(4)
    x = rng.normal(size=(1, 3, 9, 17))
    y = rng.normal(size=(1, 1, 9, 17))
    # loss_and_grads with the default channel list needs the default shapes;
    # check the tiny network through forward() and the definition of the MSE
    out = unet.forward(p, torch.as_tensor(x), channels=TINY).numpy()
    assert out.shape == (1, 1, 9, 17)
    assert _loss(p, x, y) == pytest.approx(((out - y) ** 2).mean(), rel=1e-15)


def test_shift_kernel_orientation_and_zero_padding():
    """A 3x3 kernel with a single one at (kh, kw) maps x to x shifted by
    (kh - 1, kw - 1) (cross-correlation), zero outside the grid."""
    import torch.nn.functional as F
    rng = np.random.default_rng(0)
    x = torch.as_tensor(rng.normal(size=(1, 1, 6, 7)))
    for kh in range(3):
        for kw in range(3):
            w = torch.zeros(1, 1, 3, 3, dtype=torch.float64)
            w[0, 0, kh, kw] = 1.0
            out = F.conv2d(x, w, None, padding=1)[0, 0].numpy()
            xs = x[0, 0].numpy()
            for i in range(6):
                for j in range(7):
                    si, sj = i + kh - 1, j + kw - 1
                    want = xs[si, sj] if 0 <= si < 6 and 0 <= sj < 7 else 0.0
                    assert out[i, j] == want


def test_identity_path_reproduces_input_channel():
    """Convolutions that pass channel 0 straight through (centre tap one,
    everything else zero) and a head reading channel 0 give relu(x0) back
    whenever x0 >= 0 on the coarse levels' nodes too."""
    p = unet.init_params(0, channels=TINY)
    for k in p:
        p[k] = np.zeros_like(p[k])
    for name, shp in unet.layer_shapes(channels=TINY):
        if shp[2] == 3:
            p[name + ".w"][0, 0, 1, 1] = 1.0
    # the decoders see [up(h), skip]: channel 0 of the concatenation is the
    # upsampled coarse path; also pass the skip (channel C_{l+1}) through
    for l in range(len(TINY) - 1):
        p[f"dec{l}a.w"][0, :, 1, 1] = 0.0
        p[f"dec{l}a.w"][0, TINY[l + 1], 1, 1] = 1.0
    p["head.w"][0, 0, 0, 0] = 1.0
    rng = np.random.default_rng(1)
    x = np.abs(rng.normal(size=(1, 3, 9, 9)))
    with torch.no_grad():
        out = unet.forward(p, torch.as_tensor(x), channels=TINY).numpy()
    assert np.array_equal(out[0, 0], x[0, 0])


def test_bilinear_upsampling_is_exact_on_bilinear_functions():
    I, J = np.meshgrid(np.arange(5.0), np.arange(7.0), indexing="ij")
    a, b, c, d = 0.3, -1.2, 0.7, 0.25
    coarse = a + b * I + c * J + d * I * J
    fi, fj = np.meshgrid(np.arange(9.0) / 2, np.arange(13.0) / 2, indexing="ij")
    fine = a + b * fi + c * fj + d * fi * fj
    up = unet._up(torch.as_tensor(coarse)[None, None], (9, 13))[0, 0].numpy()
    assert np.allclose(up, fine, rtol=0, atol=1e-14)


def test_zero_network_closed_form():
    """All convolution weights and biases zero, head bias c: the output is c
    everywhere, the loss is mean((c - y)^2), d loss / d c = 2 mean(c - y),
    and every other gradient is zero (relu'(0) = 0)."""
    p = unet.init_params(0)
    for k in p:
        p[k] = np.zeros_like(p[k])
    c = 0.37
    p["head.b"][0] = c
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 3, 17, 33))
    y = rng.normal(size=(2, 1, 17, 33))
    loss, g = unet.loss_and_grads(p, x, y)
    assert loss == pytest.approx(((c - y) ** 2).mean(), rel=1e-14)
    assert g["head.b"][0] == pytest.approx(2 * (c - y).mean(), rel=1e-12)
    for k, v in g.items():
        if k != "head.b":
            assert not np.any(v), k


def test_parameter_count_near_three_hundred_thousand():
    n = unet.n_params(unet.init_params(0))
    assert n == 302849
    # the conv layers of the full network, counted from the level structure:
    # encoder 3->16->16, 16->32->32, 32->64->64, 64->64->64; decoder
    # (64+64)->64->64, (64+32)->32->32, (32+16)->16->16; head 16->1
    convs = [(3, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 64), (64, 64),
             (128, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]
    assert n == sum(ci * co * 9 + co for ci, co in convs) + 16 + 1
