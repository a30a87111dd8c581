"""FP64 CPU reference of the learned warm-start network (test infrastructure
only: the tests compare the CUDA layer kernels and the whole network's
gradients against it; the product never imports it).

The network maps a cell's material field to a temperature correction
relative to the linear profile between the walls (the temperature-difference
axis is z).  Layers follow one written specification shared with the CUDA
path only through this docstring:

  input  x: 7 channels = 6 tensor components (xx, yy, zz, yz, xz, xy) divided
            by the largest diagonal entry, and the linear profile T_lin(z)
  channels per level c_0 = 32, c_1, ..., c_L (default 32, 64, 128)
  encoder level i: [avgpool2 if i > 0], conv3(. -> c_i) relu, conv3(c_i -> c_i)
            relu -> s_i
  decoder level i = L-1 .. 0: upsample2, concat[up, s_i],
            conv3(c_(i+1) + c_i -> c_i) relu, conv3(c_i -> c_i) relu
  conv1(32->1)                                          -> dT, T = T_lin + dT

conv3: 3x3x3 cross-correlation with bias, periodic (circular) padding in x
and y, zero padding in z.  relu: leaky, slope 0.01 below zero.  avgpool2: mean of 2x2x2 blocks.  upsample2:
nearest neighbour.  Loss: mean squared error of T over all voxels.

Plain PyTorch CPU ops in float64; reverse-mode differentiation of those ops
gives the reference gradients.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CHANS = (32, 64, 128)


def conv_layers(chans=CHANS, cin=7):
    """(cin, cout) of the 3x3x3 convolutions in order: two per encoder level,
    two per decoder level."""
    L = len(chans) - 1
    layers = [(cin, chans[0]), (chans[0], chans[0])]
    for i in range(1, L + 1):
        layers += [(chans[i - 1], chans[i]), (chans[i], chans[i])]
    for i in range(L - 1, -1, -1):
        layers += [(chans[i + 1] + chans[i], chans[i]), (chans[i], chans[i])]
    return layers


CONV3 = conv_layers()
HEAD = (32, 1)


def init_params(seed: int = 0, chans=CHANS):
    """He-normal weights (torch layout [Cout, Cin, 3, 3, 3]) and zero biases."""
    g = np.random.default_rng(seed)
    params = []
    for ci, co in conv_layers(chans):
        w = g.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci))
        params.append((w, np.zeros(co)))
    ci, co = HEAD
    params.append((g.standard_normal((co, ci, 1, 1, 1)) * np.sqrt(1.0 / ci), np.zeros(co)))
    return params


def conv3(x, w, b):
    """x [N, C, D, H, W]; circular pad in H, W (y, x), zero pad in D (z)."""
    xp = F.pad(x, (1, 1, 1, 1, 0, 0), mode="circular")
    xp = F.pad(xp, (0, 0, 0, 0, 1, 1))
    return F.conv3d(xp, w, b)


def forward(params, x, chans=CHANS):
    """x: torch float64 [N, 7, D, H, W] -> dT [N, 1, D, H, W]."""
    p = [(torch.as_tensor(w), torch.as_tensor(b)) for w, b in params]
    L = len(chans) - 1
    k = 0
    h = x
    skips = []
    for i in range(L + 1):
        if i > 0:
            h = F.avg_pool3d(h, 2)
        h = F.leaky_relu(conv3(h, *p[k]), 0.01); k += 1
        h = F.leaky_relu(conv3(h, *p[k]), 0.01); k += 1
        skips.append(h)
    for i in range(L - 1, -1, -1):
        h = F.interpolate(h, scale_factor=2, mode="nearest")
        h = torch.cat([h, skips[i]], dim=1)
        h = F.leaky_relu(conv3(h, *p[k]), 0.01); k += 1
        h = F.leaky_relu(conv3(h, *p[k]), 0.01); k += 1
    return F.conv3d(h, *p[k])


def loss_and_grads(params, x, t_lin, target, chans=CHANS):
    """MSE of T = T_lin + dT against target; returns (loss, [(dW, db), ...])."""
    p = [(torch.tensor(w, requires_grad=True), torch.tensor(b, requires_grad=True))
         for w, b in params]
    dT = forward([(w, b) for w, b in p], torch.as_tensor(x), chans)
    T = torch.as_tensor(np.array(t_lin)) + dT
    loss = ((T - torch.as_tensor(target)) ** 2).mean()
    loss.backward()
    return float(loss.detach()), [(w.grad.numpy(), b.grad.numpy()) for w, b in p]


def conv3_np(x_ndhwc, w_t, b):
    """Single layer in the device layout: x [N, D, H, W, Cin], w_t torch
    layout [Cout, Cin, 3, 3, 3] -> y [N, D, H, W, Cout] (no activation)."""
    x = torch.as_tensor(np.moveaxis(x_ndhwc, -1, 1))
    y = conv3(x, torch.as_tensor(w_t), torch.as_tensor(b))
    return np.moveaxis(y.numpy(), 1, -1)
