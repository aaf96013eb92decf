"""CPU reference of the learned warm start's network (float64 PyTorch ops).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs use it.

The network is the one the library's sea_unet_* entry points describe: a
3-level 3D U-Net of width c on D^3 patches (D = 32 in the library; any
multiple of 4 here), input channels (b / s, box mask), output v / s.

  e1 = relu(conv3(x; 2 -> c)),  s1 = relu(conv3(e1; c -> c))
  e2 = relu(conv3(pool(s1); c -> 2c)),  s2 = relu(conv3(e2; 2c -> 2c))
  b4 = relu(conv3(pool(s2); 2c -> 4c)),  b5 = relu(conv3(b4; 4c -> 4c))
  d2 = relu(conv3(cat(up(b5), s2); 6c -> 2c)),  d2' = relu(conv3(d2; 2c -> 2c))
  d1 = relu(conv3(cat(up(d2'), s1); 3c -> c)),  d1' = relu(conv3(d1; c -> c))
  y  = conv1(d1'; c -> 1)

conv3: 3x3x3 cross-correlation with zero padding, tap k = 9 kz + 3 ky + kx
at offset (kz - 1, ky - 1, kx - 1) in (z, y, x); pool: 2x average; up:
nearest 2x.  Weights as the library stores them: per layer W[cout][cin][k]
then b[cout] in one flat array; the library computes with W rounded to
BF16 (round to nearest even) and b as FP32, so ``unpack`` applies the same
rounding.  Loss: sum m (y - t)^2 / sum m, m = input channel 1.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F


def layer_dims(c: int):
    """(cin, cout, k) per layer, in storage order."""
    return [(2, c, 3), (c, c, 3), (c, 2 * c, 3), (2 * c, 2 * c, 3), (2 * c, 4 * c, 3),
            (4 * c, 4 * c, 3), (6 * c, 2 * c, 3), (2 * c, 2 * c, 3), (3 * c, c, 3), (c, c, 3),
            (c, 1, 1)]


def num_weights(c: int) -> int:
    return sum(co * ci * (27 if k == 3 else 1) + co for ci, co, k in layer_dims(c))


def unpack(w, c: int, requires_grad=False):
    """Flat FP32 weights -> [(W, b)] float64 tensors (W rounded to BF16)."""
    w = torch.as_tensor(np.asarray(w, dtype=np.float32))
    out, off = [], 0
    for ci, co, k in layer_dims(c):
        nw = co * ci * (27 if k == 3 else 1)
        W = w[off:off + nw].to(torch.bfloat16).to(torch.float64)
        W = W.reshape(co, ci, 3, 3, 3) if k == 3 else W.reshape(co, ci, 1, 1, 1)
        off += nw
        b = w[off:off + co].to(torch.float64)
        off += co
        if requires_grad:
            W.requires_grad_(True)
            b.requires_grad_(True)
        out.append((W, b))
    return out


def forward(x, params):
    """x: [B][2][D][D][D] float64 -> y: [B][D][D][D]."""
    def c3(t, i, relu=True):
        W, b = params[i]
        y = F.conv3d(t, W, b, padding=1 if W.shape[-1] == 3 else 0)
        return F.relu(y) if relu else y

    e1 = c3(x, 0)
    s1 = c3(e1, 1)
    e2 = c3(F.avg_pool3d(s1, 2), 2)
    s2 = c3(e2, 3)
    b4 = c3(F.avg_pool3d(s2, 2), 4)
    b5 = c3(b4, 5)
    d2 = c3(torch.cat([F.interpolate(b5, scale_factor=2, mode="nearest"), s2], dim=1), 6)
    d2 = c3(d2, 7)
    d1 = c3(torch.cat([F.interpolate(d2, scale_factor=2, mode="nearest"), s1], dim=1), 8)
    d1 = c3(d1, 9)
    return c3(d1, 10, relu=False)[:, 0]


def loss(y, t, mask):
    return ((mask * (y - t) ** 2).sum()) / mask.sum().clamp_min(1e-300)


def loss_and_grad(w, c: int, x, t):
    """Loss and its gradient w.r.t. the flat weights (float64), the
    gradient of W taken w.r.t. the BF16-rounded values the forward uses."""
    params = unpack(w, c, requires_grad=True)
    x = torch.as_tensor(np.asarray(x, dtype=np.float64))
    t = torch.as_tensor(np.asarray(t, dtype=np.float64))
    y = forward(x, params)
    L = loss(y, t, x[:, 1])
    L.backward()
    g = []
    for W, b in params:
        g.append(W.grad.reshape(-1))
        g.append(b.grad.reshape(-1))
    return float(L.detach()), torch.cat(g).numpy(), y.detach().numpy()


def conv3_direct(x, W, b):
    """The conv3 of one batch element by its definition (loops; tiny inputs)."""
    ci_n, D = x.shape[0], x.shape[1]
    co_n = W.shape[0]
    y = np.zeros((co_n, D, D, D))
    for co in range(co_n):
        for z in range(D):
            for yy in range(D):
                for xx in range(D):
                    s = b[co]
                    for ci in range(ci_n):
                        for k in range(27):
                            kz, ky, kx = k // 9, (k // 3) % 3, k % 3
                            gz, gy, gx = z + kz - 1, yy + ky - 1, xx + kx - 1
                            if 0 <= gz < D and 0 <= gy < D and 0 <= gx < D:
                                s += W[co, ci, k] * x[ci, gz, gy, gx]
                    y[co, z, yy, xx] = s
    return y
