"""Pins of the oracle's warm-start network (CPU): the convolution's tap
layout against its loop definition, the gradient against finite
differences, the architecture's parameter count and its pooling/upsampling
inverse relation."""
import numpy as np
import pytest
import torch

from oracle import unet as U


def test_conv3_layout_matches_definition(rng):
    ci, co, D = 2, 3, 5
    x = rng.standard_normal((ci, D, D, D))
    W = rng.standard_normal((co, ci, 27))
    b = rng.standard_normal(co)
    ref = U.conv3_direct(x, W, b)
    got = torch.nn.functional.conv3d(torch.as_tensor(x)[None], torch.as_tensor(W).reshape(co, ci, 3, 3, 3),
                                     torch.as_tensor(b), padding=1)[0].numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_num_weights():
    # c = 16, counted by hand: 880 + 6928 + 13856 + 27680 + 55360 + 110656 +
    # 82976 + 27680 + 20752 + 6928 + 17
    assert U.num_weights(16) == 353713
    assert U.num_weights(1) == sum(co * ci * (27 if k == 3 else 1) + co
                                   for ci, co, k in U.layer_dims(1))


def test_gradient_matches_finite_differences(rng):
    c, D, B = 1, 8, 2
    n = U.num_weights(c)
    # weights exactly representable in BF16, so the rounding inside unpack
    # does not move them
    w = (rng.integers(-64, 64, n) / 64.0).astype(np.float32)
    x = rng.standard_normal((B, 2, D, D, D))
    x[:, 1] = (rng.random((B, D, D, D)) > 0.3)
    t = rng.standard_normal((B, D, D, D))
    params = [(W.detach().clone().requires_grad_(True), bb.detach().clone().requires_grad_(True))
              for W, bb in U.unpack(w, c)]
    flat = [p for pair in params for p in pair]

    def f(*ps):
        it = iter(ps)
        pr = [(next(it), next(it)) for _ in params]
        y = U.forward(torch.as_tensor(x), pr)
        return U.loss(y, torch.as_tensor(t), torch.as_tensor(x[:, 1]))

    assert torch.autograd.gradcheck(f, tuple(flat), eps=1e-6, atol=1e-6, rtol=1e-4)


def test_loss_and_grad_is_consistent(rng):
    c, D, B = 1, 8, 1
    w = (rng.integers(-64, 64, U.num_weights(c)) / 64.0).astype(np.float32)
    x = rng.standard_normal((B, 2, D, D, D))
    x[:, 1] = 1.0
    t = rng.standard_normal((B, D, D, D))
    L, g, y = U.loss_and_grad(w, c, x, t)
    assert np.isclose(L, np.mean((y - t) ** 2))
    assert g.shape == (U.num_weights(c),)
    # the output bias gradient is the mean residual times 2
    assert np.isclose(g[-1], 2 * np.mean(y - t))


def test_up_then_pool_is_identity(rng):
    x = torch.as_tensor(rng.standard_normal((1, 3, 4, 4, 4)))
    y = torch.nn.functional.avg_pool3d(torch.nn.functional.interpolate(x, scale_factor=2, mode="nearest"), 2)
    assert (x - y).abs().max() <= 4e-16 * x.abs().max()
