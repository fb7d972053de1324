"""Pins of the network oracle: each operation against its definition written
as loops on tiny inputs, and the autograd gradients against finite
differences."""
import itertools

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import unet_oracle as U

torch.manual_seed(0)


def test_param_count():
    assert U.param_count() == 523654


def test_circular_conv3_against_loops():
    x = torch.randn(1, 2, 4, 3, 5, dtype=torch.float64)
    w = torch.randn(3, 2, 3, 3, 3, dtype=torch.float64)
    b = torch.randn(3, dtype=torch.float64)
    y = U.conv3_circ(x, w, b)
    _, ci, nz, ny, nx = x.shape
    for co in range(3):
        for z, yy, xx in itertools.product(range(nz), range(ny), range(nx)):
            acc = float(b[co])
            for c, kz, ky, kx in itertools.product(range(ci), range(3), range(3), range(3)):
                acc += float(w[co, c, kz, ky, kx]) * float(
                    x[0, c, (z + kz - 1) % nz, (yy + ky - 1) % ny, (xx + kx - 1) % nx])
            assert abs(float(y[0, co, z, yy, xx]) - acc) < 1e-12


def test_transposed_conv_and_pool_against_loops():
    x = torch.randn(1, 3, 2, 3, 2, dtype=torch.float64)
    w = torch.randn(3, 4, 2, 2, 2, dtype=torch.float64)
    b = torch.randn(4, dtype=torch.float64)
    y = F.conv_transpose3d(x, w, b, stride=2)
    assert y.shape == (1, 4, 4, 6, 4)
    for co in range(4):
        for z, yy, xx in itertools.product(range(4), range(6), range(4)):
            acc = float(b[co]) + sum(float(x[0, c, z // 2, yy // 2, xx // 2]) *
                                     float(w[c, co, z % 2, yy % 2, xx % 2]) for c in range(3))
            assert abs(float(y[0, co, z, yy, xx]) - acc) < 1e-12
    p = F.avg_pool3d(y, 2)
    for co in range(4):
        for z, yy, xx in itertools.product(range(2), range(3), range(2)):
            blk = y[0, co, 2 * z:2 * z + 2, 2 * yy:2 * yy + 2, 2 * xx:2 * xx + 2]
            assert abs(float(p[0, co, z, yy, xx]) - float(blk.mean())) < 1e-12


def test_network_gradients_against_finite_differences():
    flat = U.init_params(1)
    gen = torch.Generator().manual_seed(11)
    x = torch.randn(1, 4, 8, 8, 8, dtype=torch.float64, generator=gen)
    t = torch.randn(1, 6, 8, 8, 8, dtype=torch.float64, generator=gen)
    flat.requires_grad_(True)
    loss = U.loss(U.forward(flat, x), t)
    g, = torch.autograd.grad(loss, flat)
    rng = np.random.default_rng(2)
    idx = rng.choice(flat.numel(), size=24, replace=False)
    with torch.no_grad():
        for i in idx:
            h = 1e-7           # small step: the leaky ReLU kink is crossed with negligible probability
            fp = flat.clone(); fp[i] += h
            fm = flat.clone(); fm[i] -= h
            fd = (U.loss(U.forward(fp, x), t) - U.loss(U.forward(fm, x), t)) / (2 * h)
            assert abs(float(fd) - float(g[i])) <= 1e-5 * max(1.0, abs(float(g[i]))) + 1e-7


def test_adam_first_step_moves_by_lr():
    flat = torch.zeros(5, dtype=torch.float64)
    g = torch.tensor([1.0, -2.0, 0.5, 0.0, 3.0], dtype=torch.float64)
    m = torch.zeros(5, dtype=torch.float64)
    v = torch.zeros(5, dtype=torch.float64)
    U.adam_step(flat, g, m, v, 1, lr=1e-3)
    # bias-corrected first step is lr * sign(g) (up to eps)
    assert torch.allclose(flat, -1e-3 * torch.sign(g), atol=1e-9)
