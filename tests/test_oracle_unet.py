"""Pins of the FP64 surrogate reference (oracle/unet.py): the convolution
against a direct loop over its definition, pooling/upsampling against their
adjoints, and the full backward pass against central finite differences."""
import numpy as np
import pytest

from oracle import unet as U


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 5, 6, 3))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = U.conv(x, W, b)
    ref = np.zeros_like(y)
    for n in range(2):
        for i in range(5):
            for j in range(6):
                for o in range(4):
                    s = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            ii, jj = i + ky - 1, j + kx - 1
                            if 0 <= ii < 5 and 0 <= jj < 6:
                                s += W[o, ky, kx] @ x[n, ii, jj]
                    ref[n, i, j, o] = s
    assert np.abs(y - ref).max() < 1e-12


def test_adjoints():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 4, 6, 3))
    y = rng.normal(size=(2, 2, 3, 3))
    assert abs((U.pool(x) * y).sum() - (x * U.pool_backward(y)).sum()) < 1e-12
    z = rng.normal(size=(2, 8, 12, 3))
    assert abs((U.up(x) * z).sum() - (x * U.up_backward(z)).sum()) < 1e-12
    # conv: <conv(x) - b, dy> = <x, dx>, and dW, db as derivatives of the bilinear form
    W = rng.normal(size=(5, 3, 3, 3))
    dy = rng.normal(size=(2, 4, 6, 5))
    dx, dW, db = U.conv_backward(x, W, dy)
    lhs = ((U.conv(x, W, np.zeros(5))) * dy).sum()
    assert abs(lhs - (x * dx).sum()) < 1e-10
    assert abs(lhs - (W * dW).sum()) < 1e-10


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = U.init_params(7) + 0.0
    sl, total = U.layer_slices()
    params[[bo + k for _, _, co, _, _, bo in sl for k in range(co)]] = 0.05 * rng.normal(
        size=sum(l[2] for l in sl))
    x = rng.normal(size=(1, 8, 16, 3))
    t = rng.normal(size=(1, 8, 16, 3))
    m = (rng.uniform(size=(1, 8, 16)) > 0.2).astype(float)
    y, cache = U.forward(params, x)
    g = U.backward(params, cache, y, t, m)
    # a few parameters of every layer (weights and biases)
    idx = []
    for name, ci, co, relu, wo, bo in sl:
        idx += list(rng.integers(wo, wo + 9 * ci * co, size=3)) + [bo + int(rng.integers(0, co))]
    h = 1e-5
    for k in idx:
        p1, p2 = params.copy(), params.copy()
        p1[k] += h
        p2[k] -= h
        fd = (U.loss(U.forward(p1, x)[0], t, m) - U.loss(U.forward(p2, x)[0], t, m)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(g[k])) + 1e-9, (k, fd, g[k])
