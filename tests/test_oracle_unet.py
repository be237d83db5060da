"""Pins of the FP64 surrogate reference (oracle/unet.py): the convolution
(zero and periodic padding along x) against a direct loop over its
definition and against shift equivariance, pooling/upsampling/convolution
against their adjoints, and the full backward pass against central finite
differences."""
import numpy as np
import pytest

from oracle import unet as U


@pytest.mark.parametrize("periodic_x", [False, True])
def test_conv_matches_direct_sum(periodic_x):
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 5, 6, 3))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = U.conv(x, W, b, periodic_x)
    ref = np.zeros_like(y)
    for n in range(2):
        for i in range(5):
            for j in range(6):
                for o in range(4):
                    s = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            ii, jj = i + ky - 1, j + kx - 1
                            if periodic_x:
                                jj %= 6
                            if 0 <= ii < 5 and 0 <= jj < 6:
                                s += W[o, ky, kx] @ x[n, ii, jj]
                    ref[n, i, j, o] = s
    assert np.abs(y - ref).max() < 1e-12


def test_periodic_conv_commutes_with_shifts_along_x():
    """A periodic channel has no preferred x origin: shifting the input along
    x shifts the output (zero padding along x breaks this at the edges)."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=(1, 4, 8, 2))
    W = rng.normal(size=(3, 3, 3, 2))
    b = rng.normal(size=3)
    for s in (1, 3, 7):
        assert np.abs(U.conv(np.roll(x, s, axis=2), W, b, True) - np.roll(U.conv(x, W, b, True), s, axis=2)).max() < 1e-12
    assert np.abs(U.conv(np.roll(x, 1, axis=2), W, b) - np.roll(U.conv(x, W, b), 1, axis=2)).max() > 1e-3


@pytest.mark.parametrize("periodic_x", [False, True])
def test_adjoints(periodic_x):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 4, 6, 3))
    y = rng.normal(size=(2, 2, 3, 3))
    assert abs((U.pool(x) * y).sum() - (x * U.pool_backward(y)).sum()) < 1e-12
    z = rng.normal(size=(2, 8, 12, 3))
    assert abs((U.up(x) * z).sum() - (x * U.up_backward(z)).sum()) < 1e-12
    # conv: <conv(x) - b, dy> = <x, dx>, and dW, db as derivatives of the bilinear form
    W = rng.normal(size=(5, 3, 3, 3))
    dy = rng.normal(size=(2, 4, 6, 5))
    dx, dW, db = U.conv_backward(x, W, dy, periodic_x)
    lhs = ((U.conv(x, W, np.zeros(5), periodic_x)) * dy).sum()
    assert abs(lhs - (x * dx).sum()) < 1e-10
    assert abs(lhs - (W * dW).sum()) < 1e-10


@pytest.mark.parametrize("cin,periodic_x", [(3, False), (5, True)])
def test_gradient_matches_finite_differences(cin, periodic_x):
    rng = np.random.default_rng(2)
    params = U.init_params(7, cin) + 0.0
    sl, total = U.layer_slices(cin)
    params[[bo + k for _, _, co, _, _, bo in sl for k in range(co)]] = 0.05 * rng.normal(
        size=sum(l[2] for l in sl))
    x = rng.normal(size=(1, 8, 16, cin))
    t = rng.normal(size=(1, 8, 16, 3))
    m = (rng.uniform(size=(1, 8, 16)) > 0.2).astype(float)
    y, cache = U.forward(params, x, periodic_x=periodic_x)
    g = U.backward(params, cache, y, t, m, periodic_x=periodic_x)
    # a few parameters of every layer (weights and biases)
    idx = []
    for name, ci, co, relu, wo, bo in sl:
        idx += list(rng.integers(wo, wo + 9 * ci * co, size=3)) + [bo + int(rng.integers(0, co))]
    # the loss is piecewise smooth (ReLU): where a pre-activation crosses zero
    # within +-h the central difference straddles a kink, but one of the
    # one-sided differences still equals the derivative on its side
    h = 1e-6
    f0 = U.loss(U.forward(params, x, periodic_x=periodic_x)[0], t, m)
    for k in idx:
        p1, p2 = params.copy(), params.copy()
        p1[k] += h
        p2[k] -= h
        f1 = U.loss(U.forward(p1, x, periodic_x=periodic_x)[0], t, m)
        f2 = U.loss(U.forward(p2, x, periodic_x=periodic_x)[0], t, m)
        tol = 1e-5 * max(1e-3, abs(g[k])) + 1e-9
        errs = [abs((f1 - f2) / (2 * h) - g[k]), abs((f1 - f0) / h - g[k]), abs((f0 - f2) / h - g[k])]
        assert min(errs) <= tol, (k, errs, g[k])


def _small_problem(seed=4, H=16, W=24, n=2, cin=3):
    rng = np.random.default_rng(seed)
    params = U.init_params(seed, cin)
    sl, _ = U.layer_slices(cin)
    for name, ci, co, relu, wo, bo in sl:
        params[bo:bo + co] = 0.05 * rng.normal(size=co)
    x = rng.normal(size=(n, H, W, cin))
    t = rng.normal(size=(n, H, W, 3))
    m = (rng.uniform(size=(n, H, W)) > 0.2).astype(np.float64)
    return params, x, t, m


def _per_layer(g, ref, cin=3):
    sl, _ = U.layer_slices(cin)
    w = {name: np.linalg.norm(g[wo:bo] - ref[wo:bo]) / np.linalg.norm(ref[wo:bo]) for name, ci, co, r, wo, bo in sl}
    b = {name: np.linalg.norm(g[bo:bo + co] - ref[bo:bo + co]) / np.linalg.norm(ref[bo:bo + co])
         for name, ci, co, r, wo, bo in sl}
    return w, b


def test_bf16_gradient_rounds_only_what_is_stored():
    """With BF16 storage emulated, the stored gradients are rounded: the
    result differs from the unrounded gradient by about BF16's resolution,
    not more (no term dropped on the way)."""
    params, x, t, m = _small_problem()
    y, cache = U.forward(params, x, storage="bf16")
    g_r = U.backward(params, cache, y, t, m, storage="bf16")
    P = U.unpack(params)
    exact = {k: (U.bf16(Wt), b) for k, (Wt, b) in P.items()}
    g_u = U.backward(U.pack(exact), cache, y, t, m)   # same rounded weights, unrounded gradients
    w, b = _per_layer(g_r, g_u)
    assert max(w.values()) < 2e-2 and max(b.values()) < 2e-2, (w, b)
    assert max(w.values()) > 1e-4


@pytest.mark.parametrize("layer", ["dec2b", "enc1b", "head"])
def test_gradient_bar_catches_a_dropped_tap(layer, monkeypatch):
    """The GPU gradient test's bar (per-layer relative L2 below 2e-2, weights
    and biases apart) against a planted mistake in the oracle: one of the
    nine taps dropped from one layer's input gradient (the adjoint
    convolution) moves the gradients of that layer's inputs by far more."""
    params, x, t, m = _small_problem()
    y, cache = U.forward(params, x, storage="bf16")
    ref = U.backward(params, cache, y, t, m, storage="bf16")
    real = U.conv_backward
    target = U.unpack(params)[layer][0].shape

    def dropped(xin, Wt, dz, periodic_x=False):
        dx, dW, db = real(xin, Wt, dz, periodic_x)
        if Wt.shape == target:
            W2 = Wt.copy()
            W2[:, 1, 2] = 0.0          # tap (ky, kx) = (1, 2) missing from the adjoint
            dx = real(xin, W2, dz, periodic_x)[0]
        return dx, dW, db

    monkeypatch.setattr(U, "conv_backward", dropped)
    bad = U.backward(params, cache, y, t, m, storage="bf16")
    w, b = _per_layer(bad, ref)
    worst = max(max(w.values()), max(b.values()))
    assert worst > 5e-2, (layer, w, b)
