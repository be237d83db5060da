"""FP64 CPU reference of the surrogate network (TEST INFRASTRUCTURE ONLY).

The surrogate maps steady-flow inputs (obstacle mask, relaxation time, force)
on an H x W grid to the steady (rho, u) fields.  Architecture (the one the GPU
kernels implement): a 4-level U-Net with widths 32/64/128/256; every level has
two 3x3 convolutions (zero padding 1, bias) each followed by ReLU; 2x2 average
pooling going down; nearest-neighbour 2x upsampling followed by a 3x3
conv + ReLU going up; concatenation [up path, skip] before the two decoder
convolutions; a linear 3x3 head with 3 outputs.  Loss: weighted mean squared
error sum(m (y - t)^2) / (3 sum m) with per-pixel weights m.  The input has
cin channels (3 by default).  Every convolution pads with zeros along y (the
height); along x (the width) it pads with zeros, or, with periodic_x, wraps
around, which is the padding of a channel periodic in x.

Tensors are NHWC float64.  Parameters use the canonical flat layout shared
with the CUDA library: for each layer in LAYERS order, W[co][ky][kx][ci]
followed by b[co].

This module is plain numpy, written from the definitions above; it shares no
code with the CUDA path.  Pins (tests/test_oracle_unet.py): the convolution
equals the direct sum over taps and channels, the backward pass is the exact
adjoint of the forward one, and the gradient matches finite differences.
"""
from __future__ import annotations

import numpy as np

BASE = 32
# (name, input channels, output channels, relu) for a 3-channel input
LAYERS = [
    ("enc1a", 3, 32, True), ("enc1b", 32, 32, True),
    ("enc2a", 32, 64, True), ("enc2b", 64, 64, True),
    ("enc3a", 64, 128, True), ("enc3b", 128, 128, True),
    ("bota", 128, 256, True), ("botb", 256, 256, True),
    ("up3", 256, 128, True), ("dec3a", 256, 128, True), ("dec3b", 128, 128, True),
    ("up2", 128, 64, True), ("dec2a", 128, 64, True), ("dec2b", 64, 64, True),
    ("up1", 64, 32, True), ("dec1a", 64, 32, True), ("dec1b", 32, 32, True),
    ("head", 32, 3, False),
]


def layers(cin=3):
    """LAYERS with cin input channels in the first layer."""
    return [(LAYERS[0][0], cin) + LAYERS[0][2:]] + LAYERS[1:]


def layer_slices(cin=3):
    """(name, cin, cout, relu, w_offset, b_offset) for each layer, and the total."""
    out, off = [], 0
    for name, ci, co, relu in layers(cin):
        out.append((name, ci, co, relu, off, off + 9 * ci * co))
        off += 9 * ci * co + co
    return out, off


def unpack(params, cin=3):
    sl, total = layer_slices(cin)
    assert params.size == total
    P = {}
    for name, ci, co, relu, wo, bo in sl:
        P[name] = (params[wo:wo + 9 * ci * co].reshape(co, 3, 3, ci), params[bo:bo + co])
    return P


def pack(P, cin=3):
    sl, total = layer_slices(cin)
    out = np.zeros(total)
    for name, ci, co, relu, wo, bo in sl:
        W, b = P[name]
        out[wo:wo + 9 * ci * co] = W.ravel()
        out[bo:bo + co] = b
    return out


def _pad(x, periodic_x):
    """One halo cell on each side: zeros along y; along x zeros, or the
    opposite edge's column when periodic_x."""
    N, H, W, C = x.shape
    xp = np.zeros((N, H + 2, W + 2, C))
    xp[:, 1:-1, 1:-1] = x
    if periodic_x:
        xp[:, 1:-1, 0] = x[:, :, W - 1]
        xp[:, 1:-1, W + 1] = x[:, :, 0]
    return xp


def _cols(x, periodic_x=False):
    """im2col of a 3x3, pad-1 convolution: (N, H, W, 9, C), tap index ky*3+kx."""
    N, H, W, C = x.shape
    xp = _pad(x, periodic_x)
    return np.stack([xp[:, ky:ky + H, kx:kx + W] for ky in range(3) for kx in range(3)], axis=3)


def conv(x, W, b, periodic_x=False):
    """y[n,i,j,o] = b[o] + sum_{ky,kx,c} W[o,ky,kx,c] x[n, i+ky-1, j+kx-1, c]
    (x[n, i', j', c] = 0 outside the grid along y; along x too, or taken at
    j' mod W when periodic_x)."""
    N, H, Wd, C = x.shape
    co = W.shape[0]
    cols = _cols(x, periodic_x).reshape(N * H * Wd, 9 * C)
    return (cols @ W.reshape(co, 9 * C).T + b).reshape(N, H, Wd, co)


def conv_backward(x, W, dy, periodic_x=False):
    """Gradients of conv: (dx, dW, db)."""
    N, H, Wd, C = x.shape
    co = W.shape[0]
    cols = _cols(x, periodic_x).reshape(N * H * Wd, 9 * C)
    g = dy.reshape(N * H * Wd, co)
    dW = (g.T @ cols).reshape(co, 3, 3, C)
    db = g.sum(axis=0)
    dcols = (g @ W.reshape(co, 9 * C)).reshape(N, H, Wd, 3, 3, C)
    dxp = np.zeros((N, H + 2, Wd + 2, C))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + H, kx:kx + Wd] += dcols[:, :, :, ky, kx]
    dx = dxp[:, 1:-1, 1:-1].copy()
    if periodic_x:
        # the halo columns are copies of the opposite edge: their gradient
        # belongs there
        dx[:, :, Wd - 1] += dxp[:, 1:-1, 0]
        dx[:, :, 0] += dxp[:, 1:-1, Wd + 1]
    return dx, dW, db


def pool(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) * 0.25


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(dy):
    N, H, W, C = dy.shape
    return dy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def relu(z):
    return np.maximum(z, 0.0)


def bf16(a):
    """Round to bfloat16, nearest-even, through float32 (the precision in
    which the GPU kernels hold a value before storing it as bfloat16)."""
    f = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x, storage="fp64", periodic_x=False):
    """Returns (y, cache).  storage="bf16" rounds the weights, the input and
    every stored activation to bfloat16 where the GPU stores them (the
    arithmetic stays FP64; biases and the head's output are not rounded).
    The input's last axis gives cin."""
    P = unpack(params, x.shape[-1])
    cache = {}
    rnd = bf16 if storage == "bf16" else (lambda a: a)
    relu_of = dict((l[0], l[3]) for l in LAYERS)

    def layer(name, inp):
        W, b = P[name]
        z = conv(inp, rnd(W), b, periodic_x)
        cache[name] = (inp, z)
        return rnd(relu(z)) if relu_of[name] else z

    x = rnd(x)
    pool_ = lambda a: rnd(pool(a))
    e1 = layer("enc1b", layer("enc1a", x))
    e2 = layer("enc2b", layer("enc2a", pool_(e1)))
    e3 = layer("enc3b", layer("enc3a", pool_(e2)))
    bb = layer("botb", layer("bota", pool_(e3)))
    u3 = layer("up3", up(bb))
    d3 = layer("dec3b", layer("dec3a", np.concatenate([u3, e3], axis=3)))
    u2 = layer("up2", up(d3))
    d2 = layer("dec2b", layer("dec2a", np.concatenate([u2, e2], axis=3)))
    u1 = layer("up1", up(d2))
    d1 = layer("dec1b", layer("dec1a", np.concatenate([u1, e1], axis=3)))
    y = layer("head", d1)
    return y, cache


def loss(y, t, m):
    """sum m (y - t)^2 / (3 sum m), m: (N, H, W) weights."""
    return float((m[..., None] * (y - t) ** 2).sum() / (3.0 * m.sum()))


def backward(params, cache, y, t, m, storage="fp64", periodic_x=False):
    """Gradient of loss(forward(params, x), t, m) with respect to params (the
    exact derivative of the forward pass).  With storage="bf16" the weights
    are the rounded ones the forward pass used, and every gradient the GPU
    stores in bfloat16 is rounded where it is stored (the arithmetic stays
    FP64): the loss gradient at the head's output; each layer's dz (the
    gradient at its pre-activation, after its ReLU's gate); the input
    gradient of a layer whose input is pooled or upsampled, before the
    pooling or upsampling adjoint; and the skip part of a concatenation,
    gated by the encoder's ReLU, before the pooling path is added to it."""
    cin = cache["enc1a"][0].shape[-1]
    P = unpack(params, cin)
    rnd = bf16 if storage == "bf16" else (lambda a: a)
    if storage == "bf16":
        P = {k: (bf16(W), b) for k, (W, b) in P.items()}
    relu_of = dict((l[0], l[3]) for l in LAYERS)
    grads = {}
    dy = rnd(2.0 * m[..., None] * (y - t) / (3.0 * m.sum()))

    def gate(name, d):
        """d times the derivative of layer `name`'s ReLU at its pre-activation"""
        return d * (cache[name][1] > 0) if relu_of[name] else d

    def back(name, dout):
        """the layer's dz (dout gated, as stored), its weight and bias
        gradients, and the gradient at its input (not gated, not rounded)"""
        inp, z = cache[name]
        dz = rnd(gate(name, dout))
        dx, dW, db = conv_backward(inp, P[name][0], dz, periodic_x)
        grads[name] = (dW, db)
        return dx

    dd1 = back("dec1a", back("dec1b", back("head", dy)))
    du1, de1 = dd1[..., :32], rnd(gate("enc1b", dd1[..., 32:]))
    dd2 = up_backward(rnd(back("up1", du1)))
    dd2 = back("dec2a", back("dec2b", dd2))
    du2, de2 = dd2[..., :64], rnd(gate("enc2b", dd2[..., 64:]))
    dd3 = up_backward(rnd(back("up2", du2)))
    dd3 = back("dec3a", back("dec3b", dd3))
    du3, de3 = dd3[..., :128], rnd(gate("enc3b", dd3[..., 128:]))
    dbb = up_backward(rnd(back("up3", du3)))
    dp3 = rnd(back("bota", back("botb", dbb)))
    de3 = de3 + pool_backward(dp3)
    dp2 = rnd(back("enc3a", back("enc3b", de3)))
    de2 = de2 + pool_backward(dp2)
    dp1 = rnd(back("enc2a", back("enc2b", de2)))
    de1 = de1 + pool_backward(dp1)
    back("enc1a", back("enc1b", de1))
    return pack(grads, cin)


def init_params(seed: int, cin=3):
    """He-normal weights (std sqrt(2 / (9 cin))), zero biases, drawn with the
    project's seeded generator (lbm_workloads.SplitMix64)."""
    import lbm_workloads as W
    rng = W.SplitMix64(seed)
    sl, total = layer_slices(cin)
    out = np.zeros(total)
    for name, ci, co, relu_, wo, bo in sl:
        std = np.sqrt(2.0 / (9 * ci)) if relu_ else np.sqrt(1.0 / (9 * ci))
        out[wo:wo + 9 * ci * co] = rng.normal(9 * ci * co) * std
    return out
