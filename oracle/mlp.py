"""Oracle of the IPM warm-start network (TEST INFRASTRUCTURE; shares no code
with the CUDA path): the 3-layer perceptron of include/rlqr_mlp.h in FP64
numpy, optionally rounding to BF16 at the points where the GPU stores BF16
(inputs, weights and biases, hidden activations, the backward signals), its
mean-squared loss, the gradient by the chain rule, and one Adam step.

Parameter vector (FP32 master order): W1 [width][16] (columns >= n_in zero),
b1 [width], W2 [width][width], b2 [width], W3 [npad][width] (rows >= n_out
zero), b3 [npad], npad = n_out rounded up to 16.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), through FP32 (the GPU
    rounds FP32 values): keep the upper 16 bits of the FP32 pattern after
    adding half an ulp of BF16 plus the tie-breaking bit."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def layout(n_out, width):
    npad = (n_out + 15) // 16 * 16
    W = width
    o = {}
    o["W1"] = (0, (W, 16))
    o["b1"] = (W * 16, (W,))
    o["W2"] = (W * 17, (W, W))
    o["b2"] = (W * 17 + W * W, (W,))
    o["W3"] = (W * 18 + W * W, (npad, W))
    o["b3"] = (W * 18 + W * W + npad * W, (npad,))
    total = W * 18 + W * W + npad * W + npad
    return o, npad, total


def unpack(p, n_out, width):
    o, npad, total = layout(n_out, width)
    assert p.size == total
    return {k: p[s:s + int(np.prod(sh))].reshape(sh) for k, (s, sh) in o.items()}


def pack(parts, n_out, width):
    o, npad, total = layout(n_out, width)
    p = np.zeros(total)
    for k, (s, sh) in o.items():
        p[s:s + int(np.prod(sh))] = np.asarray(parts[k], float).ravel()
    return p


def forward(p, x, n_out, width, rounding=True):
    """Returns (y [rows][n_out], cache)."""
    r = bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    P = {k: r(v) for k, v in unpack(p, n_out, width).items()}
    rows, n_in = x.shape
    a0 = np.zeros((rows, 16))
    a0[:, :n_in] = x
    a0 = r(a0)
    h1 = r(np.maximum(0.0, a0 @ P["W1"].T + P["b1"]))
    h2 = r(np.maximum(0.0, h1 @ P["W2"].T + P["b2"]))
    y = h2 @ P["W3"].T + P["b3"]
    return y[:, :n_out], dict(P=P, a0=a0, h1=h1, h2=h2, y=y)


def loss_and_grad(p, x, t, n_out, width, rounding=True):
    """Mean of (y - t)^2 over rows and the n_out columns, and its gradient in
    the parameter order (the backward signals rounded to BF16 where the GPU
    stores them)."""
    r = bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    y, c = forward(p, x, n_out, width, rounding)
    rows = x.shape[0]
    d = y - t
    loss = float(np.mean(d * d))
    npad = c["y"].shape[1]
    dy = np.zeros((rows, npad))
    dy[:, :n_out] = 2.0 * d / (rows * n_out)
    dy = r(dy)
    g = {"W3": dy.T @ c["h2"], "b3": dy.sum(axis=0)}
    dz2 = r((dy @ c["P"]["W3"]) * (c["h2"] > 0))
    g["W2"], g["b2"] = dz2.T @ c["h1"], dz2.sum(axis=0)
    dz1 = r((dz2 @ c["P"]["W2"]) * (c["h1"] > 0))
    g["W1"], g["b1"] = dz1.T @ c["a0"], dz1.sum(axis=0)
    return loss, pack(g, n_out, width)


def abs_scales(p, x, t, n_out, width):
    """Per-element magnitudes for element-wise comparisons: for the output and
    every gradient entry, the sum of the absolute values of the terms that
    form it (the same chain rule as loss_and_grad with |.| on every factor,
    no rounding).  An FP32-accumulated value agrees with its FP64 oracle to a
    few units of roundoff times this scale; BF16 storage of an intermediate
    adds about 2^-8 times it."""
    y, c = forward(p, x, n_out, width, rounding=False)
    P = {k: np.abs(v) for k, v in c["P"].items()}
    a0, h1, h2 = np.abs(c["a0"]), np.abs(c["h1"]), np.abs(c["h2"])
    rows = x.shape[0]
    ys = h2 @ P["W3"].T + P["b3"]
    npad = c["y"].shape[1]
    dy = np.zeros((rows, npad))
    dy[:, :n_out] = 2.0 * (np.abs(y) + np.abs(t)) / (rows * n_out)
    g = {"W3": dy.T @ h2, "b3": dy.sum(axis=0)}
    dz2 = (dy @ P["W3"]) * (c["h2"] > 0)
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"]) * (c["h1"] > 0)
    g["W1"], g["b1"] = dz1.T @ a0, dz1.sum(axis=0)
    return ys[:, :n_out], pack(g, n_out, width)


def adam(p, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (Kingma and Ba, 2015); returns new p, m, v."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
