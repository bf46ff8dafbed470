"""Pins of the warm-start network's oracle (oracle/mlp.py), CPU only: BF16
rounding against torch's bfloat16 conversion, the chain-rule gradient
against central differences (FP64, no rounding), the packing order, and the
first Adam step against its closed form."""
import numpy as np
import torch

import oracle.mlp as M


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-20, 20, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 65504.0]]).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16_round(a), ref)


def _problem(seed, n_in=7, width=32, n_out=20, rows=24):
    rng = np.random.default_rng(seed)
    o, npad, total = M.layout(n_out, width)
    parts = {"W1": np.zeros((width, 16)), "b1": rng.normal(size=width) * 0.1,
             "W2": rng.normal(size=(width, width)) / np.sqrt(width),
             "b2": rng.normal(size=width) * 0.1, "W3": np.zeros((npad, width)),
             "b3": np.zeros(npad)}
    parts["W1"][:, :n_in] = rng.normal(size=(width, n_in))
    parts["W3"][:n_out] = rng.normal(size=(n_out, width)) / np.sqrt(width)
    parts["b3"][:n_out] = rng.normal(size=n_out) * 0.1
    p = M.pack(parts, n_out, width)
    x = rng.normal(size=(rows, n_in))
    t = rng.normal(size=(rows, n_out))
    return p, x, t, n_out, width


def test_gradient_matches_central_differences():
    p, x, t, n_out, width = _problem(1)
    loss, g = M.loss_and_grad(p, x, t, n_out, width, rounding=False)
    rng = np.random.default_rng(2)
    o, npad, total = M.layout(n_out, width)
    live = [i for i in range(total) if abs(p[i]) > 0 or i >= o["b1"][0] and i < o["W2"][0]
            or i >= o["b2"][0] and i < o["W3"][0] or i >= o["b3"][0] and i < o["b3"][0] + n_out]
    h = 1e-6
    for i in rng.choice(live, 60, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        fp = M.loss_and_grad(p + e, x, t, n_out, width, rounding=False)[0]
        fm = M.loss_and_grad(p - e, x, t, n_out, width, rounding=False)[0]
        assert abs((fp - fm) / (2 * h) - g[i]) <= 1e-6 * max(1.0, abs(g[i]))
    # the padding never receives a gradient
    assert np.all(g[o["b3"][0] + n_out:] == 0)
    W1g = g[:width * 16].reshape(width, 16)
    assert np.all(W1g[:, x.shape[1]:] == 0)


def test_pack_unpack_roundtrip_and_sizes():
    p, *_ , n_out, width = _problem(3)
    parts = M.unpack(p, n_out, width)
    np.testing.assert_array_equal(M.pack(parts, n_out, width), p)
    assert M.layout(902, 256)[2] == 256 * 18 + 256 * 256 + 912 * 256 + 912


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(4)
    p, g = rng.normal(size=50), rng.normal(size=50)
    p1, m1, v1 = M.adam(p, np.zeros(50), np.zeros(50), g, 1, 1e-3)
    np.testing.assert_allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)
