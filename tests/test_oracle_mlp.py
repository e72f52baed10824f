"""Pins for the oracle's cost-model perceptron: a closed form for a one-unit
network computed by hand, linearity in the output layer, and finite
differences for every weight's gradient."""
import math

import numpy as np


def test_mlp_one_unit_closed_form(orc):
    F, H = 1, 1
    # W1, b1, W2, b2, w3, b3
    w = np.array([0.7, -0.2, 1.3, 0.4, -2.0, 0.25])
    x = np.array([[0.5], [-1.5]])
    got = orc.mlp_forward(F, H, w, x)
    for xi, yi in zip(x[:, 0], got):
        want = -2.0 * math.tanh(1.3 * math.tanh(0.7 * xi - 0.2) + 0.4) + 0.25
        assert abs(yi - want) < 1e-15


def test_mlp_output_layer_is_affine(orc):
    F, H = 3, 4
    rng = np.random.Generator(np.random.PCG64(1))
    w = rng.normal(size=orc.mlp_nweights(F, H))
    x = rng.normal(size=(5, F))
    y0 = orc.mlp_forward(F, H, w, x)
    w2 = w.copy()
    w2[-1] += 0.75   # b3
    assert np.allclose(orc.mlp_forward(F, H, w2, x), y0 + 0.75, rtol=0, atol=1e-14)
    w3 = w.copy()
    w3[-1 - H:-1] *= 2.0
    w3[-1] *= 2.0     # doubling w3 and b3 doubles y
    assert np.allclose(orc.mlp_forward(F, H, w3, x), 2 * y0, rtol=0, atol=1e-13)


def test_mlp_gradient_matches_finite_differences(orc):
    F, H, B = 4, 5, 7
    rng = np.random.Generator(np.random.PCG64(2))
    w = rng.normal(size=orc.mlp_nweights(F, H)) * 0.7
    x = rng.normal(size=(B, F))
    t = rng.normal(size=B)
    loss, g = orc.mlp_loss_grad(F, H, w, x, t)
    y = orc.mlp_forward(F, H, w, x)
    assert abs(loss - 0.5 * np.mean((y - t) ** 2)) < 1e-15
    h = 1e-6
    for k in range(len(w)):
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (orc.mlp_loss_grad(F, H, wp, x, t)[0] - orc.mlp_loss_grad(F, H, wm, x, t)[0]) / (2 * h)
        assert abs(g[k] - fd) < 1e-8, k
