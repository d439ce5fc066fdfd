"""Pins of the FP64 network reference (oracle/cnn.py): convolutions against
scipy's correlation, backpropagation against finite differences, BF16
rounding against torch's conversion and known ties, Adam's first step in
closed form."""
import numpy as np
import pytest
import scipy.signal as ss

from oracle import cnn


def rand_params(rng, scale=0.3):
    return rng.standard_normal(cnn.N_PARAMS) * scale


def kernel(Wt):
    """[27] tap weights -> [3][3][3] correlation kernel indexed [dz][dy][dx],
    with the documented tap index t = (dx+1) + 3 (dy+1) + 9 (dz+1)."""
    K = np.zeros((3, 3, 3))
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                K[dz + 1, dy + 1, dx + 1] = Wt[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)]
    return K


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((2, 10, 10, 10))
    W = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    out = cnn.conv(X, W, b, True)
    for co in range(3):
        ref = b[co] + sum(ss.correlate(X[ci], kernel(W[co, ci]), mode="valid") for ci in range(2))
        assert np.allclose(out[co], ref, rtol=1e-12, atol=1e-12)
    A = rng.standard_normal((4, 8, 8, 8))
    W = rng.standard_normal((2, 4, 27))
    out = cnn.conv(A, W, np.zeros(2), False)
    for co in range(2):
        ref = sum(ss.correlate(A[ci], kernel(W[co, ci]), mode="same") for ci in range(4))
        assert np.allclose(out[co], ref, rtol=1e-12, atol=1e-12)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = rand_params(rng)
    Xs = [rng.standard_normal((2, 10, 10, 10)) for _ in range(2)]
    ts = [rng.standard_normal((8, 8, 8)) for _ in range(2)]
    L, g = cnn.loss_and_grad(p, Xs, ts)
    idx = np.concatenate([rng.choice(cnn.N_PARAMS, 40, replace=False),
                          [cnn.N_PARAMS - 1, cnn.N_W1 + 3, cnn.N_W1 + 16 + cnn.N_W2 + 5]])
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        fd = (cnn.loss_and_grad(p + e, Xs, ts)[0] - cnn.loss_and_grad(p - e, Xs, ts)[0]) / (2 * eps)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), i


def test_bf16_rounding():
    import torch
    rng = np.random.default_rng(4)
    x = (rng.standard_normal(20000) * 10.0 ** rng.integers(-5, 5, 20000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16(x), ref)
    one = np.float32(1.0)
    assert cnn.bf16(one + np.float32(2 ** -8)) == 1.0                 # tie -> even
    assert cnn.bf16(one + np.float32(3 * 2 ** -8)) == 1.0 + 2 ** -6   # tie -> even (up)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(5)
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    w1, m, v = cnn.adam(w, np.zeros(50), np.zeros(50), g, 1, 1e-3)
    assert np.allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_constant_gradient_steps():
    """With a constant gradient the bias-corrected moments equal g and g^2
    at every step, so each Adam step moves w by lr g / (|g| + eps)."""
    rng = np.random.default_rng(6)
    w0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    w, m, v = w0, np.zeros(50), np.zeros(50)
    for step in range(1, 6):
        w, m, v = cnn.adam(w, m, v, g, step, 1e-3)
        assert np.allclose(w, w0 - step * 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-14)


def test_loss_is_mean_over_boxes_and_cells():
    """The zero network predicts 0 everywhere: the loss is the mean of t^2
    over all boxes and cells, and its bias gradient -2 mean(t)."""
    rng = np.random.default_rng(7)
    Xs = [rng.standard_normal((2, 10, 10, 10)) for _ in range(3)]
    ts = [rng.standard_normal((8, 8, 8)) for _ in range(3)]
    L, g = cnn.loss_and_grad(np.zeros(cnn.N_PARAMS), Xs, ts)
    allt = np.stack(ts)
    assert L == pytest.approx(np.mean(allt ** 2), rel=1e-13)
    assert g[-1] == pytest.approx(-2.0 * np.mean(allt), rel=1e-12)


def test_forward_rounds_hidden_activations_to_bf16():
    """With round_acts both hidden activations are BF16 values, the
    rounding of the FP64 ReLU outputs (the operands the next layer
    multiplies on the tensor cores)."""
    rng = np.random.default_rng(8)
    p = rand_params(rng)
    X = rng.standard_normal((2, 10, 10, 10))
    z1, a1, z2, a2, out = cnn.forward(p, X, True)
    assert np.array_equal(a1, cnn.bf16(np.maximum(z1, 0.0)))
    assert np.array_equal(a2, cnn.bf16(np.maximum(z2, 0.0)))
    assert not np.array_equal(a2, np.maximum(z2, 0.0))
