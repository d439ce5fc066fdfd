"""FP64 reference of the per-box convolutional network of the learned warm
start (test infrastructure only).

Network (one 8^3 box): input X with 2 channels on the 10^3 box-with-ghosts
region; conv 3x3x3 "valid" 2->16 + ReLU; conv 3x3x3 "same" (zero padding)
16->16 + ReLU; conv 3x3x3 "same" 16->1.  Operands are BF16 values (weights
and activations rounded to nearest even), arithmetic here is FP64; the GPU
accumulates in FP32.  Gradients of the mean squared error and one Adam step
follow the textbook definitions.

Array layouts: X [2][10][10][10]; activations [16][8][8][8]; weights
W1 [16][2][27], W2 [16][16][27], W3 [16][27] with tap index
t = (dx+1) + 3 (dy+1) + 9 (dz+1), arrays indexed [z][y][x].
"""
from __future__ import annotations

import numpy as np

N_W1, N_W2, N_W3 = 16 * 2 * 27, 16 * 16 * 27, 16 * 27
N_PARAMS = N_W1 + 16 + N_W2 + 16 + N_W3 + 1

TAPS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    W1 = p[i:i + N_W1].reshape(16, 2, 27); i += N_W1
    b1 = p[i:i + 16]; i += 16
    W2 = p[i:i + N_W2].reshape(16, 16, 27); i += N_W2
    b2 = p[i:i + 16]; i += 16
    W3 = p[i:i + N_W3].reshape(16, 27); i += N_W3
    b3 = p[i:i + 1]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def shift(a, dx, dy, dz, valid):
    """View of a [..][z][y][x] array at offset (dx,dy,dz) over the 8^3
    output region: `valid` reads a 10^3 input, else a zero-padded 8^3."""
    if valid:
        return a[..., 1 + dz:9 + dz, 1 + dy:9 + dy, 1 + dx:9 + dx]
    p = np.pad(a, [(0, 0)] * (a.ndim - 3) + [(1, 1)] * 3)
    return p[..., 1 + dz:9 + dz, 1 + dy:9 + dy, 1 + dx:9 + dx]


def conv(a, W, b, valid):
    """out[co] = b[co] + sum_t sum_ci W[co][ci][t] a[ci] shifted by tap t."""
    co = W.shape[0]
    out = np.zeros((co, 8, 8, 8)) + b[:, None, None, None]
    for t, (dx, dy, dz) in enumerate(TAPS):
        s = shift(a, dx, dy, dz, valid)
        out += np.einsum("oc,czyx->ozyx", W[:, :, t], s)
    return out


def forward(p, X, round_acts=True):
    """Layer outputs of one box: z1 (pre-ReLU), a1, z2, a2, out."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    z1 = conv(X, W1, b1, True)
    a1 = np.maximum(z1, 0.0)
    if round_acts:
        a1 = bf16(a1)
    z2 = conv(a1, W2, b2, False)
    a2 = np.maximum(z2, 0.0)
    if round_acts:
        a2 = bf16(a2)
    out = conv(a2, W3[None], b3, False)[0]
    return z1, a1, z2, a2, out


def conv_input_grad(g, W, valid):
    """d/d(input) of conv for output gradient g [co][8][8][8]: the input
    region is 10^3 when valid, else 8^3."""
    ci = W.shape[1]
    if valid:
        gi = np.zeros((ci, 10, 10, 10))
        for t, (dx, dy, dz) in enumerate(TAPS):
            gi[:, 1 + dz:9 + dz, 1 + dy:9 + dy, 1 + dx:9 + dx] += np.einsum("oc,ozyx->czyx", W[:, :, t], g)
        return gi
    gi = np.zeros((ci, 10, 10, 10))
    for t, (dx, dy, dz) in enumerate(TAPS):
        gi[:, 1 + dz:9 + dz, 1 + dy:9 + dy, 1 + dx:9 + dx] += np.einsum("oc,ozyx->czyx", W[:, :, t], g)
    return gi[:, 1:9, 1:9, 1:9]


def conv_weight_grad(a, g, valid):
    """dW[co][ci][t] = sum over outputs of g[co] * input shifted by tap t."""
    co, ci = g.shape[0], a.shape[0]
    dW = np.zeros((co, ci, 27))
    for t, (dx, dy, dz) in enumerate(TAPS):
        s = shift(a, dx, dy, dz, valid)
        dW[:, :, t] = np.einsum("ozyx,czyx->oc", g, s)
    return dW


def backward(p, X, a1, a2, out, target, scale):
    """Gradient of sum(scale*(out - target)^2) w.r.t. the parameters, given
    the layer activations a1, a2 (whose sign decides the ReLU derivative)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    g3 = 2.0 * scale * (out - target)
    dW3 = conv_weight_grad(a2, g3[None], False)[0]
    db3 = np.array([g3.sum()])
    d2 = conv_input_grad(g3[None], W3[None], False) * (a2 > 0)
    dW2 = conv_weight_grad(a1, d2, False)
    db2 = d2.sum(axis=(1, 2, 3))
    d1 = conv_input_grad(d2, W2, False) * (a1 > 0)
    dW1 = conv_weight_grad(X, d1, True)
    db1 = d1.sum(axis=(1, 2, 3))
    return pack(dW1, db1, dW2, db2, dW3, db3)


def loss_and_grad(p, Xs, targets, round_acts=False):
    """Mean squared error over boxes and cells and its gradient (FP64)."""
    n = len(Xs)
    scale = 1.0 / (n * 512)
    L = 0.0
    g = np.zeros(N_PARAMS)
    for X, t in zip(Xs, targets):
        z1, a1, z2, a2, out = forward(p, X, round_acts)
        L += scale * np.sum((out - t) ** 2)
        g += backward(p, X, a1, a2, out, t, scale)
    return L, g


def adam(w, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected first and second moments)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
