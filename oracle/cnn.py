"""Oracle: the learned proposal network, plain numpy FP64, forward and backward by hand.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). The paper has no learned component (it
compares against a different network, Section 4.1); this is the restatement, in FP64 and without
any blocking, of the network the device trains in BF16, used to check the device's outputs and
gradients.

Network (channels last, batch B):
  x [B, 256, 2]  (normalised flux, data mask)
  conv k=5: 2 -> 64, stride 1, pad 2, GELU    -> [B, 256, 64]
  conv k=5: 64 -> 64, stride 2, pad 2, GELU   -> [B, 128, 64]
  conv k=5: 64 -> 64, stride 2, pad 2, GELU   -> [B, 64, 64]
  conv k=5: 64 -> 64, stride 2, pad 2, GELU   -> [B, 32, 64]   (flattened l-major: 2048)
  dense 2048 -> 128, GELU; dense 128 -> 12    -> means mu[6], log-variances s[6]
Loss: the Gaussian negative log-likelihood of the 6 targets, mean over the batch:
  L = mean_b sum_j 0.5 ((y_j - mu_j)^2 exp(-s_j) + s_j).
A convolution weight is stored as a [k * C_in, C_out] matrix, row kk * C_in + c.
GELU is the exact one, x Phi(x).

Pinned by tests/test_oracle_cnn.py against torch's CPU float64 conv1d / linear / gelu and its
autograd gradients, and against central finite differences of the oracle's own loss.
"""
from __future__ import annotations

import math

import numpy as np

L_IN, C_IN, WIDTH, KSIZE, HIDDEN, N_OUT = 256, 2, 64, 5, 128, 12
CONVS = [(C_IN, WIDTH, 1), (WIDTH, WIDTH, 2), (WIDTH, WIDTH, 2), (WIDTH, WIDTH, 2)]  # (C_in, C_out, stride)
PAD = 2
FLAT = 32 * WIDTH

# parameter tensors in the order of the flat vector: (name, shape)
SHAPES = []
for _i, (_ci, _co, _s) in enumerate(CONVS):
    SHAPES += [(f"W{_i + 1}", (KSIZE * _ci, _co)), (f"b{_i + 1}", (_co,))]
SHAPES += [("W5", (FLAT, HIDDEN)), ("b5", (HIDDEN,)), ("W6", (HIDDEN, N_OUT)), ("b6", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o : o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def flatten(params):
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in SHAPES])


_erf = np.vectorize(math.erf)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def out_len(L, stride):
    return (L + 2 * PAD - KSIZE) // stride + 1


def im2col(x, stride):
    """Rows (b, l), columns kk * C + c: x[b, l * stride + kk - PAD, c], zero outside."""
    B, L, C = x.shape
    Lo = out_len(L, stride)
    cols = np.zeros((B, Lo, KSIZE * C))
    for kk in range(KSIZE):
        for l in range(Lo):
            i = l * stride + kk - PAD
            if 0 <= i < L:
                cols[:, l, kk * C : (kk + 1) * C] = x[:, i, :]
    return cols


def col2im(dcols, L, C, stride):
    """Adjoint of im2col: scatter-add the column gradient back onto the input positions."""
    B, Lo, _ = dcols.shape
    dx = np.zeros((B, L, C))
    for kk in range(KSIZE):
        for l in range(Lo):
            i = l * stride + kk - PAD
            if 0 <= i < L:
                dx[:, i, :] += dcols[:, l, kk * C : (kk + 1) * C]
    return dx


def forward(params, x):
    """Network outputs [B, 12] and the cache the backward pass needs."""
    p = params if isinstance(params, dict) else unflatten(params)
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for i, (_, _, stride) in enumerate(CONVS):
        cols = im2col(h, stride)
        z = cols @ p[f"W{i + 1}"] + p[f"b{i + 1}"]
        cache.append((h.shape, cols, z, stride))
        h = gelu(z)
    B = h.shape[0]
    f = h.reshape(B, FLAT)
    z5 = f @ p["W5"] + p["b5"]
    h5 = gelu(z5)
    out = h5 @ p["W6"] + p["b6"]
    return out, (cache, f, z5, h5)


def nll(out, y):
    """Loss and its gradient with respect to the outputs."""
    B = out.shape[0]
    mu, s = out[:, :6], out[:, 6:]
    r = y - mu
    e = np.exp(-s)
    loss = np.sum(0.5 * (r * r * e + s)) / B
    dout = np.empty_like(out)
    dout[:, :6] = -r * e / B
    dout[:, 6:] = 0.5 * (1.0 - r * r * e) / B
    return loss, dout


def backward(params, ctx, dout):
    """Gradients of the loss with respect to every parameter (same dict layout)."""
    p = params if isinstance(params, dict) else unflatten(params)
    cache, f, z5, h5 = ctx
    g = {}
    g["W6"] = h5.T @ dout
    g["b6"] = dout.sum(0)
    dz5 = (dout @ p["W6"].T) * gelu_grad(z5)
    g["W5"] = f.T @ dz5
    g["b5"] = dz5.sum(0)
    dh = (dz5 @ p["W5"].T).reshape(f.shape[0], 32, WIDTH)
    for i in reversed(range(len(CONVS))):
        shape, cols, z, stride = cache[i]
        dz = dh * gelu_grad(z)
        B, Lo, Co = dz.shape
        g[f"W{i + 1}"] = cols.reshape(B * Lo, -1).T @ dz.reshape(B * Lo, Co)
        g[f"b{i + 1}"] = dz.sum((0, 1))
        if i > 0:
            dcols = dz @ p[f"W{i + 1}"].T
            dh = col2im(dcols, shape[1], shape[2], stride)
    return g


def loss_and_grad(flat, x, y):
    out, ctx = forward(flat, x)
    loss, dout = nll(out, y)
    return loss, flatten(backward(flat, ctx, dout))
