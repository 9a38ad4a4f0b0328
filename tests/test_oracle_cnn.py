"""Pins of the proposal network's oracle: torch's CPU float64 primitives and autograd (an
independent implementation of convolution, dense layers, GELU and differentiation) and central
finite differences of the oracle's own loss."""
import numpy as np
import pytest

from oracle import cnn

torch = pytest.importorskip("torch")


def _params(seed, scale=0.3):
    g = np.random.default_rng(seed)
    return g.normal(0.0, scale, cnn.N_PARAMS) / np.sqrt(np.concatenate(
        [np.full(int(np.prod(s)), s[0] if len(s) == 2 else 1.0) for _, s in cnn.SHAPES]))


def _data(seed, B):
    g = np.random.default_rng(seed)
    x = g.normal(0, 1, (B, cnn.L_IN, cnn.C_IN))
    y = g.uniform(0, 1, (B, 6))
    return x, y


def _torch_loss(flat, x, y):
    p = {k: torch.tensor(v, requires_grad=True) for k, v in cnn.unflatten(flat).items()}
    h = torch.tensor(x).permute(0, 2, 1)  # [B, C, L]
    for i, (ci, co, stride) in enumerate(cnn.CONVS):
        W = p[f"W{i + 1}"].reshape(cnn.KSIZE, ci, co).permute(2, 1, 0)  # [C_out, C_in, k]
        h = torch.nn.functional.gelu(torch.nn.functional.conv1d(h, W, p[f"b{i + 1}"], stride=stride, padding=cnn.PAD))
    f = h.permute(0, 2, 1).reshape(h.shape[0], -1)  # l-major flatten, like the oracle
    h5 = torch.nn.functional.gelu(f @ p["W5"] + p["b5"])
    out = h5 @ p["W6"] + p["b6"]
    yt = torch.tensor(y)
    mu, s = out[:, :6], out[:, 6:]
    loss = (0.5 * ((yt - mu) ** 2 * torch.exp(-s) + s)).sum() / out.shape[0]
    loss.backward()
    grads = np.concatenate([p[name].grad.numpy().ravel() for name, _ in cnn.SHAPES])
    return out.detach().numpy(), loss.item(), grads


def test_parameter_count():
    assert cnn.N_PARAMS == 640 + 64 + 3 * (320 * 64 + 64) + 2048 * 128 + 128 + 128 * 12 + 12


def test_forward_matches_torch():
    flat = _params(1)
    x, y = _data(2, 3)
    out, _ = cnn.forward(flat, x)
    ref, _, _ = _torch_loss(flat, x, y)
    np.testing.assert_allclose(out, ref, rtol=1e-10, atol=1e-12)


def test_gradients_match_torch_autograd():
    flat = _params(3)
    x, y = _data(4, 3)
    loss, g = cnn.loss_and_grad(flat, x, y)
    _, ref_loss, ref_g = _torch_loss(flat, x, y)
    assert loss == pytest.approx(ref_loss, rel=1e-12)
    np.testing.assert_allclose(g, ref_g, rtol=1e-9, atol=1e-12)


def test_gradients_match_finite_differences():
    flat = _params(5)
    x, y = _data(6, 2)
    _, g = cnn.loss_and_grad(flat, x, y)
    rng = np.random.default_rng(7)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in cnn.SHAPES])
    idx = np.concatenate([rng.choice(np.arange(offs[k], offs[k + 1]), 3, replace=False) for k in range(len(cnn.SHAPES))])
    for i in idx:
        h = 1e-6
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        num = (cnn.loss_and_grad(fp, x, y)[0] - cnn.loss_and_grad(fm, x, y)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, num, g[i])


def test_col2im_is_the_adjoint_of_im2col():
    g = np.random.default_rng(8)
    x = g.normal(size=(2, 64, 5))
    d = g.normal(size=cnn.im2col(x, 2).shape)
    lhs = np.sum(cnn.im2col(x, 2) * d)
    rhs = np.sum(x * cnn.col2im(d, 64, 5, 2))
    assert lhs == pytest.approx(rhs, rel=1e-12)
