"""The learned proposal on the device against its oracle (oracle/cnn.py, oracle/proposal.py):
initial weights, network outputs and gradients (BF16 tensor-core kernels against FP64), AdamW,
the training-curve generator, binning of observed curves, seed sampling, the seeded batched fit,
and training on the device."""
import math

import numpy as np
import pytest
import torch

from oracle import cnn as ocnn
from oracle import proposal as op
from oracle import sblm as osb
from paper_1208_4830_gb300 import synth

pytestmark = pytest.mark.gpu

# BF16 operands (8-bit mantissa) with FP32 accumulation against FP64: normwise relative error of a
# tensor of products, and the cosine between gradient tensors
BF16_REL = 3e-2
COS_MIN = 0.999


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _cos(a, b):
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))


# element-wise check: BF16 unit roundoff, FP32 accumulation; errors taken as random (root of the
# sum of squares of the independent rounding contributions) and checked at ELEM_SIGMAS of that scale
U_BF16 = 2.0 ** -8
U_F32 = 2.0 ** -24
ELEM_SIGMAS = 8.0


def _gelu_dd(z):
    """Second derivative of x Phi(x): phi(x) (2 - x^2)."""
    return np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi) * (2.0 - z * z)


def _rss(a, b):
    """sqrt(sum_k a_k^2 b_k^2) of every dot product of a @ b."""
    return np.sqrt((a * a) @ (b * b))


def _q(*terms):
    return np.sqrt(sum(t * t for t in terms))


def _elementwise_scales(w, x, y):
    """Error scale of every network output and every gradient element when each product's
    operands are rounded to BF16 (unit roundoff u = 2^-8, both operands), products accumulate in
    FP32, activations and backward signals are stored in BF16, and the errors of earlier layers
    propagate through the weights, GELU', GELU'' and the loss's derivatives. Rounding errors are
    treated as independent, so a dot product sum_k a_k b_k gets
    sqrt(sum_k (da_k b_k)^2 + (a_k db_k)^2) + sqrt(2) u sqrt(sum_k (a_k b_k)^2): the size of the
    error a correct BF16 computation makes, element by element, while an element computed wrongly
    is off by a sizeable part of its value. The scales follow the oracle's own passes."""
    p = ocnn.unflatten(w)
    u, r2 = U_BF16, math.sqrt(2.0)
    out, (cache, f, z5, h5) = ocnn.forward(w, x)
    h, e_h = np.asarray(x, float), U_BF16 * np.abs(x)
    hs, ezs = [], []
    for i, (_, _, stride) in enumerate(ocnn.CONVS):
        W = p[f"W{i + 1}"]
        cols, cols_e = ocnn.im2col(h, stride), ocnn.im2col(e_h, stride)
        K = cols.shape[-1]
        e_z = _q(_rss(cols_e, W), (r2 * u + K * U_F32) * _rss(cols, W))
        z = cache[i][2]
        hs.append((h, e_h))
        ezs.append(e_z)
        h = ocnn.gelu(z)
        e_h = _q(ocnn.gelu_grad(z) * e_z, u * h)
    B = h.shape[0]
    fv, fe = h.reshape(B, -1), e_h.reshape(B, -1)
    W5, W6 = p["W5"], p["W6"]
    e_z5 = _q(_rss(fe, W5), (r2 * u + fv.shape[1] * U_F32) * _rss(fv, W5))
    e_h5 = _q(ocnn.gelu_grad(z5) * e_z5, u * h5)
    e_out = _q(_rss(e_h5, W6), (r2 * u + 128 * U_F32) * _rss(h5, W6))
    # backward
    _, dout = ocnn.nll(out, y)
    mu, sv = out[:, :6], out[:, 6:]
    r, ex = y - mu, np.exp(-sv)
    e_mu, e_s = e_out[:, :6], e_out[:, 6:]
    e_dout = np.empty_like(dout)
    e_dout[:, :6] = _q(ex / B * e_mu, r * ex / B * e_s, u * dout[:, :6])
    e_dout[:, 6:] = _q(r * ex / B * e_mu, 0.5 * r * r * ex / B * e_s, u * dout[:, 6:])
    g = {}
    g["W6"] = _q(_rss(e_h5.T, dout), _rss(h5.T, e_dout), (r2 * u + B * U_F32) * _rss(h5.T, dout))
    g["b6"] = _q(np.sqrt((e_dout ** 2).sum(0)), B * U_F32 * np.sqrt((dout ** 2).sum(0)))
    dh5 = dout @ W6.T
    e_dh5 = _q(_rss(e_dout, W6.T), (r2 * u + 12 * U_F32) * _rss(dout, W6.T))
    gd5 = ocnn.gelu_grad(z5)
    dz5 = dh5 * gd5
    e_dz5 = _q(e_dh5 * gd5, dh5 * _gelu_dd(z5) * e_z5, u * dz5)
    g["W5"] = _q(_rss(fe.T, dz5), _rss(fv.T, e_dz5), (r2 * u + B * U_F32) * _rss(fv.T, dz5))
    g["b5"] = _q(np.sqrt((e_dz5 ** 2).sum(0)), B * U_F32 * np.sqrt((dz5 ** 2).sum(0)))
    dh = (dz5 @ W5.T).reshape(B, 32, ocnn.WIDTH)
    e_dh = _q(_rss(e_dz5, W5.T), (r2 * u + 128 * U_F32) * _rss(dz5, W5.T)).reshape(B, 32, ocnn.WIDTH)
    for i in reversed(range(len(ocnn.CONVS))):
        shape, cols, z, stride = cache[i]
        e_z = ezs[i]
        hin, e_hin = hs[i]
        gd = ocnn.gelu_grad(z)
        dz = dh * gd
        e_dz = _q(e_dh * gd, dh * _gelu_dd(z) * e_z, u * dz)
        Bq, Lo, Co = dz.shape
        cv = cols.reshape(Bq * Lo, -1)
        ce = ocnn.im2col(e_hin, stride).reshape(Bq * Lo, -1)
        dzv, edz = dz.reshape(Bq * Lo, Co), e_dz.reshape(Bq * Lo, Co)
        g[f"W{i + 1}"] = _q(_rss(ce.T, dzv), _rss(cv.T, edz), (r2 * u + Bq * Lo * U_F32) * _rss(cv.T, dzv))
        g[f"b{i + 1}"] = _q(np.sqrt((edz ** 2).sum(0)), Bq * Lo * U_F32 * np.sqrt((dzv ** 2).sum(0)))
        if i > 0:
            W = p[f"W{i + 1}"]
            dcols = dz @ W.T
            e_dcols = _q(_rss(e_dz, W.T), (r2 * u + Co * U_F32) * _rss(dz, W.T))
            dh = ocnn.col2im(dcols, shape[1], shape[2], stride)
            e_dh = np.sqrt(ocnn.col2im(e_dcols ** 2, shape[1], shape[2], stride))
    return e_out, ocnn.flatten(g)


def _weights(seed, bias_scale=0.1):
    """Oracle initial weights with non-zero biases, so every term of the gradient is exercised."""
    w = op.init_params(seed)
    g = np.random.default_rng(seed + 100)
    p = ocnn.unflatten(w)
    for name, shape in ocnn.SHAPES:
        if name.startswith("b"):
            p[name] = g.normal(0.0, bias_scale, shape)
    return ocnn.flatten(p)


def _inputs(seed, B):
    g = np.random.default_rng(seed)
    x = np.zeros((B, 256, 2))
    x[:, :, 1] = g.uniform(size=(B, 256)) > 0.15
    x[:, :, 0] = np.where(x[:, :, 1] > 0, g.normal(0, 0.7, (B, 256)), 0.0)
    y = np.stack([g.uniform(-0.4, 0.4, B), g.uniform(-3, 0.4, B), g.uniform(0, 1, B), g.uniform(0, 1, B),
                  g.uniform(-1.2, 1.1, B), g.uniform(-4, 0, B)], axis=1)
    return x, y


def test_init_matches_oracle(lib):
    w = lib.cnn_init(seed=3).cpu().numpy()
    np.testing.assert_allclose(w, op.init_params(3), rtol=2e-7, atol=1e-30)


@pytest.mark.parametrize("B", [1, 5, 37])
def test_forward_matches_oracle(lib, B):
    w = _weights(1)
    x, _ = _inputs(2 + B, B)
    out = lib.cnn_forward(torch.tensor(w, dtype=torch.float32, device="cuda"),
                          torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    ref, _ = ocnn.forward(w, x)
    assert _rel(out, ref) <= BF16_REL, _rel(out, ref)
    e_out, _ = _elementwise_scales(w, x, np.zeros((B, 6)))
    ratio = np.abs(out - ref) / (e_out + 1e-30)
    assert ratio.max() <= ELEM_SIGMAS, ratio.max()


@pytest.mark.parametrize("B", [3, 64, 130])
def test_gradients_match_oracle(lib, B):
    w = _weights(4)
    x, y = _inputs(5 + B, B)
    wt = torch.tensor(w, dtype=torch.float32, device="cuda")
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    loss, g = lib.cnn_loss_grad(wt, xt, yt)
    g = g.cpu().numpy().astype(np.float64)
    ref_loss, ref_g = ocnn.loss_and_grad(w, x, y)
    assert loss == pytest.approx(ref_loss, rel=BF16_REL)
    # element by element: every gradient element within ELEM_SIGMAS of its own rounding scale
    _, e_g = _elementwise_scales(w, x, y)
    ratio = np.abs(g - ref_g) / (e_g + 1e-30)
    assert ratio.max() <= ELEM_SIGMAS, (int(np.argmax(ratio)), ratio.max())
    o = 0
    for name, shape in ocnn.SHAPES:
        n = int(np.prod(shape))
        a, b = g[o : o + n], ref_g[o : o + n]
        assert _rel(a, b) <= BF16_REL, (name, _rel(a, b))
        assert _cos(a, b) >= COS_MIN, (name, _cos(a, b))
        o += n
    # the reduction order is fixed: a second call is bit-identical
    loss2, g2 = lib.cnn_loss_grad(wt, xt, yt)
    assert loss2 == loss and np.array_equal(g2.cpu().numpy(), g.astype(np.float32))


def test_adamw_matches_oracle(lib):
    N = ocnn.N_PARAMS
    rng = np.random.default_rng(0)
    w = rng.normal(size=N).astype(np.float32)
    m = (0.01 * rng.normal(size=N)).astype(np.float32)
    v = (1e-4 * rng.uniform(size=N)).astype(np.float32)
    grad = rng.normal(size=N).astype(np.float32)
    p = lib.cnn_train_params(lr=3e-3, n_steps=100, warmup=10)
    wt = torch.tensor(w, device="cuda")
    st = torch.tensor(np.concatenate([m, v]), device="cuda")
    lib.cnn_adamw(wt, st, torch.tensor(grad, device="cuda"), p, 7)
    lr = op.lr_at(7, 100, 10, 3e-3)
    w2, m2, v2 = op.adamw(w.astype(np.float64), m.astype(np.float64), v.astype(np.float64), grad.astype(np.float64),
                          7, lr, 0.9, 0.999, 1e-8, 1e-4)
    np.testing.assert_allclose(wt.cpu().numpy(), w2, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(st[:N].cpu().numpy(), m2, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(st[N:].cpu().numpy(), v2, rtol=1e-6, atol=1e-15)


@pytest.mark.parametrize("forced", [0.0, 0.5])
def test_make_batch_matches_oracle_fp64(lib, forced):
    B = 24
    x, y, th = lib.cnn_make_batch(seed=9, step=3, batch=B, forced_frac=forced, precision="fp64")
    X, Y, TH, infos = op.make_batch(9, 3, B, forced)
    np.testing.assert_allclose(th.cpu().numpy(), TH, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(y.cpu().numpy(), Y, rtol=2e-6, atol=1e-6)
    xd = x.cpu().numpy()
    assert np.array_equal(xd[:, :, 1], X[:, :, 1])  # mask decisions are taken in FP64 on both sides
    np.testing.assert_allclose(xd[:, :, 0], X[:, :, 0], atol=1e-5)
    if forced:
        assert sum(i["forced"] for i in infos) >= 5


def test_make_batch_mixed_generator(lib):
    B = 64
    x, _, th = lib.cnn_make_batch(seed=2, step=11, batch=B, forced_frac=0.1, precision="mixed")
    X, _, TH, _ = op.make_batch(2, 11, B, 0.1)
    xd = x.cpu().numpy()
    assert np.array_equal(xd[:, :, 1], X[:, :, 1])
    err = np.abs(xd[:, :, 0] - X[:, :, 0])
    assert np.quantile(err, 0.995) <= 1e-3 and np.all(np.isfinite(xd))


def test_bin_matches_oracle(lib):
    b = synth.seasonal_batch(6, seed=12, n_min=100, n_max=2500, span=(-100.0, 100.0), season=80.0, gap=30.0)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(6)])
    flux, sigma = b.observe(A)
    x, win = lib.cnn_bin(torch.tensor(b.t, device="cuda"), torch.tensor(flux, device="cuda"),
                         torch.tensor(sigma, device="cuda"), torch.tensor(b.offsets, device="cuda"))
    x, win = x.cpu().numpy(), win.cpu().numpy()
    for i in range(6):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        X, (c, h) = op.bin_lightcurve(b.t[sl], flux[sl], sigma[sl])
        assert win[i, 0] == pytest.approx(c, rel=1e-15, abs=1e-13) and win[i, 1] == pytest.approx(h, rel=1e-15)
        assert np.array_equal(x[i, :, 1], X[:, 1])
        np.testing.assert_allclose(x[i, :, 0], X[:, 0], atol=1e-6)
    # host buffers give the same inputs
    xh, _ = lib.cnn_bin(b.t, flux, sigma, b.offsets)
    assert np.array_equal(xh, x)


def test_propose_matches_oracle(lib):
    rng = np.random.default_rng(3)
    n_lc, n_seed = 5, 33
    out = np.concatenate([rng.normal(0, 0.5, (n_lc, 6)), rng.normal(-2, 1, (n_lc, 6))], axis=1).astype(np.float32)
    out[2, 1] = 30.0  # far outside the tE bounds: clamped
    win = np.stack([rng.uniform(-10, 10, n_lc), rng.uniform(40, 120, n_lc)], axis=1)
    g = lib.cnn_propose(torch.tensor(out, device="cuda"), torch.tensor(win, device="cuda"), synth.FIT_LO, synth.FIT_HI,
                        n_seed, seed=5).cpu().numpy()
    ref = op.propose_genes(out, win, synth.FIT_LO, synth.FIT_HI, n_seed, 5)
    np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-12)
    assert g.min() >= 0 and g.max() <= 1 and np.all(g[2, :, 1] == 1.0)


def _batch(n_lc, seed, n_min, n_max):
    b = synth.seasonal_batch(n_lc, seed=seed, n_min=n_min, n_max=n_max, span=(-100.0, 100.0), season=80.0, gap=30.0)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(n_lc)])
    flux, sigma = b.observe(A)
    return b, flux, sigma


def _genes(theta):
    v = theta.copy()
    v[..., 5] = np.log10(v[..., 5])
    return (v - synth.FIT_LO) / (synth.FIT_HI - synth.FIT_LO)


def test_seeded_rows_enter_the_first_population(lib):
    """With the encoded truth among the seed rows and a single generation, the best chi^2 found
    is at most the truth's (the first generation evaluates every seeded row)."""
    b, flux, sigma = _batch(4, seed=21, n_min=150, n_max=300)
    p = lib.params(n_pop=64, n_gen=1, precision="fp64", seed=1)
    seeds = np.repeat(_genes(b.truth)[:, None, :], 3, axis=1)
    seeds[:, 1:] = np.clip(seeds[:, 1:] + 0.05, 0, 1)
    _, chi = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p, seed_genes=seeds)
    _, chi_plain = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    for i in range(4):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        c_true = osb.chi2(b.truth[i : i + 1], b.t[sl], flux[sl], sigma[sl])[0]
        assert chi[i] <= c_true * (1 + 1e-9) + 1e-9, (i, chi[i], c_true)
        assert chi_plain[i] > c_true  # one random generation does not find the truth
    # n_seed = 0 and no seeds: the paper's fitter, identical to sblm_fit_batch
    best0, chi0 = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p,
                                seed_genes=np.zeros((4, 0, 6)))
    np.testing.assert_array_equal(chi0, chi_plain)


def test_training_on_device_reduces_the_loss(lib):
    w = lib.cnn_init(seed=0)
    st = torch.zeros(2 * lib.cnn_num_params(), device="cuda")
    p = lib.cnn_train_params(batch=128, n_steps=400, warmup=40, seed=4)
    hist = lib.cnn_train(w, st, p)
    assert hist.shape == (400,) and np.all(np.isfinite(hist))
    assert hist[-50:].mean() < hist[:20].mean() - 1.0, (hist[:20].mean(), hist[-50:].mean())
    # resuming continues the same schedule and data stream
    w2 = lib.cnn_init(seed=0)
    st2 = torch.zeros_like(st)
    h1 = lib.cnn_train(w2, st2, p, first_step=0, n_run=150)
    h2 = lib.cnn_train(w2, st2, p, first_step=150, n_run=250)
    np.testing.assert_allclose(np.concatenate([h1, h2]), hist, rtol=1e-5, atol=1e-5)


def test_proposal_gain_on_heldout_curves(lib):
    """What the trained network gains over the paper's random initialisation, on held-out curves
    (500 epochs, 2% noise, truths from the sweep priors): (1) its means of t0', ln tE' and u0 are
    far closer than the prior's spread, (2) the first generation of a seeded population is fitter
    than a random one on most curves, (3) short fits reach lower chi^2 with the seeds."""
    w = lib.cnn_init(seed=0)
    st = torch.zeros(2 * lib.cnn_num_params(), device="cuda")
    lib.cnn_train(w, st, lib.cnn_train_params(batch=1024, n_steps=2048, warmup=100, seed=3))
    n = 96
    b = synth.heldout_batch(n, seed=91)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(n)])
    flux, sigma = b.observe(A)
    sl = [slice(b.offsets[i], b.offsets[i + 1]) for i in range(n)]
    chi_true = np.array([osb.chi2(b.truth[i : i + 1], b.t[s], flux[s], sigma[s])[0] for i, s in enumerate(sl)])
    dev = [torch.tensor(v, device="cuda") for v in (b.t, flux, sigma, b.offsets)]
    x, win = lib.cnn_bin(*dev)
    out = lib.cnn_forward(w, x).cpu().numpy()
    win = win.cpu().numpy()
    tgt = np.stack([(b.truth[:, 0] - win[:, 0]) / win[:, 1], np.log(b.truth[:, 1] / win[:, 1]), b.truth[:, 2]], 1)
    err = np.median(np.abs(out[:, :3] - tgt), axis=0)
    prior_spread = np.array([40 / 120 / np.sqrt(12), np.log(20) / np.sqrt(12), 1 / np.sqrt(12)])
    assert np.all(err < 0.35 * prior_spread), (err, prior_spread)

    def fits(n_pop, n_gen, frac):
        p = lib.params(n_pop=n_pop, n_gen=n_gen, precision="mixed", seed=4)
        return lib.fit_batch_cnn(*dev, synth.FIT_LO, synth.FIT_HI, p, w, seed_frac=frac)[1] - chi_true

    g0_plain, g0_seed = fits(128, 1, 0.0), fits(128, 1, 0.5)
    assert np.mean(g0_seed < g0_plain) >= 0.75, np.mean(g0_seed < g0_plain)
    d_plain, d_seed = fits(128, 20, 0.0), fits(128, 20, 0.5)
    assert np.median(d_seed) < np.median(d_plain), (np.median(d_seed), np.median(d_plain))
    assert np.mean(d_seed <= 1.0) >= np.mean(d_plain <= 1.0)


def test_training_batch_size_properties(lib):
    """At the training batch of 1024: network outputs of sampled rows against the FP64 oracle, and
    the whole-batch gradient against the mean of the gradients of its eight 128-curve chunks (the
    loss is a mean over curves; the 1/B scalings are powers of two, so the BF16 operands of each
    curve are the same and only the FP32 summation order differs)."""
    x, y, _ = lib.cnn_make_batch(seed=1, step=0, batch=1024, precision="fp32")
    w = lib.cnn_init(seed=2)
    out = lib.cnn_forward(w, x).cpu().numpy()
    wn = w.cpu().numpy().astype(np.float64)
    rows = [0, 137, 511, 1023]
    ref, _ = ocnn.forward(wn, x[rows].cpu().numpy().astype(np.float64))
    assert _rel(out[rows], ref) <= BF16_REL
    L, g = lib.cnn_loss_grad(w, x, y)
    parts = [lib.cnn_loss_grad(w, x[i * 128 : (i + 1) * 128].contiguous(), y[i * 128 : (i + 1) * 128].contiguous())
             for i in range(8)]
    Lm = np.mean([p[0] for p in parts])
    gm = np.mean([p[1].cpu().numpy().astype(np.float64) for p in parts], axis=0)
    assert L == pytest.approx(Lm, rel=1e-6)
    assert _rel(g.cpu().numpy().astype(np.float64), gm) <= 1e-5


def test_bounded_wait_gives_up_and_reports(lib):
    """The tensor-core kernels bound every mbarrier wait. A block waiting on a barrier that nothing
    arrives on must give up after its poll budget, set the device flag, and the entry points'
    check must turn it into SBLM_ETIMEOUT and clear it: the next call on the device succeeds."""
    assert lib.cnn_selftest_timeout(polls=1000) == 4  # SBLM_ETIMEOUT
    assert lib.cnn_selftest_timeout(polls=1) == 4
    w = _weights(1)
    x, y = _inputs(3, 4)
    f32 = dict(dtype=torch.float32, device="cuda")
    loss, _ = lib.cnn_loss_grad(torch.tensor(w, **f32), torch.tensor(x, **f32), torch.tensor(y, **f32))
    assert np.isfinite(loss)

