"""Pins of the proposal's data path in the oracle (oracle/proposal.py): caustic crossings checked
through the images' Jacobian, draws against their distributions, binning against hand-made
curves, AdamW against torch's implementation, sampling against its limits."""
import math

import numpy as np
import pytest

from oracle import cnn
from oracle import proposal as op
from oracle import sblm as osb


def test_bin_centres_span_the_window():
    s = op.bin_centres()
    assert s.size == 256 and s[0] == pytest.approx(-1 + 1 / 256) and s[-1] == pytest.approx(1 - 1 / 256)
    np.testing.assert_allclose(np.diff(s), 2 / 256)


def test_normalise_by_hand():
    F = np.full(256, 2.0)
    kept = np.ones(256, bool)
    kept[:6] = False
    F[10] = 4.0  # one bin at twice the median
    x = op.normalise(F, kept)
    assert x[10, 0] == pytest.approx(math.asinh(10.0) / 3.0)
    assert np.all(x[11:, 0] == 0.0) and np.all(x[:6] == 0.0) and np.all(x[6:, 1] == 1.0)
    # even count of bins with data: the mean of the middle two
    F2 = np.zeros(256)
    k2 = np.zeros(256, bool)
    F2[:4] = [1.0, 2.0, 4.0, 8.0]
    k2[:4] = True
    x2 = op.normalise(F2, k2)
    assert x2[0, 0] == pytest.approx(math.asinh(10 * (1 / 3 - 1)) / 3)


def test_bin_lightcurve_by_hand():
    t = np.array([0.0, 0.02, 5.0, 9.99, 10.0])
    flux = np.array([1.0, 3.0, 2.0, 5.0, 7.0])
    sigma = np.array([1.0, 0.5, 1.0, 1.0, 2.0])
    x, (c, h) = op.bin_lightcurve(t, flux, sigma)
    assert (c, h) == (5.0, 5.0)
    # bin 0 holds t=0 and t=0.02 (width 10/256): weights 1 and 4
    F0 = (1 * 1.0 + 4 * 3.0) / 5
    # the last bin holds t=9.99 and t=10 (clamped): weights 1, 1/4
    F255 = (5.0 + 0.25 * 7.0) / 1.25
    F128 = 2.0
    med = F0  # median of (F0 = 2.6, F128 = 2.0, F255 = 5.4)
    assert x[0, 0] == 0.0
    assert x[128, 0] == pytest.approx(math.asinh(10 * (F128 / med - 1)) / 3)
    assert x[255, 0] == pytest.approx(math.asinh(10 * (F255 / med - 1)) / 3)
    assert x[:, 1].sum() == 3 and x[128, 1] == 1 and x[1, 1] == 0


def test_training_draws_cover_the_prior():
    th = np.array([op.sample_theta(3, 0, i, 0.0)[0] for i in range(400)])
    assert th[:, 0].min() >= -0.4 and th[:, 0].max() <= 0.4
    assert th[:, 1].min() >= 0.04 and th[:, 1].max() <= 1.5
    assert th[:, 4].min() >= 0.3 and th[:, 4].max() <= 3.0
    assert th[:, 5].min() >= 1e-4 and th[:, 5].max() <= 1.0
    # log-uniform in d: the mean of ln d is the centre of [ln 0.3, ln 3]
    assert np.mean(np.log(th[:, 4])) == pytest.approx(0.5 * math.log(0.9), abs=0.12)


def test_forced_trajectories_cross_a_caustic():
    """Crossing a fold caustic changes the image count by two (Section 2.2: 3 or 5 images), so the
    oracle's own image solver must see different counts just before and just after the drawn
    crossing time (a crossing through a cusp point is the rare exception)."""
    hits = 0
    for i in range(60):
        theta, info = op.sample_theta(11, 2, i, 1.0)
        assert info["forced"]
        t0, tE, u0, alpha, d, q = theta
        assert u0 >= 0.0 and 0.0 <= alpha < 2 * math.pi
        eps = 1e-6 * tE
        t = np.array([info["t_cross"] - eps, info["t_cross"] + eps])
        _, inf = osb.magnification(theta[None], t, return_info=True)
        hits += int(inf["n"][0, 0] != inf["n"][0, 1])
    assert hits >= 55, hits
    # unforced draws cross far less often
    miss = 0
    for i in range(60):
        theta, info = op.sample_theta(11, 2, i, 0.0)
        t = np.array([0.3 - 1e-6 * theta[1], 0.3 + 1e-6 * theta[1]])
        _, inf = osb.magnification(theta[None], t, return_info=True)
        miss += int(inf["n"][0, 0] == inf["n"][0, 1])
    assert miss >= 58


def test_noise_is_unit_normal_and_mask_rates():
    from scipy import stats

    zs, kept_frac = [], []
    for i in range(40):
        _, info = op.sample_theta(5, 1, i, 0.1)
        z, kept = op.noise_and_mask(5, 1, i, info)
        zs.append(z)
        kept_frac.append(kept.mean())
        if info["gw"] == 0.0 and kept.sum() >= op.MIN_KEPT:
            # without a gap only dropout removes bins: about 1 - p_drop kept
            assert abs(kept.mean() - (1 - info["p_drop"])) < 0.12
    assert stats.kstest(np.concatenate(zs), "norm").pvalue > 1e-3
    assert min(kept_frac) >= op.MIN_KEPT / 256


def test_make_batch_inputs_and_targets():
    X, Y, TH, infos = op.make_batch(1, 0, 6)
    assert X.shape == (6, 256, 2) and Y.shape == (6, 6)
    for i in range(6):
        np.testing.assert_allclose(Y[i], op.targets(TH[i]))
        # flux channel vanishes where the mask does
        assert np.all(X[i, X[i, :, 1] == 0, 0] == 0)
        # the noiseless part of the curve is the magnification: rebuild it from A
        A = osb.magnification(TH[i][None], op.bin_centres())[0]
        z, kept = op.noise_and_mask(1, 0, i, infos[i])
        F = A * (1 + infos[i]["sigma"] * z)
        med = np.median(F[kept])
        np.testing.assert_allclose(np.sinh(3 * X[i, kept, 0]) / 10 + 1, F[kept] / med, rtol=1e-12)


def test_init_params_statistics():
    w = op.init_params(0)
    p = cnn.unflatten(w)
    for name, shape in cnn.SHAPES:
        if name.startswith("b"):
            assert np.all(p[name] == 0)
        elif name != "W6" and p[name].size > 1000:
            assert np.std(p[name]) == pytest.approx(math.sqrt(2 / shape[0]), rel=0.06)
    assert abs(np.std(p["W6"]) - 0.1 / math.sqrt(128)) < 0.003
    assert not np.array_equal(op.init_params(1), w)


def test_adamw_matches_torch():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(0)
    w = g.normal(size=50)
    wt = torch.tensor(w.copy(), requires_grad=True)
    opt = torch.optim.AdamW([wt], lr=3e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=1e-4)
    m = np.zeros(50)
    v = np.zeros(50)
    for t in range(1, 6):
        grad = g.normal(size=50)
        w, m, v = op.adamw(w, m, v, grad, t, 3e-3)
        wt.grad = torch.tensor(grad)
        opt.step()
        np.testing.assert_allclose(w, wt.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_lr_schedule_shape():
    assert op.lr_at(1, 100, 10, 1e-3) == pytest.approx(1e-4)
    assert op.lr_at(10, 100, 10, 1e-3) == pytest.approx(1e-3 * (0.1 + 0.45 * (1 + math.cos(math.pi * 0.09))))
    assert op.lr_at(101, 100, 10, 1e-3) == pytest.approx(1e-4)


def test_propose_genes_limits():
    lo = np.array([-20.0, 5.0, 0.0, 0.0, 0.3, -4.0])
    hi = np.array([20.0, 100.0, 1.0, 2 * math.pi, 3.0, 0.0])
    mu = np.array([0.1, math.log(0.5), 0.3, 0.25, math.log(1.2), -2.0])
    out = np.concatenate([mu, np.full(6, -60.0)])[None]  # vanishing variance: the mean itself
    G = op.propose_genes(out, [(5.0, 40.0)], lo, hi, 3, seed=1)
    want = (np.array([5 + 40 * 0.1, 20.0, 0.3, math.pi / 2, 1.2, -2.0]) - lo) / (hi - lo)
    for r in range(3):
        np.testing.assert_allclose(G[0, r], want, rtol=1e-12)
    # log-variance -4: standard deviation e^-2, read back from the u0 gene (identity map, inside [0, 1])
    out2 = np.concatenate([np.array([0, 0, 0.5, 0, 0, -2.0]), np.array([0, 0, -4.0, 0, 0, 0])])[None]
    G2 = op.propose_genes(out2, [(0.0, 1.0)], lo, hi, 4000, seed=2)
    y2 = G2[0, :, 2]
    assert np.mean(y2) == pytest.approx(0.5, abs=0.01) and np.std(y2) == pytest.approx(math.exp(-2.0), rel=0.05)
    # clamping and the non-finite rule
    out3 = np.concatenate([np.array([np.nan, 50, -50, 0, 0, 0.0]), np.full(6, -60.0)])[None]
    G3 = op.propose_genes(out3, [(0.0, 1.0)], lo, hi, 1, seed=0)
    assert G3[0, 0, 0] == 0.5 and G3[0, 0, 1] == 1.0 and G3[0, 0, 2] == 0.0
