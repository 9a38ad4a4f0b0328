"""Shapes of the synthetic inputs that stand in for the paper's workloads (no method arithmetic)."""
import numpy as np

from paper_1208_4830_gb300 import synth


def test_paper_batch_follows_the_paper_test_setup():
    b = synth.paper_batch(40, seed=5)
    assert b.offsets[-1] == 40 * 100 and np.all(np.diff(b.offsets) == 100)
    for i in range(40):
        t = b.t[b.offsets[i] : b.offsets[i + 1]]
        t0, tE = b.truth[i, 0], b.truth[i, 1]
        assert -3 < (t[0] - t0) / tE < -2 and 2 < (t[-1] - t0) / tE < 3
        np.testing.assert_allclose(np.diff(t), np.diff(t)[0], rtol=1e-9)  # evenly spaced
    g = b.truth.copy()
    g[:, 5] = np.log10(g[:, 5])
    assert np.all((g >= synth.PAPER_LO) & (g <= synth.PAPER_HI))
    assert b.truth[:, 5].min() >= 0.1
    assert abs(synth.PAPER_SIGMA_FRAC - 0.00921034) < 1e-7  # 0.01 mag as a flux fraction


def test_count_peaks():
    x = np.linspace(0, 1, 2001)
    one = 1 + np.exp(-((x - 0.5) / 0.05) ** 2)
    two = one + 0.5 * np.exp(-((x - 0.8) / 0.02) ** 2)
    assert synth.count_peaks(one) == 1 and synth.count_peaks(two) == 2
    ripple = one + 1e-4 * np.sin(200 * x)  # bumps below 1% prominence are not peaks
    assert synth.count_peaks(ripple) == 1


def test_heldout_truths_inside_the_fit_domain():
    b = synth.heldout_batch(200, seed=3, n_ep=50)
    g = b.truth.copy()
    g[:, 5] = np.log10(g[:, 5])
    assert np.all((g >= synth.FIT_LO) & (g <= synth.FIT_HI))
    assert b.offsets[-1] == 200 * 50


def test_noisy_blended_batch_follows_the_paper_setup():
    """Section 4.4's changes to the test: random epochs, the noise model of Section 2.4, blending."""
    b = synth.noisy_blended_batch(50, seed=6)
    assert b.offsets[-1] == 50 * 100
    assert np.all((b.f > 0) & (b.f <= 1)) and np.all((b.m0 >= 18) & (b.m0 <= 22))
    for i in range(50):
        t = b.t[b.offsets[i] : b.offsets[i + 1]]
        t0, tE = b.truth[i, 0], b.truth[i, 1]
        assert np.all(np.diff(t) >= 0) and (t[0] - t0) / tE > -3 and (t[-1] - t0) / tE < 3
        assert np.std(np.diff(t)) > 0.1 * np.mean(np.diff(t))  # not evenly spaced
    # m0 is the source's unlensed magnitude (Section 2), so at baseline (A = 1) the light is the
    # unlensed blend of magnitude m0 + 2.5 log10 f, and its error is the noise model's there:
    # log10 sigma = 0.3416 m - 7.7095
    flux, sigma = b.observe(np.ones(b.t.size))
    n = np.diff(b.offsets)
    m_base = np.repeat(b.m0 + 2.5 * np.log10(b.f), n)
    np.testing.assert_allclose(sigma, 0.4 * np.log(10) * 10 ** (0.3416 * m_base - 7.7095), rtol=1e-12)
    r = -2.5 * np.log10(flux) / 10 ** (0.3416 * m_base - 7.7095)
    np.testing.assert_allclose(r, b.z, atol=1e-9)
    # an unblended source (f = 1) at baseline has magnitude m0; the blend is brighter than the source
    b1 = synth.noisy_blended_batch(50, seed=6)
    b1.f[:] = 1.0
    _, s1 = b1.observe(np.ones(b1.t.size))
    np.testing.assert_allclose(s1, 0.4 * np.log(10) * 10 ** (0.3416 * np.repeat(b1.m0, n) - 7.7095), rtol=1e-12)
    assert np.all(sigma <= s1)
    # f dilutes the source magnification: F - 1 = f (A - 1) without noise
    b.z[:] = 0.0
    A = np.linspace(1.0, 30.0, b.t.size)
    flux, _ = b.observe(A)
    np.testing.assert_allclose(flux - 1, np.repeat(b.f, n) * (A - 1), rtol=1e-9, atol=1e-12)
