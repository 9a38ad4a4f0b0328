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
