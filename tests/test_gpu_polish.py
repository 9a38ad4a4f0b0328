"""The amoeba fine-tuning on the device (sblm_polish_batch, and the polish_fev stage of the
fitters) against the oracle's downhill simplex (oracle/polish.py)."""
import numpy as np
import pytest
import torch

from oracle import polish as opo
from oracle import sblm as osb
from paper_1208_4830_gb300 import synth

pytestmark = pytest.mark.gpu


def _curves(n_lc, seed):
    b = synth.heldout_batch(n_lc, seed=seed, n_ep=300)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(n_lc)])
    flux, sigma = b.observe(A)
    return b, flux, sigma


def _genes(theta):
    v = theta.copy()
    v[..., 5] = np.log10(v[..., 5])
    return (v - synth.FIT_LO) / (synth.FIT_HI - synth.FIT_LO)


def test_fp64_polish_follows_the_oracle_simplex(lib):
    """In FP64 both sides take the same simplex steps: the same vertex after 60 evaluations."""
    b, flux, sigma = _curves(4, seed=31)
    start = np.clip(_genes(b.truth) + np.random.default_rng(0).normal(0, 0.01, (4, 6)), 0, 1)
    g, c = lib.polish_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, start, 60, "fp64")
    for i in range(4):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        rg, rc, _ = opo.polish_sblm(b.t[sl], flux[sl], sigma[sl], synth.FIT_LO, synth.FIT_HI, start[i], 60)
        np.testing.assert_allclose(g[i], rg, rtol=0, atol=1e-9)
        assert c[i] == pytest.approx(rc, rel=1e-10)


def test_mixed_polish_improves_and_recovers_near_misses(lib):
    b, flux, sigma = _curves(8, seed=32)
    start = np.clip(_genes(b.truth) + np.random.default_rng(1).normal(0, 0.004, (8, 6)), 0, 1)
    dev = [torch.tensor(x, device="cuda") for x in (b.t, flux, sigma, b.offsets, start)]
    g, c = lib.polish_batch(*dev[:4], synth.FIT_LO, synth.FIT_HI, dev[4], 1500, "mixed")
    ok = 0
    for i in range(8):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        c0 = osb.chi2(osb_theta(start[i]), b.t[sl], flux[sl], sigma[sl])[0]
        ct = osb.chi2(b.truth[i : i + 1], b.t[sl], flux[sl], sigma[sl])[0]
        cr = osb.chi2(osb_theta(g[i]), b.t[sl], flux[sl], sigma[sl])[0]
        assert c[i] == pytest.approx(cr, rel=1e-4)  # the reported chi^2 is that of the returned genes
        assert cr <= c0 * (1 + 1e-6)
        ok += cr - ct <= 1.0
    assert ok >= 6, ok


def osb_theta(g):
    from oracle import ea

    return ea.sblm_theta(np.asarray(g)[None, :], synth.FIT_LO, synth.FIT_HI)


def test_fitters_with_polish_never_lose(lib):
    b, flux, sigma = _curves(6, seed=33)
    p0 = lib.params(n_pop=64, n_gen=15, precision="fp64", seed=2)
    p1 = lib.params(n_pop=64, n_gen=15, precision="fp64", seed=2, polish_fev=400)
    best0, chi0 = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p0)
    best1, chi1 = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p1)
    assert np.all(chi1 <= chi0) and np.any(chi1 < chi0)
    for i in range(6):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        assert chi1[i] == pytest.approx(osb.chi2(best1[i : i + 1], b.t[sl], flux[sl], sigma[sl])[0], rel=1e-10)
    # the single-lightcurve driver runs the same stage
    sl = slice(b.offsets[0], b.offsets[1])
    th0, c0 = lib.fit(b.t[sl], flux[sl], sigma[sl], synth.FIT_LO, synth.FIT_HI, p0)
    th1, c1 = lib.fit(b.t[sl], flux[sl], sigma[sl], synth.FIT_LO, synth.FIT_HI, p1)
    assert c1 <= c0 and c1 == pytest.approx(osb.chi2(th1[None], b.t[sl], flux[sl], sigma[sl])[0], rel=1e-10)
