"""The persistent batched fitter (sblm_fit_batch): every lightcurve's fit must be the EA of
Appendix A with that lightcurve's stream id. In FP64 this is checked step for step against the
single-population entry points (sblm_ea_init, sblm_chi2_genes, sblm_ea_generation) driven from
the host; in MIXED by the consistency of each returned chi^2 with the oracle's and by recovery."""
import numpy as np
import pytest
import torch

from oracle import sblm as osb
from paper_1208_4830_gb300 import synth

pytestmark = pytest.mark.gpu


def _batch(n_lc, seed, n_min, n_max):
    b = synth.seasonal_batch(n_lc, seed=seed, n_min=n_min, n_max=n_max, span=(-100.0, 100.0), season=80.0, gap=30.0)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(n_lc)])
    flux, sigma = b.observe(A)
    return b, flux, sigma


def _emulate(lib, t, flux, sigma, p, stream_id):
    """The same fit from the host, one generation at a time."""
    n_pop = p.n_pop
    P = torch.empty((n_pop, 6), dtype=torch.float64, device="cuda")
    state = lib.new_state_buffer("cuda")
    lib.ea_init(P, 6, p, stream_id, state)
    td, fd, sd = (torch.tensor(x, device="cuda") for x in (t, flux, sigma))
    chi = torch.empty(n_pop, dtype=torch.float64, device="cuda")
    for g in range(p.n_gen):
        lib.chi2_genes(P, td, fd, sd, synth.FIT_LO, synth.FIT_HI, p.precision, out=chi)
        lib.ea_generation(P, chi, p, stream_id, g, state)
    s = lib.read_state(state)
    genes = np.array(s.best_genes[:6])
    a = synth.FIT_LO + (synth.FIT_HI - synth.FIT_LO) * genes
    a[5] = 10.0 ** a[5]
    return a, s.best_chi2


def test_fp64_batch_equals_host_driven_generations(lib):
    b, flux, sigma = _batch(4, seed=2, n_min=60, n_max=300)
    p = lib.params(n_pop=48, n_gen=12, precision="fp64", seed=7)
    best, chi = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    for i in range(4):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        th, c = _emulate(lib, b.t[sl], flux[sl], sigma[sl], p, i)
        assert chi[i] == pytest.approx(c, rel=1e-12)
        np.testing.assert_allclose(best[i], th, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("tuning", [(8, 256), (32, 512), (16, 128)])
def test_launch_shapes_agree_in_fp64(lib, tuning):
    b, flux, sigma = _batch(3, seed=3, n_min=100, n_max=400)
    p = lib.params(n_pop=32, n_gen=6, precision="fp64", seed=1)
    ref = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    got = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p, tuning=tuning)
    np.testing.assert_allclose(got[1], ref[1], rtol=1e-12)


def test_mixed_batch_chi2_consistent_with_oracle(lib):
    b, flux, sigma = _batch(10, seed=4, n_min=200, n_max=1500)
    p = lib.params(n_pop=128, n_gen=20, precision="mixed", seed=3)
    best, chi = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    for i in range(10):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        ref = osb.chi2(best[i : i + 1], b.t[sl], flux[sl], sigma[sl])[0]
        assert abs(chi[i] - ref) <= 1e-4 * ref + 1e-6, (i, chi[i], ref)
    # repeated call replays the captured graph with the same arguments: same answers
    best2, chi2 = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    np.testing.assert_allclose(chi2, chi, rtol=1e-9)


def test_device_buffers_and_one_lightcurve(lib):
    b, flux, sigma = _batch(1, seed=5, n_min=300, n_max=300)
    p = lib.params(n_pop=64, n_gen=10, precision="mixed", seed=2)
    dev = [torch.tensor(x, device="cuda") for x in (b.t, flux, sigma, b.offsets)]
    best, chi = lib.fit_batch(*dev, synth.FIT_LO, synth.FIT_HI, p)
    ref = osb.chi2(best, b.t, flux, sigma)[0]
    assert abs(chi[0] - ref) <= 1e-4 * ref


def test_batch_recovers_injected_events(lib):
    """32 short seasonal lightcurves, 0.5-5% noise, N_pop 512 x 150 generations: most fits reach
    delta chi^2 <= 1 against the injected truth (25 of 32 when this test was written)."""
    b, flux, sigma = _batch(32, seed=6, n_min=200, n_max=400)
    p = lib.params(n_pop=512, n_gen=150, precision="mixed", seed=0)
    best, chi = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    ok = 0
    for i in range(32):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        chi_true = osb.chi2(b.truth[i : i + 1], b.t[sl], flux[sl], sigma[sl])[0]
        ok += chi[i] - chi_true <= 1.0
    assert ok >= 20, ok


def test_batch_rejects_bad_layouts(lib):
    b, flux, sigma = _batch(2, seed=7, n_min=50, n_max=60)
    p = lib.params(n_pop=16, n_gen=2, precision="fp32")
    bad = b.offsets.copy()
    bad[0] = 1
    with pytest.raises(lib.SBLMError, match="offsets"):
        lib.fit_batch(b.t, flux, sigma, bad, synth.FIT_LO, synth.FIT_HI, p)
    bad = b.offsets.copy()
    bad[1] = bad[0]
    with pytest.raises(lib.SBLMError, match="no epochs"):
        lib.fit_batch(b.t, flux, sigma, bad, synth.FIT_LO, synth.FIT_HI, p)
    long_t = np.sort(np.random.default_rng(0).uniform(-60, 60, 20000))
    with pytest.raises(lib.SBLMError, match="staging"):
        lib.fit_batch(long_t, np.ones(20000), np.full(20000, 0.01), np.array([0, 20000], dtype=np.int64),
                      synth.FIT_LO, synth.FIT_HI, lib.params(n_pop=1024, n_gen=1, precision="fp64"))


def test_autotuner_returns_a_valid_shape(lib, tmp_path):
    b, flux, sigma = _batch(4, seed=8, n_min=100, n_max=200)
    p = lib.params(n_pop=64, n_gen=5, precision="mixed")
    cache = str(tmp_path / "tune.json")
    t1 = lib.autotune_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p, cache=cache)
    assert t1.group in (8, 16, 32) and t1.block in (256, 512)
    t2 = lib.autotune_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p, cache=cache)
    assert (t2.group, t2.block) == (t1.group, t1.block)
    lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p, tuning=t1)
