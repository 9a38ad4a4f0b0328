"""The island EA of Section 5.3 in the batched fitter (sblm_ea_params.n_islands,
migration_interval): every island is Appendix A's EA on its own stream (lightcurve l, island i:
stream id l + i n_lc), and every migration_interval generations the elite of island i replaces the
last row of island i + 1 (a ring; oracle/ea.py: migrate_ring). In FP64 the device must equal the
host replaying the islands one generation at a time with sblm_ea_init / sblm_chi2_genes /
sblm_ea_generation and the oracle's migration step."""
import numpy as np
import pytest
import torch

from oracle import ea as oea
from oracle import sblm as osb
from paper_1208_4830_gb300 import synth

pytestmark = pytest.mark.gpu


def _batch(n_lc, seed):
    b = synth.seasonal_batch(n_lc, seed=seed, n_min=60, n_max=200, span=(-100.0, 100.0), season=80.0, gap=30.0)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(n_lc)])
    flux, sigma = b.observe(A)
    return b, flux, sigma


def _replay(lib, t, flux, sigma, p, lc, n_lc, n_isl, interval):
    td, fd, sd = (torch.tensor(x, device="cuda") for x in (t, flux, sigma))
    Ps, states = [], []
    for i in range(n_isl):
        P = torch.empty((p.n_pop, 6), dtype=torch.float64, device="cuda")
        st = lib.new_state_buffer("cuda")
        lib.ea_init(P, 6, p, lc + i * n_lc, st)
        Ps.append(P)
        states.append(st)
    for g in range(p.n_gen):
        elites = []
        for i in range(n_isl):
            c = lib.chi2_genes(Ps[i], td, fd, sd, synth.FIT_LO, synth.FIT_HI, "fp64")
            cn = np.nan_to_num(c.cpu().numpy(), nan=np.inf)
            elites.append(Ps[i].cpu().numpy()[int(np.argmin(cn))])
            lib.ea_generation(Ps[i], c, p, lc + i * n_lc, g, states[i])
        if g + 1 < p.n_gen and interval > 0 and (g + 1) % interval == 0:
            nxt = oea.migrate_ring([P.cpu().numpy() for P in Ps], elites)
            for P, Q in zip(Ps, nxt):
                P.copy_(torch.tensor(Q, device="cuda"))
    s = [lib.read_state(x) for x in states]
    bi = int(np.argmin([x.best_chi2 for x in s]))
    a = synth.FIT_LO + (synth.FIT_HI - synth.FIT_LO) * np.array(s[bi].best_genes[:6])
    a[5] = 10.0 ** a[5]
    return a, s[bi].best_chi2


@pytest.mark.parametrize("n_isl,interval", [(3, 4), (2, 1), (4, 0)])
def test_fp64_islands_equal_host_replay(lib, n_isl, interval):
    b, flux, sigma = _batch(3, seed=31)
    p = lib.params(n_pop=24, n_gen=14, precision="fp64", seed=6, n_islands=n_isl, migration_interval=interval)
    best, chi = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    for i in range(3):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        th, c = _replay(lib, b.t[sl], flux[sl], sigma[sl], p, i, 3, n_isl, interval)
        assert chi[i] == pytest.approx(c, rel=1e-12)
        np.testing.assert_allclose(best[i], th, rtol=1e-12, atol=1e-12)


def test_one_island_is_the_default_fitter(lib):
    b, flux, sigma = _batch(2, seed=32)
    p = lib.params(n_pop=32, n_gen=10, precision="mixed", seed=1)
    ref = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    p.n_islands = 1
    got = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    np.testing.assert_array_equal(got[1], ref[1])
    np.testing.assert_array_equal(got[0], ref[0])


def test_mixed_islands_with_polish_report_the_oracle_chi2(lib):
    b, flux, sigma = _batch(6, seed=33)
    p = lib.params(n_pop=64, n_gen=40, precision="mixed", seed=2, n_islands=4, migration_interval=10,
                   polish_fev=200)
    best, chi = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    for i in range(6):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        ref = osb.chi2(best[i : i + 1], b.t[sl], flux[sl], sigma[sl])[0]
        assert abs(chi[i] - ref) <= 1e-4 * ref + 1e-6


def test_islands_are_checked(lib):
    b, flux, sigma = _batch(1, seed=34)
    with pytest.raises(lib.SBLMError):
        lib.fit(b.t, flux, sigma, synth.FIT_LO, synth.FIT_HI, lib.params(n_pop=16, n_gen=2, n_islands=2))
    with pytest.raises(lib.SBLMError):
        lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI,
                      lib.params(n_pop=16, n_gen=2, n_islands=65))
