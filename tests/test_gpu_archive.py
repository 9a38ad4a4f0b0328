"""The persistent fitter's solution archive (sblm_fit_batch_archived) against the oracle's
SolutionArchive (oracle/ea.py) fed the same ranked populations: in FP64 the batched fitter is the
EA of Appendix A step for step (tests/test_gpu_batch.py), so replaying each lightcurve's
generations from the host with the single-population entry points and offering every ranked
population to the oracle's archive must give the device's archive."""
import numpy as np
import pytest
import torch

from oracle import ea as oea
from oracle import sblm as osb
from paper_1208_4830_gb300 import synth

pytestmark = pytest.mark.gpu


def _decode(genes):
    a = synth.FIT_LO + (synth.FIT_HI - synth.FIT_LO) * np.asarray(genes)
    a[..., 5] = 10.0 ** a[..., 5]
    return a


def _replay_archive(lib, t, flux, sigma, p, stream_id, size, radius, top):
    n_pop = p.n_pop
    P = torch.empty((n_pop, 6), dtype=torch.float64, device="cuda")
    state = lib.new_state_buffer("cuda")
    lib.ea_init(P, 6, p, stream_id, state)
    td, fd, sd = (torch.tensor(x, device="cuda") for x in (t, flux, sigma))
    chi = torch.empty(n_pop, dtype=torch.float64, device="cuda")
    arc = oea.SolutionArchive(size, radius)
    for g in range(p.n_gen):
        lib.chi2_genes(P, td, fd, sd, synth.FIT_LO, synth.FIT_HI, p.precision, out=chi)
        Ph, ch = P.cpu().numpy(), chi.cpu().numpy()
        key = np.where(np.isnan(ch), np.inf, ch)
        order = np.argsort(key, kind="stable")
        arc.offer_ranked(Ph[order], key[order], top=top or None)
        lib.ea_generation(P, chi, p, stream_id, g, state)
    return arc


@pytest.mark.parametrize("size,radius,top", [(5, 0.02, 10), (3, 0.2, 0), (8, 0.005, 40)])
def test_fp64_archive_equals_oracle_replay(lib, size, radius, top):
    b = synth.seasonal_batch(3, seed=9, n_min=80, n_max=250, span=(-100.0, 100.0), season=80.0, gap=30.0)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(3)])
    flux, sigma = b.observe(A)
    p = lib.params(n_pop=48, n_gen=14, precision="fp64", seed=5)
    best, chi, a_th, a_c, a_n = lib.fit_batch_archived(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p,
                                                       size=size, radius=radius, top=top)
    for i in range(3):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        arc = _replay_archive(lib, b.t[sl], flux[sl], sigma[sl], p, i, size, radius, top)
        n = len(arc.chi2)
        assert a_n[i] == n
        np.testing.assert_allclose(a_c[i, :n], arc.chi2, rtol=1e-12)
        np.testing.assert_allclose(a_th[i, :n], _decode(np.array(arc.genes)), rtol=1e-12, atol=1e-12)
        assert np.all(np.isnan(a_c[i, n:])) and np.all(np.isnan(a_th[i, n:]))
        # the first entry is the EA's best (no polish here); entries are distinct and sorted
        assert a_c[i, 0] == pytest.approx(chi[i], rel=1e-12)
        assert np.all(np.diff(a_c[i, :n]) >= 0)


def test_mixed_archive_holds_distinct_solutions(lib):
    """MIXED, islands: the archive is sorted, its entries pairwise distinct in the genes, its first
    entry the best of the fit, and its chi^2 values those of the oracle for the archived rows."""
    b = synth.heldout_batch(4, seed=41, n_ep=300)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(4)])
    flux, sigma = b.observe(A)
    p = lib.params(n_pop=128, n_gen=40, precision="mixed", seed=2, n_islands=2, migration_interval=10)
    best, chi, a_th, a_c, a_n = lib.fit_batch_archived(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p,
                                                       size=6, radius=0.05)
    for i in range(4):
        n = a_n[i]
        assert 1 <= n <= 6 and np.all(np.diff(a_c[i, :n]) >= 0)
        assert a_c[i, 0] == pytest.approx(chi[i], rel=1e-12)
        g = (np.column_stack([a_th[i, :n, :5], np.log10(a_th[i, :n, 5])]) - synth.FIT_LO) / (synth.FIT_HI - synth.FIT_LO)
        for j in range(n):
            for k in range(j + 1, n):
                assert np.max(np.abs(g[j] - g[k])) > 0.05 - 1e-9
        sl = slice(b.offsets[i], b.offsets[i + 1])
        ref = osb.chi2(a_th[i, :n], b.t[sl], flux[sl], sigma[sl])
        np.testing.assert_allclose(a_c[i, :n], ref, rtol=1e-3)


def test_archive_rejects_bad_settings(lib):
    b = synth.seasonal_batch(2, seed=3, n_min=50, n_max=60)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(2)])
    flux, sigma = b.observe(A)
    p = lib.params(n_pop=16, n_gen=2, precision="fp64")
    for kw in ({"size": 0}, {"size": 65}, {"radius": 0.0}, {"top": -1}):
        args = dict(size=4, radius=0.05, top=0)
        args.update(kw)
        with pytest.raises(lib.SBLMError):
            lib.fit_batch_archived(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p, **args)


def test_polish_from_several_starts(lib):
    """polish_starts = K: the amoeba runs from each of the K fittest distinct solutions the EA
    evaluated (the archive rule) and the fittest result is returned. In FP64 that equals polishing
    each entry of the archive the same fit returns (sblm_polish_batch) and keeping the best; it is
    never worse than the single start of the paper's EA + amoeba."""
    b = synth.heldout_batch(6, seed=51, n_ep=300)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(6)])
    flux, sigma = b.observe(A)
    args = (b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI)
    p1 = lib.params(n_pop=96, n_gen=25, precision="fp64", seed=3, polish_fev=300)
    pk = lib.params(n_pop=96, n_gen=25, precision="fp64", seed=3, polish_fev=300, polish_starts=4,
                    polish_radius=0.05)
    _, c1 = lib.fit_batch(*args, p1)
    best_k, ck = lib.fit_batch(*args, pk)
    assert np.all(ck <= c1 * (1 + 1e-12))
    # host replay: the archive of the same EA, every entry polished, the fittest kept
    p0 = lib.params(n_pop=96, n_gen=25, precision="fp64", seed=3)
    _, c_ea, a_th, a_c, a_n = lib.fit_batch_archived(*args, p0, size=4, radius=0.05)
    for i in range(6):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        n = int(a_n[i])
        g = np.column_stack([a_th[i, :n, :5], np.log10(a_th[i, :n, 5])])
        g = (g - synth.FIT_LO) / (synth.FIT_HI - synth.FIT_LO)
        off = np.array([0] + [sl.stop - sl.start] * n, dtype=np.int64).cumsum()
        tt, ff, ss = (np.tile(x[sl], n) for x in (b.t, flux, sigma))
        _, cp = lib.polish_batch(tt, ff, ss, off, synth.FIT_LO, synth.FIT_HI, np.ascontiguousarray(g), 300, "fp64")
        assert ck[i] == pytest.approx(min(cp.min(), c_ea[i]), rel=1e-9)


def test_polish_starts_validation(lib):
    b = synth.seasonal_batch(2, seed=3, n_min=50, n_max=60)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(2)])
    flux, sigma = b.observe(A)
    for kw in ({"polish_starts": 65}, {"polish_starts": 3, "polish_radius": 0.0}):
        p = lib.params(n_pop=16, n_gen=2, precision="fp64", polish_fev=10, **kw)
        with pytest.raises(lib.SBLMError):
            lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
