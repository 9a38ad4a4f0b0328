"""The success monitor of the batched fitter (sblm_fit_batch_monitored): Section 4.2 counts a
run as successful when some returned model has delta chi^2 / nu < 1 and every parameter within
10% of the truth, and Appendix A's EA returns every population of every generation. The device
tests each evaluated row as it is produced; here the same EA is replayed from the host one
generation at a time (sblm_ea_init / sblm_ea_generation, fitness from sblm_chi2_genes or
sblm_chi2_blend), every population is checked with a plain numpy statement of the criterion, and
the first generation with a match must equal the device's."""
import numpy as np
import pytest
import torch

from oracle import ea as oea
from oracle import sblm as osb
from paper_1208_4830_gb300 import synth

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.tensor(x, device="cuda")


def _match(theta, ref, tol, f=None, f_ref=None):
    """Rows of theta [n, 6] within tol of ref (Section 4.2, errors as in the bench's criterion)."""
    da = np.abs((theta[:, 3] - ref[3] + np.pi) % (2 * np.pi) - np.pi)
    ok = (np.abs(theta[:, 0] - ref[0]) < tol * ref[1]) & (np.abs(theta[:, 1] - ref[1]) < tol * ref[1])
    ok &= (np.abs(theta[:, 2] - ref[2]) < tol * ref[2]) & (da < tol * 2 * np.pi)
    ok &= (np.abs(theta[:, 4] - ref[4]) < tol * ref[4]) & (np.abs(theta[:, 5] - ref[5]) < tol * ref[5])
    if f_ref is not None:
        ok &= np.abs(f - f_ref) < tol * f_ref
    return ok


def _replay(lib, t, flux, sigma, lo, hi, p, stream_id, ref, bound, tol, blend=False, f_ref=None):
    P = torch.empty((p.n_pop, 6), dtype=torch.float64, device="cuda")
    state = lib.new_state_buffer("cuda")
    lib.ea_init(P, 6, p, stream_id, state)
    td, fd, sd = dev(t), dev(flux), dev(sigma)
    first = -1
    for g in range(p.n_gen):
        theta = oea.sblm_theta(P.cpu().numpy(), lo, hi)
        if blend:
            c, f = lib.chi2_blend(dev(theta), td, fd, sd, "fp64")
            f = f.cpu().numpy()
        else:
            c = lib.chi2_genes(P, td, fd, sd, lo, hi, "fp64")
            f = None
        if first < 0:
            hit = (c.cpu().numpy() < bound) & _match(theta, ref, tol, f, f_ref)
            if hit.any():
                first = g
        lib.ea_generation(P, c, p, stream_id, g, state)
    return first


def test_monitor_equals_host_replay(lib):
    b = synth.seasonal_batch(4, seed=12, n_min=80, n_max=200, span=(-100.0, 100.0), season=80.0, gap=30.0)
    A = np.concatenate([osb.magnification(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]])[0]
                        for i in range(4)])
    flux, sigma = b.observe(A)
    p = lib.params(n_pop=48, n_gen=30, precision="fp64", seed=3)
    sl = [slice(b.offsets[i], b.offsets[i + 1]) for i in range(4)]
    chi_true = np.array([osb.chi2(b.truth[i : i + 1], b.t[s], flux[s], sigma[s])[0] for i, s in enumerate(sl)])
    best0, chi0 = lib.fit_batch(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p)
    seen = set()
    for tol, scale in ((0.5, 40.0), (0.3, 20.0), (0.05, 2.0)):
        bound = scale * chi_true
        best, chi, first = lib.fit_batch_monitored(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p,
                                                   b.truth, bound, rel_tol=tol)
        # the monitor does not steer the search
        np.testing.assert_array_equal(chi, chi0)
        np.testing.assert_array_equal(best, best0)
        for i, s in enumerate(sl):
            want = _replay(lib, b.t[s], flux[s], sigma[s], synth.FIT_LO, synth.FIT_HI, p, i, b.truth[i], bound[i], tol)
            assert first[i] == want, (tol, i, first[i], want)
            seen.add(want > 0 if want >= 0 else -1)
    assert len(seen) >= 2  # the cases cover a match after generation 0 and no match (or at 0)


def test_monitor_with_the_blended_model(lib):
    bb = synth.noisy_blended_batch(3, seed=13)
    A = np.concatenate([osb.magnification(bb.truth[i : i + 1], bb.t[bb.offsets[i] : bb.offsets[i + 1]])[0]
                        for i in range(3)])
    flux, sigma = bb.observe(A)
    sl = [slice(bb.offsets[i], bb.offsets[i + 1]) for i in range(3)]
    chi_true = np.array([osb.chi2_blend(bb.truth[i : i + 1], bb.t[s], flux[s], sigma[s])[0][0]
                         for i, s in enumerate(sl)])
    p = lib.params(n_pop=40, n_gen=25, precision="fp64+blend", seed=4)
    q = lib.params(n_pop=40, n_gen=25, precision="fp64", seed=4)
    bound = chi_true + 93.0
    for tol in (0.6, 0.3):
        _, _, first = lib.fit_batch_monitored(bb.t, flux, sigma, bb.offsets, synth.PAPER_LO, synth.PAPER_HI, p,
                                              bb.truth, bound, f_ref=bb.f, rel_tol=tol)
        for i, s in enumerate(sl):
            want = _replay(lib, bb.t[s], flux[s], sigma[s], synth.PAPER_LO, synth.PAPER_HI, q, i, bb.truth[i],
                           bound[i], tol, blend=True, f_ref=bb.f[i])
            assert first[i] == want, (tol, i, first[i], want)


def test_monitor_arguments_are_checked(lib):
    b = synth.seasonal_batch(2, seed=14, n_min=50, n_max=60, span=(-100.0, 100.0), season=80.0, gap=30.0)
    flux, sigma = b.observe(np.ones(b.t.size))
    p = lib.params(n_pop=16, n_gen=2, precision="mixed")
    with pytest.raises(lib.SBLMError):
        lib.fit_batch_monitored(b.t, flux, sigma, b.offsets, synth.FIT_LO, synth.FIT_HI, p, b.truth, np.ones(2),
                                rel_tol=0.0)
