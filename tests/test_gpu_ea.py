"""Parity of the device EA operators (sblm_ea_init, sblm_ea_generation) with the oracle's, and
end-to-end behaviour of sblm_fit.

Given the same population, fitness and Philox key, the device must draw the same numbers and
take the same integer decisions (ranks, parents, modes, jumps, restarts); genes then agree bit
for bit except where exp() enters the creep step, where they may differ by an ulp or two.
"""
import numpy as np
import pytest
import torch

from oracle import ea as oea
from oracle import sblm as osb
from paper_1208_4830_gb300 import synth

pytestmark = pytest.mark.gpu
GENE_TOL = 1e-15  # two ulps of the largest gene value


def dev(x):
    return torch.tensor(x, device="cuda")


def oparams(n_pop, seed, stream, **kw):
    return oea.EAParams(n_pop=n_pop, seed=seed, stream=stream, **kw)


@pytest.mark.parametrize("n_pop,n_par,seed,stream", [(64, 6, 0, 0), (37, 5, 9, 3), (1024, 6, 2**40 + 1, 7), (5, 3, 1, 1)])
def test_init_bit_exact(lib, n_pop, n_par, seed, stream):
    P = torch.empty((n_pop, n_par), dtype=torch.float64, device="cuda")
    state = lib.new_state_buffer("cuda")
    lib.ea_init(P, n_par, lib.params(n_pop=n_pop, seed=seed), stream, state)
    ref = oea.init_population(n_pop, n_par, oparams(n_pop, seed, stream), 0)
    assert np.array_equal(P.cpu().numpy(), ref)
    s = lib.read_state(state)
    assert s.p_mut == 0.01 and s.n_hist == 0 and np.isinf(s.best_chi2)


def _fitness(rng, n_pop):
    chi = rng.uniform(0, 100, n_pop)
    if n_pop >= 8:
        chi[rng.choice(n_pop, 3, replace=False)] = np.nan
        chi[5] = chi[7]  # a tie: broken by row order
        chi[2] = np.inf
    return chi


@pytest.mark.parametrize("n_pop,n_par", [(64, 6), (65, 6), (1000, 6), (8, 16), (2, 6), (4096, 6)])
def test_generation_matches_oracle(lib, n_pop, n_par):
    rng = np.random.default_rng(n_pop)
    op = oparams(n_pop, 11, 2)
    P0 = oea.init_population(n_pop, n_par, op, 0)
    chi = _fitness(rng, n_pop)
    P = dev(P0)
    state = lib.new_state_buffer("cuda")
    p = lib.params(n_pop=n_pop, seed=11, p_mut0=0.05)
    lib.ea_init(torch.empty_like(P), n_par, p, 2, state)
    lib.ea_generation(P, dev(chi), p, 2, 0, state)
    op.p_mut0 = 0.05
    st = oea.new_state(op)
    ref = oea.generation(P0, chi, st, op, 0)
    got = P.cpu().numpy()
    assert np.abs(got - ref).max() <= GENE_TOL
    assert np.mean(got == ref) > 0.9
    s = lib.read_state(state)
    assert s.p_mut == st.p_mut and s.stag_run == st.stag_run and s.best_chi2 == st.best_chi2
    assert np.array_equal(np.array(s.best_genes[:n_par]), st.best_genes)


def test_chained_generations_with_restart(lib):
    """Constant fitness stagnates: the 10th consecutive stagnant generation (t = 19) restarts
    the population from the initialisation of generation 20."""
    n_pop, n_par = 48, 6
    op = oparams(n_pop, 4, 0)
    p = lib.params(n_pop=n_pop, seed=4)
    P0 = oea.init_population(n_pop, n_par, op, 0)
    P = dev(P0)
    state = lib.new_state_buffer("cuda")
    lib.ea_init(torch.empty_like(P), n_par, p, 0, state)
    st = oea.new_state(op)
    ref = P0
    chi = np.full(n_pop, 7.0)
    for g in range(22):
        lib.ea_generation(P, dev(chi), p, 0, g, state)
        ref = oea.generation(ref, chi, st, op, g)
        got = P.cpu().numpy()
        assert np.abs(got - ref).max() <= GENE_TOL, g
        ref = got  # continue from the device's population so ulp differences do not accumulate
        s = lib.read_state(state)
        assert s.n_restarts == st.n_restarts and s.p_mut == st.p_mut and s.stag_run == st.stag_run, g
    assert st.n_restarts == 1
    assert np.array_equal(oea.init_population(n_pop, n_par, op, 20),
                          oea.init_population(n_pop, n_par, op, 20))


def test_sphere_driven_by_device_operators(lib):
    """An external fitness (a sphere, evaluated with torch on the GPU) drives the device EA."""
    target = torch.tensor([0.3, 0.7, 0.11, 0.93, 0.5, 0.42], device="cuda", dtype=torch.float64)
    p = lib.params(n_pop=64, seed=1)
    P = torch.empty((64, 6), dtype=torch.float64, device="cuda")
    state = lib.new_state_buffer("cuda")
    lib.ea_init(P, 6, p, 0, state)
    for g in range(200):
        chi = ((P - target) ** 2).sum(1)
        lib.ea_generation(P, chi, p, 0, g, state)
    s = lib.read_state(state)
    assert s.best_chi2 < 1e-6


def _config1():
    lc = synth.single_fit_lightcurve(0)
    A = osb.magnification(lc.truth[None, :], lc.t)[0]
    flux, sigma = lc.observe(A)
    chi_true = osb.chi2(lc.truth[None, :], lc.t, flux, sigma)[0]
    return lc, flux, sigma, chi_true


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fit_trace_and_result_consistent(lib, prec):
    lc, flux, sigma, _ = _config1()
    p = lib.params(n_pop=64, n_gen=100, precision=prec, seed=0)
    best, best_chi2, tr = lib.fit(lc.t, flux, sigma, synth.FIT_LO, synth.FIT_HI, p, trace=True)
    # the archive is monotone and ends at the returned value
    assert np.all(np.diff(tr[:, 3]) <= 0) and tr[-1, 3] == best_chi2
    # the returned parameters reproduce the returned chi^2 (oracle)
    ref = osb.chi2(best[None, :], lc.t, flux, sigma)[0]
    assert abs(ref - best_chi2) <= (1e-9 if prec == "fp64" else 1e-4) * ref
    assert np.all(best >= [-20, 5, 0, 0, 0.3, 1e-4]) and np.all(best <= [20, 100, 1, 2 * np.pi, 3, 1])


def test_fit_recovers_injected_event(lib):
    """Recovery of the single-lightcurve event, judged by delta chi^2 <= 1 against the truth: the EA
    with the amoeba of Section 4.1 (without it the EA alone stopped at delta chi^2 = 2.5 next to the
    truth in one build: its last digits are not converged by a generation budget)."""
    lc, flux, sigma, chi_true = _config1()
    p = lib.params(n_pop=1024, n_gen=300, precision="mixed", seed=0, polish_fev=2000)
    best, best_chi2 = lib.fit(lc.t, flux, sigma, synth.FIT_LO, synth.FIT_HI, p)
    assert best_chi2 - chi_true <= 1.0, (best, best_chi2, chi_true)


@pytest.mark.parametrize("n_pops,n_pop,n_par", [(5, 64, 6), (3, 37, 5), (2, 1024, 6)])
def test_batched_generation_equals_single_calls(lib, n_pops, n_pop, n_par):
    """sblm_ea_generation_batch: n_pops populations in one launch per operator equal n_pops calls of
    sblm_ea_generation with stream ids stream_id0 + b, over generations that include a restart
    (constant fitness makes every generation stagnant)."""
    p = lib.params(n_pop=n_pop, seed=11, restart_after=2, stag_window=2)
    P0 = torch.empty((n_pops * n_pop, n_par), dtype=torch.float64, device="cuda")
    states = torch.stack([lib.new_state_buffer("cuda") for _ in range(n_pops)])
    for b in range(n_pops):
        lib.ea_init(P0[b * n_pop : (b + 1) * n_pop], n_par, p, 4 + b, states[b])
    Pb, sb = P0.clone(), states.clone()
    Ps, ss = P0.clone(), states.clone()
    g = np.random.default_rng(3)
    for gen in range(7):
        chi = g.uniform(0, 100, n_pops * n_pop) if gen % 3 else np.full(n_pops * n_pop, 5.0)
        chi[::17] = np.nan
        chi_d = dev(chi)
        lib.ea_generation_batch(Pb, chi_d, p, 4, gen, sb)
        for b in range(n_pops):
            rows = slice(b * n_pop, (b + 1) * n_pop)
            lib.ea_generation(Ps[rows], chi_d[rows], p, 4 + b, gen, ss[b])
        assert torch.equal(Pb, Ps)
        assert torch.equal(sb, ss)
    assert any(lib.read_state(ss[b]).n_restarts > 0 for b in range(n_pops))
