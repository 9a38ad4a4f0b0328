"""Pins of the oracle's EA operators (Appendix A) against closed forms, invariants and
hand-worked sequences."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import ea

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def params(**kw):
    base = dict(n_pop=64, n_gen=10, seed=3, stream=0)
    base.update(kw)
    return ea.EAParams(**base)


def test_initialisation_is_antithetic_and_uniform():
    p = params(n_pop=100)
    P = ea.init_population(100, 6, p, 0)
    flat = np.sort(P.ravel())
    assert np.all((flat >= 0) & (flat <= 1))
    # every value X has its complement 1 - X somewhere else (exactly: 1 - X is exact for X = k 2^-53)
    assert np.array_equal(flat + flat[::-1], np.ones_like(flat))
    assert stats.kstest(flat, "uniform").pvalue > 1e-3
    # partners are random elements: the share sharing a row is near (N_par - 1)/(M - 1)
    same_row = 0
    vals = P.ravel()
    for r in range(100):
        row = P[r]
        for v in row:
            same_row += np.count_nonzero(np.isclose(row, 1 - v, rtol=0, atol=0)) > 0
    assert same_row / vals.size < 0.05


def test_initialisation_odd_count_and_fresh_draws():
    P = ea.init_population(5, 3, params(n_pop=5), 0)  # 15 elements: 7 pairs + 1 plain draw
    flat = np.sort(P.ravel())
    sums = flat[:, None] + flat[None, :]
    n_pairs = sum(np.count_nonzero(sums[i] == 1.0) > 0 for i in range(15))
    assert n_pairs >= 14
    assert not np.array_equal(P, ea.init_population(5, 3, params(n_pop=5), 1))


def test_rank_is_stable_and_nan_last():
    P = np.arange(12.0).reshape(6, 2)
    chi2 = np.array([3.0, np.nan, 1.0, 3.0, 0.5, np.inf])
    Pr, cr, order = ea.rank(P, chi2)
    assert list(order) == [4, 2, 0, 3, 1, 5]
    assert np.isinf(cr[-2:]).all()


@pytest.mark.parametrize("n_pop,k", [(64, 3), (1000, 40), (10, 1)])
def test_tournament_rank_distribution(n_pop, k):
    """min of k uniform draws from {0..N-1}: P(rank <= r) = 1 - (1 - (r+1)/N)^k."""
    ranks = ea.tournament(n_pop, k, 40000, params(n_pop=n_pop), 7)
    r = np.arange(n_pop)
    cdf = 1 - (1 - (r + 1) / n_pop) ** k
    emp = np.searchsorted(np.sort(ranks), r, side="right") / ranks.size
    assert np.max(np.abs(emp - cdf)) < 0.015


def test_default_tournament_size():
    assert params(n_pop=1000).tournament_size() == 40
    assert params(n_pop=64).tournament_size() == 3
    assert params(n_pop=1024).tournament_size() == 41


def test_reproduction_modes_and_invariants():
    g = np.random.default_rng(0)
    n_pop, n_par = 301, 6
    Pr = g.uniform(0, 1, (n_pop, n_par))
    parents = g.integers(0, n_pop, 2 * (n_pop // 2))
    children, modes = ea.reproduce(Pr, parents, params(n_pop=n_pop), 4)
    assert children.shape == (n_pop - 1, n_par)
    freq = np.bincount(modes, minlength=3) / modes.size
    assert np.all(np.abs(freq - 1 / 3) < 0.1)
    for k, m in enumerate(modes):
        a, b = Pr[parents[2 * k]], Pr[parents[2 * k + 1]]
        c1, c2 = children[2 * k], children[2 * k + 1]
        assert np.allclose(c1 + c2, a + b, rtol=0, atol=4e-16)  # convex combinations with F and I - F
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        assert np.all((c1 >= lo - 1e-16) & (c1 <= hi + 1e-16))
        if m == 2:  # f = 1: clones
            assert np.array_equal(c1, a) and np.array_equal(c2, b)
        if m == 1:  # f in {0, 1}: genes swapped, never blended
            assert np.all((c1 == a) | (c1 == b))
            assert np.all(np.where(c1 == a, c2 == b, c2 == a))


def test_creep_step_is_log_uniform():
    n = 20000
    off = np.full((n, 1), 0.5)
    out, jumped = ea.mutate(off, 0.0, params(n_pop=n + 1), 2)
    assert not jumped.any()
    step = np.abs(out[:, 0] - 0.5) * 2.0  # X, since the distance to either bound is 0.5
    u = np.log(step) / ea.LN_EPS  # ln X ~ U(ln eps, 0)  <=>  ln X / ln eps ~ U(0, 1)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    up = np.mean(out[:, 0] > 0.5)
    assert abs(up - 0.5) < 0.02
    assert ea.LN_EPS == np.log(2.0**-52)


def test_creep_stays_in_unit_interval():
    g = np.random.default_rng(5)
    off = np.concatenate([g.uniform(0, 1, (3000, 4)), np.zeros((10, 4)), np.ones((10, 4))])
    out, _ = ea.mutate(off, 0.0, params(n_pop=off.shape[0] + 1), 9)
    assert np.all((out >= 0) & (out <= 1))


def test_jump_rate_is_binomial_and_uniform():
    n, n_par, pm = 2000, 6, 0.1
    off = np.full((n, n_par), 0.5)
    out, jumped = ea.mutate(off, pm, params(n_pop=n + 1), 11)
    mean, sd = n * n_par * pm, np.sqrt(n * n_par * pm * (1 - pm))
    assert abs(jumped.sum() - mean) < 5 * sd
    assert stats.kstest(out[jumped], "uniform").pvalue > 1e-3


def test_stagnation_sequence_golden():
    rows = np.loadtxt(os.path.join(GOLDEN, "stagnation_constant.txt"))
    p = params(n_pop=64, p_mut0=0.01)
    st = ea.new_state(p)
    for g, best, pm, run, restart in rows:
        got_restart = ea.stagnation_update(st, best, p, 6)
        if got_restart:  # the driver's restart bookkeeping
            st.p_mut, st.hist, st.stag_run = p.p_mut0, [], 0
        assert st.p_mut == pytest.approx(pm, rel=1e-15), g
        assert st.stag_run == run and bool(got_restart) == bool(restart), g


def test_stagnation_threshold():
    p = params(n_pop=64)
    # 2% better every generation: never stagnant
    st = ea.new_state(p)
    assert not any(ea.stagnation_update(st, 100 * 0.98**g, p, 6) for g in range(40))
    assert st.stag_run == 0
    # 0.1% better every generation: 10 generations improve by < 1%, stagnant from g = 10
    st = ea.new_state(p)
    flags = [ea.stagnation_update(st, 100 * 0.999**g, p, 6) for g in range(25)]
    assert flags.index(True) == 19


def test_elitism_and_archive_monotone():
    target = np.array([0.2, 0.9, 0.4])
    trace = []
    ea.run(lambda P: ((P - target) ** 2).sum(1), 3, params(n_pop=40, n_gen=150), trace)
    for (g0, b0, _, r0), (g1, b1, _, r1) in zip(trace, trace[1:]):
        if r0 == r1:  # no restart in between: the elite survives unchanged
            assert b1 <= b0


def test_converges_on_sphere():
    target = np.array([0.3, 0.7, 0.11, 0.93, 0.5, 0.42])
    st = ea.run(lambda P: ((P - target) ** 2).sum(1), 6, params(n_pop=64, n_gen=200, seed=1))
    assert st.best_chi2 < 1e-6
    assert np.allclose(st.best_genes, target, atol=1e-3)


def test_generation_draws_depend_on_stream_and_generation():
    P = ea.init_population(16, 6, params(n_pop=16), 0)
    chi2 = np.arange(16.0)
    outs = []
    for stream, gen in [(0, 0), (1, 0), (0, 1)]:
        p = params(n_pop=16, stream=stream)
        st = ea.new_state(p)
        outs.append(ea.generation(P, chi2, st, p, gen))
    assert np.array_equal(outs[0][0], P[0])  # elite row unchanged
    assert not np.array_equal(outs[0], outs[1]) and not np.array_equal(outs[0], outs[2])


def test_sblm_decoding():
    from paper_1208_4830_gb300 import synth

    P = np.array([[0.0] * 6, [1.0] * 6, [0.5] * 6])
    th = ea.sblm_theta(P, synth.FIT_LO, synth.FIT_HI)
    assert np.allclose(th[0], [-20, 5, 0, 0, 0.3, 1e-4])
    assert np.allclose(th[1], [20, 100, 1, 2 * np.pi, 3, 1.0])
    assert np.allclose(th[2], [0, 52.5, 0.5, np.pi, 1.65, 1e-2])


def test_one_island_is_the_panmictic_ea():
    f = lambda P: ((P - 0.3) ** 2).sum(1)  # noqa: E731
    p = params(n_pop=24, n_gen=40, seed=2, stream=5)
    st = ea.run(f, 4, p)
    (si,) = ea.run_islands(f, 4, p, 1, 7)
    assert si.best_chi2 == st.best_chi2 and np.array_equal(si.best_genes, st.best_genes)


def test_islands_without_migration_are_independent_runs():
    f = lambda P: np.abs(np.sin(9 * P)).sum(1)  # noqa: E731
    p = params(n_pop=20, n_gen=30, seed=3, stream=2)
    states = ea.run_islands(f, 3, p, 3, 0, n_lc=10)
    for i, s in enumerate(states):
        ref = ea.run(f, 3, params(n_pop=20, n_gen=30, seed=3, stream=2 + 10 * i))
        assert s.best_chi2 == ref.best_chi2 and np.array_equal(s.best_genes, ref.best_genes)


def test_ring_migration_by_hand():
    P = [np.full((3, 2), float(k)) for k in range(3)]
    elites = [np.array([10.0 * k, 10.0 * k + 1]) for k in range(3)]
    out = ea.migrate_ring(P, elites)
    for k in range(3):
        src = (k - 1) % 3
        assert np.array_equal(out[k][-1], elites[src])  # last row from the previous island
        assert np.array_equal(out[k][:-1], P[k][:-1])  # the rest untouched
        assert np.array_equal(P[k], np.full((3, 2), float(k)))  # inputs not modified


def test_migrants_reach_the_neighbour():
    """Island 1 optimises a far target; island 0's fitness is the same function, but island 0
    starts far away. After a migration the neighbour evaluates the migrant, so every island's
    archive is at least as good as the best elite it was sent."""
    target = np.array([0.9, 0.1, 0.8])
    calls = []

    def f(P):
        calls.append(P.copy())
        return ((P - target) ** 2).sum(1)

    p = params(n_pop=16, n_gen=25, seed=4)
    states = ea.run_islands(f, 3, p, 3, 5)
    # populations are evaluated island by island, generation by generation
    pops = [calls[g * 3 : g * 3 + 3] for g in range(25)]
    for g in range(4, 24, 5):  # migrations after generations 4, 9, 14, 19
        for i in range(3):
            chi = ((pops[g][i] - target) ** 2).sum(1)
            elite = pops[g][i][int(np.argmin(chi))]
            assert np.array_equal(pops[g + 1][(i + 1) % 3][-1], elite)
            assert states[(i + 1) % 3].best_chi2 <= chi.min()


def test_solution_archive_by_hand():
    arc = ea.SolutionArchive(size=3, radius=0.1)
    steps = [([0.5, 0.5], 10.0), ([0.55, 0.5], 8.0), ([0.9, 0.9], 12.0), ([0.1, 0.1], 5.0), ([0.3, 0.3], 20.0),
             ([0.3, 0.3], 9.0), ([0.62, 0.45], 7.0), ([0.65, 0.5], 6.5), ([0.64, 0.48], 6.6), ([0.2, 0.9], np.nan)]
    for g, c in steps:
        arc.offer(g, c)
    # 0.55 replaced 0.5 (same solution, fitter); 12 was pushed out by 9; 0.62 then 0.65 replaced
    # the 0.55 entry; 6.6 matched but was not fitter; NaN is never archived
    assert arc.chi2 == [5.0, 6.5, 9.0]
    np.testing.assert_array_equal(np.array(arc.genes), [[0.1, 0.1], [0.65, 0.5], [0.3, 0.3]])
    # a fitter solution matching two entries takes the first and absorbs the other
    arc = ea.SolutionArchive(size=4, radius=0.1)
    arc.offer([0.1, 0.1], 5.0)
    arc.offer([0.3, 0.3], 9.0)
    arc.offer([0.2, 0.2], 4.0)
    assert arc.chi2 == [4.0] and np.array_equal(arc.genes[0], [0.2, 0.2])


def test_solution_archive_over_a_run():
    """Over a whole run on a function with three wells: the archive's first entry is the run's
    best, entries are sorted and pairwise distinct."""
    wells = np.array([[0.2, 0.2, 0.5], [0.8, 0.3, 0.5], [0.5, 0.85, 0.2]])
    depth = np.array([0.0, 0.001, 0.002])

    def f(P):
        d2 = ((P[:, None, :] - wells[None]) ** 2).sum(-1) + depth[None]
        return d2.min(1)

    arc = ea.SolutionArchive(size=8, radius=0.05)
    st = ea.run(f, 3, params(n_pop=40, n_gen=120, seed=5), solutions=arc)
    assert arc.chi2[0] == st.best_chi2 and np.array_equal(arc.genes[0], st.best_genes)
    assert arc.chi2 == sorted(arc.chi2) and len(arc.chi2) == 8
    for i in range(8):
        for j in range(i + 1, 8):
            assert np.max(np.abs(arc.genes[i] - arc.genes[j])) > 0.05
