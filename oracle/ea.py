"""Oracle: the evolutionary algorithm of Appendix A (Rajpaul 2012), operator by operator.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Every random number comes from Philox4x64-10 (``oracle.philox``) with key (seed, stream), where
``stream`` numbers the population (one per lightcurve of a batch), and counter
(generation, operator, index, sub-index). The device draws the same words for the same counter,
so operators can be compared exactly.

Sequence per generation t (Appendix A, "basic evolutionary sequence"):
  decode P(t) -> A(t) (Eq. EMMA-encoding) and evaluate the external fitness (chi^2);
  rank the rows of P(t) (Appendix A, "Fitness evaluation and ranking");
  tournament selection (Appendix A, "Selection");
  reproduction with a per-pairing weighting matrix F and elitism (Eq. rep1, Eq. rep2,
  Appendix A, "Reproduction");
  creep then jump mutation of the offspring (Appendix A, "Creep and jump mutation");
  stagnation check, jump-rate boost/throttle, restart (Appendix A, "Stagnation checks").

Readings where the paper is silent or loose:
* initialisation pairs element pi(2k) with pi(2k+1) of a random permutation pi of all
  N_pop*N_par elements; pi sorts the elements by a key made of the top 44 bits of one Philox
  word per element with the element index in the low 20 bits (so no two keys are equal and
  N_pop*N_par < 2^20); the first of a pair gets X ~ U(0,1), the second 1 - X; an odd leftover
  element gets a plain U(0,1);
* ranking is a stable sort on chi^2 with NaN treated as +inf (ties keep row order);
* the N_tourn tournament draws are with replacement, and a parent may pair with itself;
* N_pop - 1 offspring come from ceil((N_pop-1)/2) pairings; the last child is dropped when
  N_pop - 1 is odd; row 0 of the next population is the unmutated elite;
* the weighting-matrix mode is drawn once per pairing, the diagonal entries independently per gene;
* creep touches every gene of every offspring (clones included), then jump may overwrite it;
  epsilon is the FP64 machine epsilon 2^-52;
* stagnation at generation t (counted from the last (re)start) means
  chi2_best(t - W) - chi2_best(t) <= r * chi2_best(t - W), W = 10 generations, r = 1%; it is
  first testable W generations after a (re)start; a stagnant generation multiplies p_mut by
  1.5, any other by 0.5, clamped to [1/(N_pop*N_par), 0.5]; the mutation of generation t uses
  the rate held before this update;
* "repeated" stagnation = ``restart_after`` (10) consecutive stagnant generations; the next
  population is then re-initialised with the generation counter t + 1, p_mut returns to its
  starting value, the window is cleared; the best solution ever seen is archived throughout.

Section 5.3's island EA (``run_islands``, ``migrate_ring``) is this sequence on several
populations with a ring migration of their elites.

Pinned by tests/test_oracle_ea.py: Philox streams, the closed-form tournament rank CDF
1 - (1 - r/N)^k, the log-uniform creep step, binomial jump counts, the antithetic pairing of the
initial population, the convex-combination invariants of the three reproduction modes, scripted
stagnation sequences worked by hand, elitist monotonicity, and convergence on analytic test
functions. Whole-run trajectories are parity unpinned (rank ties flip under floating-point
reordering) and are judged by recovery of the injected parameters.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import philox as ph

# operator identifiers (counter word 1)
OP_INIT_PERM = 1
OP_INIT_U = 2
OP_SELECT = 3
OP_MODE = 4
OP_F = 5
OP_MUT = 6

LN_EPS = float(np.log(np.finfo(np.float64).eps))  # ln(2^-52)
P_MUT_MAX = 0.5
INIT_INDEX_LIMIT = 1 << 20  # population elements addressable by the initialisation keys


@dataclass
class EAParams:
    n_pop: int = 1000            # Appendix A default population size
    n_gen: int = 100
    p_mut0: float = 0.01         # Appendix A default starting jump probability
    n_tourn: int = 0             # 0 -> ceil(N_pop / 25)
    stag_window: int = 10        # generations in the stagnation test
    stag_rel: float = 0.01       # "improved by more than 1%"
    restart_after: int = 10      # consecutive stagnant generations before a restart
    seed: int = 0
    stream: int = 0

    def tournament_size(self):
        return self.n_tourn if self.n_tourn > 0 else -(-self.n_pop // 25)


@dataclass
class EAState:
    p_mut: float
    hist: list = field(default_factory=list)   # best chi^2 of the last stag_window+1 generations
    stag_run: int = 0
    n_restarts: int = 0
    best_chi2: float = math.inf
    best_genes: np.ndarray | None = None


def _draw(params, gen, op, index, sub):
    return ph.philox4x64(gen, op, index, sub, params.seed, params.stream)


# ---------------------------------------------------------------------------------------------
# Appendix A, "Initialisation"
# ---------------------------------------------------------------------------------------------
def init_population(n_pop, n_par, params, gen):
    """Half the elements get X ~ U(0,1); each remaining element gets 1 - X of another random one."""
    m = n_pop * n_par
    assert m < INIT_INDEX_LIMIT
    e = np.arange(m, dtype=np.uint64)
    words = _draw(params, gen, OP_INIT_PERM, e, 0)[:, 0]
    keys = ((words >> np.uint64(20)) << np.uint64(20)) | e
    perm = np.argsort(keys)
    n_pairs = m // 2
    x = ph.u01(_draw(params, gen, OP_INIT_U, np.arange(n_pairs + (m % 2), dtype=np.uint64), 0)[:, 0])
    flat = np.empty(m)
    flat[perm[0 : 2 * n_pairs : 2]] = x[:n_pairs]
    flat[perm[1 : 2 * n_pairs : 2]] = 1.0 - x[:n_pairs]
    if m % 2:
        flat[perm[m - 1]] = x[n_pairs]
    return flat.reshape(n_pop, n_par)


# ---------------------------------------------------------------------------------------------
# Eq. (EMMA-encoding)
# ---------------------------------------------------------------------------------------------
def decode(P, lo, hi):
    """a_ij = alpha_j + (beta_j - alpha_j) p_ij."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return lo + (hi - lo) * P


def sblm_theta(P, lo, hi):
    """Decode SBLM genes (t0, tE, u0, alpha, d, log10 q) to theta = (t0, tE, u0, alpha, d, q)."""
    a = decode(P, lo, hi)
    theta = a.copy()
    theta[:, 5] = 10.0 ** a[:, 5]
    return theta


# ---------------------------------------------------------------------------------------------
# Appendix A, "Fitness evaluation and ranking"
# ---------------------------------------------------------------------------------------------
def rank(P, chi2):
    """Rows sorted best first: stable sort on chi^2, NaN counted as +inf."""
    key = np.where(np.isnan(chi2), np.inf, chi2)
    order = np.argsort(key, kind="stable")
    return P[order], key[order], order


# ---------------------------------------------------------------------------------------------
# Appendix A, "Selection"
# ---------------------------------------------------------------------------------------------
def tournament(n_pop, n_tourn, n_slots, params, gen):
    """Parent ranks (0 = fittest): each is the minimum of n_tourn uniform draws from {0..N_pop-1}."""
    slots = np.arange(n_slots, dtype=np.uint64)[:, None]
    k = np.arange(n_tourn)
    words = _draw(params, gen, OP_SELECT, slots, (k // 4).astype(np.uint64)[None, :])
    w = np.take_along_axis(words, (k % 4)[None, :, None], axis=-1)[..., 0]
    return ph.uniform_int(w, n_pop).min(axis=1).astype(np.int64)


# ---------------------------------------------------------------------------------------------
# Appendix A, "Reproduction", Eq. (rep1), Eq. (rep2)
# ---------------------------------------------------------------------------------------------
def pairing_modes(n_pairs, params, gen):
    """0: f ~ U(0,1) (interpolants), 1: f ~ Bin(1, 1/2) (gene swap), 2: f = 1 (clones)."""
    w = _draw(params, gen, OP_MODE, np.arange(n_pairs, dtype=np.uint64), 0)[:, 0]
    return ph.uniform_int(w, 3).astype(np.int64)


def weights(modes, n_par, params, gen):
    """Diagonal of the weighting matrix F for every pairing, shape (n_pairs, n_par)."""
    n_pairs = modes.shape[0]
    w = _draw(params, gen, OP_F, np.arange(n_pairs, dtype=np.uint64)[:, None],
              np.arange(n_par, dtype=np.uint64)[None, :])[..., 0]
    f_interp = ph.u01(w)
    f_swap = ph.bit(w).astype(np.float64)
    m = modes[:, None]
    return np.where(m == 0, f_interp, np.where(m == 1, f_swap, 1.0))


def reproduce(P_ranked, parent_ranks, params, gen):
    """Offspring rows 1..N_pop-1: p_i F + p_j (I - F) and p_j F + p_i (I - F) per pairing."""
    n_pop, n_par = P_ranked.shape
    n_off = n_pop - 1
    n_pairs = (n_off + 1) // 2
    modes = pairing_modes(n_pairs, params, gen)
    F = weights(modes, n_par, params, gen)
    pa = P_ranked[parent_ranks[0::2]]
    pb = P_ranked[parent_ranks[1::2]]
    c1 = pa * F + pb * (1.0 - F)
    c2 = pb * F + pa * (1.0 - F)
    children = np.empty((2 * n_pairs, n_par))
    children[0::2] = c1
    children[1::2] = c2
    return children[:n_off], modes


# ---------------------------------------------------------------------------------------------
# Appendix A, "Creep and jump mutation"
# ---------------------------------------------------------------------------------------------
def mutate(offspring, p_mut, params, gen):
    """Creep every gene (p - p X or p + (1 - p) X, ln X ~ U(ln eps, 0)), then jump with p_mut.

    ``offspring`` holds population rows 1..N_pop-1; the counter's row index is the population row.
    """
    n_off, n_par = offspring.shape
    rows = np.arange(1, n_off + 1, dtype=np.uint64)[:, None]
    cols = np.arange(n_par, dtype=np.uint64)[None, :]
    w = _draw(params, gen, OP_MUT, rows, cols)
    X = np.exp(LN_EPS * ph.u01(w[..., 0]))
    up = ph.bit(w[..., 1]) == 1
    p = offspring
    crept = np.where(up, p + (1.0 - p) * X, p - p * X)
    crept = np.minimum(np.maximum(crept, 0.0), 1.0)
    jump = ph.u01(w[..., 2]) < p_mut
    return np.where(jump, ph.u01(w[..., 3]), crept), jump


# ---------------------------------------------------------------------------------------------
# Appendix A, "Stagnation checks"
# ---------------------------------------------------------------------------------------------
def stagnation_update(state, best, params, n_par):
    """Boost or throttle p_mut from the best chi^2 of this generation; return True on restart."""
    state.hist.append(best)
    if len(state.hist) > params.stag_window + 1:
        state.hist.pop(0)
    stagnant = False
    if len(state.hist) == params.stag_window + 1:
        old = state.hist[0]
        stagnant = math.isfinite(old) and (old - best) <= params.stag_rel * old
    p_min = 1.0 / (params.n_pop * n_par)
    if stagnant:
        state.p_mut = min(state.p_mut * 1.5, P_MUT_MAX)
        state.stag_run += 1
    else:
        state.p_mut = max(state.p_mut * 0.5, p_min)
        state.stag_run = 0
    return state.stag_run >= params.restart_after


def new_state(params):
    return EAState(p_mut=params.p_mut0)


def archive(state, P_ranked, chi2_ranked):
    """Keep the best solution ever evaluated (elitism within a run, archive across restarts)."""
    if chi2_ranked[0] < state.best_chi2:
        state.best_chi2 = float(chi2_ranked[0])
        state.best_genes = P_ranked[0].copy()


def generation(P, chi2, state, params, gen):
    """Everything after fitness evaluation in generation ``gen``; returns P(gen + 1)."""
    n_pop, n_par = P.shape
    Pr, cr, _ = rank(P, chi2)
    archive(state, Pr, cr)
    n_pairs = n_pop // 2  # == ceil((n_pop - 1) / 2)
    parents = tournament(n_pop, params.tournament_size(), 2 * n_pairs, params, gen)
    children, _ = reproduce(Pr, parents, params, gen)
    children, _ = mutate(children, state.p_mut, params, gen)
    P_next = np.vstack([Pr[:1], children])
    if stagnation_update(state, float(cr[0]), params, n_par):
        P_next = init_population(n_pop, n_par, params, gen + 1)
        state.p_mut = params.p_mut0
        state.hist = []
        state.stag_run = 0
        state.n_restarts += 1
    return P_next


def run(fitness, n_par, params, trace=None, solutions=None):
    """Reference driver: N_gen evaluations of ``fitness(P) -> chi^2``; returns the archive.
    ``solutions`` (a SolutionArchive) is offered each generation's ranked population."""
    state = new_state(params)
    P = init_population(params.n_pop, n_par, params, 0)
    for g in range(params.n_gen):
        chi2 = np.asarray(fitness(P), dtype=np.float64)
        if trace is not None:
            trace.append((g, float(np.nanmin(chi2)), state.p_mut, state.n_restarts))
        if solutions is not None:
            Pr, cr, _ = rank(P, chi2)
            solutions.offer_ranked(Pr, cr)
        if g == params.n_gen - 1:
            Pr, cr, _ = rank(P, chi2)
            archive(state, Pr, cr)
        else:
            P = generation(P, chi2, state, params, g)
    return state


# ---------------------------------------------------------------------------------------------
# Several solutions (Section 3.1: the explored phenotypes that meet a fitness criterion, rather
# than only the fittest; Appendix A, "Outputs")
# ---------------------------------------------------------------------------------------------
class SolutionArchive:
    """The ``size`` fittest mutually distinct solutions seen during a run. The paper leaves the
    rule open; the reading here: two solutions are the same when every gene differs by at most
    ``radius``; an offered row that matches an archived solution replaces it when fitter (and is
    dropped otherwise); a new solution enters while there is room, or in place of the least fit
    one when it is fitter. After a replacement the archive is merged again, so that it stays
    free of matching pairs. Entries are kept sorted by chi^2 (stable)."""

    def __init__(self, size, radius):
        self.size, self.radius = int(size), float(radius)
        self.genes, self.chi2 = [], []

    def _same(self, a, b):
        return bool(np.all(np.abs(np.asarray(a) - np.asarray(b)) <= self.radius))

    def offer(self, genes, chi2):
        chi2 = float(chi2)
        if not math.isfinite(chi2):
            return
        genes = np.array(genes, dtype=np.float64)
        for k, g in enumerate(self.genes):
            if self._same(g, genes):
                if chi2 < self.chi2[k]:
                    self.genes[k], self.chi2[k] = genes, chi2
                    self._merge(k)
                    self._sort()
                return
        if len(self.genes) < self.size:
            self.genes.append(genes)
            self.chi2.append(chi2)
        elif chi2 < self.chi2[-1]:
            self.genes[-1], self.chi2[-1] = genes, chi2
        else:
            return
        self._sort()

    def _merge(self, k):
        """Drop the entries that now match entry k (it is the fitter of each such pair)."""
        keep = [i for i in range(len(self.genes)) if i == k or not self._same(self.genes[i], self.genes[k])]
        self.genes = [self.genes[i] for i in keep]
        self.chi2 = [self.chi2[i] for i in keep]

    def _sort(self):
        order = sorted(range(len(self.chi2)), key=lambda i: self.chi2[i])
        self.genes = [self.genes[i] for i in order]
        self.chi2 = [self.chi2[i] for i in order]

    def offer_ranked(self, P_ranked, chi2_ranked, top=None):
        """Offer the ``top`` fittest rows of a ranked population (all rows by default), fittest first."""
        n = len(chi2_ranked) if top is None else min(top, len(chi2_ranked))
        for i in range(n):
            self.offer(P_ranked[i], chi2_ranked[i])


# ---------------------------------------------------------------------------------------------
# Section 5.3, "island" EAs: several populations evolve side by side with periodic migration
# ---------------------------------------------------------------------------------------------
def migrate_ring(P_next, elites):
    """One migration step: the elite of island i (its best row of the generation just ranked)
    replaces the last row of island (i + 1) mod n of the next populations. The paper names the
    scheme without its settings; the ring, one migrant and the last row are this build's reading."""
    n = len(P_next)
    out = [P.copy() for P in P_next]
    for i in range(n):
        out[(i + 1) % n][-1] = elites[i]
    return out


def run_islands(fitness, n_par, params, n_islands, interval, n_lc=1):
    """Island EA: population i uses stream id params.stream + i * n_lc; each generation every
    island is evaluated and advanced by ``generation``; when (g + 1) is a multiple of
    ``interval`` (> 0) the elites migrate by ``migrate_ring``. Returns the island states; the
    run's best is the lowest best_chi2 (the lowest island on ties)."""
    isl = []
    for i in range(n_islands):
        p = EAParams(**{**params.__dict__, "stream": params.stream + i * n_lc})
        isl.append([p, new_state(p), init_population(p.n_pop, n_par, p, 0)])
    for g in range(params.n_gen):
        last = g == params.n_gen - 1
        nexts, elites = [], []
        for p, state, P in isl:
            chi2 = np.asarray(fitness(P), dtype=np.float64)
            Pr, cr, _ = rank(P, chi2)
            elites.append(Pr[0].copy())
            if last:
                archive(state, Pr, cr)
                nexts.append(P)
            else:
                nexts.append(generation(P, chi2, state, p, g))
        if not last and interval > 0 and (g + 1) % interval == 0:
            nexts = migrate_ring(nexts, elites)
        for k, P in enumerate(nexts):
            isl[k][2] = P
    return [state for _, state, _ in isl]


def fit_sblm(t, flux, sigma, lo, hi, params, trace=None):
    """Fit the SBLM to a lightcurve: genes (t0, tE, u0, alpha, d, log10 q) within [lo, hi]."""
    from . import sblm

    def fitness(P):
        return sblm.chi2(sblm_theta(P, lo, hi), t, flux, sigma)

    state = run(fitness, 6, params, trace)
    theta = sblm_theta(state.best_genes[None, :], lo, hi)[0]
    return theta, state.best_chi2, state
