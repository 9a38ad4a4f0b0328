"""Seeded synthetic inputs shaped like the paper's workloads.

This module feeds both the CUDA library and the CPU oracle. It draws parameters, epochs, noise
and batch layouts; it computes no magnification, no quintic and no EA operator, so a mistake in
either side's arithmetic cannot hide here. Observed fluxes are assembled by the caller as
F = A_true * (1 + s * z) from the unit-normal draws ``z`` returned here and a magnification
computed by whichever side is being exercised.

The one geometric step it does take is input shaping: to force a trajectory through a caustic it
picks a point of the critical curve (the quartic e^{i phi} z^2 (z - d)^2 - (1 + q) z^2 + 2 d z - d^2 = 0,
i.e. det J = 0) and maps it to the source plane. That is the image-to-source direction of the lens
map, which the hot path never evaluates (the hot path inverts it).

Parameter rows are theta = (t0, tE, u0, alpha, d, q) (Section 2.1: t_m, t_E, b, theta, a, q);
fits encode genes (t0, tE, u0, alpha, d, log10 q).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# gene bounds of the single-lightcurve fit: t0 (Table 1 range of t_m), tE, u0, alpha, d, log10 q
FIT_LO = np.array([-20.0, 5.0, 0.0, 0.0, 0.3, -4.0])
FIT_HI = np.array([20.0, 100.0, 1.0, 2.0 * np.pi, 3.0, 0.0])


def _rng(seed):
    return np.random.Generator(np.random.Philox(seed))


def uniform_epochs(n_ep, seed, lo=-60.0, hi=60.0):
    """n_ep sorted epochs drawn uniformly in [lo, hi] days."""
    return np.sort(_rng(seed).uniform(lo, hi, n_ep))


def prior_theta(n, seed):
    """Parameter rows from the sweep priors: q log-uniform [1e-4, 1], d log-uniform [0.3, 3],
    u0 U[0, 1], alpha U[0, 2 pi), tE U[5, 100] d, t0 U[-20, 20] d."""
    g = _rng(seed)
    theta = np.empty((n, 6))
    theta[:, 0] = g.uniform(-20.0, 20.0, n)
    theta[:, 1] = g.uniform(5.0, 100.0, n)
    theta[:, 2] = g.uniform(0.0, 1.0, n)
    theta[:, 3] = g.uniform(0.0, 2.0 * np.pi, n)
    theta[:, 4] = np.exp(g.uniform(np.log(0.3), np.log(3.0), n))
    theta[:, 5] = 10.0 ** g.uniform(-4.0, 0.0, n)
    return theta


def _caustic_point(d, q, phi, pick):
    """A source-plane caustic point of lens (d, q): root number ``pick`` (0..3) of the critical
    quartic for phase phi, mapped through the image-to-source lens map."""
    e = np.exp(1j * phi)
    # e z^2 (z-d)^2 - (1+q) z^2 + 2 d z - d^2, descending powers of z
    coeffs = [e, -2.0 * d * e, e * d * d - (1.0 + q), 2.0 * d, -d * d]
    zc = np.roots(coeffs)[pick]
    zb = np.conj(zc)
    return zc - 1.0 / zb + q / (d - zb)


def force_caustics(theta, frac, seed, t_lo=-50.0, t_hi=50.0):
    """Re-aim a fraction ``frac`` of the rows so that their trajectory crosses a caustic at a time
    drawn in [t_lo, t_hi]. The trajectory is zeta(tau) = tau v + u0 w with w = e^{i alpha} and
    v = -i w, so a crossing point zeta_c fixes u0 = Re(zeta_c conj(w)) and tau_c = Re(zeta_c conj(v));
    alpha is turned by pi when that u0 is negative. Returns (theta, forced_mask, t_cross), with
    t_cross NaN for rows left alone."""
    theta = np.array(theta, dtype=np.float64, copy=True)
    n = theta.shape[0]
    g = _rng(seed)
    forced = np.zeros(n, dtype=bool)
    idx = g.choice(n, size=int(round(frac * n)), replace=False)
    forced[idx] = True
    t_cross = np.full(n, np.nan)
    for i in np.sort(idx):
        d, q, tE, alpha = theta[i, 4], theta[i, 5], theta[i, 1], theta[i, 3]
        zc = _caustic_point(d, q, g.uniform(0.0, 2.0 * np.pi), int(g.integers(0, 4)))
        w = np.exp(1j * alpha)
        v = -1j * w
        u0 = float(np.real(zc * np.conj(w)))
        tau_c = float(np.real(zc * np.conj(v)))
        if u0 < 0.0:
            alpha = (alpha + np.pi) % (2.0 * np.pi)
            u0, tau_c = -u0, -tau_c
        t_c = g.uniform(t_lo, t_hi)
        theta[i, 0] = t_c - tau_c * tE
        theta[i, 2] = u0
        theta[i, 3] = alpha
        t_cross[i] = t_c
    return theta, forced, t_cross


@dataclass
class Lightcurve:
    t: np.ndarray          # epochs [d]
    z: np.ndarray          # unit-normal noise draws, one per epoch
    sigma_frac: np.ndarray  # per-epoch sigma as a fraction of the true flux
    truth: np.ndarray      # theta of the injected event

    def observe(self, A_true):
        """Observed flux and sigma from a magnification of the truth (any implementation)."""
        sigma = self.sigma_frac * A_true
        return A_true + sigma * self.z, sigma


def single_fit_lightcurve(seed=0):
    """One lightcurve: truth (t0, tE, u0, alpha, d, q) = (0, 30, 0.1, 1.0, 1.2, 0.01), 400 epochs
    uniform in [-60, 60] d, Gaussian noise of 1% of the true flux."""
    g = _rng(seed)
    t = np.sort(g.uniform(-60.0, 60.0, 400))
    z = g.standard_normal(400)
    truth = np.array([0.0, 30.0, 0.1, 1.0, 1.2, 0.01])
    return Lightcurve(t=t, z=z, sigma_frac=np.full(400, 0.01), truth=truth)


@dataclass
class Sweep:
    theta: np.ndarray      # (n_cand, 6)
    forced: np.ndarray     # (n_cand,) trajectories aimed through a caustic
    t: np.ndarray          # (n_ep,)
    truth: np.ndarray      # theta whose magnification (plus noise) is the observed flux
    z: np.ndarray          # (n_ep,) unit-normal noise draws
    sigma_frac: float


def forward_sweep(n_cand=4096, n_ep=2000, seed=0, caustic_frac=0.1):
    """Candidates from the sweep priors, 10% forced through caustics, epochs uniform in
    [-60, 60] d; the observed flux is a prior draw plus 1% noise."""
    theta = prior_theta(n_cand, seed)
    theta, forced, _ = force_caustics(theta, caustic_frac, seed + 1)
    t = uniform_epochs(n_ep, seed + 2)
    truth = prior_theta(1, seed + 3)[0]
    z = _rng(seed + 4).standard_normal(n_ep)
    return Sweep(theta=theta, forced=forced, t=t, truth=truth, z=z, sigma_frac=0.01)


@dataclass
class Batch:
    t: np.ndarray           # concatenated epochs
    z: np.ndarray           # unit-normal noise draws, one per epoch
    sigma_frac: np.ndarray  # per-epoch sigma as a fraction of the true flux
    offsets: np.ndarray     # int64 [n_lc + 1]
    truth: np.ndarray       # (n_lc, 6)

    def observe(self, A_true):
        """Observed flux and sigma from the truths' magnifications (concatenated)."""
        sigma = self.sigma_frac * A_true
        return A_true + sigma * self.z, sigma


def seasonal_batch(n_lc=512, seed=0, n_min=200, n_max=5000, span=(-300.0, 300.0), season=245.0, gap=120.0,
                   sig_lo=0.005, sig_hi=0.05):
    """Lightcurves of uneven length with seasonal gaps: epoch counts uniform in [n_min, n_max];
    epochs uniform inside observing seasons of `season` days separated by `gap`-day gaps (random
    phase) within `span`; per-point sigma uniform in [sig_lo, sig_hi] of the true flux; truths
    from the sweep priors. A lightcurve with no epoch inside |t - t0| < tE is redrawn."""
    g = _rng(seed)
    ts, zs, ss, offs, truths = [], [], [], [0], []
    period = season + gap
    while len(truths) < n_lc:
        th = prior_theta(1, int(g.integers(0, 2**62)))[0]
        n = int(g.integers(n_min, n_max + 1))
        phase = g.uniform(0.0, period)
        t = np.empty(0)
        while t.size < n:
            x = g.uniform(span[0], span[1], 2 * n)
            x = x[np.mod(x - span[0] + phase, period) < season]
            t = np.concatenate([t, x])
        t = np.sort(t[:n])
        if not np.any(np.abs(t - th[0]) < th[1]):
            continue
        ts.append(t)
        zs.append(g.standard_normal(n))
        ss.append(g.uniform(sig_lo, sig_hi, n))
        offs.append(offs[-1] + n)
        truths.append(th)
    return Batch(t=np.concatenate(ts), z=np.concatenate(zs), sigma_frac=np.concatenate(ss),
                 offsets=np.array(offs, dtype=np.int64), truth=np.array(truths))


def heldout_batch(n_lc=2000, seed=0, n_ep=500, sigma_frac=0.02, caustic_frac=0.1, lo=-60.0, hi=60.0):
    """Held-out lightcurves for the learned proposal: truths from the sweep priors with a fraction
    re-aimed through a caustic (rows whose re-aimed t0 or u0 leaves the fit domain FIT_LO..FIT_HI
    are dropped and drawn again, so every truth is reachable by the fitter), n_ep epochs uniform
    in [lo, hi] d per curve, noise of sigma_frac of the true flux."""
    rows = []
    k = 0
    while len(rows) < n_lc:
        theta = prior_theta(n_lc, seed + 7919 * k)
        theta, _, _ = force_caustics(theta, caustic_frac, seed + 1 + 7919 * k)
        genes = theta.copy()
        genes[:, 5] = np.log10(genes[:, 5])
        inside = np.all((genes >= FIT_LO) & (genes <= FIT_HI), axis=1)
        rows.extend(theta[inside][: n_lc - len(rows)])
        k += 1
    theta = np.array(rows)
    g = _rng(seed + 2)
    t = np.sort(g.uniform(lo, hi, (n_lc, n_ep)), axis=1).ravel()
    z = g.standard_normal(n_lc * n_ep)
    offsets = np.arange(n_lc + 1, dtype=np.int64) * n_ep
    return Batch(t=t, z=z, sigma_frac=np.full(n_lc * n_ep, sigma_frac), offsets=offsets, truth=theta)


# Table 1 of the paper: the ranges of its simulated lightcurves and fits (d = a, u0 = b, alpha =
# theta, t0 = t_m), as genes (t0, tE, u0, alpha, d, log10 q)
PAPER_LO = np.array([-20.0, 5.0, 0.001, 0.0, 0.6, -1.0])
PAPER_HI = np.array([20.0, 50.0, 1.0, 2.0 * np.pi, 1.7, 0.0])


@dataclass
class PaperBatch:
    t: np.ndarray        # concatenated epochs
    offsets: np.ndarray  # int64 [n_lc + 1]
    truth: np.ndarray    # (n_lc, 6)
    sigma_frac: float    # sigma of each flux point as a fraction of the true flux (noise-free curves)

    def sigma(self, A_true):
        return self.sigma_frac * np.asarray(A_true)


# the paper's sigma of 0.01 (in magnitudes: it fits magnitudes with a baseline-magnitude
# parameter) as a fraction of the flux, 0.4 ln(10) x 0.01
PAPER_SIGMA_FRAC = 0.4 * np.log(10.0) * 0.01


def paper_batch(n_lc=512, seed=0, n_ep=100):
    """Noise-free test curves shaped like the paper's (Section 4.2): parameters uniform over the
    Table 1 ranges (q uniform in [0.1, 1]), n_ep evenly spaced epochs from t_start to t_end with
    (t_start - t0)/tE uniform in (-3, -2) and (t_end - t0)/tE uniform in (2, 3); the flux is the
    magnification itself, with sigma = 0.01 mag (0.92% of the flux) for chi^2."""
    g = _rng(seed)
    u = g.uniform(size=(n_lc, 6))
    v = PAPER_LO + (PAPER_HI - PAPER_LO) * u
    theta = v.copy()
    theta[:, 5] = 0.1 + 0.9 * u[:, 5]  # q uniform in [0.1, 1]
    a = g.uniform(-3.0, -2.0, n_lc)
    b = g.uniform(2.0, 3.0, n_lc)
    ts = [np.linspace(th[0] + ai * th[1], th[0] + bi * th[1], n_ep) for th, ai, bi in zip(theta, a, b)]
    offsets = np.arange(n_lc + 1, dtype=np.int64) * n_ep
    return PaperBatch(t=np.concatenate(ts), offsets=offsets, truth=theta, sigma_frac=PAPER_SIGMA_FRAC)


def count_peaks(A, rel_prominence=0.01):
    """Peaks of a lightcurve sampled finely: local maxima that rise above the higher of the two
    neighbouring minima by more than rel_prominence of their height."""
    A = np.asarray(A, dtype=np.float64)
    n = 0
    for i in range(1, A.size - 1):
        if A[i] > A[i - 1] and A[i] >= A[i + 1]:
            left = A[: i + 1][::-1]
            right = A[i:]
            lmin = np.minimum.accumulate(left)
            rmin = np.minimum.accumulate(right)
            # walk down each side until a higher point appears (or the end)
            li = np.argmax(left > A[i]) if np.any(left > A[i]) else left.size
            ri = np.argmax(right > A[i]) if np.any(right > A[i]) else right.size
            base = max(lmin[li - 1], rmin[ri - 1])
            if A[i] - base > rel_prominence * A[i]:
                n += 1
    return n


# Section 2.4's photometric noise model: log10 sigma_I = slope * m_I + intercept (magnitudes)
NOISE_SLOPE, NOISE_INTERCEPT = 0.3416, -7.7095
M0_RANGE = (18.0, 22.0)  # Table 1: unlensed magnitude of the source


@dataclass
class NoisyBlendedBatch:
    t: np.ndarray        # concatenated epochs (sorted within each curve)
    offsets: np.ndarray  # int64 [n_lc + 1]
    truth: np.ndarray    # (n_lc, 6) lens and trajectory
    f: np.ndarray        # (n_lc,) blending fraction: source flux / total unlensed flux
    m0: np.ndarray       # (n_lc,) unlensed magnitude of the source (blended light excluded)
    z: np.ndarray        # unit-normal draws, one per epoch

    def observe(self, A_true):
        """(flux, sigma) normalised to the total unlensed flux, from the truths' source
        magnifications (concatenated, any implementation). m0 is the source's unlensed magnitude
        (Section 2's parameter list), so the unlensed blend of source and other light has
        magnitude m0 + 2.5 log10 f and the true magnitude is m = m0 - 2.5 log10(A + (1 - f)/f);
        it gets Gaussian noise of the noise model's sigma_m(m); the observed flux is
        10^(-0.4 (m_obs - m_blend)) and its sigma the first-order image 0.4 ln 10 F sigma_m of the
        magnitude error at the true flux F = f A + 1 - f."""
        n = np.diff(self.offsets)
        f = np.repeat(self.f, n)
        m0 = np.repeat(self.m0, n)
        F = f * np.asarray(A_true) + (1.0 - f)
        m_blend = m0 + 2.5 * np.log10(f)
        m = m_blend - 2.5 * np.log10(F)
        s_m = 10.0 ** (NOISE_SLOPE * m + NOISE_INTERCEPT)
        flux = 10.0 ** (-0.4 * (m + s_m * self.z - m_blend))
        return flux, 0.4 * np.log(10.0) * s_m * F


def noisy_blended_batch(n_lc=512, seed=0, n_ep=100):
    """Curves shaped like the paper's noisy, blended test (Section 4.4): parameters as in
    paper_batch (Table 1 ranges, q uniform in [0.1, 1]), the source's unlensed magnitude m0
    uniform over Table 1's [18, 22], a blending fraction f uniform on (0, 1], and n_ep epochs
    drawn uniformly on (t_start, t_end) (sorted), with (t_start - t0)/tE in (-3, -2) and
    (t_end - t0)/tE in (2, 3)."""
    g = _rng(seed)
    u = g.uniform(size=(n_lc, 6))
    theta = PAPER_LO + (PAPER_HI - PAPER_LO) * u
    theta[:, 5] = 0.1 + 0.9 * u[:, 5]
    a = g.uniform(-3.0, -2.0, n_lc)
    b = g.uniform(2.0, 3.0, n_lc)
    f = 1.0 - g.uniform(size=n_lc)
    m0 = g.uniform(*M0_RANGE, size=n_lc)
    ts = [np.sort(g.uniform(th[0] + ai * th[1], th[0] + bi * th[1], n_ep)) for th, ai, bi in zip(theta, a, b)]
    z = g.standard_normal(n_lc * n_ep)
    offsets = np.arange(n_lc + 1, dtype=np.int64) * n_ep
    return NoisyBlendedBatch(t=np.concatenate(ts), offsets=offsets, truth=theta, f=f, m0=m0, z=z)
