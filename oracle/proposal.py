"""Oracle: the learned proposal's data path around the network, plain numpy FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). The paper fits by evolutionary search
alone (Appendix A) and mentions a trained network only as a competing method (Section 4.1); the
proposal that seeds half of each initial population is this project's addition. This module
restates, step by step and without any blocking, what the device does around the network:

* ``make_batch``      training curves drawn from the sweep priors in window units, magnified by
                      the forward model of Section 2.2, 10% aimed through a caustic, with noise,
                      data gaps and the input normalisation;
* ``bin_lightcurve``  an observed lightcurve resampled to the network's 256 bins over its own span;
* ``init_params``     He-normal initial weights;
* ``adamw``           one decoupled-weight-decay Adam step and the learning-rate schedule;
* ``propose_genes``   seed rows for the EA drawn from the network's Gaussian outputs and encoded
                      as genes of Eq. (EMMA-encoding).

Random numbers come from Philox4x64-10 (``oracle.philox``) with the counters listed below, so
the device draws the same numbers; normal deviates by the Box-Muller transform
(z0, z1) = sqrt(-2 ln(1 - u0)) (cos 2 pi u1, sin 2 pi u1).

Window units: a curve observed on [c - h, c + h] is binned over that window; the bin centres are
s_j = -1 + (2 j + 1) / 256, and the network's targets are t0' = (t0 - c) / h, ln(tE / h), u0,
alpha / 2 pi, ln d, log10 q. Since the trajectory depends on time only through (t - t0) / tE,
a curve in window units is the curve of the parameters (t0', tE / h, u0, alpha, d, q) on the
grid s_j, which is how training curves are generated.

Pinned by tests/test_oracle_proposal.py (caustic crossings checked by the images' Jacobian,
noise and mask statistics, hand-binned curves, torch's AdamW, sampling limits).
"""
from __future__ import annotations

import math

import numpy as np

from . import philox as ph
from . import sblm as osb
from .cnn import SHAPES, N_PARAMS

N_BIN = 256
OP_CNN_INIT, OP_CNN_GEN, OP_CNN_NOISE, OP_CNN_SAMPLE = 7, 8, 9, 10

# training prior in window units
T0_RANGE = (-0.4, 0.4)
LN_TE_RANGE = (math.log(0.04), math.log(1.5))
LN_D_RANGE = (math.log(0.3), math.log(3.0))
LOG10Q_RANGE = (-4.0, 0.0)
T_CROSS_RANGE = (-0.8, 0.8)
LN_SIGMA_RANGE = (math.log(1e-4), math.log(0.05))
DROP_MAX = 0.7
GAP_PROB = 0.5
GAP_MAX = 0.4
MIN_KEPT = 16
FLUX_GAIN = 10.0
FLUX_SCALE = 3.0


def bin_centres():
    j = np.arange(N_BIN, dtype=np.float64)
    return -1.0 + (2.0 * j + 1.0) / N_BIN


def box_muller(x0, x1):
    r = np.sqrt(-2.0 * np.log(1.0 - ph.u01(x0)))
    a = 2.0 * math.pi * ph.u01(x1)
    return r * np.cos(a), r * np.sin(a)


def normalise(F, kept):
    """Network input [256, 2]: asinh(10 (F / median - 1)) / 3 on bins with data, and the data mask.
    The median is over the bins with data (mean of the middle two for an even count); a
    non-positive median is replaced by 1."""
    F = np.asarray(F, dtype=np.float64)
    kept = np.asarray(kept, dtype=bool)
    med = float(np.median(F[kept])) if kept.any() else 1.0
    if not (med > 0.0 and math.isfinite(med)):
        med = 1.0
    x = np.zeros((N_BIN, 2))
    x[kept, 0] = np.arcsinh(FLUX_GAIN * (F[kept] / med - 1.0)) / FLUX_SCALE
    x[kept, 1] = 1.0
    return x


def bin_lightcurve(t, flux, sigma):
    """Resample one observed lightcurve to the 256 bins over its own span [t_min, t_max]:
    inverse-variance weighted mean flux per bin, summed in epoch order. Returns (x, (c, h))."""
    t = np.asarray(t, dtype=np.float64)
    tmin, tmax = float(t.min()), float(t.max())
    span = tmax - tmin
    if not span > 0.0:
        span = 1.0
    sw = np.zeros(N_BIN)
    swf = np.zeros(N_BIN)
    for te, fe, se in zip(t, flux, sigma):
        j = min(N_BIN - 1, int(math.floor((te - tmin) / span * N_BIN)))
        w = 1.0 / (se * se)
        sw[j] += w
        swf[j] += w * fe
    kept = sw > 0.0
    F = np.where(kept, swf / np.where(kept, sw, 1.0), 0.0)
    return normalise(F, kept), (0.5 * (tmin + tmax), 0.5 * span)


def critical_point(d, q, phi, pick):
    """Caustic point: root number `pick` (roots ordered by real part) of the critical quartic
    e^{i phi} z^2 (z - d)^2 - (1 + q) z^2 + 2 d z - d^2 = 0 (det J = 0, Section 2.2), mapped to the
    source plane by the lens equation."""
    e = np.exp(1j * phi)
    roots = np.roots([e, -2.0 * d * e, e * d * d - (1.0 + q), 2.0 * d, -d * d])
    roots = roots[np.lexsort((roots.imag, roots.real))]
    return osb.lens_map(roots[pick], d, q)


def draws(seed, step, i):
    """The four Philox blocks of training sample i at optimiser step `step` (counter word 1 is the
    operator, word 2 the sample, word 3 the block)."""
    return [ph.philox4x64(step, OP_CNN_GEN, i, k, seed, 0) for k in range(4)]


def sample_theta(seed, step, i, forced_frac):
    """Parameters of training sample i in window units, with its noise and mask settings."""
    r = draws(seed, step, i)
    u = [ph.u01(r[k][j]) for k in range(4) for j in range(4)]
    t0 = T0_RANGE[0] + (T0_RANGE[1] - T0_RANGE[0]) * u[0]
    tE = math.exp(LN_TE_RANGE[0] + (LN_TE_RANGE[1] - LN_TE_RANGE[0]) * u[1])
    u0 = u[2]
    alpha = 2.0 * math.pi * u[3]
    d = math.exp(LN_D_RANGE[0] + (LN_D_RANGE[1] - LN_D_RANGE[0]) * u[4])
    lq = LOG10Q_RANGE[0] + (LOG10Q_RANGE[1] - LOG10Q_RANGE[0]) * u[5]
    q = 10.0 ** lq
    forced = u[6] < forced_frac
    t_cross = math.nan
    if forced:
        phi = 2.0 * math.pi * u[7]
        pick = int(ph.uniform_int(r[2][0], 4))
        zc = complex(critical_point(d, q, phi, pick))
        w = complex(math.cos(alpha), math.sin(alpha))
        v = -1j * w
        u0 = (zc * w.conjugate()).real
        tau_c = (zc * v.conjugate()).real
        if u0 < 0.0:
            alpha = alpha + math.pi
            if alpha >= 2.0 * math.pi:
                alpha -= 2.0 * math.pi
            u0, tau_c = -u0, -tau_c
        t_cross = T_CROSS_RANGE[0] + (T_CROSS_RANGE[1] - T_CROSS_RANGE[0]) * u[9]
        t0 = t_cross - tau_c * tE
    sig = math.exp(LN_SIGMA_RANGE[0] + (LN_SIGMA_RANGE[1] - LN_SIGMA_RANGE[0]) * u[10])
    p_drop = DROP_MAX * u[11]
    gap = u[12] < GAP_PROB
    g0 = N_BIN * u[13]
    gw = GAP_MAX * N_BIN * u[14] if gap else 0.0
    theta = np.array([t0, tE, u0, alpha, d, q])
    return theta, dict(forced=forced, t_cross=t_cross, sigma=sig, p_drop=p_drop, g0=g0, gw=gw)


def noise_and_mask(seed, step, i, info):
    """Unit-normal noise per bin and the bins with data."""
    m = np.arange(N_BIN // 2)
    r = ph.philox4x64(step, OP_CNN_NOISE, i, m, seed, 0)
    z0, z1 = box_muller(r[:, 0], r[:, 1])
    z = np.empty(N_BIN)
    z[0::2], z[1::2] = z0, z1
    ud = np.empty(N_BIN)
    ud[0::2], ud[1::2] = ph.u01(r[:, 2]), ph.u01(r[:, 3])
    j = np.arange(N_BIN, dtype=np.float64)
    dj = j - info["g0"]
    dj = np.where(dj < 0.0, dj + N_BIN, dj)
    kept = (ud >= info["p_drop"]) & ~(dj < info["gw"])
    if kept.sum() < MIN_KEPT:
        kept[:] = True
    return z, kept


def targets(theta):
    t0, tE, u0, alpha, d, q = theta
    return np.array([t0, math.log(tE), u0, alpha / (2.0 * math.pi), math.log(d), math.log10(q)])


def make_batch(seed, step, B, forced_frac=0.1):
    """Training batch: inputs x [B, 256, 2], targets y [B, 6], parameters theta [B, 6] in window
    units, and the per-sample settings."""
    s = bin_centres()
    X = np.zeros((B, N_BIN, 2))
    Y = np.zeros((B, 6))
    TH = np.zeros((B, 6))
    infos = []
    for i in range(B):
        theta, info = sample_theta(seed, step, i, forced_frac)
        A = osb.magnification(theta[None, :], s)[0]
        z, kept = noise_and_mask(seed, step, i, info)
        F = A * (1.0 + info["sigma"] * z)
        X[i] = normalise(F, kept)
        Y[i] = targets(theta)
        TH[i] = theta
        infos.append(info)
    return X, Y, TH, infos


def init_params(seed):
    """He-normal weights (std sqrt(2 / fan_in), fan_in = the matrix's rows) for every layer but the
    last, whose std is 0.1 sqrt(1 / fan_in); zero biases. Parameter p draws block p >> 1 and takes
    the cosine (even p) or sine (odd p) deviate."""
    p = np.arange(N_PARAMS)
    r = ph.philox4x64(p >> 1, OP_CNN_INIT, 0, 0, seed, 0)
    z0, z1 = box_muller(r[:, 0], r[:, 1])
    z = np.where(p % 2 == 0, z0, z1)
    w = np.zeros(N_PARAMS)
    o = 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        if name.startswith("W"):
            std = math.sqrt(2.0 / shape[0]) if name != "W6" else 0.1 * math.sqrt(1.0 / shape[0])
            w[o : o + n] = z[o : o + n] * std
        o += n
    return w


def lr_at(t, n_steps, warmup, lr0):
    """Learning rate of step t (1-based): linear warm-up over `warmup` steps, then a cosine decay
    from lr0 to 0.1 lr0 at step n_steps."""
    warm = min(1.0, t / warmup) if warmup > 0 else 1.0
    frac = min(1.0, (t - 1) / max(1, n_steps))
    return lr0 * warm * (0.1 + 0.45 * (1.0 + math.cos(math.pi * frac)))


def adamw(w, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4):
    """One AdamW step (Loshchilov & Hutter): decay w by lr * weight_decay, then the bias-corrected
    Adam step. t is the 1-based step number. Returns new (w, m, v)."""
    w = w * (1.0 - lr * weight_decay)
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def propose_genes(out, window, lo, hi, n_seed, seed, round=0):
    """Seed rows for lightcurve l in draw round `round` (counter word 0; the fitter seeds its first
    population with round 0): row 0 is the network's mean; row r >= 1 draws y = mu + exp(s / 2) n with n six
    standard normal deviates (key (seed, l), counter (round, OP_CNN_SAMPLE, r, block)). y is
    mapped from window units to physical parameters (t0 = c + h y0, tE = h e^{y1}, u0 = y2,
    alpha = 2 pi y3 wrapped to [0, 2 pi), d = e^{y4}, log10 q = y5), then to genes
    (v - lo) / (hi - lo) clamped to [0, 1]; a non-finite gene is 0.5. Returns [n_lc, n_seed, 6]."""
    out = np.asarray(out, dtype=np.float64)
    n_lc = out.shape[0]
    G = np.zeros((n_lc, n_seed, 6))
    rows = np.arange(n_seed)
    for l in range(n_lc):
        ra = ph.philox4x64(round, OP_CNN_SAMPLE, rows, 0, seed, l)
        rb = ph.philox4x64(round, OP_CNN_SAMPLE, rows, 1, seed, l)
        n = np.empty((n_seed, 6))
        n[:, 0], n[:, 1] = box_muller(ra[:, 0], ra[:, 1])
        n[:, 2], n[:, 3] = box_muller(ra[:, 2], ra[:, 3])
        n[:, 4], n[:, 5] = box_muller(rb[:, 0], rb[:, 1])
        n[0] = 0.0
        mu, s = out[l, :6], out[l, 6:]
        y = mu + np.exp(0.5 * s) * n
        c, h = window[l]
        a = 2.0 * math.pi * y[:, 3]
        a = a - 2.0 * math.pi * np.floor(a / (2.0 * math.pi))
        v = np.stack([c + h * y[:, 0], h * np.exp(y[:, 1]), y[:, 2], a, np.exp(y[:, 4]), y[:, 5]], axis=1)
        g = (v - lo) / (hi - lo)
        g = np.where(np.isfinite(g), np.clip(g, 0.0, 1.0), 0.5)
        G[l] = g
    return G
