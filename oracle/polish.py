"""Oracle: amoeba fine-tuning of the fittest EA solution, plain Python in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Section 4.1 couples the EA with the
downhill-simplex ("amoeba") method of Nelder & Mead (1965), in the modern form of Lagarias,
Reeds, Wright & Wright (1998), applied to the fittest solution the EA returns. This module states
that search for a box-bounded problem in the encoded genes, step by step:

* start simplex: x0 and x0 + delta e_j, with -delta where x0_j + delta would leave [0, 1];
* each step orders the vertices by objective (stable), reflects the worst through the centroid
  of the others (coefficient 1), then expands (2), contracts outside or inside (1/2), or shrinks
  every vertex halfway towards the best; trial points are clamped to [0, 1];
* when every vertex lies within 1e-9 of the best in every gene the simplex is rebuilt around the
  best vertex (restarted);
* the search stops once maxfev objective values have been taken (a step in progress may take up
  to n more); the result is the best vertex, never worse than the start.

Pinned by tests/test_oracle_polish.py: minima of convex quadratics inside and on the edge of the
box, the Rosenbrock valley, monotone improvement, the evaluation budget, and one hand-checked
reflection step.
"""
from __future__ import annotations

import math

import numpy as np

DELTA = 0.03
COLLAPSE = 1e-9


def nelder_mead(fun, x0, f0=None, maxfev=1000, delta=DELTA):
    """Minimise fun over [0, 1]^n from x0; returns (x_best, f_best, fev)."""
    x0 = np.asarray(x0, dtype=np.float64)
    n = x0.size
    clamp = lambda v: np.minimum(1.0, np.maximum(0.0, v))  # noqa: E731
    X = [x0.copy()]
    F = [float(f0) if f0 is not None and math.isfinite(f0) else float(fun(x0))]
    X += [None] * n
    F += [math.inf] * n
    fev = 0
    build = True
    f_start = F[0]
    while fev < maxfev:
        if build:
            for k in range(n):
                v = X[0].copy()
                v[k] = X[0][k] + (delta if X[0][k] + delta <= 1.0 else -delta)
                X[k + 1] = v
                F[k + 1] = float(fun(v))
            fev += n
            build = False
        # stable insertion sort by objective
        for i in range(1, n + 1):
            k = i
            while k > 0 and F[k] < F[k - 1]:
                F[k], F[k - 1] = F[k - 1], F[k]
                X[k], X[k - 1] = X[k - 1], X[k]
                k -= 1
        spread = max(float(np.max(np.abs(X[k] - X[0]))) for k in range(1, n + 1))
        if spread <= COLLAPSE:
            if fev + n > maxfev:
                break
            build = True
            continue
        xb = np.zeros(n)
        for k in range(n):  # centroid of every vertex but the worst, summed in order
            xb = xb + X[k]
        xb = xb / n
        xr = clamp(2.0 * xb - X[n])
        fr = float(fun(xr))
        fev += 1
        shrink = False
        if fr < F[0]:
            xe = clamp(3.0 * xb - 2.0 * X[n])
            fe = float(fun(xe))
            fev += 1
            X[n], F[n] = (xe, fe) if fe < fr else (xr, fr)
        elif fr < F[n - 1]:
            X[n], F[n] = xr, fr
        else:
            outside = fr < F[n]
            to = xr if outside else X[n]
            xc = clamp(xb + 0.5 * (to - xb))
            fc = float(fun(xc))
            fev += 1
            if (fc <= fr) if outside else (fc < F[n]):
                X[n], F[n] = xc, fc
            else:
                shrink = True
        if shrink:
            for k in range(1, n + 1):
                X[k] = X[0] + 0.5 * (X[k] - X[0])
                F[k] = float(fun(X[k]))
            fev += n
    best = int(np.argmin(F))
    if F[best] < f_start:
        return X[best], F[best], fev
    return x0, f_start, fev


def polish_sblm(t, flux, sigma, lo, hi, genes, maxfev, chi2_start=None, blend=False):
    """Amoeba fine-tuning of one SBLM solution given by its genes: (genes, chi^2, evaluations).
    With ``blend`` the objective is the chi^2 of the blended model of Section 4.4 with the
    blending fraction profiled out (``sblm.chi2_blend``)."""
    from . import ea, sblm

    def fun(g):
        theta = ea.sblm_theta(np.asarray(g)[None, :], lo, hi)
        c = (sblm.chi2_blend(theta, t, flux, sigma)[0] if blend else sblm.chi2(theta, t, flux, sigma))[0]
        return c if math.isfinite(c) else math.inf

    return nelder_mead(fun, genes, chi2_start, maxfev)
