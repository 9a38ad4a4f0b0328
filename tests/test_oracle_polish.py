"""Pins of the amoeba oracle (oracle/polish.py) against known minima and a hand-checked step."""
import math

import numpy as np
import pytest

from oracle import polish as opo


def test_quadratic_minimum_inside_the_box():
    c = np.array([0.3, 0.6, 0.45, 0.2, 0.7, 0.55])
    w = np.array([1.0, 3.0, 0.5, 2.0, 1.5, 4.0])
    x, f, fev = opo.nelder_mead(lambda x: float(np.sum(w * (x - c) ** 2)), np.full(6, 0.5), maxfev=3000)
    np.testing.assert_allclose(x, c, atol=1e-6)
    assert f < 1e-11 and fev <= 3006


def test_minimum_on_the_edge_of_the_box():
    c = np.array([1.3, -0.2, 0.5, 0.5, 0.5, 0.5])  # outside in genes 0 and 1: the box corner is optimal
    x, f, _ = opo.nelder_mead(lambda x: float(np.sum((x - c) ** 2)), np.full(6, 0.5), maxfev=3000)
    np.testing.assert_allclose(x, [1.0, 0.0, 0.5, 0.5, 0.5, 0.5], atol=1e-6)
    assert np.all((x >= 0) & (x <= 1))


def test_rosenbrock_valley():
    def rosen(x):
        y = 2.0 * x - 0.5  # minimum at x = 0.75
        return float(np.sum(100.0 * (y[1:] - y[:-1] ** 2) ** 2 + (1.0 - y[:-1]) ** 2))

    x, f, _ = opo.nelder_mead(rosen, np.full(6, 0.3), maxfev=20000)
    assert f < 1e-8
    np.testing.assert_allclose(x, 0.75, atol=1e-4)


def test_never_worse_and_budget():
    g = np.random.default_rng(0)
    A = g.normal(size=(6, 6))
    fun = lambda x: float(np.sum(np.sin(7 * A @ x)) + np.sum(x**2))  # noqa: E731
    calls = []

    def counted(x):
        calls.append(1)
        return fun(x)

    x0 = g.uniform(size=6)
    x, f, fev = opo.nelder_mead(counted, x0, maxfev=200)
    assert f <= fun(x0) and fev <= 206 and len(calls) == fev + 1


def test_first_step_by_hand():
    """Two genes, f = x0 + 2 x1 from (0.5, 0.5): the start simplex is (0.5,0.5), (0.53,0.5),
    (0.5,0.53); the worst (0.5,0.53) reflects through the centroid (0.515, 0.5) to (0.53, 0.47),
    which beats the best, so the expansion (0.545, 0.44) is tried and kept."""
    seen = []

    def f(x):
        seen.append(x.copy())
        return float(x[0] + 2 * x[1])

    opo.nelder_mead(f, np.array([0.5, 0.5]), maxfev=4)
    np.testing.assert_allclose(seen[1], [0.53, 0.5])
    np.testing.assert_allclose(seen[2], [0.5, 0.53])
    np.testing.assert_allclose(seen[3], [0.53, 0.47])
    np.testing.assert_allclose(seen[4], [0.545, 0.44])
    assert math.isclose(f(seen[4]), 0.545 + 0.88)


def test_blended_objective_recovers_a_blended_curve():
    """Section 4.4's blended model: from near the truth of a noise-free curve diluted to f = 0.35,
    the amoeba on the profiled-f objective returns to the truth (chi^2 ~ 0, f recovered), while
    the unblended objective is left with a large chi^2."""
    from oracle import ea
    from oracle import sblm as osb

    lo = np.array([-20.0, 5.0, 0.0, 0.0, 0.3, -4.0])
    hi = np.array([20.0, 100.0, 1.0, 2 * np.pi, 3.0, 0.0])
    truth = np.array([[1.5, 22.0, 0.15, 0.9, 1.2, 0.25]])
    t = np.linspace(-50.0, 50.0, 120)
    A = osb.magnification(truth, t)[0]
    flux = 0.35 * A + 0.65
    sigma = 0.01 * flux
    g_true = (np.array([1.5, 22.0, 0.15, 0.9, 1.2, np.log10(0.25)]) - lo) / (hi - lo)
    start = g_true + np.array([0.004, -0.003, 0.002, 0.001, -0.002, 0.003])
    g, c, _ = opo.polish_sblm(t, flux, sigma, lo, hi, start, 1500, blend=True)
    c_start = osb.chi2_blend(ea.sblm_theta(start[None, :], lo, hi), t, flux, sigma)[0][0]
    assert c < 1e-2 * c_start and c < 1.0
    _, f = osb.chi2_blend(ea.sblm_theta(np.asarray(g)[None, :], lo, hi), t, flux, sigma)
    assert f[0] == pytest.approx(0.35, rel=2e-2)
    _, c_plain, _ = opo.polish_sblm(t, flux, sigma, lo, hi, start, 300)
    assert c_plain > 100 * max(c, 1.0)
