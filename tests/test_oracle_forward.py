"""Pins of the oracle's forward model against what the paper and the mathematics fix.

None of these tests re-types the oracle's quintic: the images are checked against the lens
equation itself (Eq. lensing), against a brute-force solver that never forms the polynomial,
against limits with closed forms, and against inverse ray shooting.
"""
import os

import numpy as np
import pytest

from oracle import sblm as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paczynski(u):
    """Single point-lens magnification (Paczynski 1986), a textbook closed form."""
    return (u * u + 2.0) / (u * np.sqrt(u * u + 4.0))


def lens_map(z, d, q):
    """Eq. (lensing), written here from the paper for the independent checks."""
    zb = np.conj(z)
    return z - 1.0 / zb + q / (d - zb)


def random_lenses(n, seed, qlo=-4.0):
    g = np.random.default_rng(seed)
    zeta = g.uniform(-1.5, 1.5, n) + 1j * g.uniform(-1.5, 1.5, n)
    d = np.exp(g.uniform(np.log(0.3), np.log(3.0), n))
    q = 10.0 ** g.uniform(qlo, 0.0, n)
    return zeta, d, q


def test_trajectory_golden():
    rows = np.loadtxt(os.path.join(GOLDEN, "trajectory.txt"))
    for t, tm, tE, b, th, re, im in rows:
        z = S.source_position(t, tm, tE, b, th * np.pi)
        assert abs(z - (re + 1j * im)) < 1e-14


def test_trajectory_geometry():
    g = np.random.default_rng(3)
    for _ in range(50):
        t0, tE, u0, al = g.uniform(-20, 20), g.uniform(5, 100), g.uniform(0, 1), g.uniform(0, 2 * np.pi)
        z0 = S.source_position(t0, t0, tE, u0, al)
        z1 = S.source_position(t0 + tE, t0, tE, u0, al)
        # closest approach b e^{i theta} at t = t_m, unit speed per t_E, velocity perpendicular to b
        assert abs(z0 - u0 * np.exp(1j * al)) < 1e-14
        assert abs(abs(z1 - z0) - 1.0) < 1e-13
        assert abs(np.real((z1 - z0) * np.conj(np.exp(1j * al)))) < 1e-13


def test_images_solve_lens_equation_count_and_parity():
    zeta, d, q = random_lenses(40000, 11)
    im = S.images(zeta, d, q)
    assert not im["flag"].any()
    n = im["n"]
    assert set(np.unique(n)) <= {3, 5}
    assert (n == 5).sum() > 50  # both image counts occur
    res = np.abs(lens_map(im["z"], d[:, None], q[:, None]) - zeta[:, None])
    scale = np.abs(im["z"]) + 1 / np.abs(im["z"]) + q[:, None] / np.abs(d[:, None] - im["z"]) + np.abs(zeta[:, None])
    assert np.all((res / scale)[im["is_image"]] <= 1e-10)
    # spurious roots are not solutions
    assert np.all((res / scale)[~im["is_image"]] > 1e-6)
    parity = np.where(im["is_image"], np.sign(im["det"]), 0).sum(-1)
    assert np.all(parity == -1)


def _brute_force_images(zeta, d, q):
    """All solutions of Eq. (lensing) by damped Newton on the real 2-D system with a
    finite-difference Jacobian, started from a dense set of points; no polynomial involved."""
    starts = []
    gx = np.linspace(-3.0, 3.0 + d, 61)
    gy = np.linspace(-3.0, 3.0, 61)
    X, Y = np.meshgrid(gx, gy)
    starts.append((X + 1j * Y).ravel())
    for c in (0.0, d):
        for r in np.geomspace(1e-5, 0.5, 24):
            ang = np.linspace(0, 2 * np.pi, 24, endpoint=False) + 0.1
            starts.append(c + r * np.exp(1j * ang))
    z = np.concatenate(starts)

    def F(z):
        w = lens_map(z, d, q) - zeta
        return np.stack([w.real, w.imag], -1)

    for _ in range(80):
        h = 1e-7 * (1.0 + np.abs(z))
        f0 = F(z)
        jx = (F(z + h) - F(z - h)) / (2 * h[:, None])
        jy = (F(z + 1j * h) - F(z - 1j * h)) / (2 * h[:, None])
        det = jx[:, 0] * jy[:, 1] - jy[:, 0] * jx[:, 1]
        det = np.where(np.abs(det) < 1e-300, 1e-300, det)
        dx = -(jy[:, 1] * f0[:, 0] - jy[:, 0] * f0[:, 1]) / det
        dy = -(-jx[:, 1] * f0[:, 0] + jx[:, 0] * f0[:, 1]) / det
        step = dx + 1j * dy
        lim = 0.2 * (np.abs(z) + 0.05)
        step = np.where(np.abs(step) > lim, step * lim / np.abs(step), step)
        z = z + np.where(np.isfinite(step), step, 0)
    w = np.abs(lens_map(z, d, q) - zeta)
    good = np.isfinite(w) & (w < 1e-11 * (1 + np.abs(zeta))) & (np.abs(z) > 1e-9) & (np.abs(z - d) > 1e-9)
    found = []
    for zz in z[good]:
        if all(abs(zz - f) > 1e-7 for f in found):
            found.append(zz)
    return np.array(found)


@pytest.mark.parametrize("case", range(12))
def test_images_match_brute_force_solver(case):
    zeta, d, q = random_lenses(12, 5, qlo=-2.0)
    zeta, d, q = zeta[case], d[case], q[case]
    im = S.images(np.array([zeta]), d, q)
    ours = im["z"][0][im["is_image"][0]]
    brute = _brute_force_images(zeta, d, q)
    assert len(brute) == len(ours), (zeta, d, q, ours, brute)
    for z in ours:
        assert np.min(np.abs(brute - z)) < 1e-7


@pytest.mark.parametrize("u", [0.05, 0.3, 1.0, 2.5])
def test_paczynski_limit_small_q(u):
    """q -> 0: the binary lens becomes a point lens of unit mass at the origin; the deviation
    is O(q)."""
    zeta = np.array([u * np.exp(0.7j)])
    e6 = S.images(zeta, 1.1, 1e-6)["A"][0] / paczynski(u) - 1
    e7 = S.images(zeta, 1.1, 1e-7)["A"][0] / paczynski(u) - 1
    assert abs(e7) < 5e-6
    assert abs(e6) < 5e-5
    if abs(e7) > 1e-12:
        assert 5.0 < e6 / e7 < 20.0  # linear in q


@pytest.mark.parametrize("d", [1e-2, 1e-3, 1e-4])
def test_merged_lens_limit(d):
    """a -> 0: both masses at one point act as one lens of mass 1 + q, whose Einstein radius is
    sqrt(1 + q) in units of the primary's; the deviation is O(a^2)."""
    q = 0.5
    for u in (0.2, 0.7, 1.5):
        zeta = np.array([u * np.exp(0.4j)])
        A = S.images(zeta, d, q)["A"][0]
        ue = abs(zeta[0] - q * d / (1 + q)) / np.sqrt(1 + q)
        assert abs(A / paczynski(ue) - 1) < 0.3 * d * d


def test_mirror_symmetry():
    zeta, d, q = random_lenses(5000, 21)
    a = S.images(zeta, d, q)
    b = S.images(np.conj(zeta), d, q)
    away = (np.where(a["is_image"], np.abs(a["det"]), np.inf).min(-1) > 1e-3)
    assert np.allclose(a["A"][away], b["A"][away], rtol=1e-10, atol=0)
    assert np.array_equal(a["n"], b["n"])


def test_far_field():
    for d, q in [(0.5, 1.0), (1.2, 0.01), (2.5, 0.3)]:
        for r in (50.0, 200.0):
            zeta = np.array([r * np.exp(1.3j)])
            A = S.images(zeta, d, q)["A"][0]
            # a lens of total mass 1+q seen from far away: A - 1 ~ 2 (1+q)^2 / |zeta|^4
            assert abs(A - 1.0) < 4 * (1 + q) ** 2 / r**4


def test_numerical_jacobian_of_lens_map():
    """|det J| from the closed form equals the determinant of the finite-difference Jacobian
    of the lens map (the map R^2 -> R^2) at every image."""
    zeta, d, q = random_lenses(300, 31)
    im = S.images(zeta, d, q)
    for i in range(300):
        for k in np.nonzero(im["is_image"][i])[0]:
            z = im["z"][i, k]
            if abs(im["det"][i, k]) < 1e-2 or abs(z - d[i]) < 1e-2 or abs(z) < 1e-2:
                continue
            h = 1e-6 * max(1e-3, min(abs(z), abs(z - d[i])))
            fx = (lens_map(z + h, d[i], q[i]) - lens_map(z - h, d[i], q[i])) / (2 * h)
            fy = (lens_map(z + 1j * h, d[i], q[i]) - lens_map(z - 1j * h, d[i], q[i])) / (2 * h)
            det = fx.real * fy.imag - fy.real * fx.imag
            assert abs(det - im["det"][i, k]) < 1e-5 * max(1.0, abs(det)), (i, k, det, im["det"][i, k])


def _ray_shoot(zeta, d, q, rho, h0=0.01, sub=40):
    """Magnification of a disc source of radius rho by counting lens-plane rays that land in it:
    A = (rays in disc) * (ray cell area) / (pi rho^2). Two-level grid: coarse cells whose
    corners map near the source are refined."""
    lo_x, hi_x, lo_y, hi_y = -3.0, 3.0 + d, -3.0, 3.0
    xs = np.arange(lo_x, hi_x, h0)
    ys = np.arange(lo_y, hi_y, h0)
    X, Y = np.meshgrid(xs, ys)
    hit = np.zeros(X.shape, dtype=bool)
    for ox in (0.0, 0.5, 1.0):
        for oy in (0.0, 0.5, 1.0):
            w = lens_map(X + ox * h0 + 1j * (Y + oy * h0), d, q)
            hit |= np.abs(w - zeta) < 4 * rho
    # grow by one cell to catch cells whose interior maps inside
    grown = hit.copy()
    grown[1:, :] |= hit[:-1, :]
    grown[:-1, :] |= hit[1:, :]
    grown[:, 1:] |= hit[:, :-1]
    grown[:, :-1] |= hit[:, 1:]
    cx, cy = X[grown], Y[grown]
    f = (np.arange(sub) + 0.5) / sub * h0
    FX, FY = np.meshgrid(f, f)
    count = 0
    for s in range(0, cx.size, 2000):
        zz = (cx[s : s + 2000, None] + FX.ravel()[None, :]) + 1j * (cy[s : s + 2000, None] + FY.ravel()[None, :])
        count += np.count_nonzero(np.abs(lens_map(zz, d, q) - zeta) < rho)
    return count * (h0 / sub) ** 2 / (np.pi * rho * rho)


@pytest.mark.parametrize("zeta,d,q", [(0.3 + 0.2j, 1.0, 0.3), (-0.5 + 0.4j, 0.7, 0.05), (0.9 - 0.1j, 1.5, 0.5)])
def test_inverse_ray_shooting(zeta, d, q):
    im = S.images(np.array([zeta]), d, q)
    assert np.where(im["is_image"], np.abs(im["det"]), np.inf).min() > 0.05  # away from caustics
    A_rays = _ray_shoot(zeta, d, q, rho=0.02)
    assert abs(A_rays / im["A"][0] - 1) < 0.02


def test_chi2_definition():
    g = np.random.default_rng(7)
    theta = np.array([[0.0, 30.0, 0.1, 1.0, 1.2, 0.01], [3.0, 12.0, 0.5, 4.0, 0.8, 0.2]])
    t = np.sort(g.uniform(-60, 60, 50))
    A = S.magnification(theta, t)
    sigma = g.uniform(0.005, 0.05, 50)
    # the truth against its own noise-free curve
    assert S.chi2(theta[:1], t, A[0], sigma)[0] == 0.0
    flux = A[0] + sigma * g.standard_normal(50)
    direct = [sum(((flux[k] - A[i, k]) / sigma[k]) ** 2 for k in range(50)) for i in range(2)]
    assert np.allclose(S.chi2(theta, t, flux, sigma), direct, rtol=1e-13)


def test_caustic_forcing_crosses_a_caustic():
    """A trajectory aimed through a caustic changes its image count (3 <-> 5) at the crossing:
    sample a short window around the crossing time finely."""
    from paper_1208_4830_gb300 import synth

    theta = synth.prior_theta(40, 5)
    forced_theta, forced, t_cross = synth.force_caustics(theta, 0.5, 6)
    assert forced.sum() == 20 and np.all(np.isfinite(t_cross[forced])) and np.all(np.isnan(t_cross[~forced]))
    for row, tc in zip(forced_theta[forced], t_cross[forced]):
        # a near-tangent crossing spends only a short chord inside the caustic: zoom in
        changes = 0
        for half_width in (1e-3, 1e-5, 1e-7):
            t = tc + np.linspace(-half_width, half_width, 2001) * row[1]
            _, info = S.magnification(row[None, :], t, return_info=True)
            changes = max(changes, np.abs(np.diff(info["n"][0])).sum())
        assert changes >= 2


def test_blend_fit_recovers_a_blended_curve():
    theta = np.array([[0.0, 20.0, 0.2, 0.7, 1.1, 0.3]])
    t = np.linspace(-40, 40, 300)
    A = S.magnification(theta, t)[0]
    sigma = 0.01 * A
    for f0 in (1.0, 0.6, 0.05):
        flux = f0 * A + (1 - f0)
        c, f = S.blend_fit(A, flux, sigma)
        assert f == pytest.approx(f0, rel=1e-12) and c < 1e-18
    # the closed form is the minimum of a brute-force scan over f
    rng = np.random.default_rng(3)
    flux = 0.4 * A + 0.6 + sigma * rng.standard_normal(t.size)
    c, f = S.blend_fit(A, flux, sigma)
    grid = np.linspace(0.001, 1.0, 20001)
    scan = [np.sum(((flux - (g * A + 1 - g)) / sigma) ** 2) for g in grid]
    assert c <= min(scan) + 1e-9 and abs(f - grid[int(np.argmin(scan))]) < 1e-4
    assert c == pytest.approx(S.chi2_from_model(f * A + 1 - f, flux, sigma), rel=1e-12)


def test_blend_fit_clamps():
    A = np.array([1.0, 2.0, 5.0, 2.0, 1.0])
    sigma = np.full(5, 0.1)
    c, f = S.blend_fit(A, 2.0 * (A - 1) + 1, sigma)  # needs f = 2: clamped to 1
    assert f == 1.0 and c == pytest.approx(np.sum(((A - 1) / 0.1) ** 2))
    c, f = S.blend_fit(A, 1 - 0.5 * (A - 1), sigma)  # anti-correlated: clamped to f_min
    assert f == S.BLEND_F_MIN
    c, f = S.blend_fit(np.ones(5), np.ones(5) * 1.1, sigma)  # flat model: f = 1 by convention
    assert f == 1.0 and c == pytest.approx(5 * 1.0)


def test_steepness_closed_form_in_the_point_lens_limit():
    """steepness = |grad_zeta ln A| max(1, |zeta|). For a single lens, A depends on u = |zeta| only
    and d ln A / du = -8 / (u (u^2 + 2) (u^2 + 4)) (differentiating Paczynski's formula), so the
    steepness of a binary with a small secondary (q = 1e-6, deviations O(q)) far from the source
    is that closed form times max(1, u): it pins the central differences, the gradient's two directions, the
    normalisation by A and the max(1, |zeta|) factor (u runs from 0.05 to 4)."""
    t = np.linspace(-30.0, 30.0, 61)
    rows = []
    for u0, alpha in ((0.05, 0.3), (0.4, 2.0), (1.2, 4.0), (2.5, 5.5)):
        rows.append([0.0, 10.0, u0, alpha, 2.9, 1e-6])
    theta = np.array(rows)
    steep = S.steepness(theta, t)
    zeta = S.source_position(t[None, :], theta[:, 0:1], theta[:, 1:2], theta[:, 2:3], theta[:, 3:4])
    u = np.abs(zeta)
    far = np.abs(zeta - 2.9) > 0.05  # away from the secondary's (tiny) caustic
    expect = 8.0 / (u * (u * u + 2.0) * (u * u + 4.0)) * np.maximum(1.0, u)
    assert far.mean() > 0.9 and u.min() < 0.1 and u.max() > 3.0
    np.testing.assert_allclose(steep[far], expect[far], rtol=1e-4)
