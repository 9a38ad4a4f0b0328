"""Oracle: static binary-lens model (SBLM), point source, FP64, plain numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the product path never imports it.

What it computes, in the paper's order (Rajpaul 2012, Section 2.2):

1. source position on a rectilinear trajectory, Eq. (sourcePos) with tau = (t - t_m)/t_E;
2. the lens equation, Eq. (lensing): zeta = z - 1/conj(z) + q/(a - conj(z)), primary lens at the
   origin, secondary of mass ratio q at z = a on the +x axis, lengths in units of the primary's
   Einstein angle (Section 2.1);
3. the complex quintic of Eq. (lensingPoly). The paper does not print its coefficients (it cites
   Witt 1990); they are derived here. Conjugating the lens equation gives
   conj(z) = N(z)/D(z) with D = z (z - a) and N = conj(zeta) D + (1 + q) z - a. Substituting that
   back into the lens equation and clearing denominators gives
       p(z) = (z - zeta) N (N - a D) - D (N - a D) - q D N,
   a quintic with leading coefficient conj(zeta) (conj(zeta) - a). It is built below by literal
   polynomial multiplication of those factors, never from hand-expanded coefficients;
4. its five roots (companion-matrix eigenvalues, a library primitive);
5. rejection of the spurious roots "by direct substitution into Eq. (lensing)": every root first
   gets a few Newton steps on the lens equation itself (not on the polynomial), then the roots
   whose relative lens-equation residual is below ``LENS_TOL`` are the images;
6. image magnification A_i = 1/|det J_i|, det J = 1 - |1/z^2 + q/(a - z)^2|^2. The paper prints the
   modulus without the square (Section 2.2, the equation for A_i); the square is required for
   the Jacobian of the lens map and for the single-lens (Paczynski) limit;
7. total magnification A = sum_i A_i (flux of a unit, unblended source), and the chi^2 of
   Section 4.1, sum_k ((F_k - A_k) / sigma_k)^2;
8. the blended model of Section 4.4, f A + (1 - f), with f profiled out in closed form
   (``blend_fit``; flux normalised to the baseline).

Readings where the paper is silent:
* the image count must be 3 or 5 (Section 2.2) and the parities must sum to -1 (image-counting
  theorem for two point lenses). When the residual test gives anything else, the 3 smallest
  residuals are kept, plus the 4th and 5th when both are below ``PAIR_TOL``, and the point is
  flagged;
* a source exactly on a lens (zeta = 0 or zeta = a) makes the leading coefficient vanish; zeta is
  then moved by ``DEGENERATE_SHIFT`` along +x and the point is flagged.

Parameter vector convention: theta = (t0, tE, u0, alpha, d, q) = (t_m, t_E, b, theta, a, q) of
Section 2.1.

Pinned by tests/test_oracle_forward.py: closed-form trajectory geometry, the lens-equation
residual of every image, the 3-or-5 image count and parity sum, the Paczynski limit for q -> 0
and for a -> 0, mirror symmetry, the far-field limit, a numerical Jacobian of the lens map at
each image, a brute-force lens-equation image search that never touches the quintic, and
inverse ray shooting on a small source; the blended fit by its exact recovery of a blended
curve, a brute-force scan over f, and its clamps.
"""
from __future__ import annotations

import numpy as np

LENS_TOL = 1e-10          # relative lens-equation residual accepting a polished root as an image
PAIR_TOL = 1e-8           # fallback: 4th and 5th roots both below this -> five images
POLISH_STEPS = 4          # Newton steps on the lens equation applied to every root
DEGENERATE_SHIFT = 1e-12  # shift of zeta when it sits on a lens (leading coefficient zero)
CHUNK = 1 << 16           # points per vectorised batch


# --------------------------------------------------------------------------------------------
# 1. trajectory, Eq. (sourcePos)
# --------------------------------------------------------------------------------------------
def source_position(t, t0, tE, u0, alpha):
    """Eq. (sourcePos): zeta = tau sin(theta) + b cos(theta) + i(-tau cos(theta) + b sin(theta)),
    with tau = (t - t_m)/t_E. Arguments broadcast against each other."""
    tau = (np.asarray(t, dtype=np.float64) - t0) / tE
    return (tau * np.sin(alpha) + u0 * np.cos(alpha)) + 1j * (-tau * np.cos(alpha) + u0 * np.sin(alpha))


# --------------------------------------------------------------------------------------------
# 2. lens equation, Eq. (lensing)
# --------------------------------------------------------------------------------------------
def lens_map(z, d, q):
    """Right-hand side of Eq. (lensing): the source position that the image position z maps to."""
    zb = np.conj(z)
    return z - 1.0 / zb + q / (d - zb)


def lens_residual(z, zeta, d, q):
    """f(z) = z - 1/conj(z) + q/(a - conj(z)) - zeta; zero exactly at the images."""
    return lens_map(z, d, q) - zeta


def relative_residual(z, zeta, d, q):
    """|f(z)| divided by the sum of the magnitudes of the terms of Eq. (lensing)."""
    scale = np.abs(z) + 1.0 / np.abs(z) + q / np.abs(d - z) + np.abs(zeta)
    return np.abs(lens_residual(z, zeta, d, q)) / scale


def shear_term(z, d, q):
    """kappa(z) = 1/z^2 + q/(a - z)^2, so that det J = 1 - |kappa|^2 (conjugation leaves |kappa| unchanged)."""
    return 1.0 / (z * z) + q / ((d - z) * (d - z))


def jacobian_det(z, d, q):
    """det J of the lens map at image z: 1 - |1/z^2 + q/(a - z)^2|^2."""
    k = shear_term(z, d, q)
    return 1.0 - (k.real * k.real + k.imag * k.imag)


# --------------------------------------------------------------------------------------------
# 3. the quintic of Eq. (lensingPoly), by polynomial multiplication
# --------------------------------------------------------------------------------------------
def _polymul(a, b):
    """Product of two batched polynomials stored in ascending order along the last axis."""
    shape = np.broadcast_shapes(a.shape[:-1], b.shape[:-1]) + (a.shape[-1] + b.shape[-1] - 1,)
    out = np.zeros(shape, dtype=np.complex128)
    for i in range(a.shape[-1]):
        for j in range(b.shape[-1]):
            out[..., i + j] += a[..., i] * b[..., j]
    return out


def _poly(*coeffs):
    """Batched polynomial from ascending coefficients (each broadcastable)."""
    arrs = np.broadcast_arrays(*[np.asarray(c, dtype=np.complex128) for c in coeffs])
    return np.stack(arrs, axis=-1)


def _padd(a, b):
    n = max(a.shape[-1], b.shape[-1])
    pa = np.zeros(a.shape[:-1] + (n,), np.complex128)
    pb = np.zeros(b.shape[:-1] + (n,), np.complex128)
    pa[..., : a.shape[-1]] = a
    pb[..., : b.shape[-1]] = b
    return pa + pb


def quintic_coefficients(zeta, d, q):
    """Ascending coefficients c_0..c_5 of p(z) = (z - zeta) N (N - a D) - D (N - a D) - q D N.

    D = z (z - a) and N = conj(zeta) D + (1 + q) z - a, from conj(z) = N/D (the conjugated lens
    equation). ``zeta``, ``d`` and ``q`` broadcast; the result has a trailing axis of length 6.
    """
    zeta = np.asarray(zeta, dtype=np.complex128)
    d = np.asarray(d, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    zbar = np.conj(zeta)
    zero = np.zeros(np.broadcast_shapes(zeta.shape, d.shape, q.shape))
    one = zero + 1.0
    z_poly = _poly(zero, one)                         # z
    D = _polymul(z_poly, _poly(-d + zero, one))       # z (z - a)
    N = _padd(zbar[..., None] * D, _poly(-d + zero, (1.0 + q) + zero))
    NmaD = _padd(N, -(d + zero)[..., None] * D)       # N - a D
    term1 = _polymul(_polymul(_poly(-zeta + zero, one), N), NmaD)
    term2 = _polymul(D, NmaD)
    term3 = (q + zero)[..., None] * _polymul(D, N)
    return _padd(term1, -_padd(term2, term3))


def quintic_roots(coeffs):
    """All five roots of each quintic (ascending coefficients on the last axis), as the
    eigenvalues of its Frobenius companion matrix."""
    c = np.asarray(coeffs, dtype=np.complex128)
    mon = c[..., :5] / c[..., 5:6]
    comp = np.zeros(c.shape[:-1] + (5, 5), dtype=np.complex128)
    for k in range(4):
        comp[..., k + 1, k] = 1.0
    comp[..., :, 4] = -mon
    return np.linalg.eigvals(comp)


# --------------------------------------------------------------------------------------------
# 5. spurious-root rejection
# --------------------------------------------------------------------------------------------
def polish(z, zeta, d, q, steps=POLISH_STEPS):
    """Newton steps on the lens equation (not on the polynomial), one root at a time.

    f(z + delta) ~ f + delta + K conj(delta), where K = 1/conj(z)^2 + q/(a - conj(z))^2 is the
    derivative of f with respect to conj(z). Solving delta + K conj(delta) = -f gives
    delta = (-f + K conj(f)) / (1 - |K|^2); a step is skipped where 1 - |K|^2 vanishes.

    Polishing only corrects the rounding error of a root. A root that would move by more than
    half its distance to the nearest other root of the same quintic is not an image that the
    polynomial resolved (a spurious root heading for a true image, or an unresolved pair next
    to a lens), so it keeps its unpolished value.
    """
    z0 = np.array(z, dtype=np.complex128, copy=True)
    n = z0.shape[-1]
    gap = np.abs(z0[..., :, None] - z0[..., None, :]) + np.where(np.eye(n, dtype=bool), np.inf, 0.0)
    cap = 0.5 * gap.min(axis=-1)
    z = z0.copy()
    for _ in range(steps):
        f = lens_residual(z, zeta, d, q)
        zb = np.conj(z)
        K = 1.0 / (zb * zb) + q / ((d - zb) * (d - zb))
        den = 1.0 - np.abs(K) ** 2
        ok = np.abs(den) >= 1e-300
        delta = np.where(ok, (-f + K * np.conj(f)) / np.where(ok, den, 1.0), 0.0)
        z = np.where(np.isfinite(delta), z + delta, z)
    keep = np.isfinite(z) & (np.abs(z - z0) <= cap)
    return np.where(keep, z, z0)


def images(zeta, d, q):
    """Images of the source(s) ``zeta`` (any shape) for lens (d, q).

    Returns a dict with ``z`` (..., 5) polished roots, ``is_image`` (..., 5), ``det`` (..., 5) the
    Jacobian determinants, ``n`` (...) the image count, ``flag`` (...) True where a fallback
    reading was taken, and ``A`` (...) the total magnification.
    """
    zeta = np.asarray(zeta, dtype=np.complex128)
    d = np.broadcast_to(np.asarray(d, dtype=np.float64), zeta.shape)
    q = np.broadcast_to(np.asarray(q, dtype=np.float64), zeta.shape)
    degenerate = (np.abs(zeta) < DEGENERATE_SHIFT) | (np.abs(zeta - d) < DEGENERATE_SHIFT)
    zeta = np.where(degenerate, zeta + DEGENERATE_SHIFT, zeta)

    roots = quintic_roots(quintic_coefficients(zeta, d, q))
    zeta5, d5, q5 = zeta[..., None], d[..., None], q[..., None]
    z = polish(roots, zeta5, d5, q5)
    r = relative_residual(z, zeta5, d5, q5)
    r = np.where(np.isfinite(r), r, np.inf)
    det = jacobian_det(z, d5, q5)

    accepted = r <= LENS_TOL
    count = accepted.sum(axis=-1)
    parity = np.where(accepted, np.sign(det), 0.0).sum(axis=-1)
    # two accepted roots on the same image would count it twice
    dz = np.abs(z[..., :, None] - z[..., None, :]) + np.where(np.eye(5, dtype=bool), np.inf, 0.0)
    both = accepted[..., :, None] & accepted[..., None, :]
    duplicate = np.any(both & (dz <= 1e-9 * (1.0 + np.abs(z[..., :, None]))), axis=(-1, -2))
    ok = ((count == 3) | (count == 5)) & (parity == -1) & ~duplicate

    # fallback: the 3 smallest residuals, plus the 4th and 5th when both are small
    order = np.argsort(r, axis=-1, kind="stable")
    r_sorted = np.take_along_axis(r, order, axis=-1)
    five = (r_sorted[..., 3] <= PAIR_TOL) & (r_sorted[..., 4] <= PAIR_TOL)
    rank = np.empty_like(order)
    np.put_along_axis(rank, order, np.arange(5), axis=-1)
    fallback = (rank < 3) | ((rank >= 3) & five[..., None])
    is_image = np.where(ok[..., None], accepted, fallback)

    A = np.where(is_image, 1.0 / np.abs(det), 0.0).sum(axis=-1)
    return {
        "z": z,
        "is_image": is_image,
        "det": det,
        "residual": r,
        "n": is_image.sum(axis=-1),
        "flag": ~ok | degenerate,
        "A": A,
    }


# --------------------------------------------------------------------------------------------
# 6-7. magnification over (candidate, epoch) and chi^2
# --------------------------------------------------------------------------------------------
def _split_theta(theta):
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    return [theta[:, k : k + 1] for k in range(6)]


def magnification(theta, t, return_info=False):
    """Point-source magnification A[cand, epoch] for parameter rows theta = (t0, tE, u0, alpha, d, q).

    With ``return_info`` also returns the per-point image count, fallback flag and the smallest
    |det J| over the images (how close the point is to a caustic).
    """
    t0, tE, u0, alpha, d, q = _split_theta(theta)
    t = np.asarray(t, dtype=np.float64)
    zeta = source_position(t[None, :], t0, tE, u0, alpha)
    dd = np.broadcast_to(d, zeta.shape).ravel()
    qq = np.broadcast_to(q, zeta.shape).ravel()
    zf = zeta.ravel()
    A = np.empty(zf.shape)
    n = np.empty(zf.shape, dtype=np.int64)
    flag = np.empty(zf.shape, dtype=bool)
    mindet = np.empty(zf.shape)
    for s in range(0, zf.size, CHUNK):
        e = min(zf.size, s + CHUNK)
        im = images(zf[s:e], dd[s:e], qq[s:e])
        A[s:e] = im["A"]
        n[s:e] = im["n"]
        flag[s:e] = im["flag"]
        mindet[s:e] = np.where(im["is_image"], np.abs(im["det"]), np.inf).min(axis=-1)
    A = A.reshape(zeta.shape)
    if not return_info:
        return A
    return A, {"n": n.reshape(zeta.shape), "flag": flag.reshape(zeta.shape), "min_det": mindet.reshape(zeta.shape)}


def chi2_from_model(model, flux, sigma):
    """chi^2 = sum_k ((F_k - model_k) / sigma_k)^2 over the last axis (Section 4.1)."""
    r = (np.asarray(flux, np.float64) - model) / np.asarray(sigma, np.float64)
    return np.sum(r * r, axis=-1)


def chi2(theta, t, flux, sigma):
    """chi^2 of each parameter row against the lightcurve (t, flux, sigma)."""
    return chi2_from_model(magnification(theta, t), flux, sigma)


BLEND_F_MIN = 1e-3  # smallest blending fraction of the profiled fit


def blend_fit(A, flux, sigma, f_min=BLEND_F_MIN):
    """Blended model of Section 4.4 (Eq. blend), A_obs = f A + (1 - f), with the fraction f
    profiled out: the paper notes that its least-squares value follows from a linear equation.
    With a = A - 1, b = F - 1 and w = 1/sigma^2, chi^2(f) = sum w (b - f a)^2 is least at
    f = sum w a b / sum w a^2, clamped to [f_min, 1]. Sums run over the last axis in order.
    Returns (chi^2, f)."""
    A = np.asarray(A, np.float64)
    a = A - 1.0
    b = np.asarray(flux, np.float64) - 1.0
    w = 1.0 / np.asarray(sigma, np.float64) ** 2
    s_ab = np.sum(w * a * b, axis=-1)
    s_aa = np.sum(w * a * a, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(s_aa > 0.0, s_ab / s_aa, 1.0)
    f = np.clip(f, f_min, 1.0)
    r = b - f[..., None] * a
    return np.sum(w * r * r, axis=-1), f


def chi2_blend(theta, t, flux, sigma, f_min=BLEND_F_MIN):
    """(chi^2, f) of each parameter row with the blending fraction profiled out."""
    return blend_fit(magnification(theta, t), flux, sigma, f_min)


def paczynski(u):
    """Single point-lens magnification (u^2 + 2) / (u sqrt(u^2 + 4)); used only by pins."""
    u = np.asarray(u, dtype=np.float64)
    return (u * u + 2.0) / (u * np.sqrt(u * u + 4.0))


def steepness(theta, t):
    """Amplification of a relative rounding of the source position into the magnification,
    |grad_zeta ln A| * max(1, |zeta|), by central differences in the source plane (used to tell
    points where the magnification is steep, near caustics, from the rest)."""
    th = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    zeta = source_position(np.asarray(t, dtype=np.float64)[None, :], th[:, 0:1], th[:, 1:2], th[:, 2:3], th[:, 3:4])
    d = np.broadcast_to(th[:, 4:5], zeta.shape).ravel()
    q = np.broadcast_to(th[:, 5:6], zeta.shape).ravel()
    z = zeta.ravel()
    h = 1e-6 * np.maximum(1.0, np.abs(z))
    A = np.empty(z.shape)
    grad2 = np.zeros(z.shape)
    for s0 in range(0, z.size, CHUNK):
        sl = slice(s0, min(z.size, s0 + CHUNK))
        A[sl] = images(z[sl], d[sl], q[sl])["A"]
        for step in (h[sl], 1j * h[sl]):
            ap = images(z[sl] + step, d[sl], q[sl])["A"]
            am = images(z[sl] - step, d[sl], q[sl])["A"]
            grad2[sl] += ((ap - am) / (2 * h[sl])) ** 2
    return (np.sqrt(grad2) / A * np.maximum(1.0, np.abs(z))).reshape(zeta.shape)
