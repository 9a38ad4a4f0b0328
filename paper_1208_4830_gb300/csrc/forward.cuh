// forward.cuh -- device forward model of the static binary-lens model (Rajpaul 2012, Section 2.2)
// for one (candidate, epoch): trajectory, quintic, roots, image selection, magnification.
//
// Geometry: primary of unit mass at the origin, secondary of mass ratio q at z = d on the +x
// axis, lengths in units of the primary's Einstein angle (Section 2.1).
#pragma once

#include "common.cuh"

namespace sblm {

// Tolerances per arithmetic. `step`: relative size of the last root correction that ends the
// iteration; `lens`: relative lens-equation residual that accepts a root as an image; `pair`:
// the fallback's bound for accepting the 4th and 5th roots together; `dup`: two accepted images
// closer than this (relative) are the same image; `shift`: a source closer than this to a
// lens is moved by it along +x (the quintic's leading coefficient vanishes there); `ambiguous`:
// a root whose residual lies between `lens` and this is neither clearly an image nor clearly
// spurious (an image pair the arithmetic could not resolve drops out with opposite parities,
// leaving the count and parity tests satisfied), so the epoch is flagged. `polish`: most Newton
// steps per root (fewer once a step is below the rounding level). `stall`: the polish also stops
// when a step left the squared residual above this fraction of the previous one (0: never), i.e.
// once the residual is at FP32's rounding level and Newton's steps only move the root within it.
// `cubic`: a root whose Aberth correction is below this (relative) is done: the iteration
// converges cubically, so after that update its error is far below the lens-equation polish's
// reach.
template <typename T>
struct Tol;
template <>
struct Tol<double> {
    static constexpr double step = 1e-13, lens = 1e-10, pair = 1e-8, dup = 1e-9, shift = 1e-12, ambiguous = 0.0,
                            cubic = 1e-13, stall = 0.0;
    static constexpr int cap_cold = 120, cap_warm = 40, polish = 2;
};
template <>
struct Tol<float> {
    static constexpr float step = 2e-6f, lens = 2e-6f, pair = 2e-5f, dup = 1e-5f, shift = 1e-6f, ambiguous = 3e-3f,
                           cubic = 1e-3f, stall = 0.81f;
    static constexpr int cap_cold = 100, cap_warm = 30, polish = 4;
};

template <typename T>
struct Eps;
template <>
struct Eps<double> {
    static constexpr double value = 1.1102230246251565e-16;  // 2^-53
};
template <>
struct Eps<float> {
    static constexpr float value = 5.9604645e-08f;  // 2^-24
};
// rounding level of a complex Horner evaluation of degree 5, in units of eps * sum |c_k||z|^k
constexpr float kNoise = 16.0f;

// flags written per (candidate, epoch)
enum : uint8_t {
    FLAG_FALLBACK = 1,     // image selection fell back to the residual ranking
    FLAG_FP64 = 2,         // MIXED: the epoch was re-solved in FP64
    FLAG_CAP = 4,          // the root iteration hit its cap
    FLAG_AMBIGUOUS = 8,    // a root's residual lay in the band between image and spurious
    FLAG_NEAR_DET = 16,    // an image has |det J| below the MIXED trigger (next to a caustic)
    FLAG_NEAR_GAP = 32     // two images are closer than the MIXED trigger
};

// ------------------------------------------------------------------------------------------
// Eq. (lensingPoly), for a lens of mass m1 at the origin and m2 at z = a:
//   zeta = z - m1/conj(z) + m2/(a - conj(z)).
// Conjugating gives conj(z) = N/D with D = z(z - a), N = conj(zeta) D + (m1 + m2) z - m1 a;
// substituting back and clearing denominators gives p(z) = (z - zeta) N M - m1 D M - m2 D N with
// M = N - a D. Expanded here in ascending powers. The paper's frame (primary at the origin) is
// (m1, m2, a) = (1, q, d); the frame centred on the secondary is (q, 1, -d) with zeta - d.
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void quintic_coefficients(cx<T> zeta, T a, T m1, T m2, cx<T> c[6]) {
    const cx<T> s = conj(zeta);
    const T m = m1 + m2;
    // N = n2 z^2 + n1 z + n0, M = k2 z^2 + k1 z + n0 (both constant terms are -m1 a)
    const cx<T> n2 = s;
    const cx<T> n1 = mk<T>(m - a * s.re, -a * s.im);
    const cx<T> k2 = mk<T>(s.re - a, s.im);
    const cx<T> k1 = mk<T>(m - a * s.re + a * a, -a * s.im);
    const T n0 = -m1 * a;
    const T m1a2 = m1 * a * a;
    // N M
    const cx<T> P4 = n2 * k2;
    const cx<T> P3 = n2 * k1 + n1 * k2;
    const cx<T> P2 = n0 * (n2 + k2) + n1 * k1;
    const cx<T> P1 = n0 * (n1 + k1);
    const T P0 = n0 * n0;
    // D M and D N with D = z^2 - a z (their z^1 terms are both m1 a^2)
    const cx<T> DM3 = k1 - a * k2, DM2 = mk<T>(n0 - a * k1.re, -a * k1.im);
    const cx<T> DN3 = n1 - a * n2, DN2 = mk<T>(n0 - a * n1.re, -a * n1.im);
    c[5] = P4;
    c[4] = P3 - zeta * P4 - m1 * k2 - m2 * n2;
    c[3] = P2 - zeta * P3 - m1 * DM3 - m2 * DN3;
    c[2] = P1 - zeta * P2 - m1 * DM2 - m2 * DN2;
    c[1] = mk<T>(-m2 * m1a2, T(0)) - zeta * P1;
    c[0] = -(P0 * zeta);
}

template <typename T>
__device__ __forceinline__ void horner2(const cx<T> c[6], cx<T> z, cx<T>& p, cx<T>& dp) {
    p = c[5];
    dp = mk<T>(T(0), T(0));
#pragma unroll
    for (int k = 4; k >= 0; --k) {
        dp = dp * z + p;
        p = p * z + c[k];
    }
}

__device__ __forceinline__ float tenth_power(float x) { return __expf(0.1f * __logf(x)); }
__device__ __forceinline__ double tenth_power(double x) { return exp(0.1 * log(x)); }

// Starting points for a cold solve: five points on a circle around the roots' centroid
// -c4/(5 c5), of radius |p(centroid)/c5|^(1/5) (the geometric mean distance of the roots from
// the centroid), turned off the real axis.
template <typename T>
__device__ __forceinline__ void cold_start(const cx<T> c[6], cx<T> z[5]) {
    const cx<T> inv5 = inv(c[5]);
    const cx<T> cg = T(-0.2) * (c[4] * inv5);
    cx<T> p, dp;
    horner2(c, cg, p, dp);
    const T r2 = norm2(p) * norm2(inv5);
    T R = (r2 > T(0) && isfinite(r2)) ? tenth_power(r2) : T(1);
    R = fmax(R, T(1e-3) * (T(1) + sqrt_(norm2(cg))));
    // cos and sin of 0.4 + 2 pi k / 5, k = 0..4
    constexpr double kc[5] = {0.9210609940028851, -0.08573535201472558, -0.9740483555854224,
                              -0.5162596384230086, 0.6549823520202719};
    constexpr double ks[5] = {0.3894183423086505, 0.9963179459464289, 0.22634001188772324,
                              -0.8564321255857609, -0.7556441745570415};
#pragma unroll
    for (int k = 0; k < 5; ++k) z[k] = cg + R * mk<T>(T(kc[k]), T(ks[k]));
}

// Aberth-Ehrlich simultaneous iteration, Gauss-Seidel sweep (each root uses the newest values
// of the others). A root stops moving once |p(z)| is at the rounding level of its Horner
// evaluation, kNoise * eps * sum_k |c_k| |z|^k (nothing finer can be resolved in T), or once its
// correction is below Tol::cubic relative. Only the roots in the bit mask `active` move; the
// others still repel them. Returns the number of sweeps, or -1 if `cap` sweeps did not converge.
// A sweep is a rolled loop that always updates z[0] and then rotates the five roots (and their
// done bits) by one place, so after five steps they are back in order: the loop body is emitted
// once instead of five times (8% faster in MIXED on the 4096 x 2000 sweep: the unrolled sweep
// stalled on instruction fetch).
template <typename T>
__device__ __forceinline__ int aberth(const cx<T> c[6], cx<T> z[5], int cap, unsigned active = 31u,
                                     T cubic = Tol<T>::cubic) {
    const T tol2 = cubic * cubic;
    T ac[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) ac[k] = sqrt_(norm2(c[k]));
    const T noise = T(kNoise) * Eps<T>::value;
    unsigned done = ~active & 31u;
    for (int it = 1; it <= cap; ++it) {
        bool all = true;
#pragma unroll 1
        for (int r = 0; r < 5; ++r) {
            if (!(done & 1u)) {
                cx<T> p, dp;
                horner2(c, z[0], p, dp);
                const T az = sqrt_(norm2(z[0]));
                T eb = ac[5];
#pragma unroll
                for (int k = 4; k >= 0; --k) eb = eb * az + ac[k];
                const T lim = noise * eb;
                if (norm2(p) <= lim * lim) {
                    done |= 1u;
                } else {
                    const cx<T> ratio = div(p, dp);
                    cx<T> S = mk<T>(T(0), T(0));
#pragma unroll
                    for (int j = 1; j < 5; ++j) S = S + inv(z[0] - z[j]);
                    cx<T> w = div(ratio, mk<T>(T(1), T(0)) - ratio * S);
                    if (!finite2(w)) w = finite2(ratio) ? ratio : mk<T>(T(0), T(0));
                    z[0] = z[0] - w;
                    const bool d0 = norm2(w) <= tol2 * norm2(z[0]);
                    done |= d0 ? 1u : 0u;
                    all = all && d0;
                }
            }
            const cx<T> z0 = z[0];
            z[0] = z[1];
            z[1] = z[2];
            z[2] = z[3];
            z[3] = z[4];
            z[4] = z0;
            done = (done >> 1) | ((done & 1u) << 4);
        }
        if (all) return it;
    }
    return -1;
}

template <typename T>
struct EpochOut {
    T A;         // sum of 1/|det J| over the images
    T min_det;   // smallest |det J| over the images
    T min_gap;   // smallest distance between two images
    T min_det_rej;  // smallest |det J| over the rejected roots that nearly solve the lens equation
                    // (relative residual below kSpurious): a pair of images that the arithmetic
                    // failed to converge sits next to the critical curve
    T min_gap_rej;  // smallest distance, relative to sqrt(1 + |z|^2), between two rejected roots with
                    // relative residuals below kSpuriousPair: an image pair just born at a fold
                    // that the iteration left as one near-double root (both roots stop at the
                    // noise level of the polynomial there)
    int sweeps;  // root-iteration sweeps spent (diagnostics)
    uint8_t flag;
};

// an epoch that MIXED re-solves in FP64: its FP32 roots (the warm start), candidate, epoch and
// the flags that triggered it
struct Deferred {
    cx<float> z[5];
    int c;
    int e;
    uint32_t why;
};

// A root of the quintic, kept either as z (origin at the primary) or, next to the secondary, as
// its offset w = z - d, so that q/(d - conj(z)) = -q/conj(w) keeps full relative precision.
template <typename T>
struct Root {
    cx<T> z, w;
    bool local;
};

template <typename T>
__device__ __forceinline__ cx<T> root_diff(const Root<T>& a, const Root<T>& b) {
    return (a.local && b.local) ? a.w - b.w : a.z - b.z;
}

// lens-equation residual f = z - 1/conj(z) + q/(d - conj(z)) - zeta and K = 1/conj(z)^2 +
// q/(d - conj(z))^2 (det J = 1 - |K|^2) at a root
template <typename T>
__device__ __forceinline__ void lens_terms(const Root<T>& r, cx<T> zeta, T d, T q, cx<T>& f, cx<T>& K, T& qterm) {
    const cx<T> ib = inv(conj(r.z));
    const cx<T> idz = r.local ? -inv(conj(r.w)) : inv(mk<T>(d - r.z.re, r.z.im));
    f = r.z - ib + q * idz - zeta;
    K = ib * ib + q * (idz * idz);
    qterm = q * sqrt_(norm2(idz));
}

// roots whose relative lens-equation residual exceeds this are spurious without a polish
constexpr float kSpurious = 0.05f;
// rejected roots with residuals below this enter the near-double-root test (min_gap_rej)
constexpr float kSpuriousPair = 0.25f;

// Spurious-root rejection (Section 2.2: substitution into Eq. (lensing)) and magnification.
// Each root gets up to `polish` Newton steps on the lens equation itself,
//   delta = (-f + K conj(f)) / (1 - |K|^2),
// fewer once a step is below the rounding level or the residual stalls (Tol::stall), and keeps
// its unpolished value if that moved it by more than half its distance to the nearest other
// root. Images: relative residual |f| / (|z| + 1/|z| + q/|d - z| + |zeta|) at
// most Tol::lens; the count must be 3 or 5, the parities (sign of det J) must sum to -1 and no
// two images may coincide; otherwise the 3 smallest residuals are taken, plus the 4th and 5th
// when both are at most Tol::pair, and the epoch is flagged.
template <typename T>
__device__ __forceinline__ EpochOut<T> select_images(const Root<T> rr[5], cx<T> zeta, T d, T q,
                                                     T* diag = nullptr) {
    T gap2[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) gap2[i] = T(INFINITY);
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i + 1; j < 5; ++j) {
            const T g = norm2(root_diff(rr[i], rr[j]));
            gap2[i] = fmin(gap2[i], g);
            gap2[j] = fmin(gap2[j], g);
        }
    const T zeta_abs = sqrt_(norm2(zeta));
    Root<T> rp[5];
    T r2[5], det[5], gp[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        gp[i] = gap2[i];
        rp[i] = rr[i];
        r2[i] = T(0);
        det[i] = T(0);
    }
    // one copy of the per-root body: the root in slot 0 is processed, every array moves down by one
    // place and the polished root and its results enter at slot 4, so after five passes rp holds
    // the polished roots at their own indices (one array serves as input and output)
#pragma unroll 1
    for (int i = 0; i < 5; ++i) {
        const Root<T> r_in = rp[0];
        Root<T> r = r_in;
        cx<T> f, K;
        T qt = T(0), f2prev = T(INFINITY);
#pragma unroll 1
        for (int s = 0; s <= Tol<T>::polish; ++s) {
            lens_terms(r, zeta, d, q, f, K, qt);
            if (s == Tol<T>::polish) break;
            if (s == 0) {
                const T az2 = norm2(r.z);
                const T sc = sqrt_(az2) + rsqrt_(az2) + qt + zeta_abs;
                if (norm2(f) > T(kSpurious) * T(kSpurious) * sc * sc) break;
            }
            if (Tol<T>::stall > T(0)) {
                const T f2 = norm2(f);
                if (f2 >= T(Tol<T>::stall) * f2prev) break;
                f2prev = f2;
            }
            const T dj = T(1) - norm2(K);
            if (!(fabs(dj) >= T(1e-30))) break;
            const cx<T> num = (K * conj(f)) - f;
            const cx<T> delta = rcp(fabs(dj)) * (dj < T(0) ? -num : num);
            if (!finite2(delta)) break;
            const T ref2 = r.local ? norm2(r.w) : norm2(r.z);
            if (norm2(delta) <= T(4) * Eps<T>::value * Eps<T>::value * ref2) break;
            if (r.local) {
                r.w = r.w + delta;
                r.z = mk<T>(d, T(0)) + r.w;
            } else {
                r.z = r.z + delta;
            }
        }
        const cx<T> moved = r.local ? r.w - r_in.w : r.z - r_in.z;
        if (!(norm2(moved) <= T(0.25) * gp[0]) || !finite2(r.z)) {
            r = r_in;
            lens_terms(r, zeta, d, q, f, K, qt);
        }
        const T az2 = norm2(r.z);
        const T scale = sqrt_(az2) + rsqrt_(az2) + qt + zeta_abs;
        const T q2 = norm2(f) / (scale * scale);
        const T r2v = isfinite(q2) ? q2 : T(INFINITY);
        const T detv = T(1) - norm2(K);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            gp[k] = gp[k + 1];
            rp[k] = rp[k + 1];
            r2[k] = r2[k + 1];
            det[k] = det[k + 1];
        }
        rp[4] = r;
        r2[4] = r2v;
        det[4] = detv;
    }
    const T lens2 = Tol<T>::lens * Tol<T>::lens;
    bool acc[5];
    int count = 0, parity = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        acc[i] = r2[i] <= lens2;
        count += acc[i];
        parity += acc[i] ? (det[i] > T(0) ? 1 : (det[i] < T(0) ? -1 : 0)) : 0;
    }
    bool dup = false;
    T min_gap2 = T(INFINITY);
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i + 1; j < 5; ++j) {
            if (acc[i] && acc[j]) {
                const T g = norm2(root_diff(rp[i], rp[j]));
                const T lim = Tol<T>::dup * (T(1) + sqrt_(norm2(rp[i].z)));
                dup = dup || (g <= lim * lim);
                min_gap2 = fmin(min_gap2, g);
            }
        }
    const bool ok = (count == 3 || count == 5) && parity == -1 && !dup;
    EpochOut<T> out;
    out.flag = 0;
    if (!ok) {
        // stable ranks of the residuals
        int rank[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            int r = 0;
#pragma unroll
            for (int j = 0; j < 5; ++j) r += (r2[j] < r2[i]) || (r2[j] == r2[i] && j < i);
            rank[i] = r;
        }
        T r3 = T(0), r4 = T(0);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if (rank[i] == 3) r3 = r2[i];
            if (rank[i] == 4) r4 = r2[i];
        }
        const T pair2 = Tol<T>::pair * Tol<T>::pair;
        const bool five = (r3 <= pair2) && (r4 <= pair2);
        min_gap2 = T(INFINITY);
#pragma unroll
        for (int i = 0; i < 5; ++i) acc[i] = rank[i] < 3 || five;
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = i + 1; j < 5; ++j)
                if (acc[i] && acc[j]) min_gap2 = fmin(min_gap2, norm2(root_diff(rp[i], rp[j])));
        out.flag = FLAG_FALLBACK;
    }
    if (diag) {  // per root: squared relative residual, det J, accepted, moved-from-raw
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            diag[4 * i] = r2[i];
            diag[4 * i + 1] = det[i];
            diag[4 * i + 2] = acc[i];
            diag[4 * i + 3] = norm2(rp[i].z - rr[i].z);
        }
    }
    T A = T(0), md = T(INFINITY), rej = T(INFINITY);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        if (acc[i]) {
            const T ad = fabs(det[i]);
            A += rcp(ad);
            md = fmin(md, ad);
        }
        rej = fmin(rej, r2[i] > lens2 ? r2[i] : T(INFINITY));
    }
    if (rej < T(Tol<T>::ambiguous) * T(Tol<T>::ambiguous)) out.flag |= FLAG_AMBIGUOUS;
    T mdr = T(INFINITY);
#pragma unroll
    for (int i = 0; i < 5; ++i)
        if (!acc[i] && r2[i] <= T(kSpurious) * T(kSpurious)) mdr = fmin(mdr, fabs(det[i]));
    out.min_det_rej = mdr;
    T mgr = T(INFINITY);
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i + 1; j < 5; ++j)
            if (!acc[i] && !acc[j] && r2[i] <= T(kSpuriousPair) * T(kSpuriousPair) &&
                r2[j] <= T(kSpuriousPair) * T(kSpuriousPair))
                mgr = fmin(mgr, norm2(root_diff(rp[i], rp[j])) / (T(1) + norm2(rp[i].z)));
    out.min_gap_rej = sqrt_(mgr);
    out.A = A;
    out.min_det = md;
    out.min_gap = sqrt_(min_gap2);
    return out;
}

// When two or more roots lie closer to the secondary than max(kLocalFrac d, min(sqrt q,
// kLocalCap d)), they are refined on the quintic written in the secondary's frame (masses (q, 1)
// at (0, -d), source zeta - d), whose low-order coefficients carry q with full relative
// precision: in the primary's frame a cluster of roots next to the secondary (a few q apart for a
// small q) is not resolved in FP32. The images of a source at the secondary's (planetary)
// caustic spread over about the secondary's Einstein radius sqrt(q), which exceeds kLocalFrac d
// when d is small; left in the primary's frame such a cluster stops at the noise level of the
// Horner evaluation with two roots far from the images.
constexpr float kLocalFrac = 0.1f;
constexpr float kLocalCap = 0.3f;

// One epoch in arithmetic T: quintic, roots (warm from the previous epoch's roots when `warm`),
// images, magnification. Updates z (the polynomial roots) and `warm`. The root iteration has a
// single call site (a short job list: warm solve, cold retry, refinement next to the secondary)
// so that the unrolled solver is emitted once per arithmetic.
// `cubic` overrides the Aberth stop rule: the MIXED re-solve starts from FP32 roots (relative
// error ~1e-6), so one cubic step already lands far below FP64 rounding.
template <typename T>
__device__ __forceinline__ EpochOut<T> solve_epoch(cx<T> zeta, T d, T q, cx<T> z[5], bool& warm,
                                                   T* diag = nullptr, T cubic = Tol<T>::cubic) {
    uint8_t extra = 0;
    if (norm2(zeta) < Tol<T>::shift * Tol<T>::shift ||
        norm2(mk<T>(zeta.re - d, zeta.im)) < Tol<T>::shift * Tol<T>::shift) {
        zeta.re += Tol<T>::shift;
        extra |= FLAG_FALLBACK;
    }
    constexpr bool kTwoFrames = sizeof(T) == sizeof(float);
    const cx<T> dd = mk<T>(d, T(0));
    cx<T> c[6], wl[5];
    int it = -1, sweeps = 0;
    unsigned local = 0;
    // job 0: primary frame, warm if possible; job 1: primary frame, cold (only when job 0 was a
    // warm solve that failed); job 2: secondary frame for the roots next to the secondary
    int job = 0;
    bool cold = !warm;
#pragma unroll 1
    while (job < 3) {
        unsigned mask = 31u;
        int cap;
        if (job < 2) {
            quintic_coefficients(zeta, d, T(1), q, c);
            if (cold) cold_start(c, z);
            cap = cold ? Tol<T>::cap_cold : Tol<T>::cap_warm;
        } else {
            quintic_coefficients(mk<T>(zeta.re - d, zeta.im), -d, q, T(1), c);
#pragma unroll
            for (int i = 0; i < 5; ++i) z[i] = z[i] - dd;
            mask = local;
            cap = Tol<T>::cap_warm;
        }
        const int r = aberth(c, z, cap, mask, cold ? Tol<T>::cubic : cubic);
        sweeps += r < 0 ? cap : r;
        if (job == 2) {
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                wl[i] = z[i];  // offsets from the secondary, at full relative precision
                z[i] = z[i] + dd;
            }
            if (r < 0) extra |= FLAG_CAP;
            break;
        }
        bool fin = true;
#pragma unroll
        for (int i = 0; i < 5; ++i) fin = fin && finite2(z[i]);
        it = fin ? r : -1;
        if (it < 0 && !cold) {  // retry from a cold start
            cold = true;
            job = 1;
            continue;
        }
        if (!kTwoFrames) break;
        const T rl = fmax(T(kLocalFrac) * d, fmin(sqrt_(q), T(kLocalCap) * d));
        const T lim2 = rl * rl;
        local = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) local |= (norm2(z[i] - dd) < lim2 ? 1u : 0u) << i;
        // a lone root next to the secondary is resolved in the primary frame; two or more are
        // a cluster that only the secondary's frame resolves in FP32
        if (__popc(local) < 2) {
            local = 0;
            break;
        }
        job = 2;
    }
    warm = it >= 0;
    Root<T> rr[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        rr[i].local = (local >> i) & 1u;
        rr[i].z = z[i];
        rr[i].w = rr[i].local ? wl[i] : z[i] - dd;
    }
    EpochOut<T> o = select_images(rr, zeta, d, q, diag);
    o.flag |= extra | (it < 0 ? FLAG_CAP : 0);
    o.sweeps = sweeps;
    return o;
}

// Per-candidate constants of the trajectory of Eq. (sourcePos): zeta = tau v + u0 w with
// w = e^{i alpha}, v = (sin alpha, -cos alpha), tau = (t - t0)/tE.
struct Cand {
    double t0, inv_tE, u0, sa, ca, d, q;
};

__device__ __forceinline__ Cand load_cand(const double* __restrict__ theta, int c) {
    Cand k;
    const double* r = theta + 6 * (size_t)c;
    k.t0 = r[0];
    k.inv_tE = 1.0 / r[1];
    k.u0 = r[2];
    sincos(r[3], &k.sa, &k.ca);
    k.d = r[4];
    k.q = r[5];
    return k;
}

__device__ __forceinline__ cx<double> zeta64(const Cand& k, double t) {
    const double tau = (t - k.t0) * k.inv_tE;
    return mk<double>(tau * k.sa + k.u0 * k.ca, -tau * k.ca + k.u0 * k.sa);
}

// (ah + al) - (bh + bl) rounded once to float: Knuth's two-sum on the high parts keeps the
// difference of two doubles accurate in FP32 even when t - t0 is small.
__device__ __forceinline__ float diff_ff(float ah, float al, float bh, float bl) {
    const float s = ah - bh;
    const float v = s - ah;
    const float e = (ah - (s - v)) + (-bh - v);
    return s + (e + (al - bl));
}

// MIXED: an epoch solved in FP32 is re-solved in FP64 when an image, or a rejected root that
// nearly solves the lens equation, has |det J| below kMixedDetTrigger (next to a caustic FP32
// loses accuracy, and an image pair it failed to converge sits next to the critical curve), when
// two images are closer than kMixedGapTrigger, when two rejected roots with residuals below
// kSpuriousPair nearly coincide (kMixedRejGapTrigger, relative to sqrt(1 + |z|^2): a pair just
// born at a fold, left as a near-double root), or when the FP32 image selection was flagged
// (fallback, cap, ambiguous).
constexpr float kMixedDetTrigger = 3e-2f;
constexpr float kMixedGapTrigger = 1e-4f;
constexpr float kMixedRejGapTrigger = 3e-2f;

template <typename T>
__device__ __forceinline__ uint8_t mixed_trigger_flags(const EpochOut<T>& o) {
    return (uint8_t)(o.flag | (fmin(o.min_det, o.min_det_rej) < T(kMixedDetTrigger) ? FLAG_NEAR_DET : 0) |
                     ((o.min_gap < T(kMixedGapTrigger) || o.min_gap_rej < T(kMixedRejGapTrigger)) ? FLAG_NEAR_GAP
                                                                                                    : 0));
}

}  // namespace sblm
