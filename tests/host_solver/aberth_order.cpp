// The library's Aberth iteration (forward.cuh: aberth, one copy of the per-root body that always
// updates z[0] and then turns the root array by one place, so that a sweep is five turns) against
// the textbook form of the same Gauss-Seidel iteration written here with plain indexing: sweeps over
// roots 0..4 that skip the roots already done, ending after the first sweep in which every visited
// root finished, or failing after `cap` sweeps. Both take the same updates in the same order, so
// with contraction off the roots and the returned sweep counts must agree bit for bit. Test
// infrastructure.
//
// Output: cases, mismatches, cases that hit the cap, cases with a partial active mask.
#include <cstdio>
#include <cstring>
#include <random>

#include "forward.cuh"

using namespace sblm;

template <typename T>
static int aberth_sweeps(const cx<T> c[6], cx<T> z[5], int cap, unsigned active, T cubic) {
    const T tol2 = cubic * cubic;
    T ac[6];
    for (int k = 0; k < 6; ++k) ac[k] = sqrt_(norm2(c[k]));
    const T noise = T(kNoise) * Eps<T>::value;
    unsigned done = ~active & 31u;
    for (int it = 1; it <= cap; ++it) {
        bool all = true;
        for (int i = 0; i < 5; ++i) {
            if ((done >> i) & 1u) continue;
            cx<T> p, dp;
            horner2(c, z[i], p, dp);
            const T az = sqrt_(norm2(z[i]));
            T eb = ac[5];
            for (int k = 4; k >= 0; --k) eb = eb * az + ac[k];
            const T lim = noise * eb;
            if (norm2(p) <= lim * lim) {
                done |= 1u << i;
                continue;
            }
            const cx<T> ratio = div(p, dp);
            cx<T> S = mk<T>(T(0), T(0));
            for (int j = 1; j < 5; ++j) S = S + inv(z[i] - z[(i + j) % 5]);
            cx<T> w = div(ratio, mk<T>(T(1), T(0)) - ratio * S);
            if (!finite2(w)) w = finite2(ratio) ? ratio : mk<T>(T(0), T(0));
            z[i] = z[i] - w;
            const bool d0 = norm2(w) <= tol2 * norm2(z[i]);
            if (d0) done |= 1u << i;
            all = all && d0;
        }
        if (all) return it;
    }
    return -1;
}

template <typename T>
static void run(std::mt19937_64& g, int n, long& cases, long& bad, long& capped, long& masked) {
    std::uniform_real_distribution<double> U(0.0, 1.0);
    for (int k = 0; k < n; ++k) {
        const T d = T(0.3 * std::exp(U(g) * std::log(10.0)));
        const T q = T(std::pow(10.0, -4.0 * U(g)));
        const cx<T> zeta = mk<T>(T(4.0 * U(g) - 2.0), T(4.0 * U(g) - 2.0));
        cx<T> c[6], z0[5];
        quintic_coefficients(zeta, d, T(1), q, c);
        cold_start(c, z0);
        // a warm start: the roots of a nearby source position
        if (U(g) < 0.5) {
            cx<T> c2[6];
            quintic_coefficients(mk<T>(zeta.re + T(0.05), zeta.im), d, T(1), q, c2);
            aberth_sweeps(c2, z0, 200, 31u, Tol<T>::cubic);
        }
        const int cap = U(g) < 0.3 ? 1 + (int)(3 * U(g)) : 100;
        unsigned active = 31u;
        if (U(g) < 0.3) {
            active = 1u + (unsigned)(30.0 * U(g));
            ++masked;
        }
        cx<T> za[5], zb[5];
        std::memcpy(za, z0, sizeof za);
        std::memcpy(zb, z0, sizeof zb);
        const int ra = aberth(c, za, cap, active, Tol<T>::cubic);
        const int rb = aberth_sweeps(c, zb, cap, active, Tol<T>::cubic);
        ++cases;
        capped += rb < 0;
        if (ra != rb || std::memcmp(za, zb, sizeof za) != 0) ++bad;
    }
}

int main() {
    std::mt19937_64 g(12345);
    long cases = 0, bad = 0, capped = 0, masked = 0;
    run<float>(g, 20000, cases, bad, capped, masked);
    run<double>(g, 20000, cases, bad, capped, masked);
    printf("%ld %ld %ld %ld\n", cases, bad, capped, masked);
    return 0;
}
