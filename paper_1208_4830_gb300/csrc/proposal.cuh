// proposal.cuh -- one seed row of the EA drawn from the proposal network's Gaussian outputs, shared
// by the sampling kernel and the batched fitter (which draws its seeded rows for the first
// population only; restarts are the paper's random initialisation).
#pragma once

#include "common.cuh"
#include "forward_launch.cuh"

namespace sblm {

constexpr uint64_t kOpCnnSample = 10;  // Philox operator id of seed rows (counter word 1)

// Row r of lightcurve lc in draw round `round` (0: the first population, k: the k-th restart):
// y = mu + exp(s / 2) n with n six Box-Muller deviates of Philox blocks (round, 10, r, 0..1) under
// key (seed, lc); row 0 takes n = 0 (the network's mean). y is mapped from window units
// (c, h) to physical parameters and encoded as genes over b, clamped to [0, 1] (non-finite: 0.5).
static __device__ __noinline__ void proposal_row(const float* __restrict__ out12, double c, double h, const Bounds& b,
                                          uint64_t seed, uint64_t lc, uint64_t r, uint64_t round, double* g) {
    constexpr double kTwoPi = 6.283185307179586;
    double n[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (r > 0) {
        const u64x4 ra = philox4x64(round, kOpCnnSample, r, 0, seed, lc);
        const u64x4 rb = philox4x64(round, kOpCnnSample, r, 1, seed, lc);
        const uint64_t w[6] = {ra.x[0], ra.x[1], ra.x[2], ra.x[3], rb.x[0], rb.x[1]};
        for (int k = 0; k < 6; k += 2) {
            const double rr = sqrt(-2.0 * log(1.0 - u01(w[k])));
            const double a = kTwoPi * u01(w[k + 1]);
            n[k] = rr * cos(a);
            n[k + 1] = rr * sin(a);
        }
    }
    double y[6];
    for (int k = 0; k < 6; ++k) y[k] = (double)out12[k] + exp(0.5 * (double)out12[6 + k]) * n[k];
    double a = kTwoPi * y[3];
    a = a - kTwoPi * floor(a / kTwoPi);
    const double v[6] = {c + h * y[0], h * exp(y[1]), y[2], a, exp(y[4]), y[5]};
    for (int k = 0; k < 6; ++k) {
        const double e = (v[k] - b.lo[k]) / (b.hi[k] - b.lo[k]);
        g[k] = isfinite(e) ? fmin(1.0, fmax(0.0, e)) : 0.5;
    }
}

}  // namespace sblm
