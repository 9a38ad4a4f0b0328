// Algorithmic operation count of the device's per-candidate epoch loop (eval_run, MIXED), from host
// copies of the library's solver headers instantiated with counting types (count_types.h).
// Test and measurement infrastructure: the FP32 and FP64 arithmetic per magnification that the
// roofline of the forward kernel is computed from.
//
// Binary input: int32 n_rows, n_ep, seg; double t[n_ep]; double F[n_ep]; double w[n_ep] (1/sigma);
// double theta[n_rows][6]. Runs of `seg` epochs start cold, as one device thread's segment does.
// With "--fp64" the FP64 mode's loop is counted instead (every epoch solved in FP64).
// Text output: epochs, FP32 operations, FP64 operations, epochs re-solved in FP64.
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "forward.cuh"
#include "count_types.h"

using namespace sblm;

// (ah + al) - (bh + bl) with Knuth's two-sum, as diff_ff in the library, in counted arithmetic
static CF diff_ff_c(CF ah, CF al, CF bh, CF bl) {
    const CF s = ah - bh;
    const CF v = s - ah;
    const CF e = (ah - (s - v)) + (-bh - v);
    return s + (e + (al - bl));
}

// "--pins": the counts of one quintic build and one Horner evaluation with derivative, for a
// test to compare with hand counts of the formulas
static int pins() {
    const cx<CF> zeta = mk<CF>(CF(0.3f), CF(-0.2f));
    cx<CF> c[6], p, dp;
    g_tally = FlopTally{};
    quintic_coefficients<CF>(zeta, CF(1.1f), CF(1.0f), CF(0.01f), c);
    const unsigned long long nq = g_tally.f32;
    g_tally = FlopTally{};
    horner2<CF>(c, mk<CF>(CF(0.5f), CF(0.5f)), p, dp);
    printf("%llu %llu\n", nq, g_tally.f32);
    return 0;
}

int main(int argc, char** argv) {
    if (argc == 2 && std::strcmp(argv[1], "--pins") == 0) return pins();
    // "--fp64 <input>": the FP64 mode's epoch loop instead of MIXED
    const bool fp64 = argc == 3 && std::strcmp(argv[1], "--fp64") == 0;
    if (argc != 2 && !fp64) return 2;
    FILE* fi = fopen(argv[argc - 1], "rb");
    if (!fi) return 2;
    int hdr[3];
    if (fread(hdr, sizeof(int), 3, fi) != 3) return 1;
    const int n_rows = hdr[0], n_ep = hdr[1], seg = hdr[2];
    std::vector<double> t(n_ep), F(n_ep), w(n_ep), th(6 * (size_t)n_rows);
    if (fread(t.data(), 8, n_ep, fi) != (size_t)n_ep) return 1;
    if (fread(F.data(), 8, n_ep, fi) != (size_t)n_ep) return 1;
    if (fread(w.data(), 8, n_ep, fi) != (size_t)n_ep) return 1;
    if (fread(th.data(), 8, th.size(), fi) != th.size()) return 1;
    unsigned long long deferred = 0;
    for (int r = 0; fp64 && r < n_rows; ++r) {
        const double* p = &th[6 * (size_t)r];
        const double t0 = p[0], inv_tE = 1.0 / p[1], u0 = p[2], d = p[4], q = p[5];
        double sa, ca;
        sincos(p[3], &sa, &ca);
        cx<CD> z[5];
        bool warm = false;
        for (int e = 0; e < n_ep; ++e) {
            if (e % seg == 0) warm = false;
            const CD tau = (CD(t[e]) - CD(t0)) * CD(inv_tE);
            const cx<CD> zeta = mk<CD>(tau * CD(sa) + CD(u0) * CD(ca), -tau * CD(ca) + CD(u0) * CD(sa));
            const EpochOut<CD> o = solve_epoch<CD>(zeta, CD(d), CD(q), z, warm);
            const CD rr = (CD(F[e]) - o.A) * CD(w[e]);
            (void)(rr * rr + CD(0.0));
        }
    }
    for (int r = 0; !fp64 && r < n_rows; ++r) {
        // the candidate's decode (once per thread group on the device) is not counted per epoch
        const double* p = &th[6 * (size_t)r];
        const double t0 = p[0], inv_tE = 1.0 / p[1], u0 = p[2], d = p[4], q = p[5];
        double sa, ca;
        sincos(p[3], &sa, &ca);
        const CF t0h = (float)t0, t0l = (float)(t0 - (double)(float)t0);
        const CF itE = (float)inv_tE, fsa = (float)sa, fca = (float)ca, fu0 = (float)u0;
        cx<CF> z[5];
        bool warm = false;
        for (int e = 0; e < n_ep; ++e) {
            if (e % seg == 0) warm = false;
            const CF thi = (float)t[e], tlo = (float)(t[e] - (double)(float)t[e]);
            const CF tau = diff_ff_c(thi, tlo, t0h, t0l) * itE;
            const cx<CF> zeta = mk<CF>(tau * fsa + fu0 * fca, -tau * fca + fu0 * fsa);
            EpochOut<CF> o = solve_epoch<CF>(zeta, CF((float)d), CF((float)q), z, warm);
            const uint8_t fl = mixed_trigger_flags(o);
            if (fl == 0) {
                const CF rr = (CF((float)F[e]) - o.A) * CF((float)w[e]);  // FP32 residual
                const CD r2 = CD((double)rr.v) * CD((double)rr.v);       // squared and summed in FP64
                (void)(r2 + CD(0.0));
            } else {  // the FP64 re-solve, warm-started from the FP32 roots
                ++deferred;
                cx<CD> zz[5];
                for (int i = 0; i < 5; ++i) zz[i] = mk<CD>(CD((double)z[i].re.v), CD((double)z[i].im.v));
                const CD tau64 = (CD(t[e]) - CD(t0)) * CD(inv_tE);
                const cx<CD> zeta64 = mk<CD>(tau64 * CD(sa) + CD(u0) * CD(ca), -tau64 * CD(ca) + CD(u0) * CD(sa));
                bool w2 = true;
                const EpochOut<CD> o2 = solve_epoch<CD>(zeta64, CD(d), CD(q), zz, w2, nullptr, CD(1e-6));
                const CD rr = (CD(F[e]) - o2.A) * CD(w[e]);
                (void)(rr * rr + CD(0.0));
            }
        }
    }
    printf("%llu %llu %llu %llu\n", (unsigned long long)n_rows * n_ep, g_tally.f32, g_tally.f64, deferred);
    return 0;
}
