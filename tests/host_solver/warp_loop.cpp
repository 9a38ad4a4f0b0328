// Per-(row, epoch) work record of the device's FP32 epoch loop (eval_run's FP32 branch with the MIXED
// triggers), from host copies of the library's solver headers instantiated with counting types and
// with counters planted at the loop bodies that lanes of a warp execute in lockstep (warp_replay.py
// plants them). Measurement infrastructure: the input of the warp-lockstep replay.
//
// Binary input: int32 n_rows, n_ep, seg; double t[n_ep]; double theta[n_rows][6]. Runs of `seg`
// epochs start cold, as one device thread's run does.
// Binary output: int32 rec[n_rows][n_ep][6] = FP32 operations, passes of the Aberth loop body,
// passes that updated a root, polish evaluations of the five root slots (3 bits per slot),
// root-finding jobs, MIXED trigger bits.
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "forward.cuh"
#include "count_types.h"

using namespace sblm;

static CF diff_ff_c(CF ah, CF al, CF bh, CF bl) {
    const CF s = ah - bh;
    const CF v = s - ah;
    const CF e = (ah - (s - v)) + (-bh - v);
    return s + (e + (al - bl));
}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* fi = fopen(argv[1], "rb");
    FILE* fo = fopen(argv[2], "wb");
    if (!fi || !fo) return 2;
    int hdr[3];
    if (fread(hdr, sizeof(int), 3, fi) != 3) return 1;
    const int n_rows = hdr[0], n_ep = hdr[1], seg = hdr[2];
    std::vector<double> t(n_ep), th(6 * (size_t)n_rows);
    if (fread(t.data(), 8, n_ep, fi) != (size_t)n_ep) return 1;
    if (fread(th.data(), 8, th.size(), fi) != th.size()) return 1;
    std::vector<int> rec((size_t)n_rows * n_ep * 6);
    for (int r = 0; r < n_rows; ++r) {
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
            g_passes = g_updates = g_polish = g_jobs = 0;
            const unsigned long long f0 = g_tally.f32;
            const CF thi = (float)t[e], tlo = (float)(t[e] - (double)(float)t[e]);
            const CF tau = diff_ff_c(thi, tlo, t0h, t0l) * itE;
            const cx<CF> zeta = mk<CF>(tau * fsa + fu0 * fca, -tau * fca + fu0 * fsa);
            const EpochOut<CF> o = solve_epoch<CF>(zeta, CF((float)d), CF((float)q), z, warm);
            int* R = &rec[((size_t)r * n_ep + e) * 6];
            R[0] = (int)(g_tally.f32 - f0);
            R[1] = g_passes;
            R[2] = g_updates;
            R[3] = g_polish;
            R[4] = g_jobs;
            R[5] = mixed_trigger_flags(o);
        }
    }
    fwrite(rec.data(), 4, rec.size(), fo);
    return fclose(fo) == 0 ? 0 : 1;
}
