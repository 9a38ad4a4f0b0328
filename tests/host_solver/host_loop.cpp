// Host build of the device's per-candidate epoch loop (the FP32 branch of eval_run plus an FP64
// solve of every epoch), compiled from host copies of the library's solver headers. Test
// infrastructure: it checks the solver's logic (root iteration, image selection, the MIXED
// re-solve triggers) on the CPU.
//
// Binary input: int32 n_rows, n_ep, seg; double t[n_ep]; double theta[n_rows][6].
// Binary output: double A32[n_rows][n_ep]; uint8 flags[n_rows][n_ep] (with the MIXED trigger
// bits); double A64[n_rows][n_ep]. Each run of `seg` epochs starts cold, as one device thread's
// segment does.
#include <cstdio>
#include <vector>

#include "forward.cuh"


using namespace sblm;

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
    std::vector<double> A32((size_t)n_rows * n_ep), A64((size_t)n_rows * n_ep);
    std::vector<unsigned char> fl((size_t)n_rows * n_ep);
    for (int r = 0; r < n_rows; ++r) {
        const double* p = &th[6 * (size_t)r];
        const double t0 = p[0], inv_tE = 1.0 / p[1], u0 = p[2], d = p[4], q = p[5];
        double sa, ca;
        sincos(p[3], &sa, &ca);
        const float t0h = (float)t0, t0l = (float)(t0 - (double)t0h);
        const float itE = (float)inv_tE, fsa = (float)sa, fca = (float)ca, fu0 = (float)u0;
        cx<float> z[5];
        cx<double> zz[5];
        bool warm = false, warm64 = false;
        for (int e = 0; e < n_ep; ++e) {
            if (e % seg == 0) warm = warm64 = false;
            const float thi = (float)t[e], tlo = (float)(t[e] - (double)thi);
            const float tau = diff_ff(thi, tlo, t0h, t0l) * itE;
            const cx<float> zeta = mk<float>(tau * fsa + fu0 * fca, -tau * fca + fu0 * fsa);
            EpochOut<float> o = solve_epoch<float>(zeta, (float)d, (float)q, z, warm);
            o.flag = mixed_trigger_flags(o);
            A32[(size_t)r * n_ep + e] = o.A;
            fl[(size_t)r * n_ep + e] = o.flag;
            const double tau64 = (t[e] - t0) * inv_tE;
            const cx<double> zeta64 = mk<double>(tau64 * sa + u0 * ca, -tau64 * ca + u0 * sa);
            A64[(size_t)r * n_ep + e] = solve_epoch<double>(zeta64, d, q, zz, warm64).A;
        }
    }
    fwrite(A32.data(), 8, A32.size(), fo);
    fwrite(fl.data(), 1, fl.size(), fo);
    fwrite(A64.data(), 8, A64.size(), fo);
    return fclose(fo) == 0 ? 0 : 1;
}
