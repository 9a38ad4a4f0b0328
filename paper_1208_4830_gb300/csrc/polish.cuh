// polish.cuh -- the amoeba fine-tuning of the fittest EA solution (Section 4.1: the EA "with
// amoeba"): a downhill-simplex (Nelder-Mead) search in the encoded genes, run by one block.
//
// Every thread of the block runs the same simplex arithmetic on its own copy of the simplex, so
// control flow stays uniform; each objective value is one block-wide chi^2 of a single candidate
// (the block's threads split the lightcurve's epochs, MIXED re-solves go through the block's
// queue, and a fixed-order reduction broadcasts the value to every thread).
//
// Simplex rules (Lagarias, Reeds, Wright & Wright 1998, standard coefficients): reflection 1,
// expansion 2, contraction 1/2 (outside or inside), shrink 1/2 towards the best vertex; trial
// points are clamped to the gene box [0, 1]^6. The start simplex is x0 and x0 + delta e_j
// (- delta where that would leave the box). When the simplex has collapsed (every vertex within
// 1e-9 of the best in every gene) it is rebuilt around the best vertex; the search stops once
// `maxfev` objective values have been taken (a step in progress may take up to 6 more).
#pragma once

#include "blend.cuh"
#include "forward_run.cuh"

namespace sblm {

constexpr int kPolishN = SBLM_NPAR;
constexpr double kPolishDelta = 0.03;
constexpr double kPolishCollapse = 1e-9;

// sum over the block in a fixed order; every thread gets the value (s_red: 33 doubles)
__device__ __forceinline__ double block_sum_bcast(double v, double* s_red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) s_red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += s_red[w];
        s_red[32] = s;
    }
    __syncthreads();
    const double r = s_red[32];
    __syncthreads();
    return r;
}

// flux and weight 1/sigma of staged epoch e
template <int MODE>
__device__ __forceinline__ void polish_fw(const LCView& v, int e, double& F, double& w) {
    if (MODE == SBLM_FP64) {
        F = v.s_f[e];
        w = v.s_w[e];
    } else {
        const float4 ep = v.s_ep[e];
        F = ep.z;
        w = ep.w;
    }
}

// chi^2 of the candidate encoded by genes g (identical in every thread), all threads of the block;
// with A_row (n_ep doubles of scratch) the chi^2 of the blended model with f profiled out.
// MIXED: every epoch's term goes to term_row (n_ep doubles of scratch), the queued epochs are
// re-solved by the whole block from the FP64 data, and the row is summed in a fixed order, so the
// value does not depend on scheduling.
template <int MODE>
__device__ double block_chi2(const double* g, const Bounds& b, const LCView& view, int n_ep, const DeferSink& sink,
                             double* term_row, double* s_red, double* A_row, double f_min) {
    const Cand k = candidate<true>(g, b, 0);
    const int seg = (n_ep + blockDim.x - 1) / blockDim.x;
    const int e0 = min(n_ep, (int)threadIdx.x * seg), e1 = min(n_ep, e0 + seg);
    if (MODE == SBLM_MIXED) {
        if (threadIdx.x == 0) *sink.queue_count = 0;
        __syncthreads();
    }
    double chi = eval_run<MODE, true, true>(k, true, 0, e0, e1, seg, view, A_row, nullptr, sink, term_row);
    if constexpr (MODE == SBLM_MIXED) {
        __syncthreads();
        const unsigned n = min(*sink.queue_count, sink.queue_cap);
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
            const Deferred q = sink.queue[i];
            term_row[q.e] = resolve_fp64(q.z, q.why, &k, view.t[q.e], view.flux[q.e], 1.0 / view.sigma[q.e], A_row,
                                         nullptr, q.e, true);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < n_ep; e += blockDim.x) chi += term_row[e];
    }
    if (A_row) {  // Section 4.4: f A + (1 - f) with f profiled out
        __syncthreads();
        double s_ab = 0.0, s_aa = 0.0;
        for (int e = threadIdx.x; e < n_ep; e += blockDim.x) {
            double F, w;
            polish_fw<MODE>(view, e, F, w);
            const double ww = w * w, aa = A_row[e] - 1.0;
            s_ab += ww * aa * (F - 1.0);
            s_aa += ww * aa * aa;
        }
        s_ab = block_sum_bcast(s_ab, s_red);
        s_aa = block_sum_bcast(s_aa, s_red);
        const double f = blend_f(s_ab, s_aa, f_min);
        chi = 0.0;
        for (int e = threadIdx.x; e < n_ep; e += blockDim.x) {
            double F, w;
            polish_fw<MODE>(view, e, F, w);
            const double r = (F - 1.0) - f * (A_row[e] - 1.0);
            chi += w * w * r * r;
        }
    }
    const double s = block_sum_bcast(chi, s_red);
    __syncthreads();  // A_row is rewritten by the next evaluation
    return isfinite(s) ? s : INFINITY;
}

__device__ __forceinline__ double clamp01(double v) { return fmin(1.0, fmax(0.0, v)); }

// Downhill simplex from (x0, f0) with at most about maxfev objective values; on return x0, f0
// hold the best vertex found (never worse than the start).
template <int MODE>
__device__ __noinline__ void block_nelder_mead(double* x0, double* f0, int maxfev, const Bounds& b, const LCView& view,
                                               int n_ep, const DeferSink& sink, double* term_row, double* s_red,
                                               double* A_row, double f_min) {
    constexpr int n = kPolishN;
    double x[n + 1][n], f[n + 1];
    double xb[n], xr[n], xt[n];
    for (int j = 0; j < n; ++j) x[0][j] = x0[j];
    f[0] = *f0;
    if (!isfinite(f[0])) f[0] = block_chi2<MODE>(x[0], b, view, n_ep, sink, term_row, s_red, A_row, f_min);
    int fev = 0;
    bool build = true;
    while (fev < maxfev) {
        if (build) {  // simplex x0 + delta e_k around the best vertex
            for (int k = 0; k < n; ++k) {
                for (int j = 0; j < n; ++j) x[k + 1][j] = x[0][j];
                x[k + 1][k] = x[0][k] + (x[0][k] + kPolishDelta <= 1.0 ? kPolishDelta : -kPolishDelta);
                f[k + 1] = block_chi2<MODE>(x[k + 1], b, view, n_ep, sink, term_row, s_red, A_row, f_min);
            }
            fev += n;
            build = false;
        }
        // order the vertices by chi^2 (stable insertion sort)
        for (int i = 1; i <= n; ++i)
            for (int k = i; k > 0 && f[k] < f[k - 1]; --k) {
                const double tf = f[k];
                f[k] = f[k - 1];
                f[k - 1] = tf;
                for (int j = 0; j < n; ++j) {
                    const double tx = x[k][j];
                    x[k][j] = x[k - 1][j];
                    x[k - 1][j] = tx;
                }
            }
        double spread = 0.0;
        for (int k = 1; k <= n; ++k)
            for (int j = 0; j < n; ++j) spread = fmax(spread, fabs(x[k][j] - x[0][j]));
        if (spread <= kPolishCollapse) {
            if (fev + n > maxfev) break;
            build = true;
            continue;
        }
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s = __dadd_rn(s, x[k][j]);
            xb[j] = __ddiv_rn(s, (double)n);
        }
        for (int j = 0; j < n; ++j) xr[j] = clamp01(__dsub_rn(__dmul_rn(2.0, xb[j]), x[n][j]));
        const double fr = block_chi2<MODE>(xr, b, view, n_ep, sink, term_row, s_red, A_row, f_min);
        ++fev;
        bool shrink = false;
        if (fr < f[0]) {  // expansion
            for (int j = 0; j < n; ++j) xt[j] = clamp01(__dsub_rn(__dmul_rn(3.0, xb[j]), __dmul_rn(2.0, x[n][j])));
            const double fe = block_chi2<MODE>(xt, b, view, n_ep, sink, term_row, s_red, A_row, f_min);
            ++fev;
            const bool take_e = fe < fr;
            for (int j = 0; j < n; ++j) x[n][j] = take_e ? xt[j] : xr[j];
            f[n] = take_e ? fe : fr;
        } else if (fr < f[n - 1]) {  // reflection
            for (int j = 0; j < n; ++j) x[n][j] = xr[j];
            f[n] = fr;
        } else {  // contraction, outside (towards the reflected point) or inside
            const bool outside = fr < f[n];
            for (int j = 0; j < n; ++j) {
                const double to = outside ? xr[j] : x[n][j];
                xt[j] = clamp01(__dadd_rn(xb[j], __dmul_rn(0.5, __dsub_rn(to, xb[j]))));
            }
            const double fc = block_chi2<MODE>(xt, b, view, n_ep, sink, term_row, s_red, A_row, f_min);
            ++fev;
            if (outside ? fc <= fr : fc < f[n]) {
                for (int j = 0; j < n; ++j) x[n][j] = xt[j];
                f[n] = fc;
            } else {
                shrink = true;
            }
        }
        if (shrink) {
            for (int k = 1; k <= n; ++k) {
                for (int j = 0; j < n; ++j) x[k][j] = __dadd_rn(x[0][j], __dmul_rn(0.5, __dsub_rn(x[k][j], x[0][j])));
                f[k] = block_chi2<MODE>(x[k], b, view, n_ep, sink, term_row, s_red, A_row, f_min);
            }
            fev += n;
        }
    }
    int best = 0;
    for (int k = 1; k <= n; ++k)
        if (f[k] < f[best]) best = k;
    if (f[best] < *f0) {
        *f0 = f[best];
        for (int j = 0; j < n; ++j) x0[j] = x[best][j];
    }
}

}  // namespace sblm
