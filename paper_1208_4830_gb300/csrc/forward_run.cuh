// forward_run.cuh -- one thread's run of consecutive epochs of one candidate: the unit of work
// that the population-wide forward kernel and the persistent batched fitter share.
#pragma once

#include "forward.cuh"
#include "forward_launch.cuh"

namespace sblm {

// the lightcurve as one thread reads it: staged in shared memory (FP64: t, F, 1/sigma; FP32
// modes: (t_hi, t_lo, F, 1/sigma) as float4) or straight from global memory
struct LCView {
    const double* t;
    const double* flux;
    const double* sigma;
    const double* s_t;
    const double* s_f;
    const double* s_w;
    const float4* s_ep;
};

// Stage n_ep epochs in `smem` (every thread of the block calls this; it ends with a barrier).
// FP32 modes split t = t_hi + t_lo so that t - t0 keeps full precision through a two-sum.
template <int MODE, bool CHI2>
__device__ __forceinline__ LCView stage_lightcurve(unsigned char* smem, const double* __restrict__ t,
                                                   const double* __restrict__ flux,
                                                   const double* __restrict__ sigma, int n_ep) {
    LCView v{t, flux, sigma, nullptr, nullptr, nullptr, nullptr};
    if (MODE == SBLM_FP64) {
        double* s_t = reinterpret_cast<double*>(smem);
        double* s_f = s_t + n_ep;
        double* s_w = s_f + (CHI2 ? n_ep : 0);
        for (int e = threadIdx.x; e < n_ep; e += blockDim.x) {
            s_t[e] = t[e];
            if (CHI2) {
                s_f[e] = flux[e];
                s_w[e] = 1.0 / sigma[e];
            }
        }
        v.s_t = s_t;
        v.s_f = s_f;
        v.s_w = s_w;
    } else {
        float4* s_ep = reinterpret_cast<float4*>(smem);
        for (int e = threadIdx.x; e < n_ep; e += blockDim.x) {
            const double te = t[e];
            const float th = (float)te;
            s_ep[e] = make_float4(th, (float)(te - (double)th), CHI2 ? (float)flux[e] : 0.f,
                                  CHI2 ? (float)(1.0 / sigma[e]) : 0.f);
        }
        v.s_ep = s_ep;
    }
    __syncthreads();
    return v;
}

template <bool FROM_GENES>
__device__ __forceinline__ Cand candidate(const double* __restrict__ src, const Bounds& b, int c) {
    if (!FROM_GENES) return load_cand(src, c);
    // Eq. (EMMA-encoding): a_j = lo_j + (hi_j - lo_j) p_j; gene 5 is log10 q
    const double* p = src + 6 * (size_t)c;
    double a[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) a[j] = b.lo[j] + (b.hi[j] - b.lo[j]) * p[j];
    Cand k;
    k.t0 = a[0];
    k.inv_tE = 1.0 / a[1];
    k.u0 = a[2];
    sincos(a[3], &k.sa, &k.ca);
    k.d = a[4];
    k.q = exp10(a[5]);
    return k;
}

// The candidate of a group of G threads (G a power of two; groups are aligned to G within the
// warp, or span whole warps when G > 32), decoded once per warp-part by its first lane and
// broadcast by shuffles: the decode's FP64 exp10, sincos and division run on the slow FP64 pipe.
// Every lane of the warp must call it.
template <bool FROM_GENES>
__device__ __forceinline__ Cand group_candidate(const double* __restrict__ src, const Bounds& b, int c, bool valid,
                                                int G) {
    const int lane = threadIdx.x & 31;
    const int src_lane = G < 32 ? (lane & ~(G - 1)) : 0;
    Cand k{};
    if (lane == src_lane && valid) k = candidate<FROM_GENES>(src, b, c);
    k.t0 = __shfl_sync(0xffffffffu, k.t0, src_lane);
    k.inv_tE = __shfl_sync(0xffffffffu, k.inv_tE, src_lane);
    k.u0 = __shfl_sync(0xffffffffu, k.u0, src_lane);
    k.sa = __shfl_sync(0xffffffffu, k.sa, src_lane);
    k.ca = __shfl_sync(0xffffffffu, k.ca, src_lane);
    k.d = __shfl_sync(0xffffffffu, k.d, src_lane);
    k.q = __shfl_sync(0xffffffffu, k.q, src_lane);
    return k;
}

// the MIXED re-solve's Aberth stop rule (relative correction), see solve_epoch
constexpr double kResolveCubic = 1e-6;

// FP64 re-solve of one deferred epoch (MIXED), warm-started from its FP32 roots; returns the
// chi^2 term from the FP64 flux fe and weight we = 1/sigma. Out of line: an FP32 lane that must
// do it in place keeps its state on the stack instead of competing with the FP64 solver for
// registers.
static __device__ __noinline__ double resolve_fp64(const cx<float>* z32, uint32_t why, const Cand* kk,
                                                   double te, double fe, double we, double* A_row,
                                                   uint8_t* f_row, int e, bool chi2) {
    cx<double> zz[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) zz[i] = mk<double>(z32[i].re, z32[i].im);
    bool w2 = true;
    const EpochOut<double> o2 = solve_epoch<double>(zeta64(*kk, te), kk->d, kk->q, zz, w2, nullptr, kResolveCubic);
    if (A_row) A_row[e] = o2.A;
    if (f_row) f_row[e] = (uint8_t)(o2.flag | FLAG_FP64 | why);
    if (!chi2) return 0.0;
    const double r = (fe - o2.A) * we;
    return r * r;
}

// Where MIXED work goes. Epochs to re-solve in FP64 are appended to `queue` (slots taken with one
// atomic per warp, so that a later pass re-solves them in full warps; an epoch that finds the queue
// full is re-solved in place, so the capacity is a speed choice only). Every epoch's chi^2 term is
// stored in the candidate's row of the dense term array (the FP32 ones here, the FP64 ones by the
// re-solve, wherever it runs), and the row is summed afterwards in a fixed order: a MIXED chi^2
// does not depend on the order in which the queue filled. `term_row` is the candidate's row
// (epoch e at term_row[e]); null when no chi^2 is wanted.
struct DeferSink {
    Deferred* queue;
    unsigned* queue_count;
    unsigned queue_cap;
};

// The thread's epochs [e0, e1) of candidate k (all lanes of a warp run `seg` iterations so that
// MIXED can reserve queue slots warp-wide). Writes A and flags when the row pointers are given.
// FP64 and FP32: returns the thread's chi^2 over its epochs, accumulated in FP64 in epoch order.
// MIXED: writes each epoch's chi^2 term to term_row (CHI2) and returns 0; `c_tag` is the candidate
// index recorded in its queue entries.
template <int MODE, bool CHI2, bool STAGED>
__device__ __forceinline__ double eval_run(const Cand& k, bool valid, int c_tag, int e0, int e1, int seg,
                                           const LCView& lc, double* A_row, uint8_t* f_row, const DeferSink& sink,
                                           double* term_row) {
    double chi = 0.0;
    if constexpr (MODE == SBLM_FP64) {
        cx<double> z[5];
        bool warm = false;
        for (int e = e0; valid && e < e1; ++e) {
            const double te = STAGED ? lc.s_t[e] : lc.t[e];
            const EpochOut<double> o = solve_epoch<double>(zeta64(k, te), k.d, k.q, z, warm);
            if (A_row) A_row[e] = o.A;
            if (f_row) f_row[e] = o.flag;
            if (CHI2) {
                const double fe = STAGED ? lc.s_f[e] : lc.flux[e];
                const double we = STAGED ? lc.s_w[e] : 1.0 / lc.sigma[e];
                const double r = (fe - o.A) * we;
                chi += r * r;
            }
        }
    } else {
        const float t0h = (float)k.t0, t0l = (float)(k.t0 - (double)t0h);
        const float itE = (float)k.inv_tE, sa = (float)k.sa, ca = (float)k.ca, u0 = (float)k.u0;
        const float d = (float)k.d, q = (float)k.q;
        const unsigned lane = threadIdx.x & 31u;
        cx<float> z[5];
        bool warm = false;
        for (int it = 0; it < seg; ++it) {
            const int e = e0 + it;
            const bool act = valid && e < e1;
            bool defer = false;
            uint8_t why = 0;
            if (act) {
                float4 ep;
                if (STAGED) {
                    ep = lc.s_ep[e];
                } else {
                    const double te = lc.t[e];
                    const float th = (float)te;
                    ep = make_float4(th, (float)(te - (double)th), CHI2 ? (float)lc.flux[e] : 0.f,
                                     CHI2 ? (float)(1.0 / lc.sigma[e]) : 0.f);
                }
                const float tau = diff_ff(ep.x, ep.y, t0h, t0l) * itE;
                const cx<float> zeta = mk<float>(tau * sa + u0 * ca, -tau * ca + u0 * sa);
                EpochOut<float> o = solve_epoch<float>(zeta, d, q, z, warm);
                o.flag = mixed_trigger_flags(o);
                if (MODE == SBLM_MIXED) defer = o.flag != 0;
                why = o.flag;
                if (A_row) A_row[e] = o.A;
                if (f_row) f_row[e] = o.flag;
                if (CHI2 && !defer) {
                    const double r = (double)((ep.z - o.A) * ep.w);
                    if (MODE == SBLM_MIXED)
                        term_row[e] = r * r;
                    else
                        chi += r * r;
                }
            }
            if constexpr (MODE == SBLM_MIXED) {
                // one atomic per warp reserves queue slots for the lanes that defer
                const unsigned b = __ballot_sync(0xffffffffu, defer);
                if (b) {
                    const int leader = __ffs(b) - 1;
                    unsigned base = 0;
                    if ((int)lane == leader) base = atomicAdd(sink.queue_count, (unsigned)__popc(b));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (defer) {
                        const unsigned slot = base + (unsigned)__popc(b & ((1u << lane) - 1u));
                        if (slot < sink.queue_cap) {
                            Deferred& qd = sink.queue[slot];
#pragma unroll
                            for (int i = 0; i < 5; ++i) qd.z[i] = z[i];
                            qd.c = c_tag;
                            qd.e = e;
                            qd.why = why;
                        } else {  // queue full: re-solve here, from the FP64 data
                            const double te = lc.t[e];
                            const double fe = CHI2 ? lc.flux[e] : 0.0, we = CHI2 ? 1.0 / lc.sigma[e] : 0.0;
                            cx<float> zc[5];  // a copy, so that z's address is never taken and z stays in registers
#pragma unroll
                            for (int i = 0; i < 5; ++i) zc[i] = z[i];
                            const double tm = resolve_fp64(zc, why, &k, te, fe, we, A_row, f_row, e, CHI2);
                            if (CHI2) term_row[e] = tm;
                        }
                    }
                }
            }
        }
    }
    return chi;
}

// MIXED: sum of a candidate's term row over the lanes of its group of G threads (G a power of two
// <= 32, groups aligned within the warp): lane g adds epochs g, g + G, ... in order, then a fixed
// butterfly combines the lanes; every lane of the group gets the sum. All lanes of the warp call it.
__device__ __forceinline__ double term_row_sum(const double* __restrict__ row, int n_ep, int g, int G, bool valid) {
    double s = 0.0;
    for (int e = g; valid && e < n_ep; e += G) s += row[e];
    for (int off = G / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
}

}  // namespace sblm
