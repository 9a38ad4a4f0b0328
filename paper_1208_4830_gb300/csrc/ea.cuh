// ea.cuh -- device side of the evolutionary algorithm of Appendix A (Rajpaul 2012).
//
// Random numbers: Philox4x64-10 with key (seed, stream id) and counter
// (generation, operator, index, sub-index); see common.cuh for the draw conventions.
// Offspring arithmetic uses explicitly rounded operations (no fused multiply-add) so that the
// same draws give bit-identical genes on every implementation that evaluates the same
// expressions in IEEE double.
#pragma once

#include <cuda_runtime.h>

#include "../../include/sblm.h"
#include "common.cuh"

namespace sblm {

constexpr int kMaxPop = 8192;          // largest N_pop of the single-block ranking
constexpr int kInitIndexBits = 20;     // element index in the low bits of the init sort keys
constexpr double kLnEps = -36.04365338911715;  // ln(2^-52), FP64 machine epsilon
constexpr double kPMutMax = 0.5;

struct EAConst {
    int n_pop, n_par, n_tourn, stag_window, restart_after;
    double p_mut0, stag_rel;
    uint64_t seed, stream;
};

struct EACtrl {
    double p_mut_used;  // jump probability of this generation's offspring
    int restart;        // 1: the next population is a fresh initialisation
    int pad;
};

// Appendix A, "Initialisation": sort key of element e (top 44 bits of a Philox word, index in
// the low bits, so that all keys differ).
__device__ __forceinline__ uint64_t init_key(const EAConst& c, uint64_t gen, uint64_t e) {
    const uint64_t w = philox4x64(gen, OP_INIT_PERM, e, 0, c.seed, c.stream).x[0];
    return ((w >> kInitIndexBits) << kInitIndexBits) | e;
}

// Value of the element whose key has rank `pos`: pairs (2k, 2k+1) of the sorted order get
// X_k and 1 - X_k; an odd leftover gets a plain draw.
__device__ __forceinline__ double init_value(const EAConst& c, uint64_t gen, uint64_t pos, uint64_t m) {
    const uint64_t n_pairs = m / 2;
    const uint64_t k = pos < 2 * n_pairs ? pos / 2 : n_pairs;
    const double x = u01(philox4x64(gen, OP_INIT_U, k, 0, c.seed, c.stream).x[0]);
    return (pos < 2 * n_pairs && (pos & 1)) ? __dsub_rn(1.0, x) : x;
}

// Appendix A, "Selection": parent rank = min of n_tourn uniform draws from {0..N_pop-1}
__device__ __forceinline__ int tournament(const EAConst& c, uint64_t gen, uint64_t slot) {
    uint32_t best = 0xffffffffu;
    u64x4 w{};
    for (int j = 0; j < c.n_tourn; ++j) {
        if ((j & 3) == 0) w = philox4x64(gen, OP_SELECT, slot, (uint64_t)(j >> 2), c.seed, c.stream);
        const uint32_t r = uniform_int(w.x[j & 3], (uint32_t)c.n_pop);
        best = r < best ? r : best;
    }
    return (int)best;
}

// Appendix A, "Creep and jump mutation" of gene j of population row `row`
__device__ __forceinline__ double mutate_gene(const EAConst& c, uint64_t gen, uint64_t row, uint64_t j, double p,
                                              double p_mut) {
    const u64x4 w = philox4x64(gen, OP_MUT, row, j, c.seed, c.stream);
    const double X = exp(__dmul_rn(kLnEps, u01(w.x[0])));
    double v = top_bit(w.x[1]) ? __dadd_rn(p, __dmul_rn(__dsub_rn(1.0, p), X)) : __dsub_rn(p, __dmul_rn(p, X));
    v = fmin(fmax(v, 0.0), 1.0);
    if (u01(w.x[2]) < p_mut) v = u01(w.x[3]);
    return v;
}

// Appendix A, "Stagnation checks", applied by one thread after the ranking of generation t.
// Returns 1 when the next population must be re-initialised.
__device__ __forceinline__ int stagnation_update(sblm_ea_state& s, const EAConst& c, double best) {
    const int W = c.stag_window;
    if (s.n_hist == W + 1) {
        for (int i = 0; i < W; ++i) s.hist[i] = s.hist[i + 1];
        s.n_hist = W;
    }
    s.hist[s.n_hist++] = best;
    bool stagnant = false;
    if (s.n_hist == W + 1) {
        const double old = s.hist[0];
        stagnant = isfinite(old) && (__dsub_rn(old, best) <= __dmul_rn(c.stag_rel, old));
    }
    const double p_min = 1.0 / (double)(c.n_pop * c.n_par);
    if (stagnant) {
        s.p_mut = fmin(__dmul_rn(s.p_mut, 1.5), kPMutMax);
        s.stag_run += 1;
    } else {
        s.p_mut = fmax(__dmul_rn(s.p_mut, 0.5), p_min);
        s.stag_run = 0;
    }
    if (s.stag_run >= c.restart_after) {
        s.p_mut = c.p_mut0;
        s.n_hist = 0;
        s.stag_run = 0;
        s.n_restarts += 1;
        return 1;
    }
    return 0;
}

// stable ascending order of (key, index) pairs: NaN fitness becomes +inf
__device__ __forceinline__ bool pair_less(double ka, int ia, double kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

}  // namespace sblm
