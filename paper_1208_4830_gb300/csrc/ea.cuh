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

// ---------------------------------------------------------------------------------------------
// Block-level building blocks, shared by the single-population kernels and the persistent
// batched fitter. Every thread of the calling block must call them (they hold barriers).
// ---------------------------------------------------------------------------------------------

// (fitness, row) pairs of the population in shared memory, NaN as +inf, padded to n2 (a power
// of two) with (+inf, INT_MAX), then sorted ascending by a bitonic network
__device__ __forceinline__ void block_rank(const double* __restrict__ chi2, int n_pop, int n2, double* skey,
                                           int* sidx) {
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        if (i < n_pop) {
            const double v = chi2[i];
            skey[i] = isnan(v) ? INFINITY : v;
            sidx[i] = i;
        } else {
            skey[i] = INFINITY;
            sidx[i] = 0x7fffffff;
        }
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const bool greater = pair_less(skey[l], sidx[l], skey[i], sidx[i]);
                    if (greater == up) {
                        const double tk = skey[i];
                        skey[i] = skey[l];
                        skey[l] = tk;
                        const int ti = sidx[i];
                        sidx[i] = sidx[l];
                        sidx[l] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// One thread's bookkeeping after the ranking of generation `gen`: archive of the best ever,
// stagnation check. Returns 1 when the next population is a fresh initialisation; *p_used is the
// jump probability of this generation's offspring.
__device__ __forceinline__ int block_bookkeeping(const EAConst& c, int gen, double best, const double* best_row,
                                                 sblm_ea_state& s, bool produce, double* p_used) {
    if (best < s.best_chi2) {
        s.best_chi2 = best;
        for (int j = 0; j < c.n_par; ++j) s.best_genes[j] = best_row[j];
    }
    *p_used = s.p_mut;
    const int restart = produce ? stagnation_update(s, c, best) : 0;
    s.generation = gen + 1;
    return restart;
}

// Reproductive pairing k of generation `gen` (Appendix A, "Selection", "Reproduction",
// "Creep and jump mutation"): two tournament parents from the ranked population (order[r] is
// the row of rank r), the weighting-matrix mode and diagonal, Eq. (rep1)/(rep2), then creep and
// jump of both children into rows 1 + 2k and 2 + 2k of P_next (the second dropped past N_pop).
__device__ __forceinline__ void offspring_pair(const EAConst& c, int gen, const double* __restrict__ P,
                                               const int* __restrict__ order, double p_mut, int k,
                                               double* __restrict__ P_next) {
    const int n_par = c.n_par;
    const uint64_t g = (uint64_t)gen;
    const int ra = tournament(c, g, 2 * (uint64_t)k);
    const int rb = tournament(c, g, 2 * (uint64_t)k + 1);
    const double* pa = P + (size_t)order[ra] * n_par;
    const double* pb = P + (size_t)order[rb] * n_par;
    const uint32_t mode = uniform_int(philox4x64(g, OP_MODE, (uint64_t)k, 0, c.seed, c.stream).x[0], 3u);
    const int row1 = 1 + 2 * k, row2 = 2 + 2 * k;
    for (int j = 0; j < n_par; ++j) {
        const uint64_t w = philox4x64(g, OP_F, (uint64_t)k, (uint64_t)j, c.seed, c.stream).x[0];
        const double f = mode == 0 ? u01(w) : (mode == 1 ? (double)top_bit(w) : 1.0);
        const double omf = __dsub_rn(1.0, f);
        const double a = pa[j], b = pb[j];
        const double c1 = __dadd_rn(__dmul_rn(a, f), __dmul_rn(b, omf));
        const double c2 = __dadd_rn(__dmul_rn(b, f), __dmul_rn(a, omf));
        P_next[(size_t)row1 * n_par + j] = mutate_gene(c, g, (uint64_t)row1, (uint64_t)j, c1, p_mut);
        if (row2 < c.n_pop)
            P_next[(size_t)row2 * n_par + j] = mutate_gene(c, g, (uint64_t)row2, (uint64_t)j, c2, p_mut);
    }
}

// Elements first + tid + k * step (k = 0, 1, ... while below m) of the initialisation of
// generation `gen`: each element's key is ranked against all m keys (read in tiles of `tile_n`
// through the shared array `tile`), and the rank gives its pairing and value. The trip counts are
// uniform over the block.
__device__ __forceinline__ void block_init_values(const EAConst& c, int gen, const uint64_t* __restrict__ keys,
                                                  int m, double* __restrict__ P, int first, int step,
                                                  uint64_t* tile, int tile_n) {
    for (int base = first; base < m; base += step) {
        const int e = base + threadIdx.x;
        const uint64_t mine = e < m ? keys[e] : 0;
        uint32_t pos = 0;
        for (int t0 = 0; t0 < m; t0 += tile_n) {
            const int n = min(tile_n, m - t0);
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) tile[i] = keys[t0 + i];
            __syncthreads();
            if (e < m)
                for (int i = 0; i < n; ++i) pos += tile[i] < mine;
        }
        if (e < m) P[e] = init_value(c, (uint64_t)gen, pos, (uint64_t)m);
        if (step >= m) break;
    }
}

__device__ __forceinline__ void state_reset(const EAConst& c, sblm_ea_state& s) {
    s.p_mut = c.p_mut0;
    s.best_chi2 = INFINITY;
    for (int i = 0; i <= SBLM_MAX_WINDOW; ++i) s.hist[i] = 0.0;
    s.n_hist = 0;
    s.stag_run = 0;
    s.n_restarts = 0;
    s.generation = 0;
    for (int j = 0; j < SBLM_MAX_NPAR; ++j) s.best_genes[j] = NAN;
}

}  // namespace sblm
