// batch.cu -- sblm_fit_batch: many lightcurves of uneven length, each with its own population
// and the whole evolutionary sequence of Appendix A, inside one persistent launch.
//
// One block per SM takes lightcurves from an atomic work counter, longest first (the host sorts
// them), and runs every generation of that lightcurve's fit in the block: the lightcurve staged
// in shared memory, the population's chi^2 by the same per-thread epoch runs as the forward
// kernel (G threads per candidate, several passes over the population), MIXED re-solves of the
// block's queue in a block-wide pass, then ranking, archive, stagnation, offspring or restart.
// No block ever waits for another, so no wait can stall the GPU. The launch is captured once in
// a CUDA graph and replayed for repeated calls with the same arguments.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>
#include <vector>

#include "../../include/sblm_cnn.h"
#include "cnn_launch.cuh"
#include "ea_launch.cuh"
#include "blend.cuh"
#include "forward_run.cuh"
#include "polish_launch.cuh"
#include "proposal.cuh"
#include "runtime.cuh"

namespace sblm {

sblm_status check_bounds(const sblm_bounds* b, Bounds* out);

namespace {

constexpr int kBatchMaxThreads = 512;
constexpr int kMaxIslands = 64;
constexpr size_t kBatchSmemBudget = 200 * 1024;  // dynamic shared memory per block

struct BatchArgs {
    const double* t;
    const double* flux;
    const double* sigma;
    const int64_t* offsets;
    const int* order;  // lightcurves, longest first
    int n_lc;
    Bounds b;
    EAConst c;  // stream is set per lightcurve
    int n_gen;
    int G;
    int n2;            // power of two >= n_pop
    double* P;         // per block: 2 x n_pop x 6
    uint64_t* keys;    // per block: n_pop x 6
    Deferred* queue;   // MIXED, per block: qcap entries
    unsigned qcap;
    double* term;      // MIXED, per block: n_pop x max_ep chi^2 terms (row per candidate)
    unsigned* next;    // work counter
    double* best_theta;
    double* best_chi2;
    int max_ep;        // longest lightcurve the staging area holds
    const double* seed;  // [n_lc][n_seed][6] genes of the seeded rows, or null
    int n_seed;          // rows n_pop - n_seed .. n_pop - 1 of the first population
    const float* prop_out;    // proposal outputs [n_lc][12] and windows [n_lc][2]: the seeded rows of the
    const double* prop_win;   // first population are drawn here (else `seed` holds them)
    uint64_t prop_seed;
    int polish_fev;      // amoeba fine-tuning of the archive's best (0: none), a separate launch
    int polish_starts;   // distinct starts of the amoeba (part of the graph's cache key)
    double* best_genes;  // [n_lc][6] genes of best_chi2
    int blend;           // chi^2 of the blended model with f profiled out (Section 4.4)
    double f_min;
    double* A_scr;       // blend: per block n_pop x max_ep magnifications
    int n_isl;           // island EA (Section 5.3): populations per lightcurve (1: the paper's panmictic EA)
    int mig_every;       // ring migration of the islands' elites every this many generations (0: never)
    sblm_ea_state* isl_state;  // n_isl > 1: per block n_isl states between generations
    double* isl_elite;         // n_isl > 1: per block n_isl x 6 genes of each island's last elite
    // success monitor (mon_theta nullptr: off)
    const double* mon_theta;  // [n_lc][6] reference rows
    const double* mon_f;      // [n_lc] reference blending fractions or nullptr
    const double* mon_chi2;   // [n_lc] chi^2 bound
    double mon_tol;
    int* mon_first;           // [n_lc] first generation with a matching row, -1 if none
    double* f_scr;            // blend with monitor: per block n_pop profiled f
    // solution archive (arc_size 0: off)
    int arc_size;
    int arc_top;              // rows offered per population and generation
    double arc_radius;
    double* arc_genes;        // [n_lc][arc_size][6] genes of the archived solutions
    double* arc_theta;        // [n_lc][arc_size][6] out
    double* arc_chi2;         // [n_lc][arc_size] out
    int* arc_count;           // [n_lc] out
};

// two encoded solutions are the same when every gene differs by at most r
__device__ __forceinline__ bool archive_same(const double* a, const double* b, double r) {
    bool s = true;
    for (int j = 0; j < SBLM_NPAR; ++j) s &= fabs(a[j] - b[j]) <= r;
    return s;
}

// stable insertion sort of the archive by chi^2
__device__ void archive_sort(double* g, double* c, int n) {
    for (int i = 1; i < n; ++i) {
        const double ci = c[i];
        double gi[SBLM_NPAR];
        for (int j = 0; j < SBLM_NPAR; ++j) gi[j] = g[i * SBLM_NPAR + j];
        int k = i;
        for (; k > 0 && c[k - 1] > ci; --k) {
            c[k] = c[k - 1];
            for (int j = 0; j < SBLM_NPAR; ++j) g[k * SBLM_NPAR + j] = g[(k - 1) * SBLM_NPAR + j];
        }
        c[k] = ci;
        for (int j = 0; j < SBLM_NPAR; ++j) g[k * SBLM_NPAR + j] = gi[j];
    }
}

// Offer one evaluated row (genes x, chi^2 v) to the archive of `size` entries holding *n (one
// thread): the rule of sblm_batch_archive in include/sblm.h
__device__ __noinline__ void archive_offer(double* g, double* c, int* n, int size, double r, const double* x,
                                           double v) {
    if (!isfinite(v)) return;
    for (int k = 0; k < *n; ++k) {
        if (!archive_same(g + k * SBLM_NPAR, x, r)) continue;
        if (!(v < c[k])) return;
        double xk[SBLM_NPAR];
        for (int j = 0; j < SBLM_NPAR; ++j) xk[j] = g[k * SBLM_NPAR + j] = x[j];
        c[k] = v;
        // drop the entries that now match entry k (it is the fitter of each such pair)
        int w = 0;
        for (int i = 0; i < *n; ++i) {
            if (i != k && archive_same(g + i * SBLM_NPAR, xk, r)) continue;
            if (w != i) {
                c[w] = c[i];
                for (int j = 0; j < SBLM_NPAR; ++j) g[w * SBLM_NPAR + j] = g[i * SBLM_NPAR + j];
            }
            ++w;
        }
        *n = w;
        archive_sort(g, c, *n);
        return;
    }
    int slot;
    if (*n < size) {
        slot = (*n)++;
    } else if (v < c[*n - 1]) {
        slot = *n - 1;
    } else {
        return;
    }
    c[slot] = v;
    for (int j = 0; j < SBLM_NPAR; ++j) g[slot * SBLM_NPAR + j] = x[j];
    archive_sort(g, c, *n);
}

// Section 4.2's strict test of one evaluated row (genes g) against the reference row: every
// parameter within tol (t0 relative to the reference tE, alpha as a wrapped difference relative
// to 2 pi, the others relative to their reference values; f too when f_ref >= 0)
__device__ __noinline__ bool monitor_match(const double* g, const Bounds& b, const double* ref, double f,
                                           double f_ref, double tol) {
    double a[SBLM_NPAR];
    for (int j = 0; j < SBLM_NPAR; ++j) a[j] = b.lo[j] + (b.hi[j] - b.lo[j]) * g[j];
    const double two_pi = 6.283185307179586;
    double da = a[3] - ref[3] + 0.5 * two_pi;
    da -= two_pi * floor(da / two_pi);
    bool ok = fabs(a[0] - ref[0]) < tol * fabs(ref[1]);
    ok &= fabs(a[1] - ref[1]) < tol * fabs(ref[1]);
    ok &= fabs(a[2] - ref[2]) < tol * fabs(ref[2]);
    ok &= fabs(da - 0.5 * two_pi) < tol * two_pi;
    ok &= fabs(a[4] - ref[4]) < tol * fabs(ref[4]);
    ok &= fabs(exp10(a[5]) - ref[5]) < tol * fabs(ref[5]);
    if (f_ref >= 0.0) ok &= fabs(f - f_ref) < tol * f_ref;
    return ok;
}

// flux and weight 1/sigma of staged epoch e
template <int MODE>
__device__ __forceinline__ void staged_fw(const LCView& v, int e, double& F, double& w) {
    if (MODE == SBLM_FP64) {
        F = v.s_f[e];
        w = v.s_w[e];
    } else {
        const float4 ep = v.s_ep[e];
        F = ep.z;
        w = ep.w;
    }
}

size_t batch_smem_bytes(int mode, int n_pop, int n2, int max_ep) {
    const size_t ep = (size_t)max_ep * (mode == SBLM_FP64 ? 3 * sizeof(double) : sizeof(float4));
    return ((ep + 15) & ~size_t(15)) + sizeof(double) * n_pop + (sizeof(double) + sizeof(int)) * n2;
}

template <int MODE>
__global__ void __launch_bounds__(kBatchMaxThreads, 1) batch_fit_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n_pop = a.c.n_pop, n_par = a.c.n_par, G = a.G;
    const size_t ep_bytes =
        ((size_t)a.max_ep * (MODE == SBLM_FP64 ? 3 * sizeof(double) : sizeof(float4)) + 15) & ~size_t(15);
    double* s_chi = reinterpret_cast<double*>(smem + ep_bytes);
    double* s_key = s_chi + n_pop;
    int* s_idx = reinterpret_cast<int*>(s_key + a.n2);
    __shared__ sblm_ea_state s_state;
    __shared__ int s_job, s_restart;
    __shared__ double s_pmut;
    __shared__ unsigned s_qcount;
    __shared__ int s_first;
    __shared__ int s_arc_n;

    const int n_isl = a.n_isl;
    uint64_t* keys = a.keys + (size_t)blockIdx.x * n_pop * n_par;
    DeferSink sink{};
    if (MODE == SBLM_MIXED) {
        sink.queue = a.queue + (size_t)blockIdx.x * a.qcap;
        sink.queue_count = &s_qcount;
        sink.queue_cap = a.qcap;
    }
    double* const term_blk = MODE == SBLM_MIXED ? a.term + (size_t)blockIdx.x * n_pop * a.max_ep : nullptr;
    const int m = n_pop * n_par;
    double* const Pi = a.P + (size_t)blockIdx.x * n_isl * 2 * m;  // island i: rows Pi + i 2m (two buffers)
    sblm_ea_state* const st_g = a.isl_state + (size_t)blockIdx.x * n_isl;
    double* const elite = a.isl_elite + (size_t)blockIdx.x * n_isl * n_par;

    for (;;) {
        if (threadIdx.x == 0) s_job = (int)atomicAdd(a.next, 1u);
        __syncthreads();
        const int job = s_job;
        __syncthreads();
        if (job >= a.n_lc) break;
        const int lc = a.order[job];
        const int64_t e_begin = a.offsets[lc];
        const int n_ep = (int)(a.offsets[lc + 1] - e_begin);
        const LCView view = stage_lightcurve<MODE, true>(smem, a.t + e_begin, a.flux + e_begin, a.sigma + e_begin, n_ep);
        EAConst c = a.c;

        // Appendix A, "Initialisation", of every island (island i: stream id lc + i n_lc); the
        // proposal rows replace the last n_seed random rows of island 0
        for (int isl = 0; isl < n_isl; ++isl) {
            c.stream = (uint64_t)lc + (uint64_t)isl * a.n_lc;
            double* const P0 = Pi + (size_t)isl * 2 * m;
            for (int e = threadIdx.x; e < m; e += blockDim.x) keys[e] = init_key(c, 0, (uint64_t)e);
            __syncthreads();
            block_init_values(c, 0, keys, m, P0, 0, blockDim.x, reinterpret_cast<uint64_t*>(s_key), a.n2);
            if (isl == 0 && a.n_seed > 0) {
                __syncthreads();
                double* dst = P0 + (size_t)(n_pop - a.n_seed) * n_par;
                if (a.prop_out) {
                    for (int r = threadIdx.x; r < a.n_seed; r += blockDim.x)
                        proposal_row(a.prop_out + 12 * (size_t)lc, a.prop_win[2 * lc], a.prop_win[2 * lc + 1], a.b,
                                     a.prop_seed, (uint64_t)lc, (uint64_t)r, 0, dst + (size_t)r * n_par);
                } else {
                    const double* sg = a.seed + (size_t)lc * a.n_seed * n_par;
                    for (int e = threadIdx.x; e < a.n_seed * n_par; e += blockDim.x) dst[e] = sg[e];
                }
            }
            if (threadIdx.x == 0) {
                state_reset(c, s_state);
                if (n_isl > 1) st_g[isl] = s_state;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s_first = -1;
            s_arc_n = 0;
        }
        __syncthreads();

        const int group = threadIdx.x / G, g = threadIdx.x % G;
        const int per_pass = blockDim.x / G;
        const int seg = (n_ep + G - 1) / G;
        const int e0 = min(n_ep, g * seg), e1 = min(n_ep, e0 + seg);
        int cur = 0;
        for (int gen = 0; gen < a.n_gen; ++gen) {
            const bool produce = gen + 1 < a.n_gen;
            for (int isl = 0; isl < n_isl; ++isl) {
                c.stream = (uint64_t)lc + (uint64_t)isl * a.n_lc;
                double* const Pc = Pi + (size_t)isl * 2 * m + (size_t)cur * m;
                double* const Pn = Pi + (size_t)isl * 2 * m + (size_t)(cur ^ 1) * m;
                // fitness of every row (decode + forward model + chi^2)
                if (threadIdx.x == 0) {
                    s_qcount = 0;
                    if (n_isl > 1) s_state = st_g[isl];
                }
                __syncthreads();
                for (int base = 0; base < n_pop; base += per_pass) {
                    const int cand = base + group;
                    const bool valid = cand < n_pop;
                    const Cand k = group_candidate<true>(Pc, a.b, cand, valid, G);
                    double* A_row =
                        (a.blend && valid) ? a.A_scr + ((size_t)blockIdx.x * n_pop + cand) * a.max_ep : nullptr;
                    double* term_row = (MODE == SBLM_MIXED && valid) ? term_blk + (size_t)cand * a.max_ep : nullptr;
                    double chi = eval_run<MODE, true, true>(k, valid, cand, e0, e1, seg, view, A_row, nullptr, sink,
                                                            term_row);
                    for (int off = G / 2; off > 0; off >>= 1) chi += __shfl_xor_sync(0xffffffffu, chi, off);
                    if (g == 0 && valid) s_chi[cand] = chi;
                }
                __syncthreads();
                if constexpr (MODE == SBLM_MIXED) {
                    // the block's queued epochs, in FP64 from the FP64 data, each term to its place
                    // in the candidate's term row; then each candidate's row summed in a fixed order
                    const unsigned n = min(s_qcount, a.qcap);
                    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
                        const Deferred q = sink.queue[i];
                        const Cand k = candidate<true>(Pc, a.b, q.c);
                        double* A_rq = a.blend ? a.A_scr + ((size_t)blockIdx.x * n_pop + q.c) * a.max_ep : nullptr;
                        const int64_t ge = e_begin + q.e;
                        term_blk[(size_t)q.c * a.max_ep + q.e] = resolve_fp64(
                            q.z, q.why, &k, a.t[ge], a.flux[ge], 1.0 / a.sigma[ge], A_rq, nullptr, q.e, true);
                    }
                    __syncthreads();
                    for (int base = 0; base < n_pop; base += per_pass) {
                        const int cand = base + group;
                        const double* row = term_blk + (size_t)min(cand, n_pop - 1) * a.max_ep;
                        const double chi = term_row_sum(row, n_ep, g, G, cand < n_pop);
                        if (g == 0 && cand < n_pop) s_chi[cand] = chi;
                    }
                    __syncthreads();
                }
                if (a.blend) {  // Section 4.4: chi^2 of f A + (1 - f) with f profiled out, per candidate
                    for (int base = 0; base < n_pop; base += per_pass) {
                        const int cand = base + group;
                        const double* Ar = a.A_scr + ((size_t)blockIdx.x * n_pop + min(cand, n_pop - 1)) * a.max_ep;
                        double s_ab = 0.0, s_aa = 0.0;
                        for (int e = g; cand < n_pop && e < n_ep; e += G) {
                            double F, w;
                            staged_fw<MODE>(view, e, F, w);
                            const double ww = w * w, aa = Ar[e] - 1.0;
                            s_ab += ww * aa * (F - 1.0);
                            s_aa += ww * aa * aa;
                        }
                        for (int off = G / 2; off > 0; off >>= 1) {
                            s_ab += __shfl_xor_sync(0xffffffffu, s_ab, off);
                            s_aa += __shfl_xor_sync(0xffffffffu, s_aa, off);
                        }
                        const double f = blend_f(s_ab, s_aa, a.f_min);
                        double chi = 0.0;
                        for (int e = g; cand < n_pop && e < n_ep; e += G) {
                            double F, w;
                            staged_fw<MODE>(view, e, F, w);
                            const double r = (F - 1.0) - f * (Ar[e] - 1.0);
                            chi += w * w * r * r;
                        }
                        for (int off = G / 2; off > 0; off >>= 1) chi += __shfl_xor_sync(0xffffffffu, chi, off);
                        if (g == 0 && cand < n_pop) {
                            s_chi[cand] = chi;
                            if (a.f_scr) a.f_scr[(size_t)blockIdx.x * n_pop + cand] = f;
                        }
                    }
                    __syncthreads();
                }
                if (a.mon_theta) {  // success monitor: every evaluated row against the reference
                    const double bound = a.mon_chi2[lc], f_ref = a.mon_f ? a.mon_f[lc] : -1.0;
                    for (int r = threadIdx.x; r < n_pop; r += blockDim.x) {
                        if (!(s_chi[r] < bound)) continue;
                        const double f = a.f_scr ? a.f_scr[(size_t)blockIdx.x * n_pop + r] : 1.0;
                        if (monitor_match(Pc + (size_t)r * n_par, a.b, a.mon_theta + (size_t)lc * SBLM_NPAR, f,
                                          f_ref, a.mon_tol))
                            atomicCAS(&s_first, -1, gen);
                    }
                }
                // ranking, archive, stagnation
                block_rank(s_chi, n_pop, a.n2, s_key, s_idx);
                if (a.arc_size > 0 && threadIdx.x == 0) {  // offers in rank order, fittest first
                    double* ag = a.arc_genes + (size_t)lc * a.arc_size * SBLM_NPAR;
                    double* ac = a.arc_chi2 + (size_t)lc * a.arc_size;
                    const int top = a.arc_top > 0 ? min(a.arc_top, n_pop) : n_pop;
                    int n = s_arc_n;
                    for (int i = 0; i < top; ++i)
                        archive_offer(ag, ac, &n, a.arc_size, a.arc_radius, Pc + (size_t)s_idx[i] * n_par, s_key[i]);
                    s_arc_n = n;
                }
                if (threadIdx.x == 0) {
                    double p_used = 0.0;
                    s_restart = block_bookkeeping(c, gen, s_key[0], Pc + (size_t)s_idx[0] * n_par, s_state, produce,
                                                  &p_used);
                    s_pmut = p_used;
                    if (n_isl > 1) {
                        st_g[isl] = s_state;
                        for (int j = 0; j < n_par; ++j) elite[isl * n_par + j] = Pc[(size_t)s_idx[0] * n_par + j];
                    }
                }
                __syncthreads();
                if (produce) {
                    if (s_restart) {
                        for (int e = threadIdx.x; e < m; e += blockDim.x)
                            keys[e] = init_key(c, (uint64_t)(gen + 1), (uint64_t)e);
                        __syncthreads();
                        block_init_values(c, gen + 1, keys, m, Pn, 0, blockDim.x, reinterpret_cast<uint64_t*>(s_key),
                                          a.n2);
                    } else {
                        if (threadIdx.x == 0) {
                            const double* e = Pc + (size_t)s_idx[0] * n_par;
                            for (int j = 0; j < n_par; ++j) Pn[j] = e[j];
                        }
                        for (int k = threadIdx.x; k < n_pop / 2; k += blockDim.x)
                            offspring_pair(c, gen, Pc, s_idx, s_pmut, k, Pn);
                    }
                    __syncthreads();
                }
            }
            if (!produce) break;
            if (n_isl > 1 && a.mig_every > 0 && (gen + 1) % a.mig_every == 0) {
                // Section 5.3, island EA: the elite of island i replaces the last row of the next
                // population of island (i + 1) mod n_isl
                for (int e = threadIdx.x; e < n_isl * n_par; e += blockDim.x) {
                    const int from = e / n_par, j = e % n_par, to = (from + 1) % n_isl;
                    Pi[(size_t)to * 2 * m + (size_t)(cur ^ 1) * m + (size_t)(n_pop - 1) * n_par + j] =
                        elite[from * n_par + j];
                }
                __syncthreads();
            }
            cur ^= 1;
        }
        if (threadIdx.x == 0) {
            if (n_isl > 1) {  // the lightcurve's best over its islands (the lowest island on ties)
                int bi = 0;
                for (int i = 1; i < n_isl; ++i)
                    if (st_g[i].best_chi2 < st_g[bi].best_chi2) bi = i;
                s_state = st_g[bi];
            }
            double av[SBLM_NPAR];
            for (int j = 0; j < SBLM_NPAR; ++j) av[j] = a.b.lo[j] + (a.b.hi[j] - a.b.lo[j]) * s_state.best_genes[j];
            double* th = a.best_theta + (size_t)lc * SBLM_NPAR;
            for (int j = 0; j < 5; ++j) th[j] = av[j];
            th[5] = exp10(av[5]);
            a.best_chi2[lc] = s_state.best_chi2;
            if (a.mon_first) a.mon_first[lc] = s_first;
            if (a.arc_size > 0) {
                const double* ag = a.arc_genes + (size_t)lc * a.arc_size * SBLM_NPAR;
                double* at = a.arc_theta + (size_t)lc * a.arc_size * SBLM_NPAR;
                double* ac = a.arc_chi2 + (size_t)lc * a.arc_size;
                for (int k = 0; k < a.arc_size; ++k) {
                    double av[SBLM_NPAR];
                    for (int j = 0; j < SBLM_NPAR; ++j)
                        av[j] = k < s_arc_n ? a.b.lo[j] + (a.b.hi[j] - a.b.lo[j]) * ag[k * SBLM_NPAR + j] : NAN;
                    for (int j = 0; j < 5; ++j) at[k * SBLM_NPAR + j] = av[j];
                    at[k * SBLM_NPAR + 5] = k < s_arc_n ? exp10(av[5]) : NAN;
                    if (k >= s_arc_n) ac[k] = NAN;
                }
                a.arc_count[lc] = s_arc_n;
            }
            for (int j = 0; j < SBLM_NPAR; ++j) a.best_genes[(size_t)lc * SBLM_NPAR + j] = s_state.best_genes[j];
        }
        __syncthreads();
    }
}

// several polish starts: the fittest polished start of each lightcurve (the first on ties)
// replaces the EA's best when it is fitter
__global__ void pick_polished_kernel(const double* __restrict__ g, const double* __restrict__ c, int n_lc, int starts,
                                     double* __restrict__ best_genes, double* __restrict__ best_chi2) {
    const int lc = blockIdx.x * blockDim.x + threadIdx.x;
    if (lc >= n_lc) return;
    int bk = -1;
    double bc = best_chi2[lc];
    for (int k = 0; k < starts; ++k) {
        const double v = c[(size_t)lc * starts + k];
        if (v < bc) {
            bc = v;
            bk = k;
        }
    }
    if (bk < 0) return;
    best_chi2[lc] = bc;
    for (int j = 0; j < SBLM_NPAR; ++j) best_genes[(size_t)lc * SBLM_NPAR + j] = g[((size_t)lc * starts + bk) * SBLM_NPAR + j];
}

// theta rows of the (polished) best genes
__global__ void genes_to_theta_kernel(const double* __restrict__ genes, int n_lc, Bounds b, double* __restrict__ theta) {
    const int lc = blockIdx.x * blockDim.x + threadIdx.x;
    if (lc >= n_lc) return;
    double av[SBLM_NPAR];
    for (int j = 0; j < SBLM_NPAR; ++j) av[j] = b.lo[j] + (b.hi[j] - b.lo[j]) * genes[(size_t)lc * SBLM_NPAR + j];
    double* th = theta + (size_t)lc * SBLM_NPAR;
    for (int j = 0; j < 5; ++j) th[j] = av[j];
    th[5] = exp10(av[5]);
}

template <int MODE>
cudaError_t launch_batch_mode(const BatchArgs& a, int blocks, int threads, size_t smem, cudaStream_t s,
                              bool attr_only) {
    auto kern = batch_fit_kernel<MODE>;
    if (attr_only) return raise_smem_limit((const void*)kern, smem);
    kern<<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

// attr_only: set the shared-memory opt-in (done before a stream capture begins)
cudaError_t launch_batch(int mode, const BatchArgs& a, int blocks, int threads, size_t smem, cudaStream_t s,
                         bool attr_only) {
    switch (mode) {
        case SBLM_FP64: return launch_batch_mode<SBLM_FP64>(a, blocks, threads, smem, s, attr_only);
        case SBLM_MIXED: return launch_batch_mode<SBLM_MIXED>(a, blocks, threads, smem, s, attr_only);
        default: return launch_batch_mode<SBLM_FP32>(a, blocks, threads, smem, s, attr_only);
    }
}

// The graph of the last call (counter reset + persistent kernel), replayed while the
// arguments stay the same.
struct GraphCache {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
};
GraphCache g_graph;

struct Prepared {
    BatchArgs a;
    int blocks, threads;
    size_t smem;
    int mode;
    PolishArgs pa;   // amoeba pass over every lightcurve when a.polish_fev > 0
    int polish_blocks;
    int max_ep;
};

// validate, stage and lay out one batch call; on success `st` has begun
sblm_status prepare(const double* t, const double* flux, const double* sigma, const int64_t* offsets, int32_t n_lc,
                    const sblm_bounds* bounds, const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                    const double* seed_genes, int n_seed, double* best_theta, double* best_chi2, Staging& st,
                    int* i_th, int* i_c, Prepared* out, size_t extra_bytes = 0, int* k_extra = nullptr,
                    const sblm_batch_monitor* mon = nullptr, int* i_mon = nullptr,
                    const sblm_batch_archive* arc = nullptr, int* i_arc = nullptr) {
    if (!params) return fail(SBLM_EINVAL, "params is NULL");
    const int mode = params->precision & ~SBLM_BLEND;
    const bool blend = (params->precision & SBLM_BLEND) != 0;
    sblm_ea_params pm = *params;
    pm.precision = mode;
    EAConst c;
    SBLM_TRY(ea_const(&pm, params->n_pop, SBLM_NPAR, 0, &c));
    if (params->n_gen < 1) return fail(SBLM_EINVAL, "n_gen must be >= 1");
    if (n_lc < 1) return fail(SBLM_EINVAL, "n_lc must be >= 1");
    if (!offsets || !best_theta || !best_chi2) return fail(SBLM_EINVAL, "offsets, best_theta and best_chi2 are required");
    Bounds b;
    SBLM_TRY(check_bounds(bounds, &b));
    // offsets are needed on the host for the layout
    std::vector<int64_t> off(n_lc + 1);
    bool off_dev = false;
    SBLM_TRY(is_device_pointer(offsets, &off_dev));
    if (off_dev)
        SBLM_CUDA(cudaMemcpy(off.data(), offsets, sizeof(int64_t) * (n_lc + 1), cudaMemcpyDeviceToHost));
    else
        std::memcpy(off.data(), offsets, sizeof(int64_t) * (n_lc + 1));
    if (off[0] != 0) return fail(SBLM_EINVAL, "offsets[0] must be 0");
    int max_ep = 0;
    for (int i = 0; i < n_lc; ++i) {
        const int64_t n = off[i + 1] - off[i];
        if (n < 1) return fail(SBLM_EINVAL, "lightcurve %d has no epochs", i);
        max_ep = (int)std::max<int64_t>(max_ep, n);
    }
    const int64_t total = off[n_lc];
    int G = tuning && tuning->group > 0 ? tuning->group : 16;
    int threads = tuning && tuning->block > 0 ? tuning->block : 512;
    if (G < 1 || G > 32 || (G & (G - 1))) return fail(SBLM_EINVAL, "tuning group must be a power of two <= 32");
    if (threads < 32 || threads > kBatchMaxThreads || threads % 32)
        return fail(SBLM_EINVAL, "tuning block must be a multiple of 32 in [32, %d]", kBatchMaxThreads);
    int n2 = 1;
    while (n2 < c.n_pop) n2 <<= 1;
    const size_t smem = batch_smem_bytes(mode, c.n_pop, n2, max_ep);
    if (smem > kBatchSmemBudget)
        return fail(SBLM_EINVAL, "longest lightcurve (%d epochs) does not fit the %zu-byte staging area with n_pop=%d",
                    max_ep, kBatchSmemBudget, c.n_pop);
    int dev = 0, sms = 0;
    SBLM_CUDA(cudaGetDevice(&dev));
    SBLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = std::min(sms, n_lc);

    int i_t, i_f, i_s, i_o;
    SBLM_TRY(st.arg(t, sizeof(double) * total, true, false, &i_t));
    SBLM_TRY(st.arg(flux, sizeof(double) * total, true, false, &i_f));
    SBLM_TRY(st.arg(sigma, sizeof(double) * total, true, false, &i_s));
    SBLM_TRY(st.arg(offsets, sizeof(int64_t) * (n_lc + 1), true, false, &i_o));
    SBLM_TRY(st.arg(best_theta, sizeof(double) * 6 * (size_t)n_lc, false, true, i_th));
    SBLM_TRY(st.arg(best_chi2, sizeof(double) * (size_t)n_lc, false, true, i_c));
    bool d1, d2, d3;
    SBLM_TRY(is_device_pointer(t, &d1));
    SBLM_TRY(is_device_pointer(flux, &d2));
    SBLM_TRY(is_device_pointer(sigma, &d3));
    if (!d1 && !d2 && !d3) SBLM_TRY(check_lightcurve_host(t, flux, sigma, (int)total));
    // per block: room for a quarter of a generation's epochs (a population gathered on a
    // caustic-crossing model defers many); epochs past this are re-solved in place, one divergent
    // lane at a time, so the size is a speed choice only
    // per block: room for a quarter of a generation's epochs (a population gathered on a
    // caustic-crossing model defers many), within 2^26 entries (~3 GB) over all blocks; epochs past
    // this are re-solved in place, one divergent lane at a time, so the size is a speed choice only
    const unsigned qcap =
        mode == SBLM_MIXED
            ? (unsigned)std::max<long>(4096, std::min<long>((long)c.n_pop * max_ep / 4, (1L << 26) / blocks))
            : 0;
    const int k_order = st.scratch(sizeof(int) * n_lc);
    const int n_isl = std::max(1, params->n_islands);
    if (n_isl > kMaxIslands) return fail(SBLM_EINVAL, "n_islands=%d outside [1, %d]", n_isl, kMaxIslands);
    const int k_P = st.scratch(sizeof(double) * 2 * (size_t)c.n_pop * SBLM_NPAR * blocks * n_isl);
    const int k_is = st.scratch(n_isl > 1 ? sizeof(sblm_ea_state) * (size_t)blocks * n_isl : 0);
    const int k_ie = st.scratch(n_isl > 1 ? sizeof(double) * SBLM_NPAR * (size_t)blocks * n_isl : 0);
    const int k_keys = st.scratch(sizeof(uint64_t) * (size_t)c.n_pop * SBLM_NPAR * blocks);
    const int k_q = st.scratch(deferred_entry_bytes() * (size_t)qcap * blocks);
    const int k_term = st.scratch(mode == SBLM_MIXED ? sizeof(double) * (size_t)c.n_pop * max_ep * blocks : 0);
    const int k_next = st.scratch(sizeof(unsigned));
    const int k_genes = st.scratch(sizeof(double) * SBLM_NPAR * (size_t)n_lc);
    const int k_A = st.scratch(blend ? sizeof(double) * (size_t)blocks * c.n_pop * max_ep : 0);
    // the amoeba from several distinct starts (polish_starts > 1): the archive of the solutions the
    // EA evaluated (the caller's, or one kept for this purpose) supplies them
    const int starts = params->polish_fev > 0 ? std::max(1, params->polish_starts) : 1;
    if (starts > 64) return fail(SBLM_EINVAL, "polish_starts must be in [1, 64]");
    if (starts > 1 && (!(params->polish_radius > 0.0) || !std::isfinite(params->polish_radius)))
        return fail(SBLM_EINVAL, "polish_radius must be > 0");
    const int arc_k = arc ? arc->size : (starts > 1 ? starts : 0);  // archive entries per lightcurve
    const int inst_per_lc = starts > 1 ? arc_k : 1;                 // polish instances per lightcurve
    const int polish_blocks = (int)std::min<long>((long)n_lc * inst_per_lc, 2L * sms);
    const int k_pg = st.scratch(starts > 1 ? sizeof(double) * SBLM_NPAR * (size_t)n_lc * inst_per_lc : 0);
    const int k_pc = st.scratch(starts > 1 ? sizeof(double) * (size_t)n_lc * inst_per_lc : 0);
    const int k_iag = st.scratch(!arc && starts > 1 ? sizeof(double) * SBLM_NPAR * (size_t)n_lc * arc_k : 0);
    const int k_iat = st.scratch(!arc && starts > 1 ? sizeof(double) * SBLM_NPAR * (size_t)n_lc * arc_k : 0);
    const int k_iac = st.scratch(!arc && starts > 1 ? sizeof(double) * (size_t)n_lc * arc_k : 0);
    const int k_ian = st.scratch(!arc && starts > 1 ? sizeof(int) * (size_t)n_lc : 0);
    const int k_pA = st.scratch(blend && params->polish_fev > 0 ? sizeof(double) * (size_t)polish_blocks * max_ep : 0);
    const PolishMixed pmx = polish_mixed_layout(max_ep);
    const int k_pq = st.scratch(mode == SBLM_MIXED && params->polish_fev > 0 ? pmx.block_bytes * polish_blocks : 0);
    if (params->polish_fev > 0 && polish_smem_bytes(mode, max_ep) > kPolishSmemBudget)
        return fail(SBLM_EINVAL, "the amoeba polish stages at most %zu bytes of epochs (longest lightcurve %d)",
                    kPolishSmemBudget, max_ep);
    if (n_seed < 0 || n_seed > c.n_pop) return fail(SBLM_EINVAL, "n_seed must be in [0, n_pop]");
    if (params->polish_fev < 0 || params->polish_fev > kPolishMaxFev)
        return fail(SBLM_EINVAL, "polish_fev must be in [0, %d]", kPolishMaxFev);
    if (n_seed > 0 && !seed_genes && !k_extra) return fail(SBLM_EINVAL, "seed_genes is NULL");
    int i_seed = -1;
    if (seed_genes) SBLM_TRY(st.arg(seed_genes, sizeof(double) * SBLM_NPAR * (size_t)n_lc * n_seed, true, false, &i_seed));
    if (k_extra) *k_extra = st.scratch(extra_bytes);
    int i_mt = -1, i_mf = -1, i_mc = -1, k_f = -1;
    if (mon) {
        if (!mon->theta_ref || !mon->chi2_max || !mon->first_gen)
            return fail(SBLM_EINVAL, "the monitor needs theta_ref, chi2_max and first_gen");
        if (!(mon->rel_tol > 0.0) || !std::isfinite(mon->rel_tol)) return fail(SBLM_EINVAL, "monitor rel_tol must be > 0");
        SBLM_TRY(st.arg(mon->theta_ref, sizeof(double) * SBLM_NPAR * (size_t)n_lc, true, false, &i_mt));
        SBLM_TRY(st.arg(mon->chi2_max, sizeof(double) * (size_t)n_lc, true, false, &i_mc));
        if (mon->f_ref) SBLM_TRY(st.arg(mon->f_ref, sizeof(double) * (size_t)n_lc, true, false, &i_mf));
        SBLM_TRY(st.arg(mon->first_gen, sizeof(int32_t) * (size_t)n_lc, false, true, i_mon));
        if (blend) k_f = st.scratch(sizeof(double) * (size_t)blocks * c.n_pop);
    }
    int k_ag = -1;
    if (arc) {
        if (arc->size < 1 || arc->size > 64) return fail(SBLM_EINVAL, "archive size must be in [1, 64]");
        if (arc->top < 0) return fail(SBLM_EINVAL, "archive top must be >= 0");
        if (!(arc->radius > 0.0) || !std::isfinite(arc->radius)) return fail(SBLM_EINVAL, "archive radius must be > 0");
        if (!arc->theta || !arc->chi2 || !arc->count) return fail(SBLM_EINVAL, "the archive needs theta, chi2 and count");
        SBLM_TRY(st.arg(arc->theta, sizeof(double) * SBLM_NPAR * (size_t)n_lc * arc->size, false, true, &i_arc[0]));
        SBLM_TRY(st.arg(arc->chi2, sizeof(double) * (size_t)n_lc * arc->size, false, true, &i_arc[1]));
        SBLM_TRY(st.arg(arc->count, sizeof(int32_t) * (size_t)n_lc, false, true, &i_arc[2]));
        k_ag = st.scratch(sizeof(double) * SBLM_NPAR * (size_t)n_lc * arc->size);
    }
    SBLM_TRY(st.begin());
    // longest first (stable): the classic longest-processing-time order for the work queue
    std::vector<int> order(n_lc);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return off[x + 1] - off[x] > off[y + 1] - off[y]; });
    SBLM_CUDA(cudaMemcpyAsync(st.scratch_ptr(k_order), order.data(), sizeof(int) * n_lc, cudaMemcpyHostToDevice,
                              st.stream()));
    BatchArgs a{};
    a.t = static_cast<const double*>(st.dev(i_t));
    a.flux = static_cast<const double*>(st.dev(i_f));
    a.sigma = static_cast<const double*>(st.dev(i_s));
    a.offsets = static_cast<const int64_t*>(st.dev(i_o));
    a.order = static_cast<const int*>(st.scratch_ptr(k_order));
    a.n_lc = n_lc;
    a.b = b;
    a.c = c;
    a.n_gen = params->n_gen;
    a.G = G;
    a.n2 = n2;
    a.P = static_cast<double*>(st.scratch_ptr(k_P));
    a.keys = static_cast<uint64_t*>(st.scratch_ptr(k_keys));
    a.queue = static_cast<Deferred*>(st.scratch_ptr(k_q));
    a.qcap = qcap;
    a.term = static_cast<double*>(st.scratch_ptr(k_term));
    a.next = static_cast<unsigned*>(st.scratch_ptr(k_next));
    a.best_theta = static_cast<double*>(st.dev(*i_th));
    a.best_chi2 = static_cast<double*>(st.dev(*i_c));
    a.max_ep = max_ep;
    a.seed = i_seed >= 0 ? static_cast<const double*>(st.dev(i_seed)) : nullptr;
    a.n_seed = n_seed;
    a.polish_fev = params->polish_fev;
    a.polish_starts = starts;
    a.best_genes = static_cast<double*>(st.scratch_ptr(k_genes));
    a.blend = blend ? 1 : 0;
    a.f_min = SBLM_BLEND_F_MIN;
    a.A_scr = blend ? static_cast<double*>(st.scratch_ptr(k_A)) : nullptr;
    a.n_isl = n_isl;
    a.mig_every = std::max(0, params->migration_interval);
    a.isl_state = n_isl > 1 ? static_cast<sblm_ea_state*>(st.scratch_ptr(k_is)) : nullptr;
    a.isl_elite = n_isl > 1 ? static_cast<double*>(st.scratch_ptr(k_ie)) : nullptr;
    if (mon) {
        a.mon_theta = static_cast<const double*>(st.dev(i_mt));
        a.mon_f = i_mf >= 0 ? static_cast<const double*>(st.dev(i_mf)) : nullptr;
        a.mon_chi2 = static_cast<const double*>(st.dev(i_mc));
        a.mon_tol = mon->rel_tol;
        a.mon_first = static_cast<int*>(st.dev(*i_mon));
        a.f_scr = k_f >= 0 ? static_cast<double*>(st.scratch_ptr(k_f)) : nullptr;
    }
    if (arc) {
        a.arc_size = arc->size;
        a.arc_top = arc->top;
        a.arc_radius = arc->radius;
        a.arc_genes = static_cast<double*>(st.scratch_ptr(k_ag));
        a.arc_theta = static_cast<double*>(st.dev(i_arc[0]));
        a.arc_chi2 = static_cast<double*>(st.dev(i_arc[1]));
        a.arc_count = static_cast<int*>(st.dev(i_arc[2]));
    } else if (starts > 1) {  // an archive kept only for the polish starts: every evaluated row offered
        a.arc_size = arc_k;
        a.arc_top = 0;
        a.arc_radius = params->polish_radius;
        a.arc_genes = static_cast<double*>(st.scratch_ptr(k_iag));
        a.arc_theta = static_cast<double*>(st.scratch_ptr(k_iat));
        a.arc_chi2 = static_cast<double*>(st.scratch_ptr(k_iac));
        a.arc_count = static_cast<int*>(st.scratch_ptr(k_ian));
    }
    out->a = a;
    PolishArgs pa{};
    pa.t = a.t;
    pa.flux = a.flux;
    pa.sigma = a.sigma;
    pa.offsets = a.offsets;
    pa.n_lc = n_lc;
    pa.b = b;
    pa.g_in = a.best_genes;
    pa.g_stride = SBLM_NPAR;
    pa.c_in = a.best_chi2;
    pa.c_stride = 1;
    pa.g_out = a.best_genes;
    pa.c_out = a.best_chi2;
    if (starts > 1) {  // every archived start (up to polish_starts of them) into separate outputs
        pa.starts = inst_per_lc;
        pa.counts = a.arc_count;
        pa.max_starts = starts;
        pa.g_in = a.arc_genes;
        pa.c_in = a.arc_chi2;
        pa.g_out = static_cast<double*>(st.scratch_ptr(k_pg));
        pa.c_out = static_cast<double*>(st.scratch_ptr(k_pc));
    }
    pa.maxfev = params->polish_fev;
    pa.mixed = st.scratch_ptr(k_pq);
    pa.mx = pmx;
    pa.blend = blend ? 1 : 0;
    pa.f_min = SBLM_BLEND_F_MIN;
    pa.A_scr = blend && params->polish_fev > 0 ? static_cast<double*>(st.scratch_ptr(k_pA)) : nullptr;
    pa.A_stride = max_ep;
    out->pa = pa;
    out->polish_blocks = polish_blocks;
    out->max_ep = max_ep;
    out->blocks = blocks;
    out->threads = threads;
    out->smem = smem;
    out->mode = mode;
    return SBLM_OK;
}

sblm_status run_graph(const Prepared& p, cudaStream_t s) {
    // the cache key: every launch argument (the graph replays exactly this launch)
    std::vector<unsigned char> key(sizeof(BatchArgs) + sizeof(int) * 3 + sizeof(size_t));
    // (the polish arguments are all derived from BatchArgs, whose bytes the key holds)
    unsigned char* w = key.data();
    std::memcpy(w, &p.a, sizeof(BatchArgs));
    w += sizeof(BatchArgs);
    std::memcpy(w, &p.blocks, sizeof(int));
    std::memcpy(w + sizeof(int), &p.threads, sizeof(int));
    std::memcpy(w + 2 * sizeof(int), &p.mode, sizeof(int));
    std::memcpy(w + 3 * sizeof(int), &p.smem, sizeof(size_t));
    int dev = 0;
    SBLM_CUDA(cudaGetDevice(&dev));
    key.insert(key.end(), reinterpret_cast<unsigned char*>(&dev), reinterpret_cast<unsigned char*>(&dev) + sizeof dev);
    if (!g_graph.exec || g_graph.key != key) {
        if (g_graph.exec) {
            cudaGraphExecDestroy(g_graph.exec);
            g_graph.exec = nullptr;
        }
        SBLM_CUDA(launch_batch(p.mode, p.a, p.blocks, p.threads, p.smem, s, true));
        if (p.a.polish_fev > 0) SBLM_CUDA(polish_prepare(p.mode, p.max_ep));
        cudaStream_t cap;
        SBLM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = cudaMemsetAsync(p.a.next, 0, sizeof(unsigned), cap);
            cudaError_t e2 = launch_batch(p.mode, p.a, p.blocks, p.threads, p.smem, cap, false);
            if (e2 == cudaSuccess && p.a.polish_fev > 0) {
                e2 = launch_polish(p.mode, p.pa, p.polish_blocks, p.max_ep, cap);
                if (e2 == cudaSuccess && p.pa.starts > 1) {
                    pick_polished_kernel<<<(p.a.n_lc + 127) / 128, 128, 0, cap>>>(
                        p.pa.g_out, p.pa.c_out, p.a.n_lc, p.pa.starts, p.a.best_genes, p.a.best_chi2);
                    e2 = cudaGetLastError();
                }
                if (e2 == cudaSuccess) {
                    genes_to_theta_kernel<<<(p.a.n_lc + 127) / 128, 128, 0, cap>>>(p.a.best_genes, p.a.n_lc, p.a.b,
                                                                                 p.a.best_theta);
                    e2 = cudaGetLastError();
                }
            }
            e = cudaStreamEndCapture(cap, &graph);
            if (e == cudaSuccess && (e1 != cudaSuccess || e2 != cudaSuccess)) {
                cudaGraphDestroy(graph);
                e = e1 != cudaSuccess ? e1 : e2;
            }
        }
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return cuda_fail(e, "capturing the batched fit");
        e = cudaGraphInstantiate(&g_graph.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g_graph.exec = nullptr;
            return cuda_fail(e, "instantiating the batched fit graph");
        }
        g_graph.key = key;
    }
    SBLM_CUDA(cudaGraphLaunch(g_graph.exec, s));
    return SBLM_OK;
}

}  // namespace
}  // namespace sblm

using namespace sblm;

extern "C" sblm_status sblm_fit_batch_seeded(const double* t, const double* flux, const double* sigma,
                                             const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                             const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                                             const double* seed_genes, int32_t n_seed, double* best_theta,
                                             double* best_chi2, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    Staging st(s);
    int i_th, i_c;
    Prepared p;
    SBLM_TRY(prepare(t, flux, sigma, offsets, n_lc, bounds, params, tuning, n_seed > 0 ? seed_genes : nullptr, n_seed,
                     best_theta, best_chi2, st, &i_th, &i_c, &p));
    SBLM_TRY(run_graph(p, s));
    SBLM_TRY(st.end());
    SBLM_CUDA(cudaStreamSynchronize(s));
    return SBLM_OK;
}

extern "C" sblm_status sblm_fit_batch_archived(const double* t, const double* flux, const double* sigma,
                                               const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                               const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                                               const sblm_batch_archive* archive, double* best_theta,
                                               double* best_chi2, void* stream) {
    if (!archive) return fail(SBLM_EINVAL, "archive is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    Staging st(s);
    int i_th, i_c, i_arc[3];
    Prepared p;
    SBLM_TRY(prepare(t, flux, sigma, offsets, n_lc, bounds, params, tuning, nullptr, 0, best_theta, best_chi2, st,
                     &i_th, &i_c, &p, 0, nullptr, nullptr, nullptr, archive, i_arc));
    SBLM_TRY(run_graph(p, s));
    SBLM_TRY(st.end());
    SBLM_CUDA(cudaStreamSynchronize(s));
    return SBLM_OK;
}

extern "C" sblm_status sblm_fit_batch_tuned(const double* t, const double* flux, const double* sigma,
                                            const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                            const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                                            double* best_theta, double* best_chi2, void* stream) {
    return sblm_fit_batch_seeded(t, flux, sigma, offsets, n_lc, bounds, params, tuning, nullptr, 0, best_theta,
                                 best_chi2, stream);
}

extern "C" sblm_status sblm_fit_batch_monitored(const double* t, const double* flux, const double* sigma,
                                                const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                                const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                                                const float* weights, double seed_frac,
                                                const sblm_batch_monitor* monitor, double* best_theta,
                                                double* best_chi2, void* stream) {
    if (!(seed_frac >= 0.0 && seed_frac <= 1.0)) return fail(SBLM_EINVAL, "seed_frac must be in [0, 1]");
    if (!params) return fail(SBLM_EINVAL, "params is NULL");
    const int n_seed = weights ? (int)std::lround(seed_frac * params->n_pop) : 0;
    if (n_seed == 0 && !monitor)
        return sblm_fit_batch_seeded(t, flux, sigma, offsets, n_lc, bounds, params, tuning, nullptr, 0, best_theta,
                                     best_chi2, stream);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    Staging st(s);
    int i_th, i_c, k_inf = -1, i_w = -1, i_mon = -1;
    if (n_seed > 0) SBLM_TRY(st.arg(weights, sizeof(float) * cnn::kNParams, true, false, &i_w));
    Prepared p;
    SBLM_TRY(prepare(t, flux, sigma, offsets, n_lc, bounds, params, tuning, nullptr, n_seed, best_theta, best_chi2, st,
                     &i_th, &i_c, &p, n_seed > 0 ? cnn::infer_scratch_bytes(n_lc, n_seed) : 0,
                     n_seed > 0 ? &k_inf : nullptr, monitor, &i_mon));
    if (n_seed > 0) {
        const cnn::InferScratch sc = cnn::infer_scratch_carve(st.scratch_ptr(k_inf), n_lc, n_seed);
        SBLM_CUDA(cnn::launch_seed_rows(p.a.t, p.a.flux, p.a.sigma, p.a.offsets, n_lc,
                                        static_cast<const float*>(st.dev(i_w)), p.a.b, n_seed, params->seed, sc, s));
        p.a.prop_out = sc.out;
        p.a.prop_win = sc.window;
        p.a.prop_seed = params->seed;
        SBLM_TRY(cnn::check_timeout(s));
    }
    SBLM_TRY(run_graph(p, s));
    SBLM_TRY(st.end());
    SBLM_CUDA(cudaStreamSynchronize(s));
    return SBLM_OK;
}

extern "C" sblm_status sblm_fit_batch(const double* t, const double* flux, const double* sigma,
                                      const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                      const sblm_ea_params* params, double* best_theta, double* best_chi2,
                                      void* stream) {
    return sblm_fit_batch_tuned(t, flux, sigma, offsets, n_lc, bounds, params, nullptr, best_theta, best_chi2,
                                stream);
}

extern "C" sblm_status sblm_autotune_batch(const double* t, const double* flux, const double* sigma,
                                           const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                           const sblm_ea_params* params, int32_t trial_generations,
                                           sblm_batch_tuning* best, double* best_ms, void* stream) {
    if (!params || !best) return fail(SBLM_EINVAL, "params and best are required");
    if (trial_generations < 1) return fail(SBLM_EINVAL, "trial_generations must be >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    sblm_ea_params p = *params;
    p.n_gen = trial_generations;
    std::vector<double> th(6 * (size_t)n_lc), ch(n_lc);
    const int groups[] = {8, 16, 32};
    const int blocks[] = {256, 512};
    double best_t = INFINITY;
    sblm_batch_tuning best_cfg{16, 512};
    for (int bl : blocks) {
        for (int gr : groups) {
            sblm_batch_tuning cfg{gr, bl};
            // warm (builds the graph), then time one replay
            SBLM_TRY(sblm_fit_batch_tuned(t, flux, sigma, offsets, n_lc, bounds, &p, &cfg, th.data(), ch.data(), stream));
            cudaEvent_t e0, e1;
            SBLM_CUDA(cudaEventCreate(&e0));
            SBLM_CUDA(cudaEventCreate(&e1));
            SBLM_CUDA(cudaEventRecord(e0, s));
            SBLM_TRY(sblm_fit_batch_tuned(t, flux, sigma, offsets, n_lc, bounds, &p, &cfg, th.data(), ch.data(), stream));
            SBLM_CUDA(cudaEventRecord(e1, s));
            SBLM_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            SBLM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (ms < best_t) {
                best_t = ms;
                best_cfg = cfg;
            }
        }
    }
    *best = best_cfg;
    if (best_ms) *best_ms = best_t;
    return SBLM_OK;
}

extern "C" sblm_status sblm_fit_batch_cnn(const double* t, const double* flux, const double* sigma,
                                          const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                          const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                                          const float* weights, double seed_frac, double* best_theta,
                                          double* best_chi2, void* stream) {
    return sblm_fit_batch_monitored(t, flux, sigma, offsets, n_lc, bounds, params, tuning, weights, seed_frac, nullptr,
                                    best_theta, best_chi2, stream);
}
