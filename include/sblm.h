/*
 * sblm.h -- C ABI of the GB300 (sm_103a) library for fitting static binary-lens (SBLM)
 * point-source microlensing lightcurves with the evolutionary algorithm of
 * Rajpaul (2012), "Evolutionary algorithm-based analysis of gravitational microlensing
 * lightcurves".
 *
 * Conventions shared by every call
 * --------------------------------
 * - Parameter rows theta = (t0, tE, u0, alpha, d, q): t0 = t_m (time of closest approach to the
 *   primary, days), tE = t_E (Einstein crossing time, days), u0 = b (impact parameter), alpha =
 *   theta (angle of the impact vector to the +x axis, radians), d = a (lens separation) and q
 *   (mass ratio), lengths in units of the primary's Einstein angle, primary at the origin,
 *   secondary on the +x axis (Section 2.1). Rows are stored row-major, 6 doubles each.
 * - Fit genes are (t0, tE, u0, alpha, d, log10 q), each encoded to [0, 1] by the linear map of
 *   Eq. (EMMA-encoding) over the bounds [lo_j, hi_j].
 * - Pointers may address device memory or host memory (pageable or pinned); the library finds
 *   out which with cudaPointerGetAttributes. Host buffers are copied through an internal
 *   per-device workspace on `stream`, and a call that touched host memory synchronises `stream`
 *   before it returns. A call whose buffers are all on the device is asynchronous on `stream`
 *   unless its description says otherwise.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). All work runs on
 *   the current CUDA device of the calling thread.
 * - The caller owns every buffer it passes. The library owns only its workspace, allocated
 *   lazily per device, grown on demand and kept until process exit; calls that use it are
 *   serialised by an internal lock.
 * - Errors are returned, never thrown: arguments are checked on the host before any launch
 *   (SBLM_EINVAL), CUDA failures map to SBLM_ECUDA, and sblm_last_error() describes the most
 *   recent failure of the calling thread.
 */
#ifndef SBLM_H
#define SBLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SBLM_OK = 0,
    SBLM_EINVAL = 1,   /* bad argument: size, pointer, bound, sigma <= 0, non-finite data */
    SBLM_ENOMEM = 2,   /* workspace allocation failed */
    SBLM_ECUDA = 3,    /* a CUDA runtime call or launch failed */
    SBLM_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    SBLM_ENUMERIC = 5  /* non-finite result where a finite one was required */
} sblm_status;

/* Arithmetic of the forward model. */
enum {
    SBLM_FP64 = 0,  /* everything in FP64 */
    SBLM_MIXED = 1, /* FP32 quintic solve; FP64 re-solve and polish of an epoch when triggered
                       (|det J| < 3e-2 at an image or at a rejected root that nearly solves
                       the lens equation, two roots closer than 1e-4, or an ambiguous image
                       classification); chi^2 accumulated in FP64 */
    SBLM_FP32 = 2   /* FP32 solve, no FP64 re-solve; chi^2 accumulated in FP64 */
};

/* OR-ed into sblm_ea_params.precision of the batched fitters (sblm_fit_batch*), or into the
 * precision argument of sblm_polish_batch: each candidate's chi^2 is that of the blended model
 * f A + (1 - f) (Section 4.4, Eq. blend; flux normalised to the baseline) with f profiled out as
 * in sblm_chi2_blend, so best_chi2 / chi2_out hold that chi^2 and the six returned parameters
 * are those of the lens; sblm_chi2_blend on them gives f. Needs 8 bytes of device scratch per
 * epoch per population row per SM. The single-lightcurve calls (sblm_fit, sblm_ea_*) reject it
 * with SBLM_EINVAL. */
#define SBLM_BLEND 16
#define SBLM_BLEND_F_MIN 1e-3 /* smallest profiled blending fraction */

#define SBLM_NPAR 6        /* SBLM genes */
#define SBLM_MAX_NPAR 16   /* largest N_par accepted by the generic EA calls */
#define SBLM_MAX_WINDOW 15 /* largest stagnation window */

/* Parameter domains [lo_j, hi_j] of Eq. (EMMA-encoding): genes t0, tE, u0, alpha, d, log10 q. */
typedef struct {
    double lo[SBLM_NPAR];
    double hi[SBLM_NPAR];
} sblm_bounds;

/* Control parameters of the EA (Appendix A); sblm_ea_params_default() fills the paper's. */
typedef struct {
    int32_t n_pop;         /* N_pop >= 2 (paper default 1000) */
    int32_t n_gen;         /* N_gen >= 1 fitness evaluations of the population */
    double p_mut0;         /* starting jump-mutation probability (paper default 0.01) */
    int32_t n_tourn;       /* tournament size; 0 -> ceil(N_pop / 25) (paper default) */
    int32_t stag_window;   /* generations of the stagnation test (10), 1..SBLM_MAX_WINDOW */
    double stag_rel;       /* stagnant if the best improved by <= stag_rel over the window (0.01) */
    int32_t restart_after; /* consecutive stagnant generations before a restart (10) */
    int32_t precision;     /* SBLM_FP64, SBLM_MIXED or SBLM_FP32 for the fitness evaluation */
    int32_t polish_fev;    /* amoeba fine-tuning of the fittest solution after the EA (Section 4.1,
                              "EA with amoeba"): at most this many chi^2 evaluations of a
                              downhill-simplex search in the genes (sblm_fit, sblm_fit_batch*);
                              0 = the EA alone (default) */
    uint64_t seed;         /* Philox4x64-10 key word 0; key word 1 is the population's stream id */
    int32_t n_islands;     /* island EA of Section 5.3 (batched fitters only): populations per
                              lightcurve, each of n_pop rows, evolved side by side; <= 1 = one
                              population (the paper's experiments, default). Island i of
                              lightcurve l draws on stream id l + i * n_lc. */
    int32_t migration_interval; /* with islands: every this many generations the elite of island i
                              replaces the last row of island (i + 1) mod n_islands (a ring);
                              <= 0 = islands never exchange rows (independent restarts) */
    int32_t polish_starts; /* batched fitters with polish_fev > 0: the amoeba starts from the
                              polish_starts fittest mutually distinct solutions the EA evaluated
                              (the archive rule of sblm_batch_archive, radius polish_radius) and the
                              best result is returned; 1 = the fittest solution only, as in the
                              paper (default); at most 64 */
    double polish_radius;  /* distinctness radius of those starts in the genes (default 0.05) */
} sblm_ea_params;

/* Dynamic state of one population between generations (Appendix A, "Stagnation checks"). */
typedef struct {
    double p_mut;                         /* current jump probability */
    double best_chi2;                     /* best fitness ever evaluated (archive across restarts) */
    double hist[SBLM_MAX_WINDOW + 1];     /* best chi^2 of the last stag_window + 1 generations */
    int32_t n_hist;                       /* entries of hist in use (generations since (re)start) */
    int32_t stag_run;                     /* consecutive stagnant generations */
    int32_t n_restarts;                   /* restarts so far */
    int32_t generation;                   /* generations completed */
    double best_genes[SBLM_MAX_NPAR];     /* encoded genes of best_chi2 */
} sblm_ea_state;

/* Human-readable name of a status code (static storage). */
const char* sblm_status_str(sblm_status s);

/* Description of the calling thread's most recent failure ("" if none). */
const char* sblm_last_error(void);

/* Fill *p with the paper's defaults: N_pop 1000, N_gen 100, p_mut0 0.01, N_tourn ceil(N_pop/25),
 * window 10, 1%, restart after 10, SBLM_MIXED, seed 0; one population (n_islands 1, migration
 * interval 20 if islands are asked for); the amoeba (when asked for) from the fittest solution
 * only (polish_starts 1, polish_radius 0.05). */
void sblm_ea_params_default(sblm_ea_params* p);

/*
 * Point-source magnification, Section 2.2: for every (candidate c, epoch k), the source position
 * of Eq. (sourcePos), the five roots of the quintic of Eq. (lensingPoly), rejection of the roots
 * that do not solve Eq. (lensing), and A = sum_i 1/|det J_i| over the images,
 * det J = 1 - |1/z^2 + q/(d - z)^2|^2.
 *   theta  [n_cand * 6]     parameter rows (see conventions), q > 0, d > 0, tE > 0
 *   t      [n_ep]           epochs in days; ascending order is fastest (roots are carried
 *                           from one epoch to the next) but not required
 *   A_out  [n_cand * n_ep]  row-major, written as FP64 whatever the precision
 *   flags  [n_cand * n_ep]  optional (NULL to skip): bit 0 = classification fell back to the
 *                           3 (or 5) smallest residuals, bit 1 = an FP64 re-solve ran (MIXED),
 *                           bit 2 = the root iteration hit its cap, bit 3 = a rejected root was
 *                           nearly an image (FP32: a close image pair may be unresolved), bit 4 =
 *                           an image (or a rejected root with a relative lens-equation residual
 *                           below 0.05) has |det J| < 3e-2, bit 5 = two images closer than 1e-4
 *                           (bits 4-5: FP32 and MIXED; in MIXED any of bits 0 and 2-5 of the FP32
 *                           solution triggers the FP64 re-solve, and they stay set beside bit 1)
 * n_cand >= 0, n_ep >= 0 (zero sizes return SBLM_OK without a launch). Host theta rows are checked
 * (finite, tE, d, q > 0); device rows are not, and an invalid row yields NaN or garbage in its
 * own outputs only.
 */
sblm_status sblm_magnification(const double* theta, int32_t n_cand, const double* t, int32_t n_ep,
                               double* A_out, uint8_t* flags, int32_t precision, void* stream);

/*
 * chi^2 of every candidate against one lightcurve (Section 4.1):
 * chi2_out[c] = sum_k ((flux_k - A_ck) / sigma_k)^2, A as in sblm_magnification, the model flux
 * of a unit, unblended source. The sum runs in FP64-grade arithmetic in every precision (FP32
 * modes accumulate each thread's epochs as a float pair) and in a fixed order, so FP64 and FP32
 * results are deterministic; in MIXED the terms of the epochs re-solved in FP64 are added
 * atomically, so the last bits of a MIXED chi^2 can vary from run to run. sigma_k > 0 and finite data are required: host buffers are checked
 * (SBLM_EINVAL); device buffers are not read back for a check, and bad data there turn into
 * non-finite chi^2 values (which the EA ranks last). n_ep == 0 gives chi^2 = 0.
 */
sblm_status sblm_chi2(const double* theta, int32_t n_cand, const double* t, const double* flux,
                      const double* sigma, int32_t n_ep, double* chi2_out, int32_t precision,
                      void* stream);

/*
 * Fitness of an encoded population (Appendix A, step (a): decode P -> A by Eq. (EMMA-encoding),
 * then the external fitness function): row i of P [n_pop * 6] holds genes in [0, 1] that decode
 * to a_j = lo_j + (hi_j - lo_j) p_ij over `bounds`, gene 5 being log10 q; chi2_out[i] is then
 * computed exactly as sblm_chi2 would for the decoded row. `bounds` is a host struct. The decode
 * runs inside the forward kernel.
 */
sblm_status sblm_chi2_genes(const double* P, int32_t n_pop, const sblm_bounds* bounds, const double* t,
                            const double* flux, const double* sigma, int32_t n_ep, double* chi2_out,
                            int32_t precision, void* stream);

/*
 * Initialisation of a population (Appendix A, "Initialisation"): half the elements of
 * P [n_pop * n_par] (row-major, encoded genes in [0, 1]) get X ~ U(0,1), the other half the
 * complement 1 - X of another random element, paired through a Philox-keyed permutation.
 * `state` (host or device, one sblm_ea_state) is reset: p_mut = p_mut0, empty window, no best.
 * Random numbers: Philox4x64-10, key (params->seed, stream_id), counter (generation 0, ...).
 */
sblm_status sblm_ea_init(double* P, int32_t n_pop, int32_t n_par, const sblm_ea_params* params,
                         uint64_t stream_id, sblm_ea_state* state, void* stream);

/*
 * Everything of one generation after the fitness evaluation (Appendix A, steps (b)-(f)):
 * rank the rows of P by chi2 (stable, NaN last), archive the best ever, tournament selection,
 * reproduction by Eq. (rep1)/(rep2) with a per-pairing weighting matrix, elitism (row 0 keeps
 * the fittest row, unmutated), creep then jump mutation of the N_pop - 1 offspring, and the
 * stagnation check (boost or throttle p_mut; re-initialise after repeated stagnation).
 *   P     [n_pop * n_par]  in: P(t) as evaluated; out: P(t+1)
 *   chi2  [n_pop]          fitness of the rows of P(t) (lower is fitter)
 *   generation             t, the Philox counter word 0 of this generation's draws
 * Problem-agnostic: any fitness computed by the caller can drive it ("external fitness
 * function", Appendix A).
 */
sblm_status sblm_ea_generation(double* P, const double* chi2, int32_t n_pop, int32_t n_par,
                               const sblm_ea_params* params, uint64_t stream_id,
                               int32_t generation, sblm_ea_state* state, void* stream);

/*
 * sblm_ea_generation for n_pops independent populations at once (no counterpart in the paper: a
 * throughput form of Appendix A's generation for callers that evolve many populations, e.g. one
 * per lightcurve, from the host). P [n_pops * n_pop * n_par], chi2 [n_pops * n_pop] and states
 * [n_pops] hold the populations back to back; population b uses stream id stream_id0 + b and is
 * ranked by its own block, all in one launch of each operator kernel. The results equal n_pops
 * calls of sblm_ea_generation (population b with stream id stream_id0 + b). 1 <= n_pops <= 65535.
 */
sblm_status sblm_ea_generation_batch(double* P, const double* chi2, int32_t n_pops, int32_t n_pop,
                                     int32_t n_par, const sblm_ea_params* params, uint64_t stream_id0,
                                     int32_t generation, sblm_ea_state* states, void* stream);

/*
 * sblm_ea_generation without any allocation. The paper has no counterpart: this is a library
 * convenience for callers that must not allocate device memory while they run, for example a
 * pipeline that reserves all of its GPU memory up front and may not grow it later, or a host
 * thread that cannot afford the device-wide synchronisation that cudaMalloc and cudaFree can
 * imply. The computation and its results are those of sblm_ea_generation; the differences:
 * - its scratch lives in one fixed device array compiled into the library (544 KiB plus
 *   256 bytes, held on every GPU that loads the library until the process exits), so
 *   n_pop <= 8192 and n_pop * n_par <= 32768; larger sizes return SBLM_EINVAL;
 * - P, chi2 and state must be device memory (host memory returns SBLM_EINVAL, since staging it
 *   would need a workspace); the call is asynchronous on `stream` and allocates nothing;
 * - the first call on a device looks the array's device address up (cudaGetSymbolAddress, with
 *   that device current); make that first call before any stream capture;
 * - every call shares the one array, which keeps the last call's contents (nothing in it has to
 *   start at zero), so calls that overlap on the GPU (other streams, other host threads on the
 *   same device) race: order them on one stream or synchronise between them;
 * - the looked-up address is cached per device for the life of the process and does not
 *   survive cudaDeviceReset of that device: after such a reset, do not call this entry point
 *   again in the same process.
 */
sblm_status sblm_ea_generation_noalloc(double* P, const double* chi2, int32_t n_pop, int32_t n_par,
                                       const sblm_ea_params* params, uint64_t stream_id,
                                       int32_t generation, sblm_ea_state* state, void* stream);

/*
 * Fit the SBLM to one lightcurve (the paper's problem statement: data, parameter domains,
 * population size, generation budget -> best-fit parameters and their chi^2). Runs the whole
 * evolutionary sequence of Appendix A on the device: N_gen evaluations of the population with
 * the forward model of sblm_chi2 in params->precision, the operators of sblm_ea_generation in
 * between. Synchronous: returns when best_theta (6 doubles: t0, tE, u0, alpha, d, q) and
 * *best_chi2 are written; they may be host or device pointers. Optional `trace`
 * [n_gen * 4] doubles (host or device, NULL to skip): per generation the best chi^2 of the
 * population, p_mut used for its offspring, restarts so far, and the best chi^2 ever.
 */
sblm_status sblm_fit(const double* t, const double* flux, const double* sigma, int32_t n_ep,
                     const sblm_bounds* bounds, const sblm_ea_params* params, double* best_theta,
                     double* best_chi2, double* trace, void* stream);

/* Launch shape of the persistent batched fitter (sblm_autotune_batch picks one). */
typedef struct {
    int32_t group; /* threads per candidate: 1, 2, 4, 8, 16 or 32 (0: default 16) */
    int32_t block; /* threads per block: a multiple of 32 up to 512 (0: default 512) */
} sblm_batch_tuning;

/*
 * Fit n_lc lightcurves of uneven length at once: lightcurve i owns epochs
 * [offsets[i], offsets[i+1]) of the concatenated t, flux, sigma arrays (offsets [n_lc + 1],
 * int64, offsets[0] = 0, non-decreasing, each lightcurve at least 1 epoch). Every lightcurve
 * gets its own population (stream id i) and the full sequence of Appendix A, all inside one
 * persistent launch. Synchronous; best_theta [n_lc * 6], best_chi2 [n_lc].
 */
sblm_status sblm_fit_batch(const double* t, const double* flux, const double* sigma,
                           const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                           const sblm_ea_params* params, double* best_theta, double* best_chi2,
                           void* stream);

/*
 * sblm_fit_batch with an explicit launch shape (NULL: the defaults). Details of the batched
 * fitter: one persistent block per SM takes lightcurves, longest first, from a work counter and
 * runs every generation of one lightcurve's fit itself (the lightcurve staged in shared memory,
 * so n_pop and the longest lightcurve must fit 200 KB of it: with n_pop = 1024 that is about
 * 7,600 epochs in FP64 and 11,000 in FP32/MIXED; SBLM_EINVAL otherwise). The launch is captured in
 * a CUDA graph the first time and replayed while every argument (pointers included) repeats.
 * Results are those of sblm_fit on each lightcurve with stream id = the lightcurve's index,
 * except that the evaluation's launch shape differs (chi^2 agree to rounding).
 */
sblm_status sblm_fit_batch_tuned(const double* t, const double* flux, const double* sigma,
                                 const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                 const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                                 double* best_theta, double* best_chi2, void* stream);

/*
 * Autotuner of the batched fitter (not part of the paper's method): times `trial_generations`
 * generations of the given batch for each launch shape in {8, 16, 32} threads per candidate x
 * {256, 512} threads per block and returns the fastest in *best (and its time in *best_ms, may
 * be NULL). The Python binding keeps a JSON cache of the results keyed by the workload's shape.
 */
sblm_status sblm_autotune_batch(const double* t, const double* flux, const double* sigma,
                                const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                const sblm_ea_params* params, int32_t trial_generations,
                                sblm_batch_tuning* best, double* best_ms, void* stream);

/*
 * Success monitor of the batched fitter (sblm_fit_batch_monitored): an evaluation instrument for
 * synthetic lightcurves whose parameters are known. Section 4.2 counts a fitting run as
 * successful when it returned at least one model with delta chi^2 / nu < 1 and every parameter
 * within 10% of the injected one, and the EA of Appendix A returns, by default, every population
 * of every generation. Instead of writing that history out (n_gen x n_pop rows per lightcurve),
 * the fitter tests each evaluated row as it is produced: chi^2 < chi2_max[l] and every parameter
 * within rel_tol of theta_ref[l] (t0 relative to the reference tE, alpha as a wrapped difference
 * relative to 2 pi, tE, u0, d and q relative to their reference values; with SBLM_BLEND and
 * f_ref given, also the profiled f relative to f_ref[l]). The monitor never steers the search.
 */
typedef struct {
    const double* theta_ref; /* [n_lc * 6] reference parameters (t0, tE, u0, alpha, d, q) */
    const double* f_ref;     /* [n_lc] reference blending fractions, or NULL */
    const double* chi2_max;  /* [n_lc] chi^2 bound (strict) */
    double rel_tol;          /* parameter tolerance, > 0 (0.1 in the paper) */
    int32_t* first_gen;      /* [n_lc] out: first generation with a matching row, -1 if none */
} sblm_batch_monitor;

/*
 * Several solutions per lightcurve (sblm_fit_batch_archived). Section 3.1 obtains multiple
 * solutions of a problem by keeping the explored phenotypes that meet a fitness criterion, and
 * Appendix A's EA returns every population. The fitter keeps, per lightcurve, the `size` fittest
 * mutually distinct solutions among the rows it evaluates: two rows are the same solution when
 * every encoded gene differs by at most `radius`. Each generation the `top` fittest rows of every
 * population (all rows when top = 0) are offered in rank order: a row that matches an archived
 * solution replaces it when its chi^2 is lower (the archive then drops the entries that now match
 * it) and is dropped otherwise; a new solution enters while there is room, or in place of the
 * least fit one when it is fitter; rows with a non-finite chi^2 are never archived. Entries are
 * kept sorted by chi^2 (ties in arrival order), so the first is the EA's best (before the amoeba
 * polish, which only refines the returned best).
 */
typedef struct {
    int32_t size;     /* solutions kept per lightcurve, 1..64 */
    int32_t top;      /* rows offered per population and generation (0: all) */
    double radius;    /* distinctness radius in the encoded genes (in [0, 1]), > 0 */
    double* theta;    /* [n_lc * size * 6] out: (t0, tE, u0, alpha, d, q); unused entries NaN */
    double* chi2;     /* [n_lc * size] out: their chi^2 (unused: NaN) */
    int32_t* count;   /* [n_lc] out: solutions kept */
} sblm_batch_archive;

/*
 * sblm_fit_batch_tuned plus the solution archive above (archive must not be NULL; its arrays follow
 * the pointer rules of the other arguments and are written when the call returns). With FP64 the
 * archive equals what offering each generation's ranked population to the archive rule gives.
 */
sblm_status sblm_fit_batch_archived(const double* t, const double* flux, const double* sigma,
                                    const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                    const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                                    const sblm_batch_archive* archive, double* best_theta, double* best_chi2,
                                    void* stream);

/*
 * chi^2 of the blended model of Section 4.4 (Eq. blend), A_obs = f A + (1 - f), for each
 * parameter row, with the blending fraction profiled out: the paper notes its least-squares value
 * follows from a linear equation. With a_k = A_k - 1, b_k = F_k - 1 and w_k = 1/sigma_k^2,
 * f = sum w a b / sum w a^2 clamped to [SBLM_BLEND_F_MIN, 1] (f = 1 when sum w a^2 = 0), and
 * chi^2 = sum w (b - f a)^2; the sums run per candidate in FP64, in a fixed order (one warp per
 * candidate, epochs strided over its lanes, then a shuffle tree), so results are reproducible.
 * A is computed as by sblm_magnification in `precision` (SBLM_FP64, SBLM_MIXED or SBLM_FP32).
 *   chi2_out [n_cand]; f_out [n_cand] (may be NULL). n_ep = 0 gives chi^2 = 0 and f = 1.
 *   Uses n_cand * n_ep * 8 bytes of device scratch. Errors: SBLM_EINVAL for negative sizes,
 *   NULL buffers, an unknown precision or non-finite host inputs.
 */
sblm_status sblm_chi2_blend(const double* theta, int32_t n_cand, const double* t, const double* flux,
                            const double* sigma, int32_t n_ep, double* chi2_out, double* f_out,
                            int32_t precision, void* stream);

/*
 * Amoeba fine-tuning (Section 4.1: the EA "with amoeba"; Nelder & Mead 1965 with the standard
 * coefficients of Lagarias et al. 1998) of given solutions: for each lightcurve (layout of
 * sblm_fit_batch), a downhill-simplex search in the genes over `bounds` starting from
 * genes_in[l] (6 genes in [0, 1]): start simplex x0 + 0.03 e_j (-0.03 where that leaves [0, 1]),
 * reflection 1, expansion 2, contraction 1/2, shrink 1/2, trial points clamped to [0, 1], the
 * simplex rebuilt around its best vertex whenever it has collapsed to 1e-9, stopped after
 * `maxfev` chi^2 evaluations (a step in progress may take up to 6 more). The chi^2 is that of
 * sblm_chi2_genes in `precision` (| SBLM_BLEND: of the blended model). genes_out [n_lc * 6] (may alias genes_in) receives the best
 * vertex, chi2_out [n_lc] its chi^2. The longest lightcurve must fit 200 KB of shared memory
 * (24 bytes per epoch in FP64, 16 otherwise). 0 <= maxfev <= 2^20.
 */
sblm_status sblm_polish_batch(const double* t, const double* flux, const double* sigma,
                              const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                              const double* genes_in, int32_t maxfev, int32_t precision,
                              double* genes_out, double* chi2_out, void* stream);

/*
 * Measured FMA throughput of the current device, in TFLOP/s (an FMA counts as 2 flop): eight
 * independent FMA chains per thread over 8 blocks of 256 threads per SM, timed with CUDA events.
 * Not part of the method: these are the denominators of the ALU roofline that the benchmark
 * reports for the forward model. Synchronous; uses the workspace.
 */
sblm_status sblm_peak_rates(double* fp32_tflops, double* fp64_tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SBLM_H */
