// fit.cu -- sblm_fit: the whole evolutionary sequence of Appendix A for one lightcurve on the
// device. Per generation: the forward model over the population (all SMs), then the ranking
// block and the offspring kernel; the host only enqueues.
#include <cmath>
#include <cstring>
#include <vector>

#include "ea_launch.cuh"
#include "forward_launch.cuh"
#include "polish_launch.cuh"
#include "runtime.cuh"

namespace sblm {

namespace {

// best genes of the archive -> theta (t0, tE, u0, alpha, d, q) and chi^2
__global__ void finish_kernel(const sblm_ea_state* __restrict__ state, Bounds b, double* __restrict__ theta,
                              double* __restrict__ chi2) {
    if (threadIdx.x != 0) return;
    double a[SBLM_NPAR];
    for (int j = 0; j < SBLM_NPAR; ++j) a[j] = b.lo[j] + (b.hi[j] - b.lo[j]) * state->best_genes[j];
    for (int j = 0; j < 5; ++j) theta[j] = a[j];
    theta[5] = exp10(a[5]);
    *chi2 = state->best_chi2;
}

// cache key of a single-lightcurve fit: every value its launches depend on, field by field
template <typename V>
void put(std::vector<unsigned char>& k, const V& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    k.insert(k.end(), p, p + sizeof(V));
}

std::vector<unsigned char> fit_graph_key(const EAConst& c, const ForwardArgs& fa, int n_gen, const double* tr,
                                         const double* th, const double* chi, const double* P0, int polish_fev,
                                         const void* polish_mixed) {
    std::vector<unsigned char> k;
    put(k, c.n_pop), put(k, c.n_par), put(k, c.n_tourn), put(k, c.stag_window), put(k, c.restart_after);
    put(k, c.p_mut0), put(k, c.stag_rel), put(k, c.seed), put(k, c.stream);
    put(k, fa.t), put(k, fa.flux), put(k, fa.sigma), put(k, fa.n_ep), put(k, fa.n_cand), put(k, fa.mode);
    put(k, fa.G), put(k, fa.chi2_out), put(k, fa.mixed), put(k, polish_mixed);
    for (int j = 0; j < SBLM_NPAR; ++j) put(k, fa.bounds.lo[j]), put(k, fa.bounds.hi[j]);
    put(k, n_gen), put(k, tr), put(k, th), put(k, chi), put(k, P0);
    put(k, polish_fev);
    int dev = 0;
    cudaGetDevice(&dev);
    put(k, dev);
    return k;
}

}  // namespace

sblm_status check_bounds(const sblm_bounds* b, Bounds* out) {
    if (!b) return fail(SBLM_EINVAL, "bounds is NULL");
    for (int j = 0; j < SBLM_NPAR; ++j) {
        if (!std::isfinite(b->lo[j]) || !std::isfinite(b->hi[j]) || !(b->lo[j] < b->hi[j]))
            return fail(SBLM_EINVAL, "bounds of gene %d must be finite with lo < hi", j);
        out->lo[j] = b->lo[j];
        out->hi[j] = b->hi[j];
    }
    if (!(b->lo[1] > 0)) return fail(SBLM_EINVAL, "tE bounds must be positive");
    if (!(b->lo[4] > 0)) return fail(SBLM_EINVAL, "d bounds must be positive");
    return SBLM_OK;
}

}  // namespace sblm

using namespace sblm;

extern "C" sblm_status sblm_fit(const double* t, const double* flux, const double* sigma, int32_t n_ep,
                                const sblm_bounds* bounds, const sblm_ea_params* params, double* best_theta,
                                double* best_chi2, double* trace, void* stream) {
    EAConst c;
    SBLM_TRY(ea_const(params, params ? params->n_pop : 0, SBLM_NPAR, 0, &c));
    if (params->n_gen < 1) return fail(SBLM_EINVAL, "n_gen must be >= 1");
    if (params->n_islands > 1) return fail(SBLM_EINVAL, "islands are run by the batched fitters (sblm_fit_batch*)");
    if (n_ep < 1) return fail(SBLM_EINVAL, "n_ep must be >= 1");
    if (!best_theta || !best_chi2) return fail(SBLM_EINVAL, "best_theta and best_chi2 are required");
    Bounds b;
    SBLM_TRY(check_bounds(bounds, &b));
    const int polish_fev = params->polish_fev;
    if (polish_fev < 0 || polish_fev > kPolishMaxFev)
        return fail(SBLM_EINVAL, "polish_fev must be in [0, %d]", kPolishMaxFev);
    if (polish_fev > 0 && polish_smem_bytes(params->precision, n_ep) > kPolishSmemBudget)
        return fail(SBLM_EINVAL, "the amoeba polish stages at most %zu bytes of epochs (n_ep=%d)", kPolishSmemBudget, n_ep);
    const int n_pop = c.n_pop, n_gen = params->n_gen, m = n_pop * SBLM_NPAR;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    Staging st(s);
    int i_t, i_f, i_s, i_th, i_c, i_tr;
    SBLM_TRY(st.arg(t, sizeof(double) * n_ep, true, false, &i_t));
    SBLM_TRY(st.arg(flux, sizeof(double) * n_ep, true, false, &i_f));
    SBLM_TRY(st.arg(sigma, sizeof(double) * n_ep, true, false, &i_s));
    SBLM_TRY(st.arg(best_theta, sizeof(double) * 6, false, true, &i_th));
    SBLM_TRY(st.arg(best_chi2, sizeof(double), false, true, &i_c));
    SBLM_TRY(st.arg(trace, trace ? sizeof(double) * 4 * (size_t)n_gen : 0, false, true, &i_tr));
    bool d1, d2, d3;
    SBLM_TRY(is_device_pointer(t, &d1));
    SBLM_TRY(is_device_pointer(flux, &d2));
    SBLM_TRY(is_device_pointer(sigma, &d3));
    if (!d1 && !d2 && !d3) SBLM_TRY(check_lightcurve_host(t, flux, sigma, n_ep));
    const int k_P0 = st.scratch(sizeof(double) * m);
    const int k_P1 = st.scratch(sizeof(double) * m);
    const int k_chi = st.scratch(sizeof(double) * n_pop);
    const int k_order = st.scratch(sizeof(int) * n_pop);
    const int k_ctrl = st.scratch(sizeof(EACtrl));
    const int k_keys = st.scratch(sizeof(uint64_t) * m);
    const int k_state = st.scratch(sizeof(sblm_ea_state));
    const int G = choose_group(n_pop, n_ep);
    const bool mixed = params->precision == SBLM_MIXED;
    const int k_mx = st.scratch(mixed ? mixed_scratch_bytes(n_pop, n_ep, true) : 0);
    const PolishMixed pmx = polish_mixed_layout(n_ep);
    const int k_pmx = st.scratch(mixed && polish_fev > 0 ? pmx.block_bytes : 0);
    SBLM_TRY(st.begin());

    double* P[2] = {static_cast<double*>(st.scratch_ptr(k_P0)), static_cast<double*>(st.scratch_ptr(k_P1))};
    double* chi = static_cast<double*>(st.scratch_ptr(k_chi));
    int* order = static_cast<int*>(st.scratch_ptr(k_order));
    EACtrl* ctrl = static_cast<EACtrl*>(st.scratch_ptr(k_ctrl));
    uint64_t* keys = static_cast<uint64_t*>(st.scratch_ptr(k_keys));
    sblm_ea_state* state = static_cast<sblm_ea_state*>(st.scratch_ptr(k_state));
    double* tr = static_cast<double*>(st.dev(i_tr));

    ForwardArgs fa{};
    fa.from_genes = true;
    fa.bounds = b;
    fa.n_cand = n_pop;
    fa.t = static_cast<const double*>(st.dev(i_t));
    fa.flux = static_cast<const double*>(st.dev(i_f));
    fa.sigma = static_cast<const double*>(st.dev(i_s));
    fa.n_ep = n_ep;
    fa.chi2_out = chi;
    fa.mode = params->precision;
    fa.G = G;
    fa.mixed = st.scratch_ptr(k_mx);
    void* polish_mixed = st.scratch_ptr(k_pmx);

    double* th_out = static_cast<double*>(st.dev(i_th));
    double* chi_out = static_cast<double*>(st.dev(i_c));
    // the whole sequence: ~3 launches per generation, captured once into a CUDA graph and
    // replayed while the arguments repeat (the host only launches the graph)
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t e = launch_init(c, 0, keys, P[0], q);
        if (e == cudaSuccess) e = launch_state_reset(c, state, q);
        int cur = 0;
        for (int g = 0; g < n_gen && e == cudaSuccess; ++g) {
            fa.src = P[cur];
            e = launch_forward(fa, q);
            const bool produce = g + 1 < n_gen;
            if (e == cudaSuccess)
                e = launch_rank(c, g, chi, P[cur], state, order, ctrl, keys, tr ? tr + 4 * (size_t)g : nullptr,
                                produce, q);
            if (e == cudaSuccess && produce) {
                e = launch_offspring(c, g, P[cur], order, ctrl, keys, P[cur ^ 1], q);
                cur ^= 1;
            }
        }
        if (e == cudaSuccess && polish_fev > 0) {  // amoeba fine-tuning of the archive's best
            PolishArgs pa{};
            pa.t = fa.t;
            pa.flux = fa.flux;
            pa.sigma = fa.sigma;
            pa.offsets = nullptr;
            pa.n_ep = n_ep;
            pa.n_lc = 1;
            pa.b = b;
            pa.g_in = state->best_genes;
            pa.g_stride = SBLM_MAX_NPAR;
            pa.c_in = &state->best_chi2;
            pa.c_stride = 1;
            pa.g_out = state->best_genes;
            pa.c_out = &state->best_chi2;
            pa.maxfev = polish_fev;
            pa.mixed = polish_mixed;
            pa.mx = pmx;
            e = launch_polish(fa.mode, pa, 1, n_ep, q);
        }
        if (e == cudaSuccess) {
            finish_kernel<<<1, 32, 0, q>>>(state, b, th_out, chi_out);
            e = cudaGetLastError();
        }
        return e;
    };
    SBLM_TRY(run_cached_graph(fit_graph_key(c, fa, n_gen, tr, th_out, chi_out, P[0], polish_fev, polish_mixed), enqueue, s));
    SBLM_TRY(st.end());
    SBLM_CUDA(cudaStreamSynchronize(s));
    return SBLM_OK;
}
