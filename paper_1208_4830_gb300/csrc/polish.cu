// polish.cu -- amoeba fine-tuning (polish.cuh) as a kernel: for sblm_fit (the archive's best of
// one population) and for sblm_polish_batch (given start genes of many lightcurves).
#include <algorithm>
#include <cstring>
#include <vector>

#include "polish.cuh"
#include "polish_launch.cuh"
#include "runtime.cuh"

namespace sblm {

namespace {

// one block per lightcurve (grid-stride over lightcurves); genes/chi^2 read from `g_in`/`c_in`
// (c_in may be null: the start is evaluated) and written to `g_out`/`c_out`
template <int MODE>
__global__ void __launch_bounds__(kPolishThreads) polish_kernel(PolishArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[33];
    __shared__ unsigned s_qcount;
    DeferSink sink{};
    double* term_row = nullptr;
    if (MODE == SBLM_MIXED) {
        char* m = static_cast<char*>(a.mixed) + (size_t)blockIdx.x * a.mx.block_bytes;
        sink.queue = reinterpret_cast<Deferred*>(m);
        sink.queue_count = &s_qcount;
        sink.queue_cap = a.mx.queue_cap;
        term_row = reinterpret_cast<double*>(m + a.mx.off_term);
    }
    const int starts = a.starts > 1 ? a.starts : 1;
    for (int inst = blockIdx.x; inst < a.n_lc * starts; inst += gridDim.x) {
        const int lc = inst / starts;
        if (starts > 1 && inst % starts >= min(a.counts[lc], a.max_starts)) {  // no such start
            if (threadIdx.x == 0) a.c_out[(size_t)inst * a.c_stride] = INFINITY;
            continue;
        }
        const int64_t e0 = a.offsets ? a.offsets[lc] : 0;
        const int n_ep = a.offsets ? (int)(a.offsets[lc + 1] - e0) : a.n_ep;
        const LCView view = stage_lightcurve<MODE, true>(smem, a.t + e0, a.flux + e0, a.sigma + e0, n_ep);
        double g[kPolishN];
        for (int j = 0; j < kPolishN; ++j) g[j] = a.g_in[(size_t)inst * a.g_stride + j];
        double f = a.c_in ? a.c_in[(size_t)inst * a.c_stride] : INFINITY;
        double* A_row = a.blend ? a.A_scr + (size_t)blockIdx.x * a.A_stride : nullptr;
        block_nelder_mead<MODE>(g, &f, a.maxfev, a.b, view, n_ep, sink, term_row, s_red, A_row, a.f_min);
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int j = 0; j < kPolishN; ++j) a.g_out[(size_t)inst * a.g_stride + j] = g[j];
            a.c_out[(size_t)inst * a.c_stride] = f;
        }
        __syncthreads();
    }
}

template <int MODE>
cudaError_t launch_mode(const PolishArgs& a, int blocks, size_t smem, cudaStream_t s) {
    cudaError_t e = raise_smem_limit((const void*)polish_kernel<MODE>, smem);
    if (e != cudaSuccess) return e;
    polish_kernel<MODE><<<blocks, kPolishThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t polish_smem_bytes(int mode, int max_ep) {
    return (size_t)max_ep * (mode == SBLM_FP64 ? 3 * sizeof(double) : sizeof(float4));
}

PolishMixed polish_mixed_layout(int max_ep) {
    PolishMixed l;
    l.queue_cap = (unsigned)std::max(max_ep, 1);
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    l.off_term = up(sizeof(Deferred) * (size_t)l.queue_cap);
    l.block_bytes = up(l.off_term + sizeof(double) * (size_t)l.queue_cap);
    return l;
}

cudaError_t polish_prepare(int mode, int max_ep) {
    const size_t smem = polish_smem_bytes(mode, max_ep);
    switch (mode) {
        case SBLM_FP64: return raise_smem_limit((const void*)polish_kernel<SBLM_FP64>, smem);
        case SBLM_MIXED: return raise_smem_limit((const void*)polish_kernel<SBLM_MIXED>, smem);
        default: return raise_smem_limit((const void*)polish_kernel<SBLM_FP32>, smem);
    }
}

cudaError_t launch_polish(int mode, const PolishArgs& a, int blocks, int max_ep, cudaStream_t s) {
    const size_t smem = polish_smem_bytes(mode, max_ep);
    switch (mode) {
        case SBLM_FP64: return launch_mode<SBLM_FP64>(a, blocks, smem, s);
        case SBLM_MIXED: return launch_mode<SBLM_MIXED>(a, blocks, smem, s);
        default: return launch_mode<SBLM_FP32>(a, blocks, smem, s);
    }
}

sblm_status check_bounds(const sblm_bounds* b, Bounds* out);

}  // namespace sblm

using namespace sblm;

extern "C" sblm_status sblm_polish_batch(const double* t, const double* flux, const double* sigma,
                                         const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                         const double* genes_in, int32_t maxfev, int32_t precision, double* genes_out,
                                         double* chi2_out, void* stream) {
    if (n_lc < 1) return fail(SBLM_EINVAL, "n_lc must be >= 1");
    if (maxfev < 0 || maxfev > kPolishMaxFev) return fail(SBLM_EINVAL, "maxfev must be in [0, %d]", kPolishMaxFev);
    const bool blend = (precision & SBLM_BLEND) != 0;
    precision &= ~SBLM_BLEND;
    if (precision < SBLM_FP64 || precision > SBLM_FP32) return fail(SBLM_EINVAL, "unknown precision %d", precision);
    if (!t || !flux || !sigma || !offsets || !genes_in || !genes_out || !chi2_out)
        return fail(SBLM_EINVAL, "NULL buffer");
    Bounds b;
    SBLM_TRY(check_bounds(bounds, &b));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    std::vector<int64_t> off(n_lc + 1);
    bool od = false;
    SBLM_TRY(is_device_pointer(offsets, &od));
    if (od)
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
    if (polish_smem_bytes(precision, max_ep) > kPolishSmemBudget)
        return fail(SBLM_EINVAL, "longest lightcurve (%d epochs) does not fit the polish staging area", max_ep);
    const size_t total = (size_t)off[n_lc];
    int dev = 0, sms = 0;
    SBLM_CUDA(cudaGetDevice(&dev));
    SBLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = std::min(n_lc, 2 * sms);
    Staging st(s);
    int i_t, i_f, i_s, i_o, i_gi, i_go, i_c;
    SBLM_TRY(st.arg(t, sizeof(double) * total, true, false, &i_t));
    SBLM_TRY(st.arg(flux, sizeof(double) * total, true, false, &i_f));
    SBLM_TRY(st.arg(sigma, sizeof(double) * total, true, false, &i_s));
    SBLM_TRY(st.arg(offsets, sizeof(int64_t) * (n_lc + 1), true, false, &i_o));
    SBLM_TRY(st.arg(genes_in, sizeof(double) * 6 * (size_t)n_lc, true, false, &i_gi));
    SBLM_TRY(st.arg(genes_out, sizeof(double) * 6 * (size_t)n_lc, false, true, &i_go));
    SBLM_TRY(st.arg(chi2_out, sizeof(double) * (size_t)n_lc, false, true, &i_c));
    const PolishMixed mx = polish_mixed_layout(max_ep);
    const int k_q = st.scratch(precision == SBLM_MIXED ? mx.block_bytes * (size_t)blocks : 0);
    const int k_A = st.scratch(blend ? sizeof(double) * (size_t)blocks * max_ep : 0);
    bool d1, d2, d3;
    SBLM_TRY(is_device_pointer(t, &d1));
    SBLM_TRY(is_device_pointer(flux, &d2));
    SBLM_TRY(is_device_pointer(sigma, &d3));
    if (!d1 && !d2 && !d3) SBLM_TRY(check_lightcurve_host(t, flux, sigma, (int)total));
    SBLM_TRY(st.begin());
    PolishArgs a{};
    a.t = static_cast<const double*>(st.dev(i_t));
    a.flux = static_cast<const double*>(st.dev(i_f));
    a.sigma = static_cast<const double*>(st.dev(i_s));
    a.offsets = static_cast<const int64_t*>(st.dev(i_o));
    a.n_lc = n_lc;
    a.b = b;
    a.g_in = static_cast<const double*>(st.dev(i_gi));
    a.g_stride = 6;
    a.c_in = nullptr;
    a.c_stride = 1;
    a.g_out = static_cast<double*>(st.dev(i_go));
    a.c_out = static_cast<double*>(st.dev(i_c));
    a.maxfev = maxfev;
    a.mixed = st.scratch_ptr(k_q);
    a.mx = mx;
    a.blend = blend ? 1 : 0;
    a.f_min = SBLM_BLEND_F_MIN;
    a.A_scr = blend ? static_cast<double*>(st.scratch_ptr(k_A)) : nullptr;
    a.A_stride = max_ep;
    SBLM_CUDA(launch_polish(precision, a, blocks, max_ep, s));
    return st.end();
}
