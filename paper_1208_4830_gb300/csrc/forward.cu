// forward.cu -- population-wide forward model: magnification and chi^2 for every
// (candidate, epoch): sblm_magnification, sblm_chi2, and the blended chi^2 of sblm_chi2_blend.
//
// Layout: G threads per candidate (a power of two, G <= 256), each owning a contiguous run of
// epochs so that a root set carries over as the warm start of the next epoch; the block's
// candidates share the lightcurve, staged once per block in shared memory. chi^2 is reduced
// over a candidate's G threads in a fixed order (shuffles, then shared memory), in FP64.
#include <algorithm>
#include <cmath>

#include "blend.cuh"
#include "forward_launch.cuh"
#include "forward_run.cuh"
#include "runtime.cuh"

namespace sblm {

namespace {

constexpr int kBlock = 256;

// MIXED, second pass: the queued epochs in full warps over the whole GPU. Each chi^2 term goes to
// its (candidate, epoch) place in the dense term array (no atomics), so the sums of the third pass
// do not depend on the order in which the queue was filled.
template <bool CHI2, bool FROM_GENES>
__global__ void __launch_bounds__(256) resolve_kernel(const double* __restrict__ src, Bounds bounds,
                                                      const double* __restrict__ t,
                                                      const double* __restrict__ flux,
                                                      const double* __restrict__ sigma, int n_ep,
                                                      const Deferred* __restrict__ queue,
                                                      const unsigned* __restrict__ count, unsigned cap,
                                                      double* __restrict__ A_out, uint8_t* __restrict__ flags,
                                                      double* __restrict__ term) {
    const unsigned n = min(*count, cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Deferred q = queue[i];
        const Cand k = candidate<FROM_GENES>(src, bounds, q.c);
        const double fe = CHI2 ? flux[q.e] : 0.0;
        const double we = CHI2 ? 1.0 / sigma[q.e] : 0.0;
        const double tm = resolve_fp64(q.z, q.why, &k, t[q.e], fe, we, A_out ? A_out + (size_t)q.c * n_ep : nullptr,
                                       flags ? flags + (size_t)q.c * n_ep : nullptr, q.e, CHI2);
        if (CHI2) term[(size_t)q.c * n_ep + q.e] = tm;
    }
}

// MIXED, third pass: chi^2 of candidate (warp) c as the sum of its term row in a fixed order
// (lane l adds epochs l, l + 32, ... in order, then a fixed butterfly)
__global__ void term_sum_kernel(int n_cand, int n_ep, const double* __restrict__ term, double* __restrict__ chi2_out) {
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (c >= n_cand) return;  // whole warps leave together
    const double s = term_row_sum(term + (size_t)c * n_ep, n_ep, lane, 32, true);
    if (lane == 0) chi2_out[c] = s;
}

// blended chi^2 of candidate (warp) c from its magnification row: lanes take epochs lane,
// lane + 32, ... in order; the sums meet in a fixed shuffle tree
__global__ void blend_kernel(const double* __restrict__ A, const double* __restrict__ flux,
                             const double* __restrict__ sigma, int n_cand, int n_ep, double f_min,
                             double* __restrict__ chi2_out, double* __restrict__ f_out) {
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (c >= n_cand) return;  // whole warps leave together
    const double* Ar = A + (size_t)c * n_ep;
    double s_ab = 0.0, s_aa = 0.0;
    for (int e = lane; e < n_ep; e += 32) {
        const double w = 1.0 / (sigma[e] * sigma[e]);
        const double a = Ar[e] - 1.0, b = flux[e] - 1.0;
        s_ab += w * a * b;
        s_aa += w * a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s_ab += __shfl_xor_sync(0xffffffffu, s_ab, o);
        s_aa += __shfl_xor_sync(0xffffffffu, s_aa, o);
    }
    const double f = blend_f(s_ab, s_aa, f_min);
    double chi = 0.0;
    for (int e = lane; e < n_ep; e += 32) {
        const double w = 1.0 / (sigma[e] * sigma[e]);
        const double r = (flux[e] - 1.0) - f * (Ar[e] - 1.0);
        chi += w * r * r;
    }
    for (int o = 16; o > 0; o >>= 1) chi += __shfl_xor_sync(0xffffffffu, chi, o);
    if (lane == 0) {
        chi2_out[c] = chi;
        if (f_out) f_out[c] = f;
    }
}

// MIXED runs three blocks per SM (80 registers and about 200 bytes of spills per thread: 24 warps
// hide more of the dependency latency than the spills cost, 1.2% on the 32-population step); the
// other modes keep two blocks
constexpr int forward_min_blocks(int mode) { return mode == SBLM_MIXED ? 3 : 2; }

template <int MODE, bool CHI2, bool STAGED, bool FROM_GENES>
__global__ void __launch_bounds__(kBlock, forward_min_blocks(MODE))
    forward_kernel(const double* __restrict__ src, Bounds bounds, int n_cand, const double* __restrict__ t,
                   const double* __restrict__ flux, const double* __restrict__ sigma, int n_ep,
                   double* __restrict__ A_out, uint8_t* __restrict__ flags, double* __restrict__ chi2_out, int G,
                   DeferSink sink, double* __restrict__ term) {
    extern __shared__ __align__(16) unsigned char smem[];
    const LCView lc = STAGED ? stage_lightcurve<MODE, CHI2>(smem, t, flux, sigma, n_ep)
                             : LCView{t, flux, sigma, nullptr, nullptr, nullptr, nullptr};
    const int group = threadIdx.x / G, g = threadIdx.x % G;
    const int per_block = blockDim.x / G;
    const int c = blockIdx.x * per_block + group;
    const bool valid = c < n_cand;
    const int seg = (n_ep + G - 1) / G;
    // a candidate wider than a warp interleaves its segments across its warps (segment lane * G/32
    // + warp), so each warp samples the whole lightcurve and the warps carry similar work
    const int gs = G > 32 ? (g & 31) * (G >> 5) + (g >> 5) : g;
    const int e0 = min(n_ep, gs * seg), e1 = min(n_ep, e0 + seg);
    const Cand k = group_candidate<FROM_GENES>(src, bounds, c, valid, G);
    double* A_row = (A_out && valid) ? A_out + (size_t)c * n_ep : nullptr;
    uint8_t* f_row = (flags && valid) ? flags + (size_t)c * n_ep : nullptr;
    double* term_row = (MODE == SBLM_MIXED && CHI2 && valid) ? term + (size_t)c * n_ep : nullptr;
    double chi = eval_run<MODE, CHI2, STAGED>(k, valid, c, e0, e1, seg, lc, A_row, f_row, sink, term_row);
    if (!CHI2 || MODE == SBLM_MIXED) return;  // MIXED: the term rows are summed after the re-solve
    // deterministic reduction over the candidate's G threads
    const int width = min(G, 32);
    for (int off = width / 2; off > 0; off >>= 1) chi += __shfl_xor_sync(0xffffffffu, chi, off);
    if (G <= 32) {
        if (g == 0 && valid) chi2_out[c] = chi;
        return;
    }
    __shared__ double s_part[kBlock / 32];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) s_part[warp] = chi;
    __syncthreads();
    if (g == 0 && valid) {
        double sum = 0.0;
        for (int w = 0; w < G / 32; ++w) sum += s_part[warp + w];
        chi2_out[c] = sum;
    }
}

template <int MODE, bool CHI2, bool STAGED, bool FROM_GENES>
cudaError_t launch_t(const ForwardArgs& a, cudaStream_t s) {
    auto kern = forward_kernel<MODE, CHI2, STAGED, FROM_GENES>;
    const size_t smem = STAGED ? staged_bytes(MODE, CHI2, a.n_ep) : 0;
    // opt in to more than 48 KB (dynamic plus the kernel's static shared memory) once per
    // device and size
    cudaError_t e = raise_smem_limit((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    const int per_block = kBlock / a.G;
    const int grid = (a.n_cand + per_block - 1) / per_block;
    DeferSink sink{};
    MixedLayout ml;
    double* term = nullptr;
    if (MODE == SBLM_MIXED) {
        ml = mixed_layout(a.n_cand, a.n_ep, CHI2);
        char* m = static_cast<char*>(a.mixed);
        sink.queue = reinterpret_cast<Deferred*>(m);
        sink.queue_count = reinterpret_cast<unsigned*>(m + ml.off_count);
        sink.queue_cap = ml.queue_cap;
        term = CHI2 ? reinterpret_cast<double*>(m + ml.off_term) : nullptr;
    }
    kern<<<grid, kBlock, smem, s>>>(a.src, a.bounds, a.n_cand, a.t, a.flux, a.sigma, a.n_ep, a.A_out, a.flags,
                                    a.chi2_out, a.G, sink, term);
    e = cudaGetLastError();
    if (e != cudaSuccess || MODE != SBLM_MIXED) return e;
    const int rgrid = (int)std::min<unsigned>((ml.queue_cap + 255) / 256, 8u * (unsigned)device_sm_count());
    resolve_kernel<CHI2, FROM_GENES><<<rgrid, 256, 0, s>>>(a.src, a.bounds, a.t, a.flux, a.sigma, a.n_ep, sink.queue,
                                                          sink.queue_count, ml.queue_cap, a.A_out, a.flags, term);
    e = cudaGetLastError();
    if (e != cudaSuccess || !CHI2) return e;
    term_sum_kernel<<<(int)(((long)a.n_cand * 32 + 255) / 256), 256, 0, s>>>(a.n_cand, a.n_ep, term, a.chi2_out);
    return cudaGetLastError();
}

template <int MODE, bool CHI2>
cudaError_t launch_m(const ForwardArgs& a, cudaStream_t s) {
    const bool staged = staged_bytes(MODE, CHI2, a.n_ep) <= kMaxStagedBytes;
    if (a.from_genes)
        return staged ? launch_t<MODE, CHI2, true, true>(a, s) : launch_t<MODE, CHI2, false, true>(a, s);
    return staged ? launch_t<MODE, CHI2, true, false>(a, s) : launch_t<MODE, CHI2, false, false>(a, s);
}

}  // namespace

size_t staged_bytes(int mode, bool chi2, int n_ep) {
    if (mode == SBLM_FP64) return (size_t)n_ep * sizeof(double) * (chi2 ? 3 : 1);
    return (size_t)n_ep * sizeof(float4);
}

int choose_group(int n_cand, int n_ep) {
    // threads to fill the GPU four times over (SMs x 2 blocks x 256 threads is one fill), at
    // least ~4 epochs per thread so warm starts pay off. On the 4096 x 2000 sweep 256 threads per
    // candidate (8 epochs each, a candidate per block) beat 64 threads (31 epochs each) by 8%:
    // more warps hide latency, and a block's warps carry similar work
    const long target = (long)device_sm_count() * 4096;
    long g = 1;
    while (g * n_cand < target && g < 256) g <<= 1;
    long cap = 1;
    while (cap * 2 <= std::max(1, n_ep / 4) && cap < 256) cap <<= 1;
    return (int)std::max(1L, std::min(g, cap));
}

MixedLayout mixed_layout(int n_cand, int n_ep, bool chi2) {
    MixedLayout l;
    if (n_cand <= 0 || n_ep <= 0) return l;
    // a queue entry for one epoch in 32 (0.55% of the sweep's epochs defer, 4.2% of those of the
    // trajectories aimed at caustics), at least 4096 and at most 2^24 entries (0.9 GB)
    const long n = (long)n_cand * n_ep;
    l.queue_cap = (unsigned)std::min<long>(std::max<long>(n / 32, 4096), 1L << 24);
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    l.off_count = up(sizeof(Deferred) * (size_t)l.queue_cap);
    l.off_term = up(l.off_count + sizeof(unsigned));
    l.bytes = up(l.off_term + (chi2 ? sizeof(double) * (size_t)n : 0));
    return l;
}

size_t deferred_entry_bytes() { return sizeof(Deferred); }

cudaError_t launch_forward(const ForwardArgs& a, cudaStream_t s) {
    if (a.n_cand <= 0 || a.n_ep <= 0) return cudaSuccess;
    if (a.mode == SBLM_MIXED) {
        if (!a.mixed) return cudaErrorInvalidValue;
        const MixedLayout ml = mixed_layout(a.n_cand, a.n_ep, a.chi2_out != nullptr);
        cudaError_t e = cudaMemsetAsync(static_cast<char*>(a.mixed) + ml.off_count, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    const bool chi2 = a.chi2_out != nullptr;
    switch (a.mode) {
        case SBLM_FP64: return chi2 ? launch_m<SBLM_FP64, true>(a, s) : launch_m<SBLM_FP64, false>(a, s);
        case SBLM_MIXED: return chi2 ? launch_m<SBLM_MIXED, true>(a, s) : launch_m<SBLM_MIXED, false>(a, s);
        default: return chi2 ? launch_m<SBLM_FP32, true>(a, s) : launch_m<SBLM_FP32, false>(a, s);
    }
}

sblm_status check_theta_host(const double* theta, int n_cand) {
    for (int c = 0; c < n_cand; ++c) {
        const double* r = theta + 6 * (size_t)c;
        for (int j = 0; j < 6; ++j)
            if (!std::isfinite(r[j])) return fail(SBLM_EINVAL, "theta[%d][%d] is not finite", c, j);
        if (!(r[1] > 0) || !(r[4] > 0) || !(r[5] > 0))
            return fail(SBLM_EINVAL, "theta[%d]: tE, d and q must be positive", c);
    }
    return SBLM_OK;
}

sblm_status check_lightcurve_host(const double* t, const double* flux, const double* sigma, int n_ep) {
    for (int e = 0; e < n_ep; ++e) {
        if (!std::isfinite(t[e])) return fail(SBLM_EINVAL, "t[%d] is not finite", e);
        if (flux && !std::isfinite(flux[e])) return fail(SBLM_EINVAL, "flux[%d] is not finite", e);
        if (sigma && !(sigma[e] > 0 && std::isfinite(sigma[e])))
            return fail(SBLM_EINVAL, "sigma[%d] must be positive and finite", e);
    }
    return SBLM_OK;
}

}  // namespace sblm

using namespace sblm;

extern "C" sblm_status sblm_magnification(const double* theta, int32_t n_cand, const double* t, int32_t n_ep,
                                          double* A_out, uint8_t* flags, int32_t precision, void* stream) {
    if (n_cand < 0 || n_ep < 0) return fail(SBLM_EINVAL, "negative size (n_cand=%d, n_ep=%d)", n_cand, n_ep);
    if (precision < SBLM_FP64 || precision > SBLM_FP32) return fail(SBLM_EINVAL, "unknown precision %d", precision);
    if (n_cand == 0 || n_ep == 0) return SBLM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    Staging st(s);
    int i_theta, i_t, i_A, i_f;
    SBLM_TRY(st.arg(theta, sizeof(double) * 6 * (size_t)n_cand, true, false, &i_theta));
    SBLM_TRY(st.arg(t, sizeof(double) * (size_t)n_ep, true, false, &i_t));
    SBLM_TRY(st.arg(A_out, sizeof(double) * (size_t)n_cand * n_ep, false, true, &i_A));
    SBLM_TRY(st.arg(flags, flags ? (size_t)n_cand * n_ep : 0, false, true, &i_f));
    const int G = choose_group(n_cand, n_ep);
    const int k_mx = st.scratch(precision == SBLM_MIXED ? mixed_scratch_bytes(n_cand, n_ep, false) : 0);
    bool on_dev = true;
    SBLM_TRY(is_device_pointer(theta, &on_dev));
    if (!on_dev) SBLM_TRY(check_theta_host(theta, n_cand));
    SBLM_TRY(is_device_pointer(t, &on_dev));
    if (!on_dev) SBLM_TRY(check_lightcurve_host(t, nullptr, nullptr, n_ep));
    SBLM_TRY(st.begin());
    ForwardArgs a{};
    a.src = static_cast<const double*>(st.dev(i_theta));
    a.n_cand = n_cand;
    a.t = static_cast<const double*>(st.dev(i_t));
    a.n_ep = n_ep;
    a.A_out = static_cast<double*>(st.dev(i_A));
    a.flags = static_cast<uint8_t*>(st.dev(i_f));
    a.mode = precision;
    a.G = G;
    a.mixed = st.scratch_ptr(k_mx);
    SBLM_CUDA(launch_forward(a, s));
    return st.end();
}

namespace sblm {
sblm_status check_bounds(const sblm_bounds* b, Bounds* out);
}

// shared by sblm_chi2 (theta rows) and sblm_chi2_genes (encoded genes)
static sblm_status chi2_impl(const double* src, bool genes, const Bounds& b, int32_t n_cand, const double* t,
                             const double* flux, const double* sigma, int32_t n_ep, double* chi2_out,
                             int32_t precision, void* stream) {
    if (n_cand < 0 || n_ep < 0) return fail(SBLM_EINVAL, "negative size (n_cand=%d, n_ep=%d)", n_cand, n_ep);
    if (precision < SBLM_FP64 || precision > SBLM_FP32) return fail(SBLM_EINVAL, "unknown precision %d", precision);
    if (n_cand == 0) return SBLM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    Staging st(s);
    int i_theta, i_t, i_f, i_s, i_c;
    SBLM_TRY(st.arg(src, sizeof(double) * 6 * (size_t)n_cand, true, false, &i_theta));
    SBLM_TRY(st.arg(t, sizeof(double) * (size_t)n_ep, true, false, &i_t));
    SBLM_TRY(st.arg(flux, sizeof(double) * (size_t)n_ep, true, false, &i_f));
    SBLM_TRY(st.arg(sigma, sizeof(double) * (size_t)n_ep, true, false, &i_s));
    SBLM_TRY(st.arg(chi2_out, sizeof(double) * (size_t)n_cand, false, true, &i_c));
    const int G = choose_group(n_cand, n_ep);
    const int k_mx = st.scratch(precision == SBLM_MIXED ? mixed_scratch_bytes(n_cand, n_ep, true) : 0);
    bool on_dev = true;
    SBLM_TRY(is_device_pointer(src, &on_dev));
    if (!on_dev && !genes) SBLM_TRY(check_theta_host(src, n_cand));
    if (n_ep > 0) {
        bool d1, d2, d3;
        SBLM_TRY(is_device_pointer(t, &d1));
        SBLM_TRY(is_device_pointer(flux, &d2));
        SBLM_TRY(is_device_pointer(sigma, &d3));
        if (!d1 && !d2 && !d3) SBLM_TRY(check_lightcurve_host(t, flux, sigma, n_ep));
    }
    SBLM_TRY(st.begin());
    if (n_ep == 0) {
        SBLM_CUDA(cudaMemsetAsync(st.dev(i_c), 0, sizeof(double) * (size_t)n_cand, s));
        return st.end();
    }
    ForwardArgs a{};
    a.src = static_cast<const double*>(st.dev(i_theta));
    a.from_genes = genes;
    a.bounds = b;
    a.n_cand = n_cand;
    a.t = static_cast<const double*>(st.dev(i_t));
    a.flux = static_cast<const double*>(st.dev(i_f));
    a.sigma = static_cast<const double*>(st.dev(i_s));
    a.n_ep = n_ep;
    a.chi2_out = static_cast<double*>(st.dev(i_c));
    a.mode = precision;
    a.G = G;
    a.mixed = st.scratch_ptr(k_mx);
    SBLM_CUDA(launch_forward(a, s));
    return st.end();
}

extern "C" sblm_status sblm_chi2_genes(const double* P, int32_t n_pop, const sblm_bounds* bounds, const double* t,
                                       const double* flux, const double* sigma, int32_t n_ep, double* chi2_out,
                                       int32_t precision, void* stream) {
    Bounds b;
    SBLM_TRY(check_bounds(bounds, &b));
    return chi2_impl(P, true, b, n_pop, t, flux, sigma, n_ep, chi2_out, precision, stream);
}

extern "C" sblm_status sblm_chi2_blend(const double* theta, int32_t n_cand, const double* t, const double* flux,
                                      const double* sigma, int32_t n_ep, double* chi2_out, double* f_out,
                                      int32_t precision, void* stream) {
    if (n_cand < 0 || n_ep < 0) return fail(SBLM_EINVAL, "negative size (n_cand=%d, n_ep=%d)", n_cand, n_ep);
    if (precision < SBLM_FP64 || precision > SBLM_FP32) return fail(SBLM_EINVAL, "unknown precision %d", precision);
    if (n_cand == 0) return SBLM_OK;
    if (!theta || !chi2_out || (n_ep > 0 && (!t || !flux || !sigma))) return fail(SBLM_EINVAL, "NULL buffer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    Staging st(s);
    int i_th, i_t, i_f, i_s, i_c, i_fo;
    SBLM_TRY(st.arg(theta, sizeof(double) * 6 * (size_t)n_cand, true, false, &i_th));
    SBLM_TRY(st.arg(t, sizeof(double) * (size_t)n_ep, true, false, &i_t));
    SBLM_TRY(st.arg(flux, sizeof(double) * (size_t)n_ep, true, false, &i_f));
    SBLM_TRY(st.arg(sigma, sizeof(double) * (size_t)n_ep, true, false, &i_s));
    SBLM_TRY(st.arg(chi2_out, sizeof(double) * (size_t)n_cand, false, true, &i_c));
    SBLM_TRY(st.arg(f_out, f_out ? sizeof(double) * (size_t)n_cand : 0, false, true, &i_fo));
    const int G = choose_group(n_cand, n_ep);
    const int k_A = st.scratch(sizeof(double) * (size_t)n_cand * n_ep);
    const int k_mx = st.scratch(precision == SBLM_MIXED ? mixed_scratch_bytes(n_cand, n_ep, false) : 0);
    bool d = true;
    SBLM_TRY(is_device_pointer(theta, &d));
    if (!d) SBLM_TRY(check_theta_host(theta, n_cand));
    if (n_ep > 0) {
        SBLM_TRY(is_device_pointer(t, &d));
        if (!d) SBLM_TRY(check_lightcurve_host(t, flux, sigma, n_ep));
    }
    SBLM_TRY(st.begin());
    ForwardArgs a{};
    a.src = static_cast<const double*>(st.dev(i_th));
    a.n_cand = n_cand;
    a.t = static_cast<const double*>(st.dev(i_t));
    a.n_ep = n_ep;
    a.A_out = static_cast<double*>(st.scratch_ptr(k_A));
    a.mode = precision;
    a.G = G;
    a.mixed = st.scratch_ptr(k_mx);
    if (n_ep > 0) SBLM_CUDA(launch_forward(a, s));
    const int threads = 256, blocks = (int)(((long)n_cand * 32 + threads - 1) / threads);
    blend_kernel<<<blocks, threads, 0, s>>>(a.A_out, static_cast<const double*>(st.dev(i_f)),
                                            static_cast<const double*>(st.dev(i_s)), n_cand, n_ep, SBLM_BLEND_F_MIN,
                                            static_cast<double*>(st.dev(i_c)), static_cast<double*>(st.dev(i_fo)));
    SBLM_CUDA(cudaGetLastError());
    return st.end();
}

extern "C" sblm_status sblm_chi2(const double* theta, int32_t n_cand, const double* t, const double* flux,
                                 const double* sigma, int32_t n_ep, double* chi2_out, int32_t precision,
                                 void* stream) {
    return chi2_impl(theta, false, Bounds{}, n_cand, t, flux, sigma, n_ep, chi2_out, precision, stream);
}
