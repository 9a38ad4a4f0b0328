// forward.cu -- population-wide forward model: magnification and chi^2 for every
// (candidate, epoch), sblm_magnification and sblm_chi2.
//
// Layout: G threads per candidate (a power of two, G <= 256), each owning a contiguous run of
// epochs so that a root set carries over as the warm start of the next epoch; the block's
// candidates share the lightcurve, staged once per block in shared memory. chi^2 is reduced
// over a candidate's G threads in a fixed order (shuffles, then shared memory), in FP64.
#include <algorithm>
#include <cmath>

#include "forward.cuh"
#include "forward_launch.cuh"
#include "runtime.cuh"

namespace sblm {

namespace {

constexpr int kBlock = 256;

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

// s + x as an unevaluated pair (hi, lo) of floats: Knuth's two-sum, then renormalisation
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float v = s - hi;
    const float e = (hi - (s - v)) + (x - v);
    const float t = lo + e;
    hi = s + t;
    lo = t - (hi - s);
}

// the MIXED re-solve's Aberth stop rule (relative correction), see solve_epoch
constexpr double kResolveCubic = 1e-6;

// FP64 re-solve of one deferred epoch (MIXED), warm-started from its FP32 roots; returns the
// chi^2 term. Out of line: an FP32 lane that must do it in place keeps its state on the stack
// instead of competing with the FP64 solver for registers.
__device__ __noinline__ double resolve_fp64(const cx<float>* z32, uint32_t why, const Cand* kk, double te,
                                            double fe, double we, double* A_out, uint8_t* flags, size_t idx,
                                            bool chi2) {
    cx<double> zz[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) zz[i] = mk<double>(z32[i].re, z32[i].im);
    bool w2 = true;
    const EpochOut<double> o2 = solve_epoch<double>(zeta64(*kk, te), kk->d, kk->q, zz, w2, nullptr, kResolveCubic);
    if (A_out) A_out[idx] = o2.A;
    if (flags) flags[idx] = (uint8_t)(o2.flag | FLAG_FP64 | why);
    if (!chi2) return 0.0;
    const double r = (fe - o2.A) * we;
    return r * r;
}

// MIXED, second pass: the queued epochs in full warps over the whole GPU. Each chi^2 term is
// added atomically to its candidate's FP32 partial sum, so the summation order of these terms
// (and the last bits of a MIXED chi^2) can vary from run to run.
template <bool CHI2, bool FROM_GENES>
__global__ void __launch_bounds__(256) resolve_kernel(const double* __restrict__ src, Bounds bounds,
                                                      const double* __restrict__ t,
                                                      const double* __restrict__ flux,
                                                      const double* __restrict__ sigma, int n_ep,
                                                      const Deferred* __restrict__ queue,
                                                      const unsigned* __restrict__ count, unsigned cap,
                                                      double* __restrict__ A_out, uint8_t* __restrict__ flags,
                                                      double* __restrict__ chi2_out) {
    const unsigned n = min(*count, cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Deferred q = queue[i];
        const Cand k = candidate<FROM_GENES>(src, bounds, q.c);
        const double fe = CHI2 ? flux[q.e] : 0.0;
        const double we = CHI2 ? 1.0 / sigma[q.e] : 0.0;
        const double term =
            resolve_fp64(q.z, q.why, &k, t[q.e], fe, we, A_out, flags, (size_t)q.c * n_ep + q.e, CHI2);
        if (CHI2) atomicAdd(&chi2_out[q.c], term);
    }
}

template <int MODE, bool CHI2, bool STAGED, bool FROM_GENES>
__global__ void __launch_bounds__(kBlock, 2) forward_kernel(const double* __restrict__ src, Bounds bounds,
                                                         int n_cand, const double* __restrict__ t,
                                                         const double* __restrict__ flux,
                                                         const double* __restrict__ sigma, int n_ep,
                                                         double* __restrict__ A_out,
                                                         uint8_t* __restrict__ flags,
                                                         double* __restrict__ chi2_out, int G,
                                                         Deferred* __restrict__ queue,
                                                         unsigned* __restrict__ queue_count, unsigned queue_cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    // staged lightcurve: FP64 mode keeps (t, F, 1/sigma) in FP64; the FP32 modes keep
    // (t_hi, t_lo, F, 1/sigma) as floats, t = t_hi + t_lo split so that t - t0 stays exact
    double* s_t = reinterpret_cast<double*>(smem);
    double* s_f = s_t + (STAGED && MODE == SBLM_FP64 ? n_ep : 0);
    double* s_w = s_f + (STAGED && MODE == SBLM_FP64 && CHI2 ? n_ep : 0);
    float4* s_ep = reinterpret_cast<float4*>(smem);
    if (STAGED) {
        for (int e = threadIdx.x; e < n_ep; e += blockDim.x) {
            const double te = t[e];
            const double fe = CHI2 ? flux[e] : 0.0;
            const double we = CHI2 ? 1.0 / sigma[e] : 0.0;
            if (MODE == SBLM_FP64) {
                s_t[e] = te;
                if (CHI2) {
                    s_f[e] = fe;
                    s_w[e] = we;
                }
            } else {
                const float th = (float)te;
                s_ep[e] = make_float4(th, (float)(te - (double)th), (float)fe, (float)we);
            }
        }
        __syncthreads();
    }
    const int group = threadIdx.x / G, g = threadIdx.x % G;
    const int per_block = blockDim.x / G;
    const int c = blockIdx.x * per_block + group;
    const bool valid = c < n_cand;
    const int seg = (n_ep + G - 1) / G;
    const int e0 = min(n_ep, g * seg), e1 = min(n_ep, e0 + seg);
    double chi = 0.0;
    Cand k{};
    if (valid) k = candidate<FROM_GENES>(src, bounds, c);
    double* A_row = (A_out && valid) ? A_out + (size_t)c * n_ep : nullptr;
    uint8_t* f_row = (flags && valid) ? flags + (size_t)c * n_ep : nullptr;
    if constexpr (MODE == SBLM_FP64) {
        cx<double> z[5];
        bool warm = false;
        for (int e = e0; valid && e < e1; ++e) {
            const double te = STAGED ? s_t[e] : t[e];
            const EpochOut<double> o = solve_epoch<double>(zeta64(k, te), k.d, k.q, z, warm);
            if (A_row) A_row[e] = o.A;
            if (f_row) f_row[e] = o.flag;
            if (CHI2) {
                const double fe = STAGED ? s_f[e] : flux[e];
                const double we = STAGED ? s_w[e] : 1.0 / sigma[e];
                const double r = (fe - o.A) * we;
                chi += r * r;
            }
        }
    } else {
        const float t0h = (float)k.t0, t0l = (float)(k.t0 - (double)t0h);
        const float itE = (float)k.inv_tE, sa = (float)k.sa, ca = (float)k.ca, u0 = (float)k.u0;
        const float d = (float)k.d, q = (float)k.q;
        const unsigned lane = threadIdx.x & 31u;
        // per-thread chi^2 of the FP32 epochs as an unevaluated float pair (hi + lo): FP64-grade
        // accumulation on the FP32 pipes; converted to FP64 for the cross-thread reduction
        float chi_hi = 0.f, chi_lo = 0.f;
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
                    ep = s_ep[e];
                } else {
                    const double te = t[e];
                    const float th = (float)te;
                    ep = make_float4(th, (float)(te - (double)th), CHI2 ? (float)flux[e] : 0.f,
                                     CHI2 ? (float)(1.0 / sigma[e]) : 0.f);
                }
                const float tau = diff_ff(ep.x, ep.y, t0h, t0l) * itE;
                const cx<float> zeta = mk<float>(tau * sa + u0 * ca, -tau * ca + u0 * sa);
                EpochOut<float> o = solve_epoch<float>(zeta, d, q, z, warm);
                o.flag |= (o.min_det < kMixedDetTrigger ? FLAG_NEAR_DET : 0) |
                          (o.min_gap < kMixedGapTrigger ? FLAG_NEAR_GAP : 0);
                if (MODE == SBLM_MIXED) defer = o.flag != 0;
                why = o.flag;
                if (A_row) A_row[e] = o.A;
                if (f_row) f_row[e] = o.flag;
                if (CHI2 && !defer) {
                    const float r = (ep.z - o.A) * ep.w;
                    ff_add(chi_hi, chi_lo, r * r);
                }
            }
            if constexpr (MODE == SBLM_MIXED) {
                // one atomic per warp reserves queue slots for the lanes that defer
                const unsigned b = __ballot_sync(0xffffffffu, defer);
                if (b) {
                    const int leader = __ffs(b) - 1;
                    unsigned base = 0;
                    if ((int)lane == leader) base = atomicAdd(queue_count, (unsigned)__popc(b));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (defer) {
                        const unsigned slot = base + __popc(b & ((1u << lane) - 1u));
                        if (slot < queue_cap) {
                            Deferred& q = queue[slot];
#pragma unroll
                            for (int i = 0; i < 5; ++i) q.z[i] = z[i];
                            q.c = c;
                            q.e = e;
                            q.why = why;
                        } else {  // queue full: re-solve here
                            double te, fe = 0.0, we = 0.0;
                            if (STAGED) {
                                const float4 ep = s_ep[e];
                                te = (double)ep.x + (double)ep.y;
                                fe = ep.z;
                                we = ep.w;
                            } else {
                                te = t[e];
                                if (CHI2) {
                                    fe = flux[e];
                                    we = 1.0 / sigma[e];
                                }
                            }
                            chi += resolve_fp64(z, why, &k, te, fe, we, A_out, flags, (size_t)c * n_ep + e, CHI2);
                        }
                    }
                }
            }
        }
        chi += (double)chi_hi + (double)chi_lo;
    }
    if (!CHI2) return;
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
    static size_t granted[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (smem > granted[dev & 63]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        granted[dev & 63] = smem;
    }
    const int per_block = kBlock / a.G;
    const int grid = (a.n_cand + per_block - 1) / per_block;
    kern<<<grid, kBlock, smem, s>>>(a.src, a.bounds, a.n_cand, a.t, a.flux, a.sigma, a.n_ep, a.A_out, a.flags,
                                    a.chi2_out, a.G, static_cast<Deferred*>(a.queue), a.queue_count, a.queue_cap);
    e = cudaGetLastError();
    if (e != cudaSuccess || MODE != SBLM_MIXED || a.queue_cap == 0) return e;
    const int rgrid = (int)std::min<unsigned>((a.queue_cap + 255) / 256, 152u * 8u);
    resolve_kernel<CHI2, FROM_GENES><<<rgrid, 256, 0, s>>>(a.src, a.bounds, a.t, a.flux, a.sigma, a.n_ep,
                                                          static_cast<const Deferred*>(a.queue), a.queue_count,
                                                          a.queue_cap, a.A_out, a.flags, a.chi2_out);
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
    // enough threads to fill the GPU, at least ~4 epochs per thread so warm starts pay off
    const long target = 152L * 1024;
    long g = 1;
    while (g * n_cand < target && g < 256) g <<= 1;
    long cap = 1;
    while (cap * 2 <= std::max(1, n_ep / 4) && cap < 256) cap <<= 1;
    return (int)std::max(1L, std::min(g, cap));
}

unsigned mixed_queue_capacity(int n_cand, int n_ep) {
    const long n = (long)n_cand * n_ep / 32;
    return (unsigned)std::min<long>(std::max<long>(n, 4096), 1L << 24);
}

size_t deferred_entry_bytes() { return sizeof(Deferred); }

cudaError_t launch_forward(const ForwardArgs& a, cudaStream_t s) {
    if (a.n_cand <= 0 || a.n_ep <= 0) return cudaSuccess;
    if (a.mode == SBLM_MIXED && a.queue_cap > 0) {
        cudaError_t e = cudaMemsetAsync(a.queue_count, 0, sizeof(unsigned), s);
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
    const unsigned qcap = precision == SBLM_MIXED ? mixed_queue_capacity(n_cand, n_ep) : 0;
    const int k_q = st.scratch(deferred_entry_bytes() * qcap), k_qc = st.scratch(sizeof(unsigned));
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
    a.G = choose_group(n_cand, n_ep);
    a.queue = st.scratch_ptr(k_q);
    a.queue_count = static_cast<unsigned*>(st.scratch_ptr(k_qc));
    a.queue_cap = qcap;
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
    const unsigned qcap = precision == SBLM_MIXED ? mixed_queue_capacity(n_cand, n_ep) : 0;
    const int k_q = st.scratch(deferred_entry_bytes() * qcap), k_qc = st.scratch(sizeof(unsigned));
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
    a.G = choose_group(n_cand, n_ep);
    a.queue = st.scratch_ptr(k_q);
    a.queue_count = static_cast<unsigned*>(st.scratch_ptr(k_qc));
    a.queue_cap = qcap;
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

extern "C" sblm_status sblm_chi2(const double* theta, int32_t n_cand, const double* t, const double* flux,
                                 const double* sigma, int32_t n_ep, double* chi2_out, int32_t precision,
                                 void* stream) {
    return chi2_impl(theta, false, Bounds{}, n_cand, t, flux, sigma, n_ep, chi2_out, precision, stream);
}
