// peaks.cu -- measured FP32 and FP64 FMA throughput of the current device: the denominators of
// the ALU roofline that the benchmark reports (the forward model has no dense contraction, so
// its roofline is the plain FP32 / FP64 pipes, not the tensor cores).
#include <cuda_runtime.h>

#include "runtime.cuh"

namespace sblm {
namespace {

// eight independent FMA chains per thread keep every FMA pipe busy; the result is stored so
// the chains cannot be removed
template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* __restrict__ out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
sblm_status rate(int sms, int iters, T* buf, cudaStream_t s, double* tflops) {
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    SBLM_CUDA(cudaEventCreate(&e0));
    SBLM_CUDA(cudaEventCreate(&e1));
    fma_chains<T><<<blocks, threads, 0, s>>>(buf, iters / 8, T(0.999999), T(1e-7));  // warm-up
    SBLM_CUDA(cudaEventRecord(e0, s));
    fma_chains<T><<<blocks, threads, 0, s>>>(buf, iters, T(0.999999), T(1e-7));
    SBLM_CUDA(cudaEventRecord(e1, s));
    SBLM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    SBLM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flop = 2.0 * 8.0 * (double)iters * blocks * threads;
    *tflops = flop / (ms * 1e-3) / 1e12;
    return SBLM_OK;
}

}  // namespace
}  // namespace sblm

using namespace sblm;

extern "C" sblm_status sblm_peak_rates(double* fp32_tflops, double* fp64_tflops, void* stream) {
    if (!fp32_tflops || !fp64_tflops) return fail(SBLM_EINVAL, "outputs are required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    int dev = 0, sms = 0;
    SBLM_CUDA(cudaGetDevice(&dev));
    SBLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    Scratch sc(s);
    const int k = sc.add(sizeof(double) * (size_t)sms * 8 * 256);
    SBLM_TRY(sc.commit());
    SBLM_TRY(rate<float>(sms, 1 << 16, static_cast<float*>(sc.ptr(k)), s, fp32_tflops));
    SBLM_TRY(rate<double>(sms, 1 << 12, static_cast<double*>(sc.ptr(k)), s, fp64_tflops));
    return SBLM_OK;
}
