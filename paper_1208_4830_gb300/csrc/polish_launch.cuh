// polish_launch.cuh -- host interface of the amoeba fine-tuning kernel (polish.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "forward.cuh"
#include "forward_launch.cuh"

namespace sblm {

constexpr int kPolishThreads = 256;
constexpr int kPolishMaxFev = 1 << 20;
constexpr size_t kPolishSmemBudget = 200 * 1024;

// MIXED scratch of one polish block: a re-solve queue with room for every epoch of the longest
// lightcurve and its chi^2 term row (forward_run.cuh: DeferSink)
struct PolishMixed {
    unsigned queue_cap = 0;
    size_t off_term = 0, block_bytes = 0;
};
PolishMixed polish_mixed_layout(int max_ep);

struct PolishArgs {
    const double* t;
    const double* flux;
    const double* sigma;
    const int64_t* offsets;  // null: one lightcurve of n_ep epochs
    int n_ep;
    int n_lc;
    Bounds b;
    int starts;          // searches per lightcurve (instance i: lightcurve i / starts); 0 or 1: one
    const int* counts;   // starts > 1: starts of lightcurve l in use: min(counts[l], max_starts)
    int max_starts;
    const double* g_in;  // start genes of instance i at g_in[i * g_stride]
    int g_stride;
    const double* c_in;  // their chi^2 at c_in[i * c_stride], or null (evaluated)
    int c_stride;
    double* g_out;       // may alias g_in
    double* c_out;       // may alias c_in; a skipped instance gets +inf
    int maxfev;
    void* mixed;         // MIXED: mx.block_bytes of scratch per block
    PolishMixed mx;      // MIXED: polish_mixed_layout(longest lightcurve)
    int blend;           // chi^2 of the blended model with f profiled out (Section 4.4)
    double f_min;
    double* A_scr;       // blend: per block A_stride magnifications
    int A_stride;
};

size_t polish_smem_bytes(int mode, int max_ep);
cudaError_t launch_polish(int mode, const PolishArgs& a, int blocks, int max_ep, cudaStream_t s);
// set the kernel's shared-memory opt-in for `max_ep` (call before a stream capture)
cudaError_t polish_prepare(int mode, int max_ep);

}  // namespace sblm
