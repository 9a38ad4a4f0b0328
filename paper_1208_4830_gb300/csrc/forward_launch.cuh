// forward_launch.cuh -- host interface of the forward-model kernels, shared by the entry points
// of forward.cu and the fit drivers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/sblm.h"

namespace sblm {

// gene domains of Eq. (EMMA-encoding), passed to kernels by value
struct Bounds {
    double lo[SBLM_NPAR];
    double hi[SBLM_NPAR];
};

// MIXED: an epoch is re-solved in FP64 when an image, or a rejected root that nearly solves the
// lens equation, has |det J| below this (next to a caustic FP32 loses accuracy, and an image pair
// it failed to converge sits next to the critical curve), when two images are closer than the
// gap trigger, or when the FP32 image selection was ambiguous
constexpr float kMixedDetTrigger = 3e-2f;
constexpr float kMixedGapTrigger = 1e-4f;

// largest lightcurve staged in shared memory per block (larger ones are read from global memory)
constexpr size_t kMaxStagedBytes = 96 * 1024;

struct ForwardArgs {
    const double* src = nullptr;   // theta rows, or encoded genes when from_genes
    bool from_genes = false;
    Bounds bounds{};
    int n_cand = 0;
    const double* t = nullptr;
    const double* flux = nullptr;
    const double* sigma = nullptr;
    int n_ep = 0;
    double* A_out = nullptr;       // optional [n_cand * n_ep]
    uint8_t* flags = nullptr;      // optional [n_cand * n_ep]
    double* chi2_out = nullptr;    // optional [n_cand]; null -> no chi^2
    int mode = SBLM_FP64;
    int G = 32;                    // threads per candidate (power of two, <= 256)
    // MIXED only: queue of epochs to re-solve in FP64 (capacity entries of
    // deferred_entry_bytes() each) and its counter; launch_forward zeroes the counter
    void* queue = nullptr;
    unsigned* queue_count = nullptr;
    unsigned queue_cap = 0;
};

// scratch of the MIXED re-solve queue: entry count sized for a few percent of the epochs (an
// epoch that finds the queue full is re-solved in place, so the size is a speed choice only)
unsigned mixed_queue_capacity(int n_cand, int n_ep);
size_t deferred_entry_bytes();

size_t staged_bytes(int mode, bool chi2, int n_ep);
int choose_group(int n_cand, int n_ep);
cudaError_t launch_forward(const ForwardArgs& a, cudaStream_t s);
sblm_status check_theta_host(const double* theta, int n_cand);
sblm_status check_lightcurve_host(const double* t, const double* flux, const double* sigma, int n_ep);

}  // namespace sblm
