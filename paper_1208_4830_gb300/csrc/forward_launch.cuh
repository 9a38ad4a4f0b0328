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
    // MIXED only: mixed_scratch_bytes(n_cand, n_ep, chi2_out != null) bytes of device scratch
    // (256-byte aligned) for the re-solve queue, its counter and the chi^2 terms; launch_forward
    // zeroes the counter
    void* mixed = nullptr;
};

// MIXED scratch of one forward pass: the re-solve queue (an entry for one epoch in 32; an epoch
// that finds it full is re-solved in place), its counter and, when chi^2 is wanted, the dense
// n_cand x n_ep array of chi^2 terms that is summed row by row in a fixed order
struct MixedLayout {
    unsigned queue_cap = 0;
    size_t off_count = 0, off_term = 0, bytes = 0;
};
MixedLayout mixed_layout(int n_cand, int n_ep, bool chi2);
inline size_t mixed_scratch_bytes(int n_cand, int n_ep, bool chi2) { return mixed_layout(n_cand, n_ep, chi2).bytes; }
size_t deferred_entry_bytes();

size_t staged_bytes(int mode, bool chi2, int n_ep);
int choose_group(int n_cand, int n_ep);
cudaError_t launch_forward(const ForwardArgs& a, cudaStream_t s);
sblm_status check_theta_host(const double* theta, int n_cand);
sblm_status check_lightcurve_host(const double* t, const double* flux, const double* sigma, int n_ep);

}  // namespace sblm
