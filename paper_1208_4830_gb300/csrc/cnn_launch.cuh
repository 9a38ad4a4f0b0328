// cnn_launch.cuh -- host interface of the proposal network used by the seeded batched fitter.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/sblm.h"
#include "forward_launch.cuh"

namespace sblm {
namespace cnn {

constexpr int kNParams = 326156;

// device buffers of one inference pass over n curves plus their seed rows, carved from one slice
struct InferScratch {
    float* x;            // [n][256][2]
    double* window;      // [n][2]
    void* wb;            // BF16 weights as stored
    void* wbt;           // BF16 weight matrices transposed
    void* act;           // BF16 activations of every layer
    float* out;          // [n][12]
    double* genes;       // [n][n_seed][6]
};
size_t infer_scratch_bytes(int n, int n_seed);
InferScratch infer_scratch_carve(void* base, int n, int n_seed);

// bin the curves, run the network and draw n_seed seed rows per curve into sc.genes
cudaError_t launch_seed_rows(const double* t, const double* flux, const double* sigma, const int64_t* offsets,
                             int n_lc, const float* weights, const Bounds& b, int n_seed, uint64_t seed,
                             const InferScratch& sc, cudaStream_t s);

// SBLM_ETIMEOUT if a tensor-core tile gave up waiting since the last check (synchronises s)
sblm_status check_timeout(cudaStream_t s);

}  // namespace cnn
}  // namespace sblm
