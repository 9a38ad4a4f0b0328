// ea_launch.cuh -- host interface of the EA kernels, shared by ea.cu and the fit drivers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ea.cuh"

namespace sblm {

// validated constants of a parameter set (n_tourn resolved)
sblm_status ea_const(const sblm_ea_params* p, int n_pop, int n_par, uint64_t stream_id, EAConst* out);

// keys[n_pop * n_par] of the initialisation of generation `gen`, then the population values
cudaError_t launch_init(const EAConst& c, int gen, uint64_t* keys, double* P, cudaStream_t s);
// reset *state to the start of a run
cudaError_t launch_state_reset(const EAConst& c, sblm_ea_state* state, cudaStream_t s);
// ranking, archive, stagnation (and restart keys); `produce` = false archives only. With n_pops > 1
// the arrays hold n_pops populations back to back (stream ids c.stream, c.stream + 1, ...; trace_row
// must then be null), ranked by one block each in one launch
cudaError_t launch_rank(const EAConst& c, int gen, const double* chi2, const double* P, sblm_ea_state* state,
                        int* order, EACtrl* ctrl, uint64_t* keys, double* trace_row, bool produce, cudaStream_t s,
                        int n_pops = 1);
// offspring (or the fresh population after a restart) into P_next, for n_pops populations
cudaError_t launch_offspring(const EAConst& c, int gen, const double* P, const int* order, const EACtrl* ctrl,
                             const uint64_t* keys, double* P_next, cudaStream_t s, int n_pops = 1);

}  // namespace sblm
