// ea.cu -- EA operator kernels (Appendix A) and the entry points sblm_ea_init and
// sblm_ea_generation.
//
// One generation after its fitness evaluation takes two launches:
//   rank_kernel      one block: stable bitonic sort of (chi^2, row) in shared memory, archive of
//                    the best ever, stagnation check; on a restart it also writes the sort keys
//                    of the fresh population;
//   offspring_kernel one thread per reproductive pairing: tournament selection, weighting
//                    matrix, Eq. (rep1)/(rep2), creep and jump mutation, elitism in row 0; on a
//                    restart instead one thread per element of the fresh population.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ea_launch.cuh"
#include "runtime.cuh"

namespace sblm {

namespace {

constexpr int kRankThreads = 1024;
constexpr int kInitTile = 2048;

__global__ void init_keys_kernel(EAConst c, int gen, uint64_t* __restrict__ keys, int m) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) keys[e] = init_key(c, (uint64_t)gen, (uint64_t)e);
}

__global__ void init_values_kernel(EAConst c, int gen, const uint64_t* __restrict__ keys, int m,
                                   double* __restrict__ P) {
    __shared__ uint64_t tile[kInitTile];
    block_init_values(c, gen, keys, m, P, blockIdx.x * blockDim.x, m, tile, kInitTile);
}

__global__ void state_reset_kernel(EAConst c, sblm_ea_state* state) {
    if (threadIdx.x != 0) return;
    sblm_ea_state s;
    memset(&s, 0, sizeof s);
    state_reset(c, s);
    *state = s;
}

// block b ranks population b of a batch (its rows, chi^2, state, order, control word and keys
// at b times the per-population strides; stream id c.stream + b); a single population is b = 0
__global__ void __launch_bounds__(kRankThreads)
    rank_kernel(EAConst c, int gen, const double* __restrict__ chi2, const double* __restrict__ P,
                sblm_ea_state* __restrict__ state, int* __restrict__ order, EACtrl* __restrict__ ctrl,
                uint64_t* __restrict__ keys, double* __restrict__ trace_row, int produce) {
    extern __shared__ __align__(16) unsigned char smem[];
    {
        const size_t b = blockIdx.x, m = (size_t)c.n_pop * c.n_par;
        chi2 += b * c.n_pop;
        P += b * m;
        state += b;
        order += b * c.n_pop;
        ctrl += b;
        keys += b * m;
        c.stream += b;
    }
    int n2 = 1;
    while (n2 < c.n_pop) n2 <<= 1;
    double* skey = reinterpret_cast<double*>(smem);
    int* sidx = reinterpret_cast<int*>(skey + n2);
    __shared__ int s_restart;
    block_rank(chi2, c.n_pop, n2, skey, sidx);
    for (int i = threadIdx.x; i < c.n_pop; i += blockDim.x) order[i] = sidx[i];
    if (threadIdx.x == 0) {
        sblm_ea_state s = *state;
        double p_used = 0.0;
        const int restart =
            block_bookkeeping(c, gen, skey[0], P + (size_t)sidx[0] * c.n_par, s, produce != 0, &p_used);
        *state = s;
        ctrl->p_mut_used = p_used;
        ctrl->restart = restart;
        if (trace_row) {
            trace_row[0] = skey[0];
            trace_row[1] = p_used;
            trace_row[2] = (double)s.n_restarts;
            trace_row[3] = s.best_chi2;
        }
        s_restart = restart;
    }
    __syncthreads();
    if (s_restart) {
        const int m = c.n_pop * c.n_par;
        for (int e = threadIdx.x; e < m; e += blockDim.x) keys[e] = init_key(c, (uint64_t)(gen + 1), (uint64_t)e);
    }
}

// grid row blockIdx.y is population y of a batch (strides as in rank_kernel)
__global__ void offspring_kernel(EAConst c, int gen, const double* __restrict__ P, const int* __restrict__ order,
                                 const EACtrl* __restrict__ ctrl, const uint64_t* __restrict__ keys,
                                 double* __restrict__ P_next) {
    {
        const size_t b = blockIdx.y, m = (size_t)c.n_pop * c.n_par;
        P += b * m;
        order += b * c.n_pop;
        ctrl += b;
        keys += b * m;
        P_next += b * m;
        c.stream += b;
    }
    if (ctrl->restart) {  // uniform over the grid row
        __shared__ uint64_t tile[kInitTile];
        const int m = c.n_pop * c.n_par;
        block_init_values(c, gen + 1, keys, m, P_next, blockIdx.x * blockDim.x, m, tile, kInitTile);
        return;
    }
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {  // elitism: the fittest row survives unmutated
        const double* e = P + (size_t)order[0] * c.n_par;
        for (int j = 0; j < c.n_par; ++j) P_next[j] = e[j];
    }
    if (k < c.n_pop / 2) offspring_pair(c, gen, P, order, ctrl->p_mut_used, k, P_next);  // ceil((N_pop-1)/2)
}

int blocks_for(int n, int b) { return (n + b - 1) / b; }

}  // namespace

sblm_status ea_const(const sblm_ea_params* p, int n_pop, int n_par, uint64_t stream_id, EAConst* out) {
    if (!p) return fail(SBLM_EINVAL, "params is NULL");
    if (n_pop < 2 || n_pop > kMaxPop) return fail(SBLM_EINVAL, "n_pop=%d outside [2, %d]", n_pop, kMaxPop);
    if (n_par < 1 || n_par > SBLM_MAX_NPAR) return fail(SBLM_EINVAL, "n_par=%d outside [1, %d]", n_par, SBLM_MAX_NPAR);
    if ((long)n_pop * n_par >= (1L << kInitIndexBits)) return fail(SBLM_EINVAL, "n_pop * n_par too large");
    if (p->stag_window < 1 || p->stag_window > SBLM_MAX_WINDOW)
        return fail(SBLM_EINVAL, "stag_window=%d outside [1, %d]", p->stag_window, SBLM_MAX_WINDOW);
    if (!(p->p_mut0 >= 0.0 && p->p_mut0 <= 1.0)) return fail(SBLM_EINVAL, "p_mut0 must lie in [0, 1]");
    if (!(p->stag_rel >= 0.0) || !std::isfinite(p->stag_rel)) return fail(SBLM_EINVAL, "stag_rel must be >= 0");
    if (p->restart_after < 1) return fail(SBLM_EINVAL, "restart_after must be >= 1");
    if (p->n_tourn < 0) return fail(SBLM_EINVAL, "n_tourn must be >= 0");
    if (p->precision & SBLM_BLEND)
        return fail(SBLM_EINVAL, "SBLM_BLEND is taken by sblm_chi2_blend, the batched fitters and sblm_polish_batch");
    if (p->precision < SBLM_FP64 || p->precision > SBLM_FP32) return fail(SBLM_EINVAL, "unknown precision");
    EAConst c;
    c.n_pop = n_pop;
    c.n_par = n_par;
    c.n_tourn = p->n_tourn > 0 ? p->n_tourn : (n_pop + 24) / 25;
    c.stag_window = p->stag_window;
    c.restart_after = p->restart_after;
    c.p_mut0 = p->p_mut0;
    c.stag_rel = p->stag_rel;
    c.seed = p->seed;
    c.stream = stream_id;
    *out = c;
    return SBLM_OK;
}

cudaError_t launch_init(const EAConst& c, int gen, uint64_t* keys, double* P, cudaStream_t s) {
    const int m = c.n_pop * c.n_par;
    init_keys_kernel<<<blocks_for(m, 256), 256, 0, s>>>(c, gen, keys, m);
    init_values_kernel<<<blocks_for(m, 256), 256, 0, s>>>(c, gen, keys, m, P);
    return cudaGetLastError();
}

cudaError_t launch_state_reset(const EAConst& c, sblm_ea_state* state, cudaStream_t s) {
    state_reset_kernel<<<1, 32, 0, s>>>(c, state);
    return cudaGetLastError();
}

cudaError_t launch_rank(const EAConst& c, int gen, const double* chi2, const double* P, sblm_ea_state* state,
                        int* order, EACtrl* ctrl, uint64_t* keys, double* trace_row, bool produce, cudaStream_t s,
                        int n_pops) {
    int n2 = 1;
    while (n2 < c.n_pop) n2 <<= 1;
    const size_t smem = (size_t)n2 * (sizeof(double) + sizeof(int));
    // opt in beyond 48 KB (with the kernel's static shared memory)
    cudaError_t e = raise_smem_limit((const void*)rank_kernel, smem);
    if (e != cudaSuccess) return e;
    rank_kernel<<<n_pops, kRankThreads, smem, s>>>(c, gen, chi2, P, state, order, ctrl, keys, trace_row,
                                                   produce ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_offspring(const EAConst& c, int gen, const double* P, const int* order, const EACtrl* ctrl,
                             const uint64_t* keys, double* P_next, cudaStream_t s, int n_pops) {
    const int m = c.n_pop * c.n_par;
    offspring_kernel<<<dim3(blocks_for(m, 256), n_pops), 256, 0, s>>>(c, gen, P, order, ctrl, keys, P_next);
    return cudaGetLastError();
}

}  // namespace sblm

using namespace sblm;

extern "C" sblm_status sblm_ea_init(double* P, int32_t n_pop, int32_t n_par, const sblm_ea_params* params,
                                    uint64_t stream_id, sblm_ea_state* state, void* stream) {
    EAConst c;
    SBLM_TRY(ea_const(params, n_pop, n_par, stream_id, &c));
    if (!P || !state) return fail(SBLM_EINVAL, "P and state are required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    Staging st(s);
    const int m = n_pop * n_par;
    int i_P, i_s;
    SBLM_TRY(st.arg(P, sizeof(double) * m, false, true, &i_P));
    SBLM_TRY(st.arg(state, sizeof(sblm_ea_state), false, true, &i_s));
    const int k_keys = st.scratch(sizeof(uint64_t) * m);
    SBLM_TRY(st.begin());
    SBLM_CUDA(launch_init(c, 0, static_cast<uint64_t*>(st.scratch_ptr(k_keys)), static_cast<double*>(st.dev(i_P)), s));
    SBLM_CUDA(launch_state_reset(c, static_cast<sblm_ea_state*>(st.dev(i_s)), s));
    return st.end();
}

extern "C" sblm_status sblm_ea_generation(double* P, const double* chi2, int32_t n_pop, int32_t n_par,
                                          const sblm_ea_params* params, uint64_t stream_id, int32_t generation,
                                          sblm_ea_state* state, void* stream) {
    EAConst c;
    SBLM_TRY(ea_const(params, n_pop, n_par, stream_id, &c));
    if (!P || !chi2 || !state) return fail(SBLM_EINVAL, "P, chi2 and state are required");
    if (generation < 0) return fail(SBLM_EINVAL, "generation must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    Staging st(s);
    const int m = n_pop * n_par;
    int i_P, i_c, i_s;
    SBLM_TRY(st.arg(P, sizeof(double) * m, true, true, &i_P));
    SBLM_TRY(st.arg(chi2, sizeof(double) * n_pop, true, false, &i_c));
    SBLM_TRY(st.arg(state, sizeof(sblm_ea_state), true, true, &i_s));
    const int k_order = st.scratch(sizeof(int) * n_pop);
    const int k_ctrl = st.scratch(sizeof(EACtrl));
    const int k_keys = st.scratch(sizeof(uint64_t) * m);
    const int k_next = st.scratch(sizeof(double) * m);
    SBLM_TRY(st.begin());
    double* dP = static_cast<double*>(st.dev(i_P));
    double* dN = static_cast<double*>(st.scratch_ptr(k_next));
    int* order = static_cast<int*>(st.scratch_ptr(k_order));
    EACtrl* ctrl = static_cast<EACtrl*>(st.scratch_ptr(k_ctrl));
    uint64_t* keys = static_cast<uint64_t*>(st.scratch_ptr(k_keys));
    SBLM_CUDA(launch_rank(c, generation, static_cast<const double*>(st.dev(i_c)), dP,
                          static_cast<sblm_ea_state*>(st.dev(i_s)), order, ctrl, keys, nullptr, true, s));
    SBLM_CUDA(launch_offspring(c, generation, dP, order, ctrl, keys, dN, s));
    SBLM_CUDA(cudaMemcpyAsync(dP, dN, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    return st.end();
}

extern "C" sblm_status sblm_ea_generation_batch(double* P, const double* chi2, int32_t n_pops, int32_t n_pop,
                                                int32_t n_par, const sblm_ea_params* params, uint64_t stream_id0,
                                                int32_t generation, sblm_ea_state* states, void* stream) {
    EAConst c;
    SBLM_TRY(ea_const(params, n_pop, n_par, stream_id0, &c));
    if (n_pops < 1 || n_pops > 65535) return fail(SBLM_EINVAL, "n_pops=%d outside [1, 65535]", n_pops);
    if (!P || !chi2 || !states) return fail(SBLM_EINVAL, "P, chi2 and states are required");
    if (generation < 0) return fail(SBLM_EINVAL, "generation must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallLock lock;
    Staging st(s);
    const size_t m = (size_t)n_pop * n_par, all = m * n_pops;
    int i_P, i_c, i_s;
    SBLM_TRY(st.arg(P, sizeof(double) * all, true, true, &i_P));
    SBLM_TRY(st.arg(chi2, sizeof(double) * (size_t)n_pop * n_pops, true, false, &i_c));
    SBLM_TRY(st.arg(states, sizeof(sblm_ea_state) * (size_t)n_pops, true, true, &i_s));
    const int k_order = st.scratch(sizeof(int) * (size_t)n_pop * n_pops);
    const int k_ctrl = st.scratch(sizeof(EACtrl) * (size_t)n_pops);
    const int k_keys = st.scratch(sizeof(uint64_t) * all);
    const int k_next = st.scratch(sizeof(double) * all);
    SBLM_TRY(st.begin());
    double* dP = static_cast<double*>(st.dev(i_P));
    double* dN = static_cast<double*>(st.scratch_ptr(k_next));
    int* order = static_cast<int*>(st.scratch_ptr(k_order));
    EACtrl* ctrl = static_cast<EACtrl*>(st.scratch_ptr(k_ctrl));
    uint64_t* keys = static_cast<uint64_t*>(st.scratch_ptr(k_keys));
    SBLM_CUDA(launch_rank(c, generation, static_cast<const double*>(st.dev(i_c)), dP,
                          static_cast<sblm_ea_state*>(st.dev(i_s)), order, ctrl, keys, nullptr, true, s, n_pops));
    SBLM_CUDA(launch_offspring(c, generation, dP, order, ctrl, keys, dN, s, n_pops));
    SBLM_CUDA(cudaMemcpyAsync(dP, dN, sizeof(double) * all, cudaMemcpyDeviceToDevice, s));
    return st.end();
}

// ---------------------------------------------------------------------------------------------
// sblm_ea_generation_noalloc: the generation above with its scratch (ranking order, control word,
// initialisation keys, next population) in one fixed device array instead of the workspace.
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxPop = 8192;      // largest N_pop
constexpr int kNoAllocMaxElems = 32768;   // largest N_pop * N_par
constexpr size_t kNoAllocOrder = 0;                                              // int32 [N_pop]
constexpr size_t kNoAllocCtrl = kNoAllocOrder + sizeof(int) * kNoAllocMaxPop;    // EACtrl
constexpr size_t kNoAllocKeys = kNoAllocCtrl + 256;                              // uint64 [M]
static_assert(sizeof(EACtrl) <= 256, "the control word's slot in the fixed scratch is 256 bytes");
constexpr size_t kNoAllocNext = kNoAllocKeys + sizeof(uint64_t) * kNoAllocMaxElems;  // double [M]
constexpr size_t kNoAllocBytes = kNoAllocNext + sizeof(double) * kNoAllocMaxElems;   // 544 KiB + 256 B

// Every GPU that loads the library holds this array until the process exits. Its name is a
// host-side stand-in in host code: kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_ea_scratch[kNoAllocBytes];

std::mutex g_noalloc_lock;
void* g_noalloc_base[64] = {};

// device address of g_ea_scratch on the current device, looked up once per device
sblm_status noalloc_base(void** out) {
    int dev = 0;
    SBLM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(SBLM_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> g(g_noalloc_lock);
    if (!g_noalloc_base[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_ea_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(SBLM_ECUDA, "cudaGetSymbolAddress of the fixed EA scratch failed: %s", cudaGetErrorString(e));
        }
        g_noalloc_base[dev] = p;
    }
    *out = g_noalloc_base[dev];
    return SBLM_OK;
}

}  // namespace

extern "C" sblm_status sblm_ea_generation_noalloc(double* P, const double* chi2, int32_t n_pop, int32_t n_par,
                                                  const sblm_ea_params* params, uint64_t stream_id,
                                                  int32_t generation, sblm_ea_state* state, void* stream) {
    EAConst c;
    SBLM_TRY(ea_const(params, n_pop, n_par, stream_id, &c));
    if (n_pop > kNoAllocMaxPop || (long)n_pop * n_par > kNoAllocMaxElems)
        return fail(SBLM_EINVAL,
                    "sblm_ea_generation_noalloc: n_pop=%d, n_par=%d exceed its fixed scratch "
                    "(n_pop <= %d and n_pop * n_par <= %d)",
                    n_pop, n_par, kNoAllocMaxPop, kNoAllocMaxElems);
    if (!P || !chi2 || !state) return fail(SBLM_EINVAL, "P, chi2 and state are required");
    if (generation < 0) return fail(SBLM_EINVAL, "generation must be >= 0");
    const void* ptrs[3] = {P, chi2, state};
    for (const void* p : ptrs) {
        bool on_dev = false;
        SBLM_TRY(is_device_pointer(p, &on_dev));
        if (!on_dev)
            return fail(SBLM_EINVAL, "sblm_ea_generation_noalloc takes device memory only (%p is host memory)", p);
    }
    void* base = nullptr;
    SBLM_TRY(noalloc_base(&base));
    char* b = static_cast<char*>(base);
    int* order = reinterpret_cast<int*>(b + kNoAllocOrder);
    EACtrl* ctrl = reinterpret_cast<EACtrl*>(b + kNoAllocCtrl);
    uint64_t* keys = reinterpret_cast<uint64_t*>(b + kNoAllocKeys);
    double* next = reinterpret_cast<double*>(b + kNoAllocNext);
    // nothing in the array has to start at zero: the ranking writes order and ctrl (and keys on
    // a restart) before the offspring kernel reads them, and the offspring kernel writes every
    // element of next before it is copied into P
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SBLM_CUDA(launch_rank(c, generation, chi2, P, state, order, ctrl, keys, nullptr, true, s));
    SBLM_CUDA(launch_offspring(c, generation, P, order, ctrl, keys, next, s));
    SBLM_CUDA(cudaMemcpyAsync(P, next, sizeof(double) * (size_t)n_pop * n_par, cudaMemcpyDeviceToDevice, s));
    SBLM_CUDA(cudaGetLastError());
    return SBLM_OK;
}
