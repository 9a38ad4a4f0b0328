// runtime.cuh -- host-side plumbing of the SBLM library: error reporting, pointer location,
// per-(device, stream) workspace and host<->device staging of call arguments.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <vector>

#include "../../include/sblm.h"

namespace sblm {

// Record a failure for sblm_last_error() and return its status.
sblm_status fail(sblm_status s, const char* fmt, ...);
sblm_status cuda_fail(cudaError_t e, const char* what);

#define SBLM_CUDA(call)                                                    \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ::sblm::cuda_fail(e_, #call);        \
    } while (0)

#define SBLM_TRY(expr)                                \
    do {                                              \
        sblm_status s_ = (expr);                      \
        if (s_ != SBLM_OK) return s_;                 \
    } while (0)

// True if the device can dereference p directly (device or managed memory of the current
// device); false for host memory, pageable or pinned. EINVAL for another device's memory.
sblm_status is_device_pointer(const void* p, bool* on_device);

// A call's scratch: one contiguous workspace per (device, stream), grown on demand (the
// stream is synchronised before an old buffer is freed). Slices are 256-byte aligned.
class Scratch {
   public:
    explicit Scratch(cudaStream_t s) : stream_(s) {}
    // reserve `bytes` and return the slice index
    int add(size_t bytes);
    // allocate (or reuse) the workspace for all slices added so far
    sblm_status commit();
    void* ptr(int slice) const { return base_ + offsets_[slice]; }
    template <typename T>
    T* as(int slice) const { return reinterpret_cast<T*>(ptr(slice)); }

   private:
    cudaStream_t stream_;
    std::vector<size_t> offsets_;
    size_t total_ = 0;
    char* base_ = nullptr;
};

// Arguments of one call: host pointers get a workspace slice with copies in before the
// kernels and out after them; device pointers are used as they are.
class Staging {
   public:
    explicit Staging(cudaStream_t s) : stream_(s), scratch_(s) {}
    // register an argument; returns its index. `bytes` may be 0 (then p may be NULL).
    sblm_status arg(const void* p, size_t bytes, bool in, bool out, int* index);
    // extra device scratch of the call
    int scratch(size_t bytes) { return scratch_.add(bytes); }
    // allocate workspace and copy inputs; afterwards dev() and scratch_ptr() are valid
    sblm_status begin();
    void* dev(int index) const;
    void* scratch_ptr(int slice) const { return scratch_.ptr(slice); }
    bool any_host() const;
    // copy outputs back and synchronise if any argument was on the host
    sblm_status end();
    cudaStream_t stream() const { return stream_; }

   private:
    struct A {
        const void* user;
        size_t bytes;
        bool in, out, host;
        int slice;
    };
    cudaStream_t stream_;
    Scratch scratch_;
    std::vector<A> args_;
};

// Runs `enqueue` through a CUDA graph: the first call with a given key captures its launches
// (on a private stream) and instantiates them; later calls with the same key replay the graph on
// `s`. The last few graphs are kept. Kernel attributes that enqueue sets are set before capture
// by a dry pass only if the caller did so itself; enqueue must only enqueue stream work.
sblm_status run_cached_graph(const std::vector<unsigned char>& key,
                             const std::function<cudaError_t(cudaStream_t)>& enqueue, cudaStream_t s);

// Raise, never lower, the dynamic shared-memory limit of kernel `func` on the current device to
// at least `bytes` (thread-safe; remembered per kernel and device). Call it before a launch, and
// before any stream capture that contains the launch.
cudaError_t raise_smem_limit(const void* func, size_t bytes);

// Streaming multiprocessors of the current device (queried once per device; 1 if unknown).
int device_sm_count();

// Serialises calls that use a workspace (the lock is per process; calls are short to enqueue).
struct CallLock {
    CallLock();
    ~CallLock();
};

}  // namespace sblm
