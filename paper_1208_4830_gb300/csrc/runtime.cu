// runtime.cu -- status strings, error reporting, pointer location, workspace, staging.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "runtime.cuh"

namespace sblm {

namespace {
thread_local std::string g_last_error;
std::recursive_mutex g_lock;

struct Workspace {
    void* ptr = nullptr;
    size_t size = 0;
};
// keyed by (device, stream); guarded by g_lock
std::map<std::pair<int, cudaStream_t>, Workspace>& workspaces() {
    static auto* m = new std::map<std::pair<int, cudaStream_t>, Workspace>();
    return *m;
}
}  // namespace

sblm_status fail(sblm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

sblm_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? SBLM_ENOMEM : SBLM_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

CallLock::CallLock() { g_lock.lock(); }
CallLock::~CallLock() { g_lock.unlock(); }

namespace {
std::mutex g_smem_lock;
std::map<std::pair<const void*, int>, size_t> g_smem_granted;
}  // namespace

int device_sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    int sms = dev < 64 ? cached[dev].load() : 0;
    if (sms > 0) return sms;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return 1;
    }
    if (dev < 64) cached[dev].store(sms);
    return sms;
}

cudaError_t raise_smem_limit(const void* func, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(g_smem_lock);
    size_t& granted = g_smem_granted[{func, dev}];
    if (bytes <= granted) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) granted = bytes;
    return e;
}

sblm_status is_device_pointer(const void* p, bool* on_device) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();  // older drivers report plain host memory as an error
        *on_device = false;
        return SBLM_OK;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        int dev = 0;
        SBLM_CUDA(cudaGetDevice(&dev));
        if (a.type == cudaMemoryTypeDevice && a.device != dev)
            return fail(SBLM_EINVAL, "pointer %p belongs to device %d, current device is %d", p, a.device, dev);
        *on_device = true;
    } else {
        *on_device = false;
    }
    return SBLM_OK;
}

int Scratch::add(size_t bytes) {
    const size_t aligned = (total_ + 255) & ~size_t(255);
    offsets_.push_back(aligned);
    total_ = aligned + bytes;
    return (int)offsets_.size() - 1;
}

sblm_status Scratch::commit() {
    if (total_ == 0) return SBLM_OK;
    int dev = 0;
    SBLM_CUDA(cudaGetDevice(&dev));
    Workspace& w = workspaces()[{dev, stream_}];
    if (w.size < total_) {
        if (w.ptr) {
            SBLM_CUDA(cudaStreamSynchronize(stream_));
            SBLM_CUDA(cudaFree(w.ptr));
            w.ptr = nullptr;
            w.size = 0;
        }
        const size_t want = total_ + total_ / 4;
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SBLM_ENOMEM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
        }
        w.ptr = p;
        w.size = want;
    }
    base_ = static_cast<char*>(w.ptr);
    return SBLM_OK;
}

sblm_status Staging::arg(const void* p, size_t bytes, bool in, bool out, int* index) {
    A a{p, bytes, in, out, false, -1};
    if (bytes > 0) {
        if (!p) return fail(SBLM_EINVAL, "NULL pointer for a buffer of %zu bytes", bytes);
        bool on_dev = false;
        SBLM_TRY(is_device_pointer(p, &on_dev));
        a.host = !on_dev;
        if (a.host) a.slice = scratch_.add(bytes);
    }
    args_.push_back(a);
    *index = (int)args_.size() - 1;
    return SBLM_OK;
}

sblm_status Staging::begin() {
    SBLM_TRY(scratch_.commit());
    for (const A& a : args_)
        if (a.host && a.in)
            SBLM_CUDA(cudaMemcpyAsync(scratch_.ptr(a.slice), a.user, a.bytes, cudaMemcpyHostToDevice, stream_));
    return SBLM_OK;
}

void* Staging::dev(int index) const {
    const A& a = args_[index];
    if (a.bytes == 0) return const_cast<void*>(a.user);
    return a.host ? scratch_.ptr(a.slice) : const_cast<void*>(a.user);
}

bool Staging::any_host() const {
    for (const A& a : args_)
        if (a.host) return true;
    return false;
}

sblm_status Staging::end() {
    SBLM_CUDA(cudaGetLastError());
    bool host = false;
    for (const A& a : args_) {
        if (a.host && a.out)
            SBLM_CUDA(cudaMemcpyAsync(const_cast<void*>(a.user), scratch_.ptr(a.slice), a.bytes,
                                      cudaMemcpyDeviceToHost, stream_));
        host = host || a.host;
    }
    if (host) SBLM_CUDA(cudaStreamSynchronize(stream_));
    return SBLM_OK;
}

namespace {
struct CachedGraph {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
};
std::vector<CachedGraph>& graph_cache() {
    static auto* v = new std::vector<CachedGraph>();
    return *v;
}
constexpr size_t kGraphCacheSize = 8;
}  // namespace

sblm_status run_cached_graph(const std::vector<unsigned char>& key,
                             const std::function<cudaError_t(cudaStream_t)>& enqueue, cudaStream_t s) {
    auto& cache = graph_cache();
    for (size_t i = 0; i < cache.size(); ++i) {
        if (cache[i].key == key) {
            SBLM_CUDA(cudaGraphLaunch(cache[i].exec, s));
            return SBLM_OK;
        }
    }
    // kernels that opt in to more shared memory set their attribute on the first launch; run the
    // launches once on the caller's stream (this is also the first execution), then capture
    SBLM_CUDA(enqueue(s));
    cudaStream_t cap;
    SBLM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t e1 = enqueue(cap);
        e = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess && e1 != cudaSuccess) e = e1;
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return SBLM_OK;  // the launches already ran directly; no graph for this key
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SBLM_OK;
    }
    if (cache.size() >= kGraphCacheSize) {
        cudaGraphExecDestroy(cache.front().exec);
        cache.erase(cache.begin());
    }
    cache.push_back({key, exec});
    return SBLM_OK;
}

}  // namespace sblm

extern "C" {

const char* sblm_status_str(sblm_status s) {
    switch (s) {
        case SBLM_OK: return "SBLM_OK";
        case SBLM_EINVAL: return "SBLM_EINVAL";
        case SBLM_ENOMEM: return "SBLM_ENOMEM";
        case SBLM_ECUDA: return "SBLM_ECUDA";
        case SBLM_ETIMEOUT: return "SBLM_ETIMEOUT";
        case SBLM_ENUMERIC: return "SBLM_ENUMERIC";
    }
    return "SBLM_UNKNOWN";
}

const char* sblm_last_error(void) { return sblm::g_last_error.c_str(); }

void sblm_ea_params_default(sblm_ea_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->n_pop = 1000;
    p->n_gen = 100;
    p->p_mut0 = 0.01;
    p->n_tourn = 0;
    p->stag_window = 10;
    p->stag_rel = 0.01;
    p->restart_after = 10;
    p->precision = SBLM_MIXED;
    p->polish_fev = 0;
    p->seed = 0;
    p->n_islands = 1;
    p->migration_interval = 20;
    p->polish_starts = 1;
    p->polish_radius = 0.05;
}

}  // extern "C"
