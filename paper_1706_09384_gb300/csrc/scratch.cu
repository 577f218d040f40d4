// scratch.cu — the library's scratch memory for solver and build temporaries.
//
// Temporaries of a solve (the GMRES basis, its small Hessenberg problem,
// partial sums) and of a build (the ACA factors and their double-float
// copies, the staged factors) come from a stream-ordered memory pool that the
// library creates per device (cudaMemPoolCreate) with its release threshold at
// the maximum, so memory freed stays reserved in the pool and the next solve
// or build, on this or any other handle, takes it back without a cudaMalloc,
// a cudaFree (tens of milliseconds for the tens of gigabytes of an ACA batch)
// or a device-wide synchronisation.  The pool's unused memory is returned to
// the device by hm_release_cached_memory and when the process exits.  Small
// pinned host buffers for reading scalars back are kept in a process-wide
// free list.
#include <mutex>
#include <vector>

#include "hm_internal.h"

namespace {

constexpr int SC_MAX_DEVICES = 64;
std::mutex g_sc_mutex;
cudaMemPool_t g_pool[SC_MAX_DEVICES] = {};

struct Pinned {
    void* p;
    size_t bytes;
    bool used;
};
std::vector<Pinned> g_pinned;

cudaMemPool_t pool_of_current_device() {
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= SC_MAX_DEVICES) hm_throw(HM_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_sc_mutex);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        HM_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t keep = ~0ull;
        HM_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pool[dev] = p;
    }
    return g_pool[dev];
}

}  // namespace

void* hm_scratch_alloc(size_t bytes, cudaStream_t st) {
    void* p = nullptr;
    cudaMemPool_t pool = pool_of_current_device();
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, pool, st);
    if (e == cudaErrorMemoryAllocation) {
        // the pool's reserved pieces may not fit this request: hand them back
        // to the device (once the stream's frees are done) and try once more
        cudaGetLastError();
        HM_CUDA(cudaStreamSynchronize(st));
        HM_CUDA(cudaMemPoolTrimTo(pool, 0));
        e = cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, pool, st);
    }
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        hm_throw(HM_ERR_OOM, "device memory exhausted (library scratch)");
    }
    HM_CUDA(e);
    return p;
}

size_t hm_scratch_cached() {
    cudaMemPool_t pool = pool_of_current_device();
    uint64_t res = 0, used = 0;
    HM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &res));
    HM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    return res > used ? (size_t)(res - used) : 0;
}

void hm_scratch_trim() {
    std::lock_guard<std::mutex> lk(g_sc_mutex);
    for (int d = 0; d < SC_MAX_DEVICES; ++d)
        if (g_pool[d]) HM_CUDA(cudaMemPoolTrimTo(g_pool[d], 0));
}

void hm_scratch_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

void* hm_pinned_take(size_t bytes) {
    std::lock_guard<std::mutex> lk(g_sc_mutex);
    for (Pinned& b : g_pinned)
        if (!b.used && b.bytes >= bytes) {
            b.used = true;
            return b.p;
        }
    void* p = nullptr;
    HM_CUDA(cudaMallocHost(&p, bytes < 4096 ? 4096 : bytes));
    g_pinned.push_back({p, bytes < 4096 ? 4096 : bytes, true});
    return p;
}

void hm_pinned_give(void* p) {
    std::lock_guard<std::mutex> lk(g_sc_mutex);
    for (Pinned& b : g_pinned)
        if (b.p == p) b.used = false;
}
