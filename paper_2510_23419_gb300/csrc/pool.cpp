// pool.cpp -- device memory and stream resources of the library: a per-device
// stream-ordered memory pool with its allocation stream, and a per-device set
// of non-blocking launch streams for batches and the request server.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "pb_handles.h"

namespace pb {

namespace {

constexpr int kMaxDevices = 64;
constexpr int kLaunchStreams = 32;

struct DeviceRes {
    bool init = false;
    cudaMemPool_t pool = nullptr;
    cudaStream_t alloc_st = nullptr;
    cudaStream_t launch[kLaunchStreams] = {};
};

std::mutex g_res_mutex;
DeviceRes g_res[kMaxDevices];

// Resources of the current device, created on first use.
DeviceRes* device_res()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_res_mutex);
    DeviceRes& r = g_res[dev];
    if (!r.init) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&r.pool, &props) != cudaSuccess) return nullptr;
        uint64_t keep = UINT64_MAX;  // keep freed memory in the pool for reuse
        cudaMemPoolSetAttribute(r.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (cudaStreamCreateWithFlags(&r.alloc_st, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        for (int k = 0; k < kLaunchStreams; ++k)
            if (cudaStreamCreateWithFlags(&r.launch[k], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        r.init = true;
    }
    return &r;
}

}  // namespace

cudaError_t pool_alloc(void** p, size_t n)
{
    DeviceRes* r = device_res();
    if (!r) return cudaErrorInitializationError;
    cudaError_t e = cudaMallocFromPoolAsync(p, n, r->pool, r->alloc_st);
    if (e != cudaSuccess) return e;
    // the allocation is usable from every stream once the allocation stream has passed it
    return cudaStreamSynchronize(r->alloc_st);
}

void pool_free(void* p)
{
    DeviceRes* r = device_res();
    if (r) cudaFreeAsync(p, r->alloc_st);
}

cudaStream_t pool_stream(int k)
{
    DeviceRes* r = device_res();
    return r ? r->launch[((k % kLaunchStreams) + kLaunchStreams) % kLaunchStreams] : nullptr;
}

int pool_streams() { return kLaunchStreams; }

}  // namespace pb
