// The library's device memory pool.
//
// Every device array the library allocates (graph arrays, tile tables, EM
// workspace, build temporaries) comes from one stream-ordered pool per device,
// created on first use.  Its release threshold is unbounded, so memory a
// destroyed graph gave back stays mapped and the next build of a batch of the
// same size reuses it instead of mapping fresh pages at every synchronisation
// (which is what a pool with threshold 0 does).  pmrf_trim_memory hands the
// unused part back to the driver.
#include "common.cuh"

#include <mutex>

namespace pmrf {
namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[MAX_DEVICES] = {};

}  // namespace

cudaMemPool_t lib_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaGetLastError();
            cudaMemPoolDestroy(p);
            return nullptr;
        }
        g_pool[dev] = p;
    }
    return g_pool[dev];
}

int pool_trim(int64_t keep_bytes) {
    cudaMemPool_t p = lib_pool();
    if (!p) return fail(PMRF_ERR_CUDA, "memory pool unavailable");
    PMRF_CUDA(cudaDeviceSynchronize());
    PMRF_CUDA(cudaMemPoolTrimTo(p, (size_t)std::max<int64_t>(keep_bytes, 0)));
    return PMRF_OK;
}

int pool_usage(int64_t* reserved, int64_t* used) {
    cudaMemPool_t p = lib_pool();
    if (!p) return fail(PMRF_ERR_CUDA, "memory pool unavailable");
    uint64_t r = 0, u = 0;
    PMRF_CUDA(cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &r));
    PMRF_CUDA(cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &u));
    if (reserved) *reserved = (int64_t)r;
    if (used) *used = (int64_t)u;
    return PMRF_OK;
}

}  // namespace pmrf
