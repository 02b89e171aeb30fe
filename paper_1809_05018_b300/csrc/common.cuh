// common.cuh -- shared helpers of the PMRF CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pmrf.h"

namespace pmrf {

// ---------------------------------------------------------------------------
// host-side error plumbing

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define PMRF_CUDA(call)                                     \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ::pmrf::cuda_fail(e_, #call); \
    } while (0)

#define PMRF_TRY(call)              \
    do {                            \
        int rc_ = (call);           \
        if (rc_ != PMRF_OK) return rc_; \
    } while (0)

// Device status word: kernels record the first error they meet (never trap).
struct DevStatus {
    int32_t code;      // pmrf_status
    int32_t where;     // kernel-specific site id
    int64_t detail;    // kernel-specific value (e.g. an index)
};

__device__ __forceinline__ void record_error(DevStatus* st, int code, int where, int64_t detail) {
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->where = where;
        st->detail = detail;
    }
}

// sites recorded in DevStatus::where
enum Site : int32_t {
    SITE_NONE = 0,
    SITE_BAD_ID = 1,
    SITE_NONFINITE = 2,
    SITE_DEGREE = 3,
    SITE_HOOD_TILE = 4,
    SITE_MCE_STACK = 5,
    SITE_SORT = 6,
    SITE_LABEL = 7,
    SITE_WAIT = 8,
    SITE_RANGE = 9,   // energies beyond the fixed point's range (non-finite bound)
};

// ---------------------------------------------------------------------------
// device helpers

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block-wide sum: fixed shuffle tree inside warps, then warp 0
// sums the per-warp values in warp order.  `sh` needs blockDim.x/32 slots.
// Every thread returns the total.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
    v = warp_sum(v);
    if (lane_id() == 0) sh[warp_id()] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    T t = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
    if (warp_id() == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    T r = sh[0];
    __syncthreads();
    return r;
}

// first index i in [lo, hi) with a[i] >= key (a ascending)
template <typename T>
__device__ __forceinline__ int64_t lower_bound_dev(const T* a, int64_t lo, int64_t hi, T key) {
    while (lo < hi) {
        int64_t m = lo + ((hi - lo) >> 1);
        if (a[m] < key) lo = m + 1; else hi = m;
    }
    return lo;
}
// last index i in [lo, hi) with a[i] <= key, i.e. upper_bound - 1
template <typename T>
__device__ __forceinline__ int64_t upper_bound_dev(const T* a, int64_t lo, int64_t hi, T key) {
    while (lo < hi) {
        int64_t m = lo + ((hi - lo) >> 1);
        if (a[m] <= key) lo = m + 1; else hi = m;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// primitives implemented in scan.cu / segsort.cu

// out[i] = sum_{j<i} in[j] for i in [0, n]; out has n+1 entries (out[n] = total).
// `in` may be int32 or int64 counts.  Scratch is allocated internally from
// the library pool on `s`.
int exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
// read one device value (synchronous)
int read_i64(const int64_t* d, int64_t* h, cudaStream_t s);

// Sort each segment [off[k], off[k+1]) of `vals` ascending, in place.  With
// `unique` set, also drop repeated values: the unique values move to the front
// of the segment and `ucount[k]` receives their number (ucount may be NULL
// when unique == false).  Segments are processed in shared memory when they
// fit, else by a per-segment bitmap over the segment's value range.
int segmented_sort_u32(uint32_t* vals, const int64_t* off, int64_t nseg, int64_t n, bool unique,
                       int32_t* ucount, DevStatus* st, cudaStream_t s);

// Kernel-launch accounting (pmrf_launch_count): every launch site calls
// note_launch(1).  While a CUDA graph is being captured the launches are
// counted into the capture's own counter instead, and each replay of the graph
// adds that count.
void note_launch(int64_t n);
void set_capture_counter(int64_t* counter);
// a device word that kernels inside conditional graph bodies add their count
// to (pmrf_launch_count adds it in); NULL when it cannot be created
unsigned long long* device_launch_counter();

// The library's stream-ordered memory pool on the current device (pool.cu):
// created on first use, it keeps the memory freed into it mapped for reuse.
// NULL when it cannot be created.
cudaMemPool_t lib_pool();
int pool_trim(int64_t keep_bytes);
int pool_usage(int64_t* reserved, int64_t* used);

// Device allocation helpers (stream ordered, from lib_pool()).
template <typename T>
int dalloc(T** p, int64_t n, cudaStream_t s) {
    *p = nullptr;
    size_t bytes = (size_t)(n > 0 ? n : 1) * sizeof(T) + 16;  // +16: padded tail for vector reads
    cudaMemPool_t pool = lib_pool();
    if (!pool) return fail(PMRF_ERR_CUDA, "device memory pool unavailable");
    cudaError_t e = cudaMallocFromPoolAsync((void**)p, bytes, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PMRF_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return PMRF_OK;
}
template <typename T>
void dfree(T*& p, cudaStream_t s) {
    if (p) cudaFreeAsync((void*)p, s);
    p = nullptr;
}

}  // namespace pmrf
