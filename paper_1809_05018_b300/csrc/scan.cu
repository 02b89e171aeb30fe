// scan.cu -- exclusive prefix sums (int64 results) used to turn per-item
// counts into CSR offsets.  Reduce-then-scan in three passes: per-block totals,
// a scan of the totals (recursively), and a per-block scan with its offset.
#include "common.cuh"

namespace pmrf {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 4096

template <typename Tin>
__global__ void __launch_bounds__(SCAN_THREADS) k_block_totals(const Tin* __restrict__ in, int64_t n,
                                                               int64_t* __restrict__ totals) {
    __shared__ int64_t sh[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t acc = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) acc += (int64_t)in[i];
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) totals[blockIdx.x] = acc;
}

// Exclusive scan of one tile of SCAN_TILE items starting at blockIdx.x*SCAN_TILE;
// adds offs[blockIdx.x] (if offs) to every output; writes out[n] = total when
// this block holds the last item.
template <typename Tin>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const Tin* __restrict__ in, int64_t n,
                                                            const int64_t* __restrict__ offs,
                                                            int64_t* __restrict__ out) {
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t tsum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + k;
        v[k] = (i < n) ? (int64_t)in[i] : 0;
        tsum += v[k];
    }
    // inclusive scan of thread sums inside the warp
    int64_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane_id() >= o) x += y;
    }
    if (lane_id() == 31) wsum[warp_id()] = x;
    __syncthreads();
    if (warp_id() == 0) {
        int64_t w = (lane_id() < SCAN_THREADS / 32) ? wsum[lane_id()] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane_id() >= o) w += y;
        }
        if (lane_id() < SCAN_THREADS / 32) wsum[lane_id()] = w;  // inclusive warp prefix
    }
    __syncthreads();
    int64_t run = (x - tsum) + (warp_id() > 0 ? wsum[warp_id() - 1] : 0) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
        if (i == n - 1) out[n] = run;
    }
}

template <typename Tin>
int scan_impl(const Tin* in, int64_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        PMRF_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return PMRF_OK;
    }
    const int64_t nb = ceil_div(n, SCAN_TILE);
    if (nb == 1) {
        k_tile_scan<Tin><<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out); ::pmrf::note_launch(1);
        PMRF_CUDA(cudaGetLastError());
        return PMRF_OK;
    }
    if (nb > 2147483647ll) return fail(PMRF_ERR_UNSUPPORTED, "scan too long");
    int64_t* totals = nullptr;
    int64_t* toffs = nullptr;
    PMRF_TRY(dalloc(&totals, nb, s));
    int rc = dalloc(&toffs, nb + 1, s);
    if (rc) { dfree(totals, s); return rc; }
    k_block_totals<Tin><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, totals); ::pmrf::note_launch(1);
    rc = scan_impl<int64_t>(totals, toffs, nb, s);
    if (!rc) {
        k_tile_scan<Tin><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, toffs, out); ::pmrf::note_launch(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "k_tile_scan");
    }
    dfree(totals, s);
    dfree(toffs, s);
    return rc;
}

}  // namespace

int exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, s);
}
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, s);
}
int read_i64(const int64_t* d, int64_t* h, cudaStream_t s) {
    PMRF_CUDA(cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PMRF_CUDA(cudaStreamSynchronize(s));
    return PMRF_OK;
}

}  // namespace pmrf
