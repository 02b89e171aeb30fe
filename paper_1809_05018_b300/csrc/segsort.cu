// segsort.cu -- segmented ascending sort (optionally with de-duplication) of
// u32 values laid out as CSR segments.  Used by the graph build for
//   * the pixel list of each region (row-major order => the region sum is
//     added in row-major order),
//   * the candidate neighbour list of each region (sort + unique => CSR
//     adjacency),
//   * the replica list of each vertex (hoods containing it, ascending).
//
// Short segments (<= 256 values) are sorted by one warp each in registers;
// medium ones (<= SMALL_MAX) by a CTA with a shared-memory bitonic network.  Larger
// segments are sorted through a bitmap over their value range (one CTA per
// segment), which requires distinct values unless `unique` is requested.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace pmrf {

namespace {

constexpr int SORT_THREADS = 512;
constexpr int SMALL_MAX = 2048;      // longest segment sorted in shared memory
constexpr int WARP_MAX = 256;        // longest segment sorted by one warp in registers

__device__ __forceinline__ void bitonic_sort_smem(uint64_t* key, int npow2) {
    for (int k = 2; k <= npow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    uint64_t a = key[i], b = key[ixj];
                    bool up = ((i & k) == 0);
                    if ((a > b) == up) {
                        key[i] = b;
                        key[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// One CTA per listed medium segment (WARP_MAX < length <= SMALL_MAX): bitonic
// sort of the segment in shared memory.
__global__ void __launch_bounds__(SORT_THREADS) k_sort_medium(uint32_t* __restrict__ vals,
                                                              const int64_t* __restrict__ off,
                                                              const int64_t* __restrict__ list, int unique,
                                                              int32_t* __restrict__ ucount) {
    __shared__ uint64_t key[SMALL_MAX];
    const int64_t k = list[blockIdx.x];
    const int64_t gstart = off[k];
    const int cnt = (int)(off[k + 1] - gstart);
    int npow2 = 1;
    while (npow2 < cnt) npow2 <<= 1;
    for (int i = threadIdx.x; i < npow2; i += blockDim.x) key[i] = (i < cnt) ? (uint64_t)vals[gstart + i] : ~0ull;
    __syncthreads();
    bitonic_sort_smem(key, npow2);
    if (!unique) {
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) vals[gstart + i] = (uint32_t)key[i];
    } else if (threadIdx.x == 0) {
        int u = 0;
        for (int i = 0; i < cnt; ++i)
            if (i == 0 || key[i] != key[i - 1]) vals[gstart + u++] = (uint32_t)key[i];
        ucount[k] = u;
    }
}

// Segments of at most 32*E values: one warp per segment, E values per lane in
// registers (lane l holds positions l*E .. l*E+E-1), bitonic network with
// in-register exchanges for distances below E and shuffles above.
template <int E>
__device__ __forceinline__ void warp_sort_seg(uint32_t* __restrict__ vals, int64_t b, int len, bool unique,
                                              int32_t* __restrict__ ucount, int64_t k) {
    constexpr int N = 32 * E;
    const int lane = lane_id();
    uint32_t a[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = lane * E + r;
        a[r] = i < len ? vals[b + i] : 0xffffffffu;
    }
#pragma unroll
    for (int kk = 2; kk <= N; kk <<= 1) {
#pragma unroll
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            if (jj >= E) {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int i = lane * E + r;
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, a[r], jj / E);
                    const bool up = (i & kk) == 0;
                    const bool lower = (i & jj) == 0;
                    a[r] = (lower == up) ? min(a[r], o) : max(a[r], o);
                }
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    if ((r & jj) == 0) {
                        const int r2 = r | jj;
                        const bool up = ((lane * E + r) & kk) == 0;
                        const uint32_t x = a[r], y = a[r2];
                        if ((x > y) == up) {
                            a[r] = y;
                            a[r2] = x;
                        }
                    }
                }
            }
        }
    }
    if (!unique) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int i = lane * E + r;
            if (i < len) vals[b + i] = a[r];
        }
        return;
    }
    // keep the first of each run of equal values
    const uint32_t prev_last = __shfl_up_sync(0xffffffffu, a[E - 1], 1);
    int c = 0;
    bool f[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = lane * E + r;
        const uint32_t prev = (r == 0) ? prev_last : a[r - 1];
        f[r] = (i < len) && (i == 0 || a[r] != prev);
        c += f[r];
    }
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    int pos = x - c;
#pragma unroll
    for (int r = 0; r < E; ++r)
        if (f[r]) vals[b + pos++] = a[r];
    if (lane == 31) ucount[k] = x;
}

__global__ void __launch_bounds__(256) k_sort_warp(uint32_t* __restrict__ vals, const int64_t* __restrict__ off,
                                                   int64_t nseg, int unique, int32_t* __restrict__ ucount) {
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); k < nseg; k += warps) {
        const int64_t b = off[k];
        const int64_t n64 = off[k + 1] - b;
        const int len = n64 > WARP_MAX ? WARP_MAX + 1 : (int)n64;
        if (len <= 1) {
            if (unique && lane_id() == 0) ucount[k] = len;
        } else if (len <= 32) {
            warp_sort_seg<1>(vals, b, len, unique, ucount, k);
        } else if (len <= 64) {
            warp_sort_seg<2>(vals, b, len, unique, ucount, k);
        } else if (len <= 128) {
            warp_sort_seg<4>(vals, b, len, unique, ucount, k);
        } else if (len <= WARP_MAX) {
            warp_sort_seg<8>(vals, b, len, unique, ucount, k);
        }
    }
}

__global__ void k_mark_long(const int64_t* __restrict__ off, int64_t nseg, int64_t* __restrict__ mlist,
                            int32_t* __restrict__ nm, int64_t* __restrict__ blist, int32_t* __restrict__ nb) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nseg) return;
    const int64_t len = off[k + 1] - off[k];
    if (len > SMALL_MAX) blist[atomicAdd(nb, 1)] = k;
    else if (len > WARP_MAX) mlist[atomicAdd(nm, 1)] = k;
}

__global__ void __launch_bounds__(1024) k_big_minmax(const uint32_t* __restrict__ vals,
                                                     const int64_t* __restrict__ off,
                                                     const int64_t* __restrict__ list,
                                                     uint32_t* __restrict__ mn, uint32_t* __restrict__ mx) {
    __shared__ uint32_t smin[32], smax[32];
    const int64_t k = list[blockIdx.x];
    uint32_t a = 0xffffffffu, b = 0;
    for (int64_t i = off[k] + threadIdx.x; i < off[k + 1]; i += blockDim.x) {
        uint32_t v = vals[i];
        a = min(a, v);
        b = max(b, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if (lane_id() == 0) { smin[warp_id()] = a; smax[warp_id()] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { a = min(a, smin[w]); b = max(b, smax[w]); }
        a = min(a, smin[0]);
        b = max(b, smax[0]);
        mn[blockIdx.x] = a;
        mx[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(1024) k_big_bitmap(uint32_t* __restrict__ vals, const int64_t* __restrict__ off,
                                                     const int64_t* __restrict__ list,
                                                     const uint32_t* __restrict__ mn,
                                                     const int64_t* __restrict__ bm_off, uint32_t* __restrict__ bm,
                                                     int unique, int32_t* __restrict__ ucount, DevStatus* st) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    const int64_t k = list[blockIdx.x];
    const int64_t b = off[k], e = off[k + 1];
    const uint32_t lo = mn[blockIdx.x];
    uint32_t* bits = bm + bm_off[blockIdx.x];
    const int64_t nwords = bm_off[blockIdx.x + 1] - bm_off[blockIdx.x];
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        uint32_t d = vals[i] - lo;
        atomicOr(&bits[d >> 5], 1u << (d & 31));
    }
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    // ordered emission: block scan of popcounts over chunks of blockDim words
    for (int64_t w0 = 0; w0 < nwords; w0 += blockDim.x) {
        int64_t w = w0 + threadIdx.x;
        uint32_t word = (w < nwords) ? bits[w] : 0u;
        int c = __popc(word);
        int x = c;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= o) x += y;
        }
        if (lane_id() == 31) wsum[warp_id()] = x;
        __syncthreads();
        if (warp_id() == 0) {
            int64_t t = (lane_id() < (int)(blockDim.x >> 5)) ? wsum[lane_id()] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane_id() >= o) t += y;
            }
            if (lane_id() < (int)(blockDim.x >> 5)) wsum[lane_id()] = t;
        }
        __syncthreads();
        int64_t pos = carry + (x - c) + (warp_id() > 0 ? wsum[warp_id() - 1] : 0);
        while (word) {
            int bit = __ffs(word) - 1;
            word &= word - 1;
            vals[b + pos++] = lo + (uint32_t)(w * 32 + bit);
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = pos;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (unique) ucount[k] = (int32_t)carry;
        else if (carry != e - b) record_error(st, PMRF_ERR_DEVICE, SITE_SORT, k);
    }
}

}  // namespace

int segmented_sort_u32(uint32_t* vals, const int64_t* off, int64_t nseg, int64_t n, bool unique, int32_t* ucount,
                       DevStatus* st, cudaStream_t s) {
    (void)n;
    if (nseg <= 0) return PMRF_OK;
    {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(nseg, 8), (int64_t)sms * 16));
        k_sort_warp<<<(unsigned)blocks, 256, 0, s>>>(vals, off, nseg, unique ? 1 : 0, ucount);
        ::pmrf::note_launch(1);
    }
    PMRF_CUDA(cudaGetLastError());

    // medium and long segments: listed first (order of the lists does not
    // matter: each segment is sorted on its own)
    int64_t *mlist = nullptr, *list = nullptr;
    int32_t* cnts = nullptr;
    PMRF_TRY(dalloc(&cnts, 2, s));
    int rc = dalloc(&mlist, nseg, s);
    if (!rc) rc = dalloc(&list, nseg, s);
    if (rc) { dfree(cnts, s); dfree(mlist, s); dfree(list, s); return rc; }
    cudaMemsetAsync(cnts, 0, 2 * sizeof(int32_t), s);
    k_mark_long<<<(unsigned)ceil_div(nseg, 256), 256, 0, s>>>(off, nseg, mlist, cnts, list, cnts + 1);
    ::pmrf::note_launch(1);
    int32_t hc[2] = {0, 0};
    cudaMemcpyAsync(hc, cnts, sizeof(hc), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { dfree(cnts, s); dfree(mlist, s); dfree(list, s); return cuda_fail(e, "segmented sort"); }
    const int32_t nmed = hc[0], nbig = hc[1];
    if (nmed > 0) {
        k_sort_medium<<<nmed, SORT_THREADS, 0, s>>>(vals, off, mlist, unique ? 1 : 0, ucount);
        ::pmrf::note_launch(1);
    }
    if (nbig > 0) {
        uint32_t *mn = nullptr, *mx = nullptr;
        int64_t* bmo = nullptr;
        uint32_t* bm = nullptr;
        rc = dalloc(&mn, nbig, s);
        if (!rc) rc = dalloc(&mx, nbig, s);
        if (!rc) rc = dalloc(&bmo, nbig + 1, s);
        if (!rc) {
            k_big_minmax<<<nbig, 1024, 0, s>>>(vals, off, list, mn, mx);
            ::pmrf::note_launch(1);
            std::vector<uint32_t> hmn(nbig), hmx(nbig);
            cudaMemcpyAsync(hmn.data(), mn, sizeof(uint32_t) * nbig, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(hmx.data(), mx, sizeof(uint32_t) * nbig, cudaMemcpyDeviceToHost, s);
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_fail(e, "segmented sort (long)");
            if (!rc) {
                std::vector<int64_t> hbo(nbig + 1, 0);
                for (int i = 0; i < nbig; ++i) hbo[i + 1] = hbo[i] + ceil_div((int64_t)hmx[i] - hmn[i] + 1, 32);
                cudaMemcpyAsync(bmo, hbo.data(), sizeof(int64_t) * (nbig + 1), cudaMemcpyHostToDevice, s);
                rc = dalloc(&bm, hbo[nbig], s);
                if (!rc) {
                    cudaMemsetAsync(bm, 0, sizeof(uint32_t) * hbo[nbig], s);
                    k_big_bitmap<<<nbig, 1024, 0, s>>>(vals, off, list, mn, bmo, bm, unique ? 1 : 0, ucount, st);
                    ::pmrf::note_launch(1);
                    e = cudaGetLastError();
                    if (e != cudaSuccess) rc = cuda_fail(e, "k_big_bitmap");
                    // the host vector hbo must outlive the async copy
                    cudaError_t e2 = cudaStreamSynchronize(s);
                    if (!rc && e2 != cudaSuccess) rc = cuda_fail(e2, "segmented sort (long)");
                }
            }
        }
        dfree(mn, s); dfree(mx, s); dfree(bmo, s); dfree(bm, s);
    }
    dfree(cnts, s);
    dfree(mlist, s);
    dfree(list, s);
    PMRF_CUDA(cudaGetLastError());
    return rc;
}

}  // namespace pmrf
