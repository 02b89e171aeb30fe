// quality.cu -- segmentation quality against a ground truth (Section 4.2.1,
// evaluation metrics): per slice, the confusion counts of predicted against
// true pixel labels, and per label the one-against-the-rest precision, recall
// and accuracy with the predicted and true phase fractions (the porosity when
// the label is the void phase).
//
// One pass over the two u8 pixel images, 4 pixels per thread and step where
// both images allow 4-byte loads; the counts are integers (exact, any order),
// gathered per warp with match_any, per block in shared memory and added to
// the slice's counters once per block.  A second, tiny kernel turns the counts
// into the ratios with IEEE double divisions.
#include <algorithm>

#include "graph.cuh"

namespace pmrf {

namespace {

constexpr int QT_THREADS = 256;
constexpr int QT_MAX_BINS = PMRF_MAX_LABELS * PMRF_MAX_LABELS;

// add one pixel pair (bin, or -1 for none) of every lane to the block's bins
__device__ __forceinline__ void warp_count(int bin, unsigned long long* s_bins) {
    const unsigned same = __match_any_sync(0xffffffffu, bin);
    const int lane = threadIdx.x & 31;
    if (bin >= 0 && lane == __ffs(same) - 1) atomicAdd(&s_bins[bin], (unsigned long long)__popc(same));
}

// bin of one (truth, prediction) pair, -1 when either label is out of range
__device__ __forceinline__ int pair_bin(unsigned t, unsigned q, int L, int64_t p, DevStatus* st) {
    if (t >= (unsigned)L || q >= (unsigned)L) {
        record_error(st, PMRF_ERR_ARG, SITE_LABEL, p);
        return -1;
    }
    return (int)(t * (unsigned)L + q);
}

__global__ void __launch_bounds__(QT_THREADS) k_confusion(const uint8_t* __restrict__ pred,
                                                          const uint8_t* __restrict__ truth,
                                                          const int64_t* __restrict__ pix_off, int L,
                                                          unsigned long long* __restrict__ conf, DevStatus* st) {
    __shared__ unsigned long long s_bins[QT_MAX_BINS];
    const int s = blockIdx.y;
    const int nb = L * L;
    for (int b = threadIdx.x; b < nb; b += QT_THREADS) s_bins[b] = 0ull;
    __syncthreads();
    const int64_t base = pix_off[s], n = pix_off[s + 1] - base;
    const int64_t stride = (int64_t)gridDim.x * QT_THREADS;
    const bool vec = ((reinterpret_cast<uintptr_t>(pred + base) | reinterpret_cast<uintptr_t>(truth + base)) & 3) == 0;
    // every lane of a warp runs the same number of steps (match_any needs
    // them all), out-of-range steps count nothing
    const int64_t first = (int64_t)blockIdx.x * QT_THREADS + (threadIdx.x & ~31);
    if (vec) {
        const int64_t nw = n >> 2;
        const uint32_t* pw = reinterpret_cast<const uint32_t*>(pred + base);
        const uint32_t* tw = reinterpret_cast<const uint32_t*>(truth + base);
        for (int64_t w0 = first; w0 < nw; w0 += stride) {
            const int64_t w = w0 + (threadIdx.x & 31);
            uint32_t a = 0, b = 0;
            const bool ok = w < nw;
            if (ok) {
                a = __ldg(pw + w);
                b = __ldg(tw + w);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int bin = ok ? pair_bin((b >> (8 * k)) & 0xffu, (a >> (8 * k)) & 0xffu, L, base + 4 * w + k, st)
                                   : -1;
                warp_count(bin, s_bins);
            }
        }
        // the ragged tail (n mod 4 pixels), one per thread of the first block
        if (blockIdx.x == 0 && threadIdx.x < 32) {
            const int64_t p = (nw << 2) + threadIdx.x;
            const int bin = p < n ? pair_bin(truth[base + p], pred[base + p], L, base + p, st) : -1;
            warp_count(bin, s_bins);
        }
    } else {
        for (int64_t p0 = first; p0 < n; p0 += stride) {
            const int64_t p = p0 + (threadIdx.x & 31);
            const int bin = p < n ? pair_bin(truth[base + p], pred[base + p], L, base + p, st) : -1;
            warp_count(bin, s_bins);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += QT_THREADS)
        if (s_bins[b]) atomicAdd(&conf[(int64_t)s * nb + b], s_bins[b]);
}

// metrics[s][l][0..4] = precision, recall, accuracy, predicted fraction, true
// fraction of label l; NaN where the denominator is 0
__global__ void k_quality_metrics(const int64_t* __restrict__ conf, const int64_t* __restrict__ pix_off, int S, int L,
                                  double* __restrict__ metrics) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S * L) return;
    const int s = i / L, l = i % L;
    const int64_t* c = conf + (int64_t)s * L * L;
    const int64_t n = pix_off[s + 1] - pix_off[s];
    const int64_t tp = c[l * L + l];
    int64_t fp = 0, fn = 0;
    for (int t = 0; t < L; ++t)
        if (t != l) fp += c[t * L + l];
    for (int q = 0; q < L; ++q)
        if (q != l) fn += c[l * L + q];
    const int64_t tn = n - tp - fp - fn;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    double* m = metrics + (int64_t)i * 5;
    m[0] = (tp + fp) > 0 ? (double)tp / (double)(tp + fp) : nan;
    m[1] = (tp + fn) > 0 ? (double)tp / (double)(tp + fn) : nan;
    m[2] = n > 0 ? (double)(tp + tn) / (double)n : nan;
    m[3] = n > 0 ? (double)(tp + fp) / (double)n : nan;
    m[4] = n > 0 ? (double)(tp + fn) / (double)n : nan;
}

}  // namespace

int quality_run(pmrf_graph* g, int32_t L, const uint8_t* pred, const uint8_t* truth, int64_t* conf, double* metrics,
                cudaStream_t s) {
    if (!pred || !truth || !conf || !metrics) return fail(PMRF_ERR_ARG, "null pointer");
    if (L < 1 || L > PMRF_MAX_LABELS) return fail(PMRF_ERR_ARG, "n_labels must be in [1, 8]");
    const int32_t S = g->S;
    if (S == 0) return PMRF_OK;
    PMRF_CUDA(cudaMemsetAsync(conf, 0, sizeof(int64_t) * (size_t)S * L * L, s));
    int64_t maxpix = 0;
    for (int i = 0; i < S; ++i) maxpix = std::max(maxpix, g->h_pix_off[i + 1] - g->h_pix_off[i]);
    if (maxpix > 0) {
        // about 16 pixels per thread; the slices share the grid's y dimension
        const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(maxpix, 16 * QT_THREADS), 65535));
        k_confusion<<<dim3(gx, (unsigned)S), QT_THREADS, 0, s>>>(pred, truth, g->d_pix_off, L,
                                                               reinterpret_cast<unsigned long long*>(conf),
                                                               g->d_status);
        note_launch(1);
        PMRF_CUDA(cudaGetLastError());
    }
    k_quality_metrics<<<(unsigned)ceil_div((int64_t)S * L, 256), 256, 0, s>>>(conf, g->d_pix_off, S, L, metrics);
    note_launch(1);
    PMRF_CUDA(cudaGetLastError());
    return PMRF_OK;
}

}  // namespace pmrf
