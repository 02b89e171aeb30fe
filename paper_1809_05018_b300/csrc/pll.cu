// pll.cu -- vertex pseudo-log-likelihood of the MRF model and its hand-written
// FP64 adjoint (the differentiable form of the model; not part of the paper's
// algorithm).  With labels x fixed, per vertex over the full neighbourhood:
//   E_v(l) = D_l(y_v) + beta * m_v(l),  m_v(l) = #{u in N(v): x_u != l}
//   PLL_s  = sum_{v in s} [ -E_v(x_v) - logsumexp_l(-E_v(l)) ]
//   dPLL/dmu_l    = sum_v (p_v(l) - [x_v = l]) (mu_l - y_v) / sigma_l^2
//   dPLL/dsigma_l = sum_v (p_v(l) - [x_v = l]) (1/sigma_l - (y_v - mu_l)^2 / sigma_l^3)
//   dPLL/dbeta    = sum_v ( sum_l p_v(l) m_v(l) - m_v(x_v) ),   p_v = softmax(-E_v)
// One pass over the vertices writes per-block partial sums (deterministic
// order); a per-slice pass adds them in block order.
#include <algorithm>
#include <string>

#include "graph.cuh"

namespace pmrf {

namespace {

constexpr int PLL_THREADS = 256;
// vertices a thread in the allocating calls (the allocation-free call keeps
// one, so its scratch bound stays S ceil(V_max / 256) (2L + 2) + S doubles)
constexpr int PLL_VPT = 4;

template <int L>
__global__ void __launch_bounds__(PLL_THREADS) k_pll(int32_t S, const int64_t* __restrict__ vert_off,
                                                     const double* __restrict__ y, const int64_t* __restrict__ adj_off,
                                                     const int32_t* __restrict__ adj, const uint8_t* __restrict__ x,
                                                     const double* __restrict__ mu, const double* __restrict__ sigma,
                                                     double beta, int64_t nchunk, int vpt,
                                                     double* __restrict__ part) {
    constexpr int NP = 2 * L + 2;  // pll, gmu[L], gsigma[L], gbeta
    __shared__ double s_mu[L], s_inv[L], s_ln[L], s_isg[L], s_isg2[L], s_isg3[L];
    __shared__ double s_acc[NP][PLL_THREADS];
    __shared__ double s_red[NP][8];
    const int s = blockIdx.y;
    const int64_t vb = vert_off[s], ve = vert_off[s + 1];
    // vpt vertices a thread, PLL_THREADS apart: block b takes the slice's
    // vertices [b vpt PLL_THREADS, (b + 1) vpt PLL_THREADS)
    const int64_t vblk = vb + (int64_t)blockIdx.x * vpt * PLL_THREADS;
    if (vblk >= ve) return;  // whole block beyond this slice
    if (threadIdx.x < L) {
        const double m = mu[(int64_t)s * L + threadIdx.x], sg = sigma[(int64_t)s * L + threadIdx.x];
        s_mu[threadIdx.x] = m;
        s_inv[threadIdx.x] = 1.0 / (2.0 * sg * sg);
        s_ln[threadIdx.x] = log(sg);
        // reciprocals for the adjoint: per-vertex divisions become products
        const double isg = 1.0 / sg;
        s_isg[threadIdx.x] = isg;
        s_isg2[threadIdx.x] = isg * isg;
        s_isg3[threadIdx.x] = isg * isg * isg;
    }
    __syncthreads();
    double acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0.0;
    for (int r = 0; r < vpt; ++r) {
        const int64_t v = vblk + (int64_t)r * PLL_THREADS + threadIdx.x;
        if (v >= ve) break;
        const double yv = y[v];
        const int xv = x[v];
        int cnt[L];
#pragma unroll
        for (int l = 0; l < L; ++l) cnt[l] = 0;
        const int64_t a0 = adj_off[v], a1 = adj_off[v + 1];
        for (int64_t j = a0; j < a1; ++j) {
            const int xl = x[adj[j]];
#pragma unroll
            for (int l = 0; l < L; ++l) cnt[l] += (xl == l);
        }
        const int d = (int)(a1 - a0);
        double E[L], dev[L], dev2[L], emin = 0.0;
#pragma unroll
        for (int l = 0; l < L; ++l) {
            dev[l] = yv - s_mu[l];
            dev2[l] = dev[l] * dev[l];
            E[l] = dev2[l] * s_inv[l] + s_ln[l] + beta * (double)(d - cnt[l]);
            emin = (l == 0 || E[l] < emin) ? E[l] : emin;
        }
        // p = softmax(-E) with the minimum shifted out; log z of the same sum
        double p[L], logz;
        if constexpr (L == 2) {
            // one exponential: z = 1 + exp(-|E_0 - E_1|)
            const double e = exp(-fabs(E[0] - E[1]));
            const double inv_z = 1.0 / (1.0 + e);
            const bool zero_min = E[0] <= E[1];
            p[0] = zero_min ? inv_z : e * inv_z;
            p[L - 1] = zero_min ? e * inv_z : inv_z;
            logz = log1p(e);
        } else {
            double z = 0.0;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                p[l] = exp(-(E[l] - emin));
                z += p[l];
            }
            const double inv_z = 1.0 / z;
#pragma unroll
            for (int l = 0; l < L; ++l) p[l] *= inv_z;
            logz = log(z);
        }
        double Ex = 0.0, mx = 0.0, eb = 0.0;
#pragma unroll
        for (int l = 0; l < L; ++l) {
            if (l == xv) { Ex = E[l]; mx = (double)(d - cnt[l]); }
            eb += p[l] * (double)(d - cnt[l]);
        }
        acc[0] += -Ex - (-emin + logz);
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const double w = p[l] - (l == xv ? 1.0 : 0.0);
            acc[1 + l] += -w * dev[l] * s_isg2[l];
            acc[1 + L + l] += w * (s_isg[l] - dev2[l] * s_isg3[l]);
        }
        acc[1 + 2 * L] += eb - mx;
    }
    // block sums in a fixed order without shuffle trees (the FP64 pipe is the
    // scarce unit): 8 threads per quantity add 32 consecutive entries each,
    // then one thread adds the 8 results
#pragma unroll
    for (int k = 0; k < NP; ++k) s_acc[k][threadIdx.x] = acc[k];
    __syncthreads();
    if (threadIdx.x < NP * 8) {
        const int k = threadIdx.x >> 3, w = threadIdx.x & 7;
        double t = 0.0;
        for (int j = 0; j < PLL_THREADS / 8; ++j) t += s_acc[k][w * (PLL_THREADS / 8) + j];
        s_red[k][w] = t;
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s_red[threadIdx.x][w];
        part[((int64_t)s * nchunk + blockIdx.x) * NP + threadIdx.x] = t;
    }
}

template <int L>
__global__ void k_pll_final(int32_t S, const int64_t* __restrict__ vert_off, int64_t nchunk, int vpt,
                            const double* __restrict__ part, double* __restrict__ pll, const double* __restrict__ gout,
                            double* __restrict__ gmu, double* __restrict__ gsigma, double* __restrict__ gbeta_s) {
    constexpr int NP = 2 * L + 2;
    const int s = blockIdx.x;
    const int64_t nb = ceil_div(vert_off[s + 1] - vert_off[s], (int64_t)PLL_THREADS * vpt);  // k_pll's blocks
    double tot[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) tot[k] = 0.0;
    for (int64_t b = threadIdx.x; b < nb; b += 32) {
#pragma unroll
        for (int k = 0; k < NP; ++k) tot[k] += part[((int64_t)s * nchunk + b) * NP + k];
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) tot[k] = warp_sum(tot[k]);
    if (threadIdx.x != 0) return;
    if (pll) pll[s] = tot[0];
    if (gout) {
        const double go = gout[s];
        for (int l = 0; l < L; ++l) {
            if (gmu) gmu[(int64_t)s * L + l] = go * tot[1 + l];
            if (gsigma) gsigma[(int64_t)s * L + l] = go * tot[1 + L + l];
        }
        gbeta_s[s] = go * tot[1 + 2 * L];
    }
}

__global__ void k_sum_slices(int32_t S, const double* __restrict__ in, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0;
    for (int s = 0; s < S; ++s) t += in[s];
    *out = t;
}

// dst may alias rep_el: each thread reads its own entry before writing it
__global__ void k_rep_hood(const uint32_t* rep_el, const int64_t* __restrict__ hood_off, int64_t C, int64_t N_el,
                           int32_t* dst) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N_el) return;
    dst[q] = (int32_t)(upper_bound_dev<int64_t>(hood_off, 0, C + 1, (int64_t)rep_el[q]) - 1);
}

template <int L>
int pll_body(pmrf_graph* g, const uint8_t* x, const double* mu, const double* sigma, double beta, double* pll,
             const double* gout, double* gmu, double* gsigma, double* gbeta, cudaStream_t s) {
    constexpr int NP = 2 * L + 2;
    int64_t maxv = 0;
    for (int i = 0; i < g->S; ++i) maxv = std::max(maxv, g->h_vert_off[i + 1] - g->h_vert_off[i]);
    const int64_t nchunk = std::max<int64_t>(1, ceil_div(maxv, (int64_t)PLL_THREADS * PLL_VPT));
    if (nchunk > 2147483647ll) return fail(PMRF_ERR_UNSUPPORTED, "slice too large");
    double* part = nullptr;
    double* gb = nullptr;
    PMRF_TRY(dalloc(&part, (int64_t)g->S * nchunk * NP, s));
    int rc = dalloc(&gb, g->S, s);
    if (rc) { dfree(part, s); return rc; }
    if (maxv > 0) {
        const dim3 grid((unsigned)nchunk, (unsigned)g->S);
        k_pll<L><<<grid, PLL_THREADS, 0, s>>>(g->S, g->d_vert_off, g->d_y, g->d_adj_off, g->d_adj, x, mu, sigma, beta,
                                             nchunk, PLL_VPT, part); ::pmrf::note_launch(1);
    }
    k_pll_final<L><<<(unsigned)g->S, 32, 0, s>>>(g->S, g->d_vert_off, nchunk, PLL_VPT, part, pll, gout, gmu, gsigma,
                                                 gb); ::pmrf::note_launch(1);
    if (gout && gbeta) { k_sum_slices<<<1, 32, 0, s>>>(g->S, gb, gbeta); ::pmrf::note_launch(1); }
    cudaError_t e = cudaGetLastError();
    dfree(part, s);
    dfree(gb, s);
    if (e != cudaSuccess) return cuda_fail(e, "pll kernels");
    return PMRF_OK;
}

}  // namespace

int pll_run(pmrf_graph* g, int32_t L, const uint8_t* x, const double* mu, const double* sigma, double beta,
            double* pll, const double* gout, double* gmu, double* gsigma, double* gbeta, cudaStream_t s) {
    if (L < 1 || L > PMRF_MAX_LABELS) return fail(PMRF_ERR_ARG, "n_labels must be in [1, 8]");
    if (!x || !mu || !sigma) return fail(PMRF_ERR_ARG, "null pointer");
    if (!std::isfinite(beta)) return fail(PMRF_ERR_ARG, "beta must be finite");
    switch (L) {
        case 1: return pll_body<1>(g, x, mu, sigma, beta, pll, gout, gmu, gsigma, gbeta, s);
        case 2: return pll_body<2>(g, x, mu, sigma, beta, pll, gout, gmu, gsigma, gbeta, s);
        case 3: return pll_body<3>(g, x, mu, sigma, beta, pll, gout, gmu, gsigma, gbeta, s);
        case 4: return pll_body<4>(g, x, mu, sigma, beta, pll, gout, gmu, gsigma, gbeta, s);
        case 5: return pll_body<5>(g, x, mu, sigma, beta, pll, gout, gmu, gsigma, gbeta, s);
        case 6: return pll_body<6>(g, x, mu, sigma, beta, pll, gout, gmu, gsigma, gbeta, s);
        case 7: return pll_body<7>(g, x, mu, sigma, beta, pll, gout, gmu, gsigma, gbeta, s);
        default: return pll_body<8>(g, x, mu, sigma, beta, pll, gout, gmu, gsigma, gbeta, s);
    }
}

int export_rep_hood(pmrf_graph* g, int32_t* dst, cudaStream_t s) {
    if (g->N_el == 0) return PMRF_OK;
    // the sorted replica list is only needed here, so it is built on demand
    // into dst's own storage (same size, 32-bit entries) and mapped in place
    static_assert(sizeof(uint32_t) == sizeof(int32_t), "in-place mapping");
    PMRF_TRY(rep_elements(g, reinterpret_cast<uint32_t*>(dst), s));
    k_rep_hood<<<(unsigned)ceil_div(g->N_el, 256), 256, 0, s>>>(reinterpret_cast<const uint32_t*>(dst),
                                                                 g->d_hood_off, g->C, g->N_el, dst);
    ::pmrf::note_launch(1);
    PMRF_CUDA(cudaGetLastError());
    return PMRF_OK;
}

}  // namespace pmrf

// ---------------------------------------------------------------------------
// Allocation-free adjoint (pmrf_pll_grad_noalloc).
//
// Some callers cannot allocate device memory at the moment they need the
// gradient: an application whose device memory is already claimed by its own
// caching allocator (a cudaMalloc would fail, or force that allocator to give
// memory back), or a latency-critical loop that must not pay for, or be
// implicitly synchronised by, an allocation.  For them the adjoint's per-block
// partial sums live in the fixed array below, which is part of the loaded
// module: every GPU that loads this library holds PMRF_PLL_NOALLOC_MAX_DOUBLES
// doubles (8 MiB) of it until the process exits.
//
// The array's name is only a stand-in in host code; its device address is
// obtained with cudaGetSymbolAddress, with the caller's device current, on
// every call (after the first call on a device has loaded the module this is a
// lookup, and it stays right if the caller resets the device between calls).
// Every call shares the array, so calls whose work overlaps on the GPU (other
// streams, other host threads) race on it and must be ordered by the caller.
// Each call writes every entry it later reads, so nothing left by an earlier
// call is used.

static __device__ __align__(256) double pmrf_pll_noalloc_scratch[PMRF_PLL_NOALLOC_MAX_DOUBLES];

namespace pmrf {

namespace {

int noalloc_scratch(double** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, pmrf_pll_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(pmrf_pll_noalloc_scratch)");
    *out = (double*)p;
    return PMRF_OK;
}

template <int L>
int pll_grad_noalloc_body(pmrf_graph* g, const uint8_t* x, const double* mu, const double* sigma, double beta,
                          const double* gout, double* gmu, double* gsigma, double* gbeta, cudaStream_t s) {
    constexpr int NP = 2 * L + 2;
    int64_t maxv = 0;
    for (int i = 0; i < g->S; ++i) maxv = std::max(maxv, g->h_vert_off[i + 1] - g->h_vert_off[i]);
    const int64_t nchunk = std::max<int64_t>(1, ceil_div(maxv, PLL_THREADS));
    const int64_t need = (int64_t)g->S * nchunk * NP + g->S;
    if (need > (int64_t)PMRF_PLL_NOALLOC_MAX_DOUBLES)
        return fail(PMRF_ERR_UNSUPPORTED, "pmrf_pll_grad_noalloc needs " + std::to_string(need) +
                                              " doubles of scratch (slices x ceil(largest slice's regions / 256) x (2 "
                                              "n_labels + 2) + slices), above its fixed " +
                                              std::to_string((int64_t)PMRF_PLL_NOALLOC_MAX_DOUBLES) +
                                              "; use pmrf_pll_grad or smaller batches");
    double* scr = nullptr;
    PMRF_TRY(noalloc_scratch(&scr));
    double* part = scr;
    double* gb = scr + (int64_t)g->S * nchunk * NP;
    if (maxv > 0) {
        const dim3 grid((unsigned)nchunk, (unsigned)g->S);
        k_pll<L><<<grid, PLL_THREADS, 0, s>>>(g->S, g->d_vert_off, g->d_y, g->d_adj_off, g->d_adj, x, mu, sigma, beta,
                                             nchunk, 1, part);
        ::pmrf::note_launch(1);
    }
    k_pll_final<L><<<(unsigned)g->S, 32, 0, s>>>(g->S, g->d_vert_off, nchunk, 1, part, nullptr, gout, gmu, gsigma, gb);
    ::pmrf::note_launch(1);
    if (gbeta) {
        k_sum_slices<<<1, 32, 0, s>>>(g->S, gb, gbeta);
        ::pmrf::note_launch(1);
    }
    PMRF_CUDA(cudaGetLastError());
    return PMRF_OK;
}

}  // namespace

int pll_grad_noalloc_run(pmrf_graph* g, int32_t L, const uint8_t* x, const double* mu, const double* sigma,
                         double beta, const double* gout, double* gmu, double* gsigma, double* gbeta, cudaStream_t s) {
    if (L < 1 || L > PMRF_MAX_LABELS) return fail(PMRF_ERR_ARG, "n_labels must be in [1, 8]");
    if (!x || !mu || !sigma || !gout) return fail(PMRF_ERR_ARG, "null pointer");
    if (!std::isfinite(beta)) return fail(PMRF_ERR_ARG, "beta must be finite");
    switch (L) {
        case 1: return pll_grad_noalloc_body<1>(g, x, mu, sigma, beta, gout, gmu, gsigma, gbeta, s);
        case 2: return pll_grad_noalloc_body<2>(g, x, mu, sigma, beta, gout, gmu, gsigma, gbeta, s);
        case 3: return pll_grad_noalloc_body<3>(g, x, mu, sigma, beta, gout, gmu, gsigma, gbeta, s);
        case 4: return pll_grad_noalloc_body<4>(g, x, mu, sigma, beta, gout, gmu, gsigma, gbeta, s);
        case 5: return pll_grad_noalloc_body<5>(g, x, mu, sigma, beta, gout, gmu, gsigma, gbeta, s);
        case 6: return pll_grad_noalloc_body<6>(g, x, mu, sigma, beta, gout, gmu, gsigma, gbeta, s);
        case 7: return pll_grad_noalloc_body<7>(g, x, mu, sigma, beta, gout, gmu, gsigma, gbeta, s);
        default: return pll_grad_noalloc_body<8>(g, x, mu, sigma, beta, gout, gmu, gsigma, gbeta, s);
    }
}

}  // namespace pmrf
