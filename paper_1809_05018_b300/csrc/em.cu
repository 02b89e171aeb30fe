// em.cu -- the EM loop of DPP-PMRF on the device (Algorithm 2 steps 3, 6-11;
// Section 3.2.2 EM steps 2-5), plus the standalone MAP sweep, parameter
// update, starts (threshold, random) and label image.
//
// One EM iteration t is three kernels over a tile table (and the loop's
// condition setter):
//   k_vertex<L, VAR> (vertex tiles) -- for every vertex v: the neighbour-label
//     masks from x^{t-1}; for every replica (hood c containing v) the
//     disagreement counts m(c,v,l) = #{u in N(v) n H_c : x_u != l} by popcount
//     of the replica's slot mask against the label masks; their minimum over
//     the replicas M_l(v); E*_v = min_l D_l(y_v) + beta * M_l(v) and x^t_v its
//     smallest minimising label.  Because beta >= 0 and rounding is monotone,
//     min_c fl(D_l + beta*m(c,v,l)) = fl(D_l + beta*min_c m(c,v,l)), so this
//     equals the lexicographic minimum of (Emin(c,v), label) over the replicas
//     (Section 3.2.2 "Update Output Labels", reading G6) while keeping all
//     per-replica work in integers.  Also writes v's hood-pass record (its
//     data terms in the slice's fixed point and its label masks) and the
//     per-tile moment partials of the parameter update.  The VAR instantiation
//     adds the sweep variants (full-neighbourhood Potts, mean-energy and vote
//     replica rules).
//   k_hood<L> (one block per hood tile) -- for every hood c: S_c = sum over
//     its members v of Emin(c,v).  The tile's element stream (member id and
//     slot mask per element) is staged in shared memory by one bulk copy;
//     adjacent lanes take each hood, gather its members' records and form the
//     element energies in integers from a record and the element's slot mask.
//     Hoods with a member of more than 32 neighbours go hood by hood through
//     their hood-local adjacency rows.  The same lanes run the hood
//     convergence test over the last W sums (ring buffer) and add the tile's
//     exact partial of T.
//   k_finalize<L> (one block per slice) -- label moments -> (n, mu, sigma, U),
//     the total T^t, the MAP and EM convergence tests, per-slice stop flags,
//     and the fixed-point unit of the next iteration.
// Energies of a slice are integers in units 2^-q, q chosen per slice and
// iteration from a bound on every element energy (slice_unit), so that all
// sums are exact and independent of order.  Slices that have stopped skip all
// work.  The loop is captured once into a CUDA graph as two conditional WHILE
// nodes in sequence, each body one iteration (the kernels read the iteration
// number from device memory): the dense loop runs one block per tile while at
// least a quarter of the tiles belong to slices still iterating, the sparse
// loop the remaining iterations with blocks that take only those tiles
// (k_vertex<L, VAR, true>, k_hood<L, true>); it ends once every slice has
// stopped.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "graph.cuh"

namespace pmrf {

namespace {

constexpr int VT_THREADS = 128;             // vertices per vertex tile = threads
// resident blocks per SM the register budget of the EM kernels must allow
// (measured on the two-label stack: the vertex pass gains from 16 blocks at 32
// registers; more labels need more registers)
__host__ __device__ constexpr int vt_min_blocks(int L) { return L <= 2 ? 16 : (L <= 4 ? 10 : 4); }
__host__ __device__ constexpr int ht_min_blocks(int L) { return L <= 4 ? 12 : 8; }
constexpr int FIN_THREADS = 256;            // finaliser block (one per slice)
constexpr int LI_THREADS = 256;             // label-image block
constexpr int HT_THREADS = 128;             // hood-pass block
constexpr int MIN_HOOD_TILE = 32;           // hoods per hood tile, limits
constexpr int MAX_HOOD_TILE = 1024;
constexpr int HT_CAP_MAX = 4096;            // largest staged tile (elements; 32 KB of shared memory)
// Per-vertex record of the hood pass, in 32-byte chunks, written by the vertex
// pass of the same iteration; energies in the slice's unit 2^-q (SliceUnit):
//   word 0        D_min(v) = min_l D_l(y_v) (each D_l rounded to the unit once)
//   words 1..L-1  the excess D_l - D_min of every label l other than amin (the
//                 lowest label attaining D_min), ascending l, saturated at
//                 DQ_SAT (larger excesses never decide a minimum); bits 61-63
//                 of word 1 hold amin
//   then          L-1 u32 masks from u32 index 2L on: which of v's adjacency
//                 slots hold label l, for l < L-1 (the last label's count
//                 follows from the slot mask)
// For L = 2 the mask differs: it marks the slots that hold the label other
// than amin.  With c_b the in-hood neighbours holding that label, c_a the
// others and k = c_b - c_a, the element's excess min(beta_q c_b, dq + beta_q
// c_a) is beta_q c_b less max(0, beta_q k - dq).
__host__ __device__ constexpr int vrec_words(int L) { return ((L + (L - 1 + 1) / 2) + 3) / 4 * 4; }
constexpr uint64_t DQ_SAT = (1ull << 61) - 1;

enum Mode : int32_t { MODE_INIT = 0, MODE_EM = 1, MODE_SWEEP = 2, MODE_PARAMS = 3 };

struct RunCfg {
    int32_t L, W, max_iters, init_from_labels;
    double beta, tol, sigma_min, init_lo, init_hi;
    int32_t scope;   // PMRF_SCOPE_*
    int32_t rule;    // PMRF_RULE_*
};

struct OutPtrs {  // outputs of one pmrf_em call (read by the closing kernel)
    uint8_t* labels;
    double* params;
    int32_t* iters;
    int32_t* conv;
    double* thist;
};

struct DevGraph {
    int32_t S;
    int32_t max_deg, max_hood;
    int64_t V, C;
    const int64_t* vert_off;
    const int64_t* hood_slice_off;
    const double* y;
    const int64_t* adj_off;
    const int32_t* adj;
    const int64_t* hood_off;
    const int32_t* hood;
    const int64_t* row_off;
    const uint32_t* row;
    const int64_t* rep_woff;
    const uint32_t* rep_mask;
    const uint2* el;
};

DevGraph view(const pmrf_graph* g) {
    DevGraph d;
    d.S = g->S;
    d.max_deg = g->max_deg;
    d.max_hood = g->max_hood;
    d.V = g->V;
    d.C = g->C;
    d.vert_off = g->d_vert_off;
    d.hood_slice_off = g->d_hood_slice_off;
    d.y = g->d_y;
    d.adj_off = g->d_adj_off;
    d.adj = g->d_adj;
    d.hood_off = g->d_hood_off;
    d.hood = g->d_hood;
    d.row_off = g->d_row_off;
    d.row = g->d_row;
    d.rep_woff = g->d_rep_woff;
    d.rep_mask = g->d_rep_mask;
    d.el = g->d_el;
    return d;
}

// initial mean of an empty label: centre of its threshold bin
__device__ __forceinline__ double bin_centre(const RunCfg& c, int l) {
    return c.init_lo + ((double)l + 0.5) * (c.init_hi - c.init_lo) / (double)c.L;
}

__device__ __forceinline__ int threshold_label(const RunCfg& c, double y) {
    double q = floor((y - c.init_lo) / (c.init_hi - c.init_lo) * (double)c.L);
    return q < 0.0 ? 0 : (q > (double)(c.L - 1) ? c.L - 1 : (int)q);
}

// 1 / (2 sigma^2) of the Gaussian data term (one expression for every caller)
__device__ __forceinline__ double inv_two_var(double sg) { return 1.0 / (2.0 * sg * sg); }

// ---------------------------------------------------------------------------
// exact energy sums in a per-slice fixed point
//
// Every energy of slice s in iteration t is an integer in units 2^-q.  q is
// chosen (slice_unit) from a bound M on |Emin(c,v)|: the data terms of the
// slice's labels at the ends of its intensity range bound the least data term
// of every vertex, and the Potts part is at most beta times the largest degree.
// With H = max(128, largest hood), 2^q M H < 2^62, so an element energy, a hood
// sum and a vertex tile's sum of vertex energies (128 vertices) all fit in 64
// bits, and every sum is exact and independent of order.  A double is rounded to the
// unit once (to_fixed: to nearest, ties away from zero); for the usual range of
// energies q is about 52, i.e. the rounding is below 1e-16.  Totals T are sums
// of hood sums in 128 bits, rounded to double once; a vertex tile's sum of its
// label's vertex energies is rounded to double once and the label's total U is
// the fixed-order FP64 sum of those.

struct SliceUnit {
    int32_t q;       // unit 2^-q of this iteration's energies
    int32_t pad;
    int64_t beta_q;  // beta in units 2^-q, rounded to nearest
    int64_t tol_q;   // smallest integer >= conv_tol * 2^q (the hood test's threshold)
};

// round(d * 2^q) for |d * 2^q| < 2^62 (saturated beyond), with integer operations
__device__ __forceinline__ int64_t to_fixed(double d, int q) {
    const long long bits = __double_as_longlong(d);
    const int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long man = (unsigned long long)bits & 0xfffffffffffffull;
    if (ex != 0) man |= 1ull << 52;
    const int sh = (ex == 0 ? 1 : ex) - 1075 + q;  // |d| 2^q = man 2^sh
    unsigned long long r;
    if (sh >= 0) {
        r = sh >= 10 ? (1ull << 62) : (man << sh);
    } else {
        r = sh < -54 ? 0ull : ((man + (1ull << (-sh - 1))) >> (-sh));
    }
    return bits < 0 ? -(long long)r : (long long)r;
}

// x * 2^-q rounded to double once (|x| < 2^64 converts with a single rounding;
// larger magnitudes take a second one from the low word)
__device__ __forceinline__ double from_fixed(__int128 x, int q) {
    const bool neg = x < 0;
    const unsigned __int128 a = neg ? -(unsigned __int128)x : (unsigned __int128)x;
    // the top bits in 63 bits, the bits shifted out kept as a sticky bit below
    // the rounding position: one conversion rounds the 128-bit value once
    int sh = 0;
    const unsigned long long hi = (unsigned long long)(a >> 64);
    if (hi) sh = 65 - __clzll((long long)hi);
    unsigned long long m = (unsigned long long)(a >> sh);
    if (sh && (a & (((unsigned __int128)1 << sh) - 1))) m |= 1ull;
    const double r = ldexp((double)m, sh - q);
    return neg ? -r : r;
}

__device__ __forceinline__ double from_fixed64(int64_t x, int q) { return ldexp((double)x, -q); }

__device__ __forceinline__ __int128 shfl_xor_i128(__int128 x, int o) {
    const long long hi = __shfl_xor_sync(0xffffffffu, (long long)(x >> 64), o);
    const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)x, o);
    return ((__int128)hi << 64) | (__int128)lo;
}

// smallest integer >= tol * 2^m (saturated), for the hood test at unit 2^-m
__device__ __forceinline__ int64_t tol_units(double tol, int m) {
    const double x = ceil(ldexp(tol, m));
    return x >= 0x1p62 ? (int64_t)(1ll << 62) : (int64_t)x;
}

// The unit of slice s for energies from parameters th [L][4] (mu, sigma at 1,
// 2): D_l(y) = (y - mu_l)^2 / (2 sigma_l^2) + ln sigma_l is convex in y, so on
// the slice's intensity range [ylo, yhi] the least data term of every vertex
// lies in [min_l ln sigma_l, min_l max(D_l(ylo), D_l(yhi))]; an element adds at
// most beta times its vertex's degree.  Margins of 2^-20 cover the rounding of
// these bounds.  ok = false when the bound is not finite.
__device__ __forceinline__ SliceUnit slice_unit(const double* __restrict__ th, int L, double ylo, double yhi,
                                                double beta, double tol, int max_deg, int max_hood, bool& ok) {
    double lo = INFINITY, up = INFINITY;
    for (int l = 0; l < L; ++l) {
        const double mu = th[4 * l + 1], sg = th[4 * l + 2];
        const double inv = inv_two_var(sg), ls = log(sg);
        const double a = ylo - mu, b = yhi - mu;
        lo = fmin(lo, ls);
        up = fmin(up, fmax(a * a * inv + ls, b * b * inv + ls));
    }
    const double B = fmax(fabs(lo), fabs(up));
    const double M = (B + beta * (double)max(32, max_deg)) * (1.0 + 0x1p-20) + 0x1p-60;
    const double P = M * (double)max(VT_THREADS, max_hood);
    SliceUnit u;
    u.pad = 0;
    ok = isfinite(P);
    int e = 0;
    frexp(ok ? P : 1.0, &e);  // P < 2^e
    u.q = max(-1000, min(1000, 62 - e));
    u.beta_q = (int64_t)llrint(ldexp(beta, u.q));
    u.tol_q = tol_units(tol, u.q);
    return u;
}

__device__ __forceinline__ void store_vrec_words(uint64_t* __restrict__ p, const uint64_t* w, int nw) {
    for (int k = 0; k < nw; k += 4)
        asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p + k), "l"(w[k]), "l"(w[k + 1]),
                     "l"(w[k + 2]), "l"(w[k + 3])
                     : "memory");
}

// For L = 2 the record is split: words 0-1 in a 16-byte array [V][2], the mask
// in a 4-byte array [V] after it, so that a hood-pass gather moves 16 + 4
// bytes (more records per cache line) instead of 32
__device__ __forceinline__ const uint32_t* vrec2_masks(const uint64_t* vrec, int64_t V) {
    return reinterpret_cast<const uint32_t*>(vrec + 2 * V);
}

template <int L>
__device__ __forceinline__ void store_vrec(uint64_t* __restrict__ vrec, int64_t V, int64_t v, const uint64_t* w) {
    if constexpr (L == 2) {
        asm volatile("st.global.v2.b64 [%0], {%1, %2};" ::"l"(vrec + 2 * v), "l"(w[0]), "l"(w[1]) : "memory");
        reinterpret_cast<uint32_t*>(vrec + 2 * V)[v] = (uint32_t)w[2];
    } else {
        constexpr int NW = vrec_words(L);
        store_vrec_words(vrec + v * NW, w, NW);
    }
}

// the data terms in the unit: every D_l rounded once, amin the lowest label
// attaining the least, each label's excess over it (saturated at DQ_SAT)
template <int L>
__device__ __forceinline__ int64_t data_fixed(const double (&D)[L], int q, uint64_t (&dq)[L], int& amin) {
    int64_t F[L];
#pragma unroll
    for (int l = 0; l < L; ++l) F[l] = to_fixed(D[l], q);
    amin = 0;
    int64_t Fmin = F[0];
#pragma unroll
    for (int l = 1; l < L; ++l)
        if (F[l] < Fmin) {
            Fmin = F[l];
            amin = l;
        }
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const uint64_t d = (uint64_t)(F[l] - Fmin);  // >= 0, < 2^63
        dq[l] = d > DQ_SAT ? DQ_SAT : d;
    }
    return Fmin;
}

// a record whose element energy is E in every hood (the full-neighbourhood
// Potts scope: every replica of v carries the same energies): D_min = E, every
// excess 0 and no label masks, so the hood pass adds E for each element
template <int L>
__device__ __forceinline__ void write_vrec_const(uint64_t* __restrict__ vrec, int64_t V, int64_t v, int64_t E) {
    constexpr int NW = vrec_words(L);
    uint64_t w[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) w[k] = 0ull;
    w[0] = (uint64_t)E;
    store_vrec<L>(vrec, V, v, w);
}

// the hood-pass record of vertex v (layout above) from its data terms in the
// slice's unit
template <int L>
__device__ __forceinline__ void write_vrec_fixed(uint64_t* __restrict__ vrec, int64_t V, int64_t v,
                                                 const int64_t (&F)[L], const uint32_t (&lmw)[L]) {
    constexpr int NW = vrec_words(L);
    uint64_t dq[L];
    int amin = 0;
    int64_t Fmin = F[0];
#pragma unroll
    for (int l = 1; l < L; ++l)
        if (F[l] < Fmin) {
            Fmin = F[l];
            amin = l;
        }
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const uint64_t d = (uint64_t)(F[l] - Fmin);
        dq[l] = d > DQ_SAT ? DQ_SAT : d;
    }
    uint64_t w[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) w[k] = 0ull;
    w[0] = (uint64_t)Fmin;
#pragma unroll
    for (int k = 0; k < L - 1; ++k) w[1 + k] = k < amin ? dq[k] : dq[k + 1];
    if (L > 1) w[1] |= (uint64_t)amin << 61;
    if constexpr (L == 2) {
        // slots holding the other label (the complement within v's slots of
        // the label-0 mask when amin = 0)
        w[2] = (uint64_t)(amin == 0 ? ~lmw[0] : lmw[0]);
    } else {
#pragma unroll
        for (int k = 0; k < L - 1; ++k) {
            const int u = 2 * L + k;
            w[u >> 1] |= (uint64_t)lmw[k] << (32 * (u & 1));
        }
    }
    store_vrec<L>(vrec, V, v, w);
}

// the same from FP64 data terms (each rounded to the unit once)
template <int L>
__device__ __forceinline__ void write_vrec(uint64_t* __restrict__ vrec, int64_t V, int64_t v, const double (&D)[L],
                                           const uint32_t (&lmw)[L], int q) {
    int64_t F[L];
#pragma unroll
    for (int l = 0; l < L; ++l) F[l] = to_fixed(D[l], q);
    write_vrec_fixed<L>(vrec, V, v, F, lmw);
}

// ---------------------------------------------------------------------------
// bulk copies into shared memory (the TMA engine) tracked by an mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// copy `bytes` (a multiple of 16, both addresses 16-byte aligned) into shared
// memory; completion is counted on bar
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// wait for the phase `parity` of bar to complete, at most ~2^20 polls; false
// (and the status word set) when the wait gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, DevStatus* st) {
    for (int it = 0; it < (1 << 20); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    record_error(st, PMRF_ERR_TIMEOUT, SITE_WAIT, 0);
    return false;
}

// ---------------------------------------------------------------------------
// which tiles a block takes
//
// Blocks launched for the tiles of stopped slices return at once, but on 512
// slices of 1024x1024 they still cost 0.06 ms (vertex pass) and 0.10 ms (hood
// pass) a pass once most slices have stopped: the rate at which blocks start.
// The sparse EM loop therefore lists the tiles of the slices still iterating
// (k_next_iter, after each iteration: cum[s] = the tiles of the active slices
// before s, cum[S] all of them) and launches one block per resident slot, each
// block taking the k-th listed tile from a counter until none is left (0.02 ms
// a pass at the end of the run).  With most tiles active the one-tile blocks
// are faster (a fully active pass took 0.74 against 0.64 ms, vertex, and 1.09
// against 0.91 ms, hood, in the listed form: its per-tile claim, binary search
// and barriers), so the dense loop keeps them.
struct TileSched {
    const int32_t* cum;  // [S+1] prefix sums over the active slices' tile counts
    const int64_t* t0;   // [S+1] first tile of each slice in the table
    int32_t* next;       // the pass's tile counter (zeroed by k_next_iter)
    int32_t S;
};

// the table index of the k-th listed tile: slice s with cum[s] <= k < cum[s+1]
// (binary search; cum is non-decreasing, cum[0] = 0 <= k < cum[S])
__device__ __forceinline__ int64_t sched_tile(const TileSched& sc, int k) {
    int lo = 0, hi = sc.S;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sc.cum[mid] <= k) lo = mid;
        else hi = mid;
    }
    return sc.t0[lo] + (k - sc.cum[lo]);
}

// run body(tile index) for each tile this block takes; body returns false to
// stop the block (a staging wait that gave up).  LISTED: the listed tiles of
// sc, the next one claimed while the current one runs, the barriers between
// tiles ending every thread's use of the shared buffers before the next tile
// writes them; otherwise tile blockIdx.x of the table (a separate kernel
// instance, so that one-tile blocks carry no loop)
template <bool LISTED, typename Body>
__device__ __forceinline__ void for_each_tile(const TileSched& sc, int* s_k, Body&& body) {
    if constexpr (!LISTED) {
        (void)sc;
        (void)s_k;
        body((int64_t)blockIdx.x);
    } else {
        if (threadIdx.x == 0) *s_k = atomicAdd(sc.next, 1);
        __syncthreads();
        int k = *s_k;
        while (k < sc.cum[sc.S]) {
            int kn = 0;
            if (threadIdx.x == 0) kn = atomicAdd(sc.next, 1);
            if (!body(sched_tile(sc, k))) return;
            __syncthreads();
            if (threadIdx.x == 0) *s_k = kn;
            __syncthreads();
            k = *s_k;
        }
    }
}

// ---------------------------------------------------------------------------
// vertex pass

// label counts among the neighbours of v in one replica with a multi-word
// slot mask (degree > 32): returns the replica's in-hood degree
template <int L>
__device__ __forceinline__ int slot_label_counts(const DevGraph& g, const uint8_t* __restrict__ x_in, int64_t a0,
                                                 int64_t r, int nw, int (&cnt)[L]) {
#pragma unroll
    for (int l = 0; l < L; ++l) cnt[l] = 0;
    int dc = 0;
    for (int w = 0; w < nw; ++w) {
        uint32_t m = g.rep_mask[r + w];
        dc += __popc(m);
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const int xl = x_in[g.adj[a0 + w * 32 + b]];
#pragma unroll
            for (int l = 0; l < L; ++l) cnt[l] += (xl == l);
        }
    }
    return dc;
}

// f(mask) for the one-word replica masks rm[r0 .. r1), read four at a time
// once the address is 16-byte aligned (fewer load requests per warp)
template <typename F>
__device__ __forceinline__ void for_each_mask(const uint32_t* __restrict__ rm, int64_t r0, int64_t r1, F&& f) {
    int64_t r = r0;
    for (; r < r1 && (r & 3); ++r) f(rm[r]);
    for (; r + 4 <= r1; r += 4) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(rm + r));
        f(q.x);
        f(q.y);
        f(q.z);
        f(q.w);
    }
    for (; r < r1; ++r) f(rm[r]);
}

constexpr int RCP_N = 65;  // replica counts whose reciprocal the vertex pass takes from a table

// The votes of all replicas of v (vote rule): each replica's least label from
// its counts k_l of in-hood neighbours not labelled l, by the exact energies in
// the slice's unit (the caller has ruled out near-ties, see vertex_variant)
template <int L>
__device__ __forceinline__ void vote_tally(const DevGraph& g, const uint8_t* __restrict__ x_in, int64_t a0, int d,
                                           int nw, int64_t r0, int64_t r1, const uint32_t (&lm)[L],
                                           const uint64_t (&dq)[L], uint64_t bq, int (&votes)[L], int (&kmin)[L]) {
#pragma unroll
    for (int l = 0; l < L; ++l) {
        votes[l] = 0;
        kmin[l] = 0x7fffffff;
    }
    auto vote = [&](const int (&k)[L]) {
        // excess <= 2^61, beta_q k below 2^62 / 32 (slice_unit): no overflow
        int b = 0;
        uint64_t eb = dq[0] + bq * (uint64_t)k[0];
#pragma unroll
        for (int l = 1; l < L; ++l) {
            const uint64_t e = dq[l] + bq * (uint64_t)k[l];
            if (e < eb) {
                eb = e;
                b = l;
            }
        }
#pragma unroll
        for (int l = 0; l < L; ++l)
            if (l == b) {
                votes[l] += 1;
                kmin[l] = min(kmin[l], k[l]);
            }
    };
    if (d <= 32) {
        for_each_mask(g.rep_mask, r0, r1, [&](uint32_t m) {
            const int dc = __popc(m);
            int k[L];
#pragma unroll
            for (int l = 0; l < L; ++l) k[l] = dc - __popc(m & lm[l]);
            vote(k);
        });
    } else {
        for (int64_t r = r0; r < r1; r += nw) {
            int cnt[L], k[L];
            const int dc = slot_label_counts<L>(g, x_in, a0, r, nw, cnt);
#pragma unroll
            for (int l = 0; l < L; ++l) k[l] = dc - cnt[l];
            vote(k);
        }
    }
}

// the vote tally of one vertex with every replica's least label taken in FP64
// (D_l + beta k_l, lower label on ties); out of line and given values only, so
// that the rare near-tie path adds nothing to the integer tally's code
template <int L>
struct VoteFP64 {
    const uint32_t* rep_mask;
    const int32_t* adj;
    const uint8_t* x_in;
    int64_t a0, r0, r1;
    int d, nw;
    double beta;
    double D[L];
    uint32_t lm[L];
    int votes[L], kmin[L];
};

template <int L>
__device__ __noinline__ VoteFP64<L> vote_tally_fp64(VoteFP64<L> a) {
#pragma unroll
    for (int l = 0; l < L; ++l) {
        a.votes[l] = 0;
        a.kmin[l] = 0x7fffffff;
    }
    for (int64_t r = a.r0; r < a.r1; r += a.nw) {
        int k[L];
        if (a.d <= 32) {
            const uint32_t m = a.rep_mask[r];
            const int dc = __popc(m);
#pragma unroll
            for (int l = 0; l < L; ++l) k[l] = dc - __popc(m & a.lm[l]);
        } else {
            int cnt[L];
#pragma unroll
            for (int l = 0; l < L; ++l) cnt[l] = 0;
            int dc = 0;
            for (int w = 0; w < a.nw; ++w) {
                uint32_t m = a.rep_mask[r + w];
                dc += __popc(m);
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    const int xl = a.x_in[a.adj[a.a0 + w * 32 + b]];
#pragma unroll
                    for (int l = 0; l < L; ++l) cnt[l] += (xl == l);
                }
            }
#pragma unroll
            for (int l = 0; l < L; ++l) k[l] = dc - cnt[l];
        }
        int b = 0;
        double best = a.D[0] + a.beta * (double)k[0];
#pragma unroll
        for (int l = 1; l < L; ++l) {
            const double x = a.D[l] + a.beta * (double)k[l];
            if (x < best) { best = x; b = l; }
        }
#pragma unroll
        for (int l = 0; l < L; ++l)
            if (l == b) {
                a.votes[l] += 1;
                a.kmin[l] = min(a.kmin[l], k[l]);
            }
    }
    return a;
}

// The sweep variants for one vertex (scope and replica rule of RunCfg; the
// same definitions as pmrf_config documents): returns the new label, sets
// Estar, writes the hood-pass record.  k_l of a replica = its in-hood
// neighbours whose label is not l (every neighbour for the full scope).
template <int L>
__device__ __forceinline__ int vertex_variant(const DevGraph& g, const RunCfg& c, const uint8_t* __restrict__ x_in,
                                           int64_t a0, int d, int64_t r0, int64_t r1, const uint32_t (&lm)[L],
                                           const double (&D)[L], uint64_t* __restrict__ vrec, int64_t v,
                                           double& Estar, const double* __restrict__ rcp, int q, int64_t beta_q) {
    int lab = 0;
    if (c.scope == PMRF_SCOPE_FULL) {
        // one set of energies for every replica: every rule picks its least label
        int M[L];
        if (d <= 32) {
#pragma unroll
            for (int l = 0; l < L; ++l) M[l] = d - __popc(lm[l]);
        } else {
            int cnt[L];
#pragma unroll
            for (int l = 0; l < L; ++l) cnt[l] = 0;
            for (int j = 0; j < d; ++j) {
                const int xl = x_in[g.adj[a0 + j]];
#pragma unroll
                for (int l = 0; l < L; ++l) cnt[l] += (xl == l);
            }
#pragma unroll
            for (int l = 0; l < L; ++l) M[l] = d - cnt[l];
        }
        Estar = D[0] + c.beta * (double)M[0];
#pragma unroll
        for (int l = 1; l < L; ++l) {
            const double e = D[l] + c.beta * (double)M[l];
            if (e < Estar) { Estar = e; lab = l; }
        }
        if (vrec) {
            // the element energy min_l (D_l + beta M_l) in the slice's fixed point
            int64_t Emin = 0;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const int64_t e = to_fixed(D[l], q) + beta_q * (int64_t)M[l];
                if (l == 0 || e < Emin) Emin = e;
            }
            write_vrec_const<L>(vrec, g.V, v, Emin);
        }
        return lab;
    }
    const int nw = d <= 32 ? 1 : (d + 31) >> 5;
    if (c.rule == PMRF_RULE_SUM) {
        // mean energy over the replicas: D_l + beta * (sum of k_l) / R
        int64_t Ks[L];
#pragma unroll
        for (int l = 0; l < L; ++l) Ks[l] = 0;
        int64_t R = 0;
        if (d <= 32) {
            R = r1 - r0;
            for_each_mask(g.rep_mask, r0, r1, [&](uint32_t m) {
                const int dc = __popc(m);
#pragma unroll
                for (int l = 0; l < L; ++l) Ks[l] += dc - __popc(m & lm[l]);
            });
        } else {
            for (int64_t r = r0; r < r1; r += nw, ++R) {
                int cnt[L];
                const int dc = slot_label_counts<L>(g, x_in, a0, r, nw, cnt);
#pragma unroll
                for (int l = 0; l < L; ++l) Ks[l] += dc - cnt[l];
            }
        }
        // every vertex lies in at least one hood; 1/R from the block's table of
        // the same correctly rounded quotients when R is small
        const double inv_R = R < RCP_N ? rcp[R] : 1.0 / (double)R;
        Estar = D[0] + c.beta * ((double)Ks[0] * inv_R);
#pragma unroll
        for (int l = 1; l < L; ++l) {
            const double e = D[l] + c.beta * ((double)Ks[l] * inv_R);
            if (e < Estar) { Estar = e; lab = l; }
        }
    } else {
        // vote: each replica's least label D_l + beta k_l with FP64 semantics:
        // the exact energies of the hood pass's fixed point (excess_l +
        // beta_q k_l in the slice's unit) decide when the least leads every
        // other label by more than both evaluations' rounding bound (as for the
        // default rule), FP64 compares the rest
        uint64_t dq[L];
        int amin;
        const int64_t Fmin = data_fixed<L>(D, q, dq, amin);
        int votes[L], kmin[L];  // set by vote_tally
        const uint64_t bq = (uint64_t)beta_q;
        // one bound for every replica of v: counts k_l <= d, so both
        // evaluations' rounding stays below 8 + 2d units plus 2^-50 of twice
        // the largest magnitude |F_l| + beta_q d
        uint64_t maxF = 0;
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const int64_t F = Fmin + (int64_t)dq[l];
            maxF = max(maxF, (uint64_t)(F < 0 ? -F : F));
        }
        const uint64_t eps = 8 + 2 * (uint64_t)d + ((2 * (maxF + bq * (uint64_t)d)) >> 50);
        // a near-tie needs two labels l, m whose energies differ by at most
        // eps in some replica: (dq_l - dq_m) + beta_q (k_l - k_m) with
        // |k_l - k_m| <= d, i.e. dq_m - dq_l within eps of a multiple beta_q
        // delta, |delta| <= d.  With beta_q > 2 eps at most the nearest
        // multiple qualifies, and a float quotient is within one of it, so
        // three exact integer checks settle it; a smaller beta_q counts as a
        // possible near-tie.  Once per vertex
        bool near = false;
#pragma unroll
        for (int l = 0; l < L; ++l)
#pragma unroll
            for (int m = l + 1; m < L; ++m) {
                const int64_t y = (int64_t)dq[m] - (int64_t)dq[l];
                const uint64_t ay = (uint64_t)(y < 0 ? -y : y);
                if (bq <= 2 * eps) {
                    near = near || ay <= bq * (uint64_t)d + eps;
                } else if (ay <= bq * (uint64_t)d + eps) {
                    const int est = (int)rintf((float)y / (float)bq);
                    for (int dd = -1; dd <= 1; ++dd) {
                        const int64_t delta = (int64_t)est + dd;
                        if (delta < -(int64_t)d || delta > (int64_t)d) continue;
                        const int64_t diff = y - (int64_t)bq * delta;
                        near = near || (uint64_t)(diff < 0 ? -diff : diff) <= eps;
                    }
                }
            }
        if (!near) {
            vote_tally<L>(g, x_in, a0, d, nw, r0, r1, lm, dq, bq, votes, kmin);
        } else {
            VoteFP64<L> a;
            a.rep_mask = g.rep_mask;
            a.adj = g.adj;
            a.x_in = x_in;
            a.a0 = a0;
            a.r0 = r0;
            a.r1 = r1;
            a.d = d;
            a.nw = nw;
            a.beta = c.beta;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                a.D[l] = D[l];
                a.lm[l] = lm[l];
            }
            a = vote_tally_fp64<L>(a);
#pragma unroll
            for (int l = 0; l < L; ++l) {
                votes[l] = a.votes[l];
                kmin[l] = a.kmin[l];
            }
        }
        int best = votes[0];
#pragma unroll
        for (int l = 1; l < L; ++l)
            if (votes[l] > best) { best = votes[l]; lab = l; }
        Estar = 0.0;
#pragma unroll
        for (int l = 0; l < L; ++l)
            if (l == lab) Estar = D[l] + c.beta * (double)kmin[l];
    }
    if (vrec) write_vrec<L>(vrec, g.V, v, D, lm, q);
    return lab;
}

// VAR: the sweep variants of RunCfg (Potts scope, replica rule) read at run
// time; without it the default (hood scope, least-energy replica) is compiled
// alone, so the variants cost the default nothing.  LISTED: each block takes
// listed tiles of sc (the sparse EM loop); otherwise tile blockIdx.x
template <int L, bool VAR, bool LISTED = false>
__global__ void __launch_bounds__(VT_THREADS, vt_min_blocks(L)) k_vertex(DevGraph g, const Tile* __restrict__ tiles, int mode,
                                                       const RunCfg* __restrict__ cfgp,
                                                       const int32_t* __restrict__ active,
                                                       const uint8_t* __restrict__ x_in0, uint8_t* __restrict__ x_out0,
                                                       const double* __restrict__ theta,
                                                       const double* __restrict__ dterm,
                                                       const double* __restrict__ E_in, double* __restrict__ E_out,
                                                       double* __restrict__ vpart, DevStatus* st,
                                                       uint64_t* __restrict__ vrec,
                                                       const SliceUnit* __restrict__ unit,
                                                       const int32_t* __restrict__ tp,
                                                       const TileSched sc) {
    __shared__ double s_mu[L], s_inv[L], s_lnsig[L], s_K[L];
    __shared__ double s_Md[33];  // (double)m for m <= 32: no int-to-FP64 conversions on the common path
    __shared__ double s_rcp[VAR ? RCP_N : 1];  // 1 / R for the mean-energy replica rule
    __shared__ double s_vq[3][VT_THREADS];
    __shared__ double s_vc[3 * L][8];
    __shared__ int s_cnt[VT_THREADS / 32][L];
    __shared__ int s_k;
    for_each_tile<LISTED>(sc, &s_k, [&](int64_t ti) -> bool {
        const Tile tile = tiles[ti];
        const int s = tile.slice;
        if (active && !active[s]) return true;
        // in a loop graph the iteration t comes from device memory: x_in,
        // x_out are the label buffers of odd t, exchanged for even t
        const bool swap = tp && !(*tp & 1);
        const uint8_t* __restrict__ x_in = swap ? x_out0 : x_in0;
        uint8_t* __restrict__ x_out = swap ? const_cast<uint8_t*>(x_in0) : x_out0;
        const RunCfg c = *cfgp;
        if (threadIdx.x < 33) s_Md[threadIdx.x] = (double)threadIdx.x;
        if (VAR && threadIdx.x < RCP_N && c.rule == PMRF_RULE_SUM)
            s_rcp[threadIdx.x] = threadIdx.x > 0 ? 1.0 / (double)threadIdx.x : 0.0;
        if (threadIdx.x < L) {
            const int l = threadIdx.x;
            if (mode == MODE_INIT) {
                s_K[l] = bin_centre(c, l);
            } else {
                const double mu = theta[((int64_t)s * L + l) * 4 + 1];
                s_mu[l] = mu;
                s_K[l] = mu;
                if (dterm) {  // the finaliser's per-slice values (EM loop)
                    s_inv[l] = dterm[((int64_t)s * L + l) * 2 + 0];
                    s_lnsig[l] = dterm[((int64_t)s * L + l) * 2 + 1];
                } else {
                    const double sg = theta[((int64_t)s * L + l) * 4 + 2];
                    s_inv[l] = inv_two_var(sg);
                    s_lnsig[l] = log(sg);
                }
            }
        }
        __syncthreads();
        const int64_t v = (int64_t)tile.a0 + threadIdx.x;
        const bool ok = v < tile.a1;
        // the slice's fixed-point unit of this iteration (records of the hood pass)
        const int uq = unit ? unit[s].q : 0;
        const int64_t ubq = unit ? unit[s].beta_q : 0;
        int vlab = 0;
        double vq0 = 0.0, vq1 = 0.0, vq2 = 0.0;  // y - K_lab, (y - K_lab)^2, E* of this vertex
        int64_t Eq = 0;                          // EM: E* in the slice's unit (exact sums within the tile)
        bool have_dev = false;                   // EM/sweep: y - mu_lab and its square already known
        if (ok) {
            const double y = g.y[v];
            int lab = 0;
            double Estar = 0.0;
            if (mode == MODE_INIT) {
                lab = c.init_from_labels ? (int)x_in[v] : threshold_label(c, y);
                if (lab >= L) { record_error(st, PMRF_ERR_ARG, SITE_LABEL, v); lab = L - 1; }
            } else if (mode == MODE_PARAMS) {
                lab = (int)x_in[v];
                if (lab >= L) { record_error(st, PMRF_ERR_ARG, SITE_LABEL, v); lab = L - 1; }
                Estar = E_in ? E_in[v] : 0.0;
            } else {
                // a caller's labels (standalone sweep) must lie in [0, L)
                if (mode == MODE_SWEEP && x_in[v] >= L) record_error(st, PMRF_ERR_ARG, SITE_LABEL, v);
                // data term D_l(y) = (y - mu_l)^2 / (2 sigma_l^2) + ln sigma_l
                double D[L], dev[L], dev2[L];
    #pragma unroll
                for (int l = 0; l < L; ++l) {
                    dev[l] = y - s_mu[l];
                    dev2[l] = dev[l] * dev[l];
                    D[l] = dev2[l] * s_inv[l] + s_lnsig[l];
                }
                const int64_t a0 = g.adj_off[v];
                const int d = (int)(g.adj_off[v + 1] - a0);
                const int64_t r0 = g.rep_woff[v], r1 = g.rep_woff[v + 1];
                int M[L];
    #pragma unroll
                for (int l = 0; l < L; ++l) M[l] = 0x7fffffff;
                uint32_t lm[L];  // label masks over v's adjacency slots (degree <= 32; else unused)
    #pragma unroll
                for (int l = 0; l < L; ++l) lm[l] = 0;
                if (d <= 32) {
                    for (int j = 0; j < d; ++j) {
                        const int xl = x_in[g.adj[a0 + j]];
    #pragma unroll
                        for (int l = 0; l < L; ++l) lm[l] |= (xl == l ? 1u : 0u) << j;
                    }
                }
                if (!VAR || (c.scope == PMRF_SCOPE_HOOD && c.rule == PMRF_RULE_MIN)) {
                    if (d <= 32) {
                        // neighbours in the hood whose label is not l, minimised over
                        // the replicas; the masks are read four at a time once the
                        // address is 16-byte aligned (fewer load requests per warp)
                        for_each_mask(g.rep_mask, r0, r1, [&](uint32_t m) {
                            const int dc = __popc(m);
    #pragma unroll
                            for (int l = 0; l < L; ++l) M[l] = min(M[l], dc - __popc(m & lm[l]));
                        });
                    } else {
                        const int nw = (d + 31) >> 5;
                        for (int64_t r = r0; r < r1; r += nw) {
                            int cnt[L];
                            const int dc = slot_label_counts<L>(g, x_in, a0, r, nw, cnt);
    #pragma unroll
                            for (int l = 0; l < L; ++l) M[l] = min(M[l], dc - cnt[l]);
                        }
                    }
                    // the hood pass of this iteration reads v's data terms and label masks
                    // every vertex lies in at least one hood, so M_l is set (and
                    // <= 32 when d <= 32).  The data terms in the slice's unit serve
                    // the hood pass's record.  The label is the least D_l + beta M_l
                    // in FP64 (ties to the lower label), the precision the oracle
                    // decides in.  The exact energies in the unit give the same
                    // label whenever the least one leads every other by more than
                    // both evaluations' rounding can move them (fixed point: half a
                    // unit per rounded term, so 1/2 + M/2; FP64: 2^-52 of the
                    // magnitude plus one unit; taken generously below); only closer
                    // labels are compared in FP64.  The label's energy in the unit
                    // enters the tile's exact sum of E*
                    int64_t F[L], e[L];
    #pragma unroll
                    for (int l = 0; l < L; ++l) {
                        F[l] = to_fixed(D[l], uq);
                        e[l] = F[l] + ubq * (int64_t)M[l];
                    }
                    if (vrec) write_vrec_fixed<L>(vrec, g.V, v, F, lm);
                    int64_t eb = e[0];
                    lab = 0;
    #pragma unroll
                    for (int l = 1; l < L; ++l)
                        if (e[l] < eb) { eb = e[l]; lab = l; }
                    uint64_t mag_b = 0;
                    int m_b = 0;
    #pragma unroll
                    for (int l = 0; l < L; ++l)
                        if (l == lab) {
                            mag_b = (uint64_t)(F[l] < 0 ? -F[l] : F[l]) + (uint64_t)ubq * (uint64_t)M[l];
                            m_b = M[l];
                        }
                    bool sure = true;
    #pragma unroll
                    for (int l = 0; l < L; ++l) {
                        const uint64_t mag = (uint64_t)(F[l] < 0 ? -F[l] : F[l]) + (uint64_t)ubq * (uint64_t)M[l];
                        const int64_t eps = 4 + M[l] + m_b + (int64_t)((mag + mag_b) >> 50);
                        if (l != lab && e[l] - eb <= eps) sure = false;
                    }
                    if (!sure) {
                        double best = D[0] + c.beta * (d <= 32 ? s_Md[M[0]] : (double)M[0]);
                        lab = 0;
    #pragma unroll
                        for (int l = 1; l < L; ++l) {
                            const double x = D[l] + c.beta * (d <= 32 ? s_Md[M[l]] : (double)M[l]);
                            if (x < best) { best = x; lab = l; }
                        }
                    }
    #pragma unroll
                    for (int l = 0; l < L; ++l)
                        if (l == lab) Eq = e[l];
                    if (E_out) {  // the chosen label's energy in FP64 (standalone sweep)
    #pragma unroll
                        for (int l = 0; l < L; ++l)
                            if (l == lab) Estar = D[l] + c.beta * (d <= 32 ? s_Md[M[l]] : (double)M[l]);
                    }
                } else {
                    lab = vertex_variant<L>(g, c, x_in, a0, d, r0, r1, lm, D, vrec, v, Estar, s_rcp, uq, ubq);
                    Eq = to_fixed(Estar, uq);
                }
                x_out[v] = (uint8_t)lab;
                if (E_out) E_out[v] = Estar;
                // K = mu here: the moments reuse y - mu_lab and its square
    #pragma unroll
                for (int l = 0; l < L; ++l)
                    if (l == lab) {
                        vq0 = dev[l];
                        vq1 = dev2[l];
                    }
                have_dev = true;
            }
            if (mode == MODE_INIT) x_out[v] = (uint8_t)lab;
            if (mode != MODE_SWEEP) {
                if (!have_dev) {
                    const double dv = y - s_K[lab];
                    vq0 = dv;
                    vq1 = dv * dv;
                }
                vlab = lab;
                vq2 = mode == MODE_EM ? __longlong_as_double(Eq) : Estar;
            }
        }
        if (mode == MODE_SWEEP) return true;
        // deterministic per-label sums of the tile: each vertex contributes to the
        // label it carries (no shuffle trees: the FP64 pipe is the scarce unit).
        // Label counts of the tile by warp ballots; each vertex's place in its
        // label's run (tile order kept) so the sums below add only that label's
        // values
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        unsigned mine = 0u;
    #pragma unroll
        for (int l = 0; l < L; ++l) {
            const unsigned b = __ballot_sync(0xffffffffu, ok && vlab == l);
            if (lane == 0) s_cnt[warp][l] = __popc(b);
            if (ok && vlab == l) mine = b;
        }
        __syncthreads();
        if (ok) {
            int pos = __popc(mine & ((1u << lane) - 1u));
            for (int l = 0; l < vlab; ++l)
                for (int w = 0; w < VT_THREADS / 32; ++w) pos += s_cnt[w][l];
            for (int w = 0; w < warp; ++w) pos += s_cnt[w][vlab];
            s_vq[0][pos] = vq0;
            s_vq[1][pos] = vq1;
            s_vq[2][pos] = vq2;
        }
        __syncthreads();
        // 8 threads per (label, quantity) add fixed consecutive chunks of the
        // label's run in order, then one thread adds the 8 results in order
        for (int job = threadIdx.x; job < 3 * L * 8; job += VT_THREADS) {  // two jobs a thread when L > 5
            const int lq = job >> 3, k = job & 7;
            const int l = lq / 3, q = lq % 3;
            int base = 0, n = 0;
            for (int m = 0; m < L; ++m)
                for (int w = 0; w < VT_THREADS / 32; ++w) {
                    const int cw = s_cnt[w][m];
                    if (m < l) base += cw;
                    if (m == l) n += cw;
                }
            const int lo = base + (k * n) / 8, hi = base + ((k + 1) * n) / 8;
            if (q == 2 && mode == MODE_EM) {
                // E* in the slice's unit: an exact integer sum (|E*| < 2^62 / 128)
                int64_t a = 0;
                for (int i = lo; i < hi; ++i) a += __double_as_longlong(s_vq[q][i]);
                s_vc[lq][k] = __longlong_as_double(a);
            } else {
                double a = 0.0;
                for (int i = lo; i < hi; ++i) a += s_vq[q][i];
                s_vc[lq][k] = a;
            }
            if (q == 0 && k == 0) vpart[(int64_t)tile.part * 4 * L + 4 * l + 0] = (double)n;
        }
        __syncthreads();
        if (threadIdx.x < 3 * L) {
            const int l = threadIdx.x / 3, q = threadIdx.x % 3;
            double a = 0.0;
            if (q == 2 && mode == MODE_EM) {
                // the tile's exact sum of E*, rounded to double once
                int64_t ai = 0;
                for (int w = 0; w < 8; ++w) ai += __double_as_longlong(s_vc[threadIdx.x][w]);
                a = from_fixed64(ai, uq);
            } else {
                for (int w = 0; w < 8; ++w) a += s_vc[threadIdx.x][w];
            }
            vpart[(int64_t)tile.part * 4 * L + 4 * l + 1 + q] = a;
        }
        return true;
    });
}

// ---------------------------------------------------------------------------
// hood pass

// decoded hood-pass record of one vertex (dq[amin] = 0)
template <int L>
struct VRec {
    int64_t Dmin;
    uint64_t dq[L];
    uint32_t lmv[L];  // lmv[L-1] unused
};

// The records are gathered (one 32-byte chunk per element for L <= 3)
template <int L>
__device__ __forceinline__ VRec<L> load_vrec(const uint64_t* __restrict__ vrec, int64_t V, int64_t v) {
    constexpr int NW = vrec_words(L);
    uint64_t w[NW];
    if constexpr (L == 2) {
        asm("ld.global.nc.v2.b64 {%0, %1}, [%2];" : "=l"(w[0]), "=l"(w[1]) : "l"(vrec + 2 * v));
        w[2] = __ldg(vrec2_masks(vrec, V) + v);
        w[3] = 0;
    } else {
        const uint64_t* p = vrec + v * NW;
#pragma unroll
        for (int k = 0; k < NW; k += 4)
            asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
                : "=l"(w[k]), "=l"(w[k + 1]), "=l"(w[k + 2]), "=l"(w[k + 3])
                : "l"(p + k));
    }
    VRec<L> R;
    R.Dmin = (int64_t)w[0];
    const int amin = L > 1 ? (int)(w[1] >> 61) : 0;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const uint64_t own = (l < L - 1) ? (w[1 + l] & DQ_SAT) : 0ull;  // stored slot l (labels below amin)
        const uint64_t up = (l >= 1) ? (w[l] & DQ_SAT) : 0ull;          // stored slot l-1 (labels above amin)
        R.dq[l] = l == amin ? 0ull : (l < amin ? own : up);
    }
    if constexpr (L == 2) {
        const uint32_t mb = (uint32_t)w[2];  // slots holding the label other than amin
        R.lmv[0] = amin == 0 ? ~mb : mb;
        R.lmv[1] = 0u;
    } else {
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const int u = 2 * L + k;  // u32 index of mask k
            R.lmv[k] = k < L - 1 ? (uint32_t)(w[u >> 1] >> (32 * (u & 1))) : 0u;
        }
    }
    return R;
}

// the element's energy above D_min at its best label: min_l [dq_l + beta_q *
// (dc - cnt_l)]; every term is >= 0 and the minimum is at most dc * beta_q
// (the amin term)
template <int L>
__device__ __forceinline__ int64_t vrec_excess(const VRec<L>& R, const int (&cnt)[L], int dc, int64_t beta_q) {
    int64_t r = INT64_MAX;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const int64_t x = (int64_t)R.dq[l] + beta_q * (int64_t)(dc - cnt[l]);
        r = x < r ? x : r;
    }
    return r;
}

// label counts among the element's in-hood neighbours, from its slot mask and
// the vertex's label masks (every label is in [0, L): the last label's count is
// what the other masks leave of the slot mask)
template <int L>
__device__ __forceinline__ int slot_counts(const VRec<L>& R, uint32_t m, int (&cnt)[L]) {
    const int dc = __popc(m);
    int rest = dc;
#pragma unroll
    for (int l = 0; l < L - 1; ++l) {
        cnt[l] = __popc(m & R.lmv[l]);
        rest -= cnt[l];
    }
    cnt[L - 1] = rest;
    return dc;
}

// Element energy Emin(c,v) in the slice's unit, from v's record and the
// element's slot mask (every neighbour of v of degree <= 32)
template <int L>
__device__ __forceinline__ int64_t element_energy(const uint64_t* __restrict__ vrec, int64_t V, uint32_t vid,
                                                  uint32_t m, int64_t beta_q) {
    if constexpr (L == 2) {
        uint64_t w0, w1;
        asm("ld.global.nc.v2.b64 {%0, %1}, [%2];" : "=l"(w0), "=l"(w1) : "l"(vrec + 2 * (int64_t)vid));
        const uint32_t mb = __ldg(vrec2_masks(vrec, V) + vid);
        const int cb = __popc(m & mb);
        const int k = 2 * cb - __popc(m);
        const int64_t dq = (int64_t)(w1 & DQ_SAT);
        const int64_t bk = beta_q * k;
        return (int64_t)w0 + beta_q * cb - (bk > dq ? bk - dq : 0);
    } else {
        const VRec<L> R = load_vrec<L>(vrec, V, (int64_t)vid);
        int cnt[L];
        const int dc = slot_counts<L>(R, m, cnt);
        return R.Dmin + vrec_excess<L>(R, cnt, dc, beta_q);
    }
}

// The hood convergence test of Section 3.2.2 (reading G9) in integers: hood c
// has converged at t iff t > W and |S^t - S^{t-k}| < tol for k = 1..W.  The
// ring holds each sum in the unit of its own iteration (qhist per slot): with
// equal units the test is exact (|a - b| < ceil(tol 2^q)); when the unit
// changed in between, both are floored to the coarser unit first (an error
// below one unit of it, about 1e-15 relative).  Equal states give identical
// sums and pass exactly.  Returns 1 when the hood is unconverged.
__device__ __forceinline__ int64_t shift_down(int64_t x, int sh) { return sh >= 63 ? (x < 0 ? -1 : 0) : (x >> sh); }

__device__ __forceinline__ int hood_history(int64_t S, int64_t c, int64_t C, int t, int W, const SliceUnit& u,
                                            const int32_t* __restrict__ qh, double tol,
                                            int64_t* __restrict__ hist) {
    int unconv = 1;
    if (t > W) {
        unconv = 0;
        for (int k = 1; k <= W; ++k) {
            const int slot = (t - k) % W;
            const int64_t prev = hist[(int64_t)slot * C + c];
            const int qp = qh[slot];
            int64_t a = S, b = prev, thr = u.tol_q;
            if (qp != u.q) {
                const int m = min(qp, u.q);
                a = shift_down(S, u.q - m);
                b = shift_down(prev, qp - m);
                thr = tol_units(tol, m);
            }
            const int64_t d = a >= b ? a - b : b - a;
            if (!(d < thr)) {
                unconv = 1;
                break;
            }
        }
    }
    hist[(int64_t)(t % W) * C + c] = S;
    return unconv;
}

// The fast-tile hood sums: P adjacent lanes per hood (1, 2, 4 or 8), each taking
// every P-th element of the hood from the tile's staged element stream, their
// partial sums added across the group (integers: exact in any order).
// energy(vertex id, slot mask) gives the element energy.
template <int P, typename Energy, typename Done>
__device__ __forceinline__ void fast_hoods(const DevGraph& g, int64_t c0, int64_t c1, int64_t e0,
                                           const uint2* __restrict__ s_el, Energy&& energy, Done&& hood_done) {
    const int sub = threadIdx.x & (P - 1);
    const unsigned gmask = P == 1 ? (1u << (threadIdx.x & 31))
                                  : (((1u << P) - 1u) << ((threadIdx.x & 31) & ~(P - 1)));
    for (int64_t c = c0 + threadIdx.x / P; c < c1; c += HT_THREADS / P) {
        const int b = (int)(g.hood_off[c] - e0), e = (int)(g.hood_off[c + 1] - e0);
        int64_t acc = 0;
#pragma unroll 2
        for (int i = b + sub; i < e; i += P) {
            const uint2 q = s_el[i];
            acc += energy(q.x & 0x7fffffffu, q.y);
        }
#pragma unroll
        for (int o = 1; o < P; o <<= 1) acc += __shfl_xor_sync(gmask, acc, o);
        if (sub == 0) hood_done(c, acc);
    }
}

template <typename Energy, typename Done>
__device__ __forceinline__ void fast_hoods_p(int lanes, const DevGraph& g, int64_t c0, int64_t c1, int64_t e0,
                                             const uint2* __restrict__ s_el, Energy&& energy, Done&& hood_done) {
    if (lanes >= 8)
        fast_hoods<8>(g, c0, c1, e0, s_el, energy, hood_done);
    else if (lanes == 4)
        fast_hoods<4>(g, c0, c1, e0, s_el, energy, hood_done);
    else if (lanes == 2)
        fast_hoods<2>(g, c0, c1, e0, s_el, energy, hood_done);
    else
        fast_hoods<1>(g, c0, c1, e0, s_el, energy, hood_done);
}

// Per-hood bookkeeping of one tile and its partials: the exact sum of the
// tile's hood sums and its number of unconverged hoods
struct TileAcc {
    __int128 T = 0;
    int unconv = 0;
};

__device__ __forceinline__ void tile_partials(TileAcc& a, int64_t part, int64_t* __restrict__ hpart,
                                              __int128* s_wT, int* s_wu) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a.T += shfl_xor_i128(a.T, o);
        a.unconv += __shfl_xor_sync(0xffffffffu, a.unconv, o);
    }
    __syncthreads();
    if (lane_id() == 0) {
        s_wT[warp_id()] = a.T;
        s_wu[warp_id()] = a.unconv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __int128 t = 0;
        int n = 0;
        for (int w = 0; w < HT_THREADS / 32; ++w) {
            t += s_wT[w];
            n += s_wu[w];
        }
        hpart[part * 3 + 0] = (int64_t)(uint64_t)(unsigned __int128)t;
        hpart[part * 3 + 1] = (int64_t)(t >> 64);
        hpart[part * 3 + 2] = n;
    }
    a.T = 0;
    a.unconv = 0;
}

// A general tile (some member of degree > 32): hood by hood, the block's lanes
// splitting the hood's elements and counting labels through the hood-local
// adjacency rows
template <int L, typename Done>
__device__ __forceinline__ void general_tile(const DevGraph& g, const RunCfg& cf, int64_t c0, int64_t c1,
                                             const uint8_t* __restrict__ x_in, const uint64_t* __restrict__ vrec,
                                             int64_t beta_q, int64_t* s_wsum, Done&& hood_done) {
    for (int64_t c = c0; c < c1; ++c) {
        const int64_t hb = g.hood_off[c];
        const int64_t k = g.hood_off[c + 1] - hb;
        const int64_t nwh = (k + 31) >> 5;
        const int64_t rb = g.row_off[c];
        int64_t part = 0;
        for (int64_t i = threadIdx.x; i < k; i += HT_THREADS) {
            const int64_t v = g.hood[hb + i];
            int cnt[L];
#pragma unroll
            for (int l = 0; l < L; ++l) cnt[l] = 0;
            int dc = 0;
            for (int64_t w = 0; w < nwh; ++w) {
                uint32_t m = g.row[rb + i * nwh + w];
                dc += __popc(m);
                while (m) {
                    const int bb = __ffs(m) - 1;
                    m &= m - 1;
                    const int xl = x_in[g.hood[hb + w * 32 + bb]];
#pragma unroll
                    for (int l = 0; l < L; ++l) cnt[l] += (xl == l);
                }
            }
            const VRec<L> R = load_vrec<L>(vrec, g.V, v);
            // full scope: the record's D_min is already the element energy
            part += cf.scope == PMRF_SCOPE_FULL ? R.Dmin : R.Dmin + vrec_excess<L>(R, cnt, dc, beta_q);
        }
        // exact integer sums: the reduction order does not matter
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        __syncthreads();
        if (lane_id() == 0) s_wsum[warp_id()] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t S = 0;
            for (int w = 0; w < HT_THREADS / 32; ++w) S += s_wsum[w];
            hood_done(c, S);
        }
    }
}

// The hood pass: one block per hood tile (consecutive hoods of one slice, their
// elements contiguous).  Fast tiles (every member of degree <= 32): the tile's
// element stream (member id and slot mask, one 8-byte word each) is staged in
// shared memory by one bulk copy (the TMA engine, completion counted on an
// mbarrier), then lanes-per-hood adjacent lanes take each hood, gather its
// members' records and sum the element energies.
// General tiles go hood by hood through the hood-local adjacency rows.
template <int L, bool LISTED = false>
__global__ void __launch_bounds__(HT_THREADS, ht_min_blocks(L)) k_hood(DevGraph g, const Tile* __restrict__ tiles,
                                                     int mode, int t, int lanes,
                                                     const RunCfg* __restrict__ cfgp,
                                                     const int32_t* __restrict__ active,
                                                     const uint8_t* __restrict__ x_in,
                                                     const uint64_t* __restrict__ vrec,
                                                     const SliceUnit* __restrict__ unit,
                                                     const int32_t* __restrict__ qhist,
                                                     int64_t* __restrict__ hist, double* __restrict__ S_out,
                                                     int64_t* __restrict__ hpart, int cap, DevStatus* st,
                                                     const uint8_t* __restrict__ x_alt,
                                                     const int32_t* __restrict__ tp,
                                                     const TileSched sc) {
    // in a loop graph t comes from device memory and x_alt holds the labels
    // that even iterations read
    if (tp) {
        t = *tp;
        if (!(t & 1)) x_in = x_alt;
    }
    // cap + 2 elements: the window plus the rest of its last hood, and one word
    // either side for the 16-byte alignment of the bulk copy
    extern __shared__ __align__(16) uint2 s_el[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int64_t s_wsum[HT_THREADS / 32];
    __shared__ __int128 s_wT[HT_THREADS / 32];
    __shared__ int s_wu[HT_THREADS / 32];
    __shared__ int s_k;
    // the staging barrier, initialised by the block's first staged tile: each
    // staged tile completes one phase of it (parity ph)
    bool bar_ready = false;
    uint32_t ph = 0;
    for_each_tile<LISTED>(sc, &s_k, [&](int64_t ti) -> bool {
        const Tile tile = tiles[ti];
        const int s = tile.slice;
        if (active && !active[s]) return true;
        const RunCfg cf = *cfgp;
        const SliceUnit u = unit[s];
        const int W = cf.W;
        const int32_t* qh = qhist ? qhist + (int64_t)s * W : nullptr;
        TileAcc acc;
        auto hood_done = [&](int64_t c, int64_t S) {
            if (mode == MODE_SWEEP) {
                if (S_out) S_out[c] = from_fixed((__int128)S, u.q);
            } else {
                acc.unconv += hood_history(S, c, g.C, t, W, u, qh, cf.tol, hist);
                acc.T += S;
            }
        };
        const int64_t c0 = tile.a0, c1 = tile.a1;
        if (c1 > c0) {
            const int64_t e0 = g.hood_off[c0];
            const int ne = (int)(g.hood_off[c1] - e0);
            if (tile.pad != 0) {
                auto energy = [&](uint32_t vid, uint32_t m) { return element_energy<L>(vrec, g.V, vid, m, u.beta_q); };
                if (ne <= cap) {
                    const int64_t ea = e0 & ~1ll, eb = (e0 + ne + 1) & ~1ll;  // 16-byte aligned bounds
                    if (!bar_ready) {  // (the same in every thread)
                        if (threadIdx.x == 0) {
                            mbar_init(&s_bar);
                            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
                        }
                        __syncthreads();  // initialised before anyone polls it
                        bar_ready = true;
                    }
                    if (threadIdx.x == 0) {
                        const uint32_t bytes = (uint32_t)((eb - ea) * 8);
                        mbar_expect(&s_bar, bytes);
                        bulk_copy(s_el, g.el + ea, bytes, &s_bar);
                    }
                    // a wait that gives up has set the status word; it waits
                    // once more (bounded) so that no copy is left in flight,
                    // and the block stops: the barrier's phase is unknown
                    // (the same decision in every thread: lanes of a hood
                    // shuffle together)
                    const bool staged = __syncthreads_and(mbar_wait(&s_bar, ph, st) || mbar_wait(&s_bar, ph, st));
                    ph ^= 1u;
                    if (!staged) return false;
                    fast_hoods_p(lanes, g, c0, c1, e0, s_el + (e0 - ea), energy, hood_done);
                } else {
                    // a tile whose last hood reaches far past its window (very
                    // large hoods): the element stream is read where it lies
                    fast_hoods<8>(g, c0, c1, e0, g.el + e0, energy, hood_done);
                }
            } else {
                general_tile<L>(g, cf, c0, c1, x_in, vrec, u.beta_q, s_wsum, hood_done);
            }
        }
        if (mode != MODE_SWEEP) tile_partials(acc, tile.part, hpart, s_wT, s_wu);
        return true;
    });
}

// ---------------------------------------------------------------------------
// per slice: intensity range, fixed-point unit, parameters and convergence

// the unit of every slice from the given parameters (standalone sweep)
__global__ void k_units(int32_t S, int L, const double* __restrict__ theta, const double* __restrict__ yr,
                        const RunCfg* __restrict__ cfgp, int max_deg, int max_hood, SliceUnit* __restrict__ unit,
                        DevStatus* st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    bool ok = true;
    unit[s] = slice_unit(theta + (int64_t)s * L * 4, L, yr[2 * s], yr[2 * s + 1], cfgp->beta, cfgp->tol, max_deg,
                         max_hood, ok);
    if (!ok) record_error(st, PMRF_ERR_UNSUPPORTED, SITE_RANGE, s);
}

// the intensity range [min y, max y] of every slice (one block per slice)
__global__ void k_yrange(const int64_t* __restrict__ vert_off, const double* __restrict__ y, double* __restrict__ yr) {
    __shared__ double s_lo[FIN_THREADS / 32], s_hi[FIN_THREADS / 32];
    const int s = blockIdx.x;
    double lo = INFINITY, hi = -INFINITY;
    const int64_t v0 = vert_off[s], v1 = vert_off[s + 1];
    // eight loads in flight per thread
    for (int64_t v = v0 + threadIdx.x; v < v1; v += 8 * (int64_t)blockDim.x) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t i = v + (int64_t)u * blockDim.x;
            x[u] = i < v1 ? y[i] : y[v];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            lo = fmin(lo, x[u]);
            hi = fmax(hi, x[u]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane_id() == 0) {
        s_lo[warp_id()] = lo;
        s_hi[warp_id()] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < FIN_THREADS / 32; ++w) {
            lo = fmin(lo, s_lo[w]);
            hi = fmax(hi, s_hi[w]);
        }
        lo = fmin(lo, s_lo[0]);
        hi = fmax(hi, s_hi[0]);
        // an empty slice: any finite range
        yr[2 * s] = lo <= hi ? lo : 0.0;
        yr[2 * s + 1] = lo <= hi ? hi : 0.0;
    }
}

template <int L>
__global__ void k_finalize(int32_t S, int mode, int t, const RunCfg* __restrict__ cfgp,
                           const int64_t* __restrict__ vt0, const int64_t* __restrict__ ht0,
                           const double* __restrict__ vpart, const int64_t* __restrict__ hpart,
                           const double* __restrict__ theta_prev, double* __restrict__ theta,
                           const int64_t* __restrict__ vert_off, int32_t* __restrict__ active,
                           int32_t* __restrict__ iters, int32_t* __restrict__ conv, double* __restrict__ Thist,
                           int32_t* __restrict__ nactive, const OutPtrs* __restrict__ op,
                           double* __restrict__ dterm, SliceUnit* __restrict__ unit, int32_t* __restrict__ qhist,
                           const double* __restrict__ yr, int max_deg, int max_hood, DevStatus* st,
                           const int32_t* __restrict__ tp) {
    if (tp) t = *tp;  // a loop graph's iteration
    constexpr int NQ = 4 * L;  // label moments
    __shared__ double s_q[FIN_THREADS / 32][NQ];
    __shared__ __int128 s_T[FIN_THREADS / 32];
    __shared__ int64_t s_u[FIN_THREADS / 32];
    const int s = blockIdx.x;
    if (s >= S) return;
    const RunCfg cf = *cfgp;
    const bool em = (mode == MODE_EM);
    if (em && !active[s]) return;
    // the slice's tile partials: a fixed thread per partial, then fixed-order
    // warp and block sums (deterministic)
    double tot[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) tot[k] = 0.0;
    for (int64_t p = vt0[s] + threadIdx.x; p < vt0[s + 1]; p += FIN_THREADS) {
#pragma unroll
        for (int k = 0; k < 4 * L; ++k) tot[k] += vpart[p * 4 * L + k];
    }
    // T: the exact sum of the tiles' exact partials (integers: independent
    // of the tiling and of the order), rounded once
    __int128 Tacc = 0;
    int64_t uacc = 0;
    if (em) {
        for (int64_t p = ht0[s] + threadIdx.x; p < ht0[s + 1]; p += FIN_THREADS) {
            Tacc += (__int128)(((unsigned __int128)(uint64_t)hpart[p * 3 + 1] << 64) | (uint64_t)hpart[p * 3 + 0]);
            uacc += hpart[p * 3 + 2];
        }
    }
#pragma unroll
    for (int k = 0; k < NQ; ++k) tot[k] = warp_sum(tot[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Tacc += shfl_xor_i128(Tacc, o);
        uacc += __shfl_xor_sync(0xffffffffu, uacc, o);
    }
    if (lane_id() == 0) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) s_q[warp_id()][k] = tot[k];
        s_T[warp_id()] = Tacc;
        s_u[warp_id()] = uacc;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        double a = 0.0;
        for (int w = 0; w < FIN_THREADS / 32; ++w) a += s_q[w][k];
        tot[k] = a;
    }
    Tacc = 0;
    uacc = 0;
    for (int w = 0; w < FIN_THREADS / 32; ++w) {
        Tacc += s_T[w];
        uacc += s_u[w];
    }
    // T^t in the unit of this iteration (the unit slot of the hood ring takes
    // the same unit); then the unit of the next iteration from theta^t
    const int q_now = (mode == MODE_EM) ? unit[s].q : 0;
    const double Tsum = em ? from_fixed(Tacc, q_now) : 0.0, unconv = (double)uacc;
    if (em) qhist[(int64_t)s * cf.W + t % cf.W] = q_now;
    for (int l = 0; l < L; ++l) {
        const double n = tot[4 * l + 0];
        double* th = theta + ((int64_t)s * L + l) * 4;
        double mu_prev, sg_prev;
        if (mode == MODE_INIT) {
            mu_prev = bin_centre(cf, l);
            sg_prev = (cf.init_hi - cf.init_lo) / (double)cf.L;
        } else {
            mu_prev = theta_prev[((int64_t)s * L + l) * 4 + 1];
            sg_prev = theta_prev[((int64_t)s * L + l) * 4 + 2];
        }
        if (mode == MODE_INIT && cf.init_from_labels == 2) {
            // the caller's starting mu and sigma (already in theta), sigma floored
            th[0] = 0.0;
            if (!(th[2] > cf.sigma_min)) th[2] = cf.sigma_min;
            th[3] = 0.0;
        } else if (n > 0.0) {
            const double m1 = tot[4 * l + 1] / n;
            const double var = fmax(tot[4 * l + 2] / n - m1 * m1, 0.0);
            const double sd = sqrt(var);
            th[0] = n;
            th[1] = mu_prev + m1;
            th[2] = sd > cf.sigma_min ? sd : cf.sigma_min;
            th[3] = (mode == MODE_INIT) ? 0.0 : tot[4 * l + 3];
        } else {
            th[0] = 0.0;
            th[1] = mu_prev;
            th[2] = sg_prev;
            th[3] = 0.0;
        }
        if (dterm) {  // read by the next vertex pass instead of recomputing them per block
            dterm[((int64_t)s * L + l) * 2 + 0] = inv_two_var(th[2]);
            dterm[((int64_t)s * L + l) * 2 + 1] = log(th[2]);
        }
    }
    if (unit && (mode == MODE_INIT || mode == MODE_EM)) {
        bool ok = true;
        unit[s] = slice_unit(theta + (int64_t)s * L * 4, L, yr[2 * s], yr[2 * s + 1], cf.beta, cf.tol, max_deg,
                             max_hood, ok);
        if (!ok) record_error(st, PMRF_ERR_UNSUPPORTED, SITE_RANGE, s);
    }
    if (mode == MODE_INIT) {
        const bool nonempty = vert_off[s + 1] > vert_off[s];
        active[s] = nonempty ? 1 : 0;
        iters[s] = 0;
        conv[s] = nonempty ? 0 : 1;
        if (!nonempty) atomicSub(nactive, 1);
        return;
    }
    if (!em) return;
    const int W = cf.W;
    bool tot_conv = false;
    if (t > W) {
        double dmax = 0.0;
        for (int k = 1; k <= W; ++k) dmax = fmax(dmax, fabs(Tsum - Thist[(int64_t)s * W + (t - k) % W]));
        tot_conv = dmax < cf.tol;
    }
    Thist[(int64_t)s * W + t % W] = Tsum;
    if (op && op->thist) op->thist[(int64_t)s * cf.max_iters + (t - 1)] = Tsum;
    const bool all_conv = (t > W) && unconv == 0.0;
    iters[s] = t;
    if (all_conv || tot_conv || t >= cf.max_iters) {
        active[s] = 0;
        conv[s] = (all_conv || tot_conv) ? 1 : 0;
        atomicSub(nactive, 1);
    }
}

// copy each slice's final labels (from the buffer its last iteration wrote)
// and the run's outputs
__global__ void k_close(DevGraph g, int L, const uint8_t* __restrict__ x0, const uint8_t* __restrict__ x1,
                        const int32_t* __restrict__ iters, const int32_t* __restrict__ conv,
                        const double* __restrict__ theta, const OutPtrs* __restrict__ op) {
    const OutPtrs o = *op;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.V; v += stride) {
        const int s = (int)(upper_bound_dev<int64_t>(g.vert_off, 0, g.S + 1, v) - 1);
        o.labels[v] = (iters[s] & 1) ? x1[v] : x0[v];
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)g.S * L * 4; i += stride)
        o.params[i] = theta[i];
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < g.S; s += stride) {
        o.iters[s] = iters[s];
        o.conv[s] = conv[s];
    }
}

__global__ void k_zero_T(const OutPtrs* __restrict__ op, int64_t n) {
    double* T = op->thist;
    if (!T) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        T[i] = 0.0;
}

__global__ void k_init_labels(DevGraph g, const RunCfg* __restrict__ cfgp, uint8_t* __restrict__ x) {
    const RunCfg c = *cfgp;
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < g.V) x[v] = (uint8_t)threshold_label(c, g.y[v]);
}

__global__ void k_label_image(const int32_t* __restrict__ ids, const int64_t* __restrict__ pix_off,
                              const int64_t* __restrict__ rank_off, const int32_t* __restrict__ rank,
                              const uint8_t* __restrict__ labels, uint8_t* __restrict__ out,
                              const int64_t* __restrict__ maxid1, DevStatus* st) {
    // four pixels a thread (256 apart, each access coalesced), their
    // id -> vertex -> label chains in flight together
    const int s = blockIdx.y;
    const int64_t b = pix_off[s], e = pix_off[s + 1], rb = rank_off[s], nr = rank_off[s + 1] - rb;
    constexpr int CHUNK = 4 * LI_THREADS;
    for (int64_t base = b + (int64_t)blockIdx.x * CHUNK + threadIdx.x; base < e; base += (int64_t)gridDim.x * CHUNK) {
        int32_t id[4], v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t p = base + k * LI_THREADS;
            id[k] = p < e ? ids[p] : -1;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (id[k] >= 0 && id[k] < nr) ? rank[rb + id[k]] : -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t p = base + k * LI_THREADS;
            if (p >= e) continue;
            if (v[k] < 0) {
                record_error(st, PMRF_ERR_ARG, SITE_BAD_ID, p);
                out[p] = 0;
            } else {
                out[p] = labels[v[k]];
            }
        }
    }
    (void)maxid1;
}

// tile table: vertex tiles then hood tiles, each grouped by slice; one warp
// per hood tile.  Hood tile j of a slice holds its hoods [j te, (j+1) te); the
// largest tile's element count goes to *maxne (the staging buffer's size)
__global__ void k_make_hood_tiles(const int64_t* __restrict__ hood_off, const int64_t* __restrict__ hood_slice_off,
                                  const uint8_t* __restrict__ hood_gen, const int64_t* __restrict__ ht_first,
                                  int32_t S, int64_t n_htiles, int32_t te, Tile* __restrict__ tiles,
                                  int64_t tile_base, unsigned long long* __restrict__ maxne) {
    __shared__ unsigned long long s_ne[8];
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (lane == 0) s_ne[warp_id()] = 0;
    // the block's largest tile goes out in one atomic (atomics on one word serialise)
    auto block_max = [&]() {
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = 0;
            for (int w = 0; w < 8; ++w) m = max(m, s_ne[w]);
            if (m) atomicMax(maxne, m);
        }
    };
    if (k >= n_htiles) {  // whole warps
        block_max();
        return;
    }
    const int s = (int)(upper_bound_dev<int64_t>(ht_first, 0, S + 1, k) - 1);
    const int64_t j = k - ht_first[s];
    const int64_t cs = hood_slice_off[s], ce = hood_slice_off[s + 1];
    const int64_t c0 = cs + j * te, c1 = min(ce, c0 + te);
    // fast when every element's vertex has degree <= 32 (the build flags the
    // hoods that do not)
    bool ok = true;
    for (int64_t c = c0 + lane; c < c1; c += 32) ok = ok && hood_gen[c] == 0;
    const bool fast = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
        Tile t;
        t.kind = 0;
        t.slice = s;
        t.a0 = (int32_t)c0;
        t.a1 = (int32_t)c1;
        t.part = (int32_t)k;
        t.pad = fast ? 1 : 0;
        tiles[tile_base + k] = t;
        s_ne[warp_id()] = (unsigned long long)(hood_off[c1] - hood_off[c0]);
    }
    block_max();
}

__global__ void k_make_vert_tiles(const int64_t* __restrict__ vert_off, const int64_t* __restrict__ vt_first,
                                  int32_t S, int64_t n_vtiles, int32_t vt, Tile* __restrict__ tiles) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_vtiles) return;
    const int s = (int)(upper_bound_dev<int64_t>(vt_first, 0, S + 1, k) - 1);
    const int64_t j = k - vt_first[s];
    Tile t;
    t.kind = 1;
    t.slice = s;
    t.a0 = (int32_t)(vert_off[s] + j * vt);
    t.a1 = (int32_t)min(vert_off[s + 1], vert_off[s] + (j + 1) * vt);
    t.part = (int32_t)k;
    t.pad = 0;
    tiles[k] = t;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side

int free_plans(pmrf_graph* g) {
    for (auto& kv : g->plans) {
        Plan& p = kv.second;
        dfree(p.d_tiles, 0);
        dfree(p.d_slice_ntiles, 0);
        dfree(p.d_slice_vt0, 0);
        dfree(p.d_slice_ht0, 0);
    }
    g->plans.clear();
    for (auto& e : g->execs)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    g->execs.clear();
    return PMRF_OK;
}

int free_em(pmrf_graph* g) {
    EMWork& w = g->em;
    void* ps[] = {w.d_x[0], w.d_x[1], w.d_hist, w.d_qhist, w.d_unit, w.d_yr, w.d_vpart, w.d_hpart, w.d_theta,
                  w.d_dterm, w.d_Thist, w.d_vrec,
                  w.d_active, w.d_iters, w.d_conv, w.d_nactive, w.d_t, w.d_sched, w.d_cfg};
    for (void* p : ps)
        if (p) cudaFreeAsync(p, 0);
    g->em = EMWork();
    for (auto& e : g->execs)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    g->execs.clear();
    return PMRF_OK;
}

namespace {

// The default hood tile and lanes per hood: one lane per hood (two for a mean
// hood size m of 16 or more, as in k-neighbourhoods) and as many hoods as the
// block has lane groups, so that every lane takes one hood in one round (128
// hoods, about 1570 elements, for the 1-neighbourhoods of a jittered-grid
// oversegmentation, m = 12.3)
int default_hood_lanes(const pmrf_graph* g) {
    const double m = g->C > 0 ? (double)g->N_el / (double)g->C : 1.0;
    return m >= 16.0 ? 2 : 1;
}

int default_hood_tile(int lanes) { return std::max(MIN_HOOD_TILE, HT_THREADS / lanes); }

// The autotuner's results for this process, keyed by the graph's shape
// (slices, regions, hood elements) and the number of labels: a graph whose
// tuning is left at 0 takes the entry of its shape when there is one
using TuneKey = std::array<int64_t, 4>;
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;

TuneKey tune_key(const pmrf_graph* g, int L) { return TuneKey{(int64_t)g->S, g->V, g->N_el, (int64_t)L}; }

int effective_tiles(const pmrf_graph* g, int L, int* te, int* lanes) {
    int ct = 0, cl = 0;
    if (g->tuning.hood_tile == 0 && g->tuning.hood_lanes == 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(tune_key(g, L));
        if (it != g_tune_cache.end()) {
            ct = it->second.first;
            cl = it->second.second;
        }
    }
    *lanes = g->tuning.hood_lanes > 0 ? g->tuning.hood_lanes : (cl > 0 ? cl : default_hood_lanes(g));
    *te = g->tuning.hood_tile > 0 ? g->tuning.hood_tile : (ct > 0 ? ct : default_hood_tile(*lanes));
    return PMRF_OK;
}

// elements a fast hood tile stages: the largest tile's (up to HT_CAP_MAX;
// larger tiles read their stream in place)
int hood_cap(const Plan* p) { return p->cap; }
size_t hood_smem(const Plan* p) { return sizeof(uint2) * (size_t)(hood_cap(p) + 2); }

int get_plan(pmrf_graph* g, int L, cudaStream_t s, Plan** out) {
    int te, lanes;
    effective_tiles(g, L, &te, &lanes);
    auto key = std::make_pair(te, lanes);
    auto it = g->plans.find(key);
    if (it != g->plans.end()) {
        *out = &it->second;
        return PMRF_OK;
    }
    const int32_t S = g->S;
    const int vt = VT_THREADS;  // one vertex per thread
    Plan p;
    p.hood_tile = te;
    p.hood_lanes = lanes;
    p.max_hood = g->max_hood;
    // the hood pass bulk-copies the element stream from 16-byte boundaries
    if (reinterpret_cast<uintptr_t>(g->d_el) & 15) return fail(PMRF_ERR_CUDA, "element stream is not 16-byte aligned");
    std::vector<int64_t> vfirst(S + 1, 0), hfirst(S + 1, 0);
    for (int i = 0; i < S; ++i) {
        const int64_t nv = g->h_vert_off[i + 1] - g->h_vert_off[i];
        const int64_t ne = g->h_el_slice_off[i + 1] - g->h_el_slice_off[i];
        const int64_t nh = g->h_hood_slice_off[i + 1] - g->h_hood_slice_off[i];
        vfirst[i + 1] = vfirst[i] + ceil_div(nv, vt);
        hfirst[i + 1] = hfirst[i] + ceil_div(nh, te);
        (void)ne;
    }
    p.n_vtiles = vfirst[S];
    p.n_htiles = hfirst[S];
    p.n_tiles = p.n_vtiles + p.n_htiles;
    if (p.n_tiles >= 2147483647ll) return fail(PMRF_ERR_UNSUPPORTED, "too many tiles");
    int ra = dalloc(&p.d_tiles, p.n_tiles, s);
    if (!ra) ra = dalloc(&p.d_slice_vt0, S + 1, s);
    if (!ra) ra = dalloc(&p.d_slice_ht0, S + 1, s);
    if (ra) {
        dfree(p.d_tiles, s);
        dfree(p.d_slice_vt0, s);
        dfree(p.d_slice_ht0, s);
        return ra;
    }
    PMRF_CUDA(cudaMemcpyAsync(p.d_slice_vt0, vfirst.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice, s));
    PMRF_CUDA(cudaMemcpyAsync(p.d_slice_ht0, hfirst.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice, s));
    if (p.n_vtiles > 0) {
        k_make_vert_tiles<<<(unsigned)ceil_div(p.n_vtiles, 256), 256, 0, s>>>(g->d_vert_off, p.d_slice_vt0, S,
                                                                              p.n_vtiles, vt, p.d_tiles);
        ::pmrf::note_launch(1);
    }
    unsigned long long maxne = 0;
    if (p.n_htiles > 0) {
        unsigned long long* d_maxne = nullptr;
        PMRF_TRY(dalloc(&d_maxne, 1, s));
        PMRF_CUDA(cudaMemsetAsync(d_maxne, 0, sizeof(unsigned long long), s));
        k_make_hood_tiles<<<(unsigned)ceil_div(p.n_htiles, 8), 256, 0, s>>>(
            g->d_hood_off, g->d_hood_slice_off, g->d_hood_gen, p.d_slice_ht0, S, p.n_htiles,
            te, p.d_tiles,
            p.n_vtiles, d_maxne);
        ::pmrf::note_launch(1);
        PMRF_CUDA(cudaMemcpyAsync(&maxne, d_maxne, sizeof(maxne), cudaMemcpyDeviceToHost, s));
        dfree(d_maxne, s);
    }
    PMRF_CUDA(cudaGetLastError());
    PMRF_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
    p.cap = (int)std::min<unsigned long long>(HT_CAP_MAX, std::max<unsigned long long>(maxne, 1));
    auto res = g->plans.emplace(key, p);
    *out = &res.first->second;
    return PMRF_OK;
}

int check_cfg(const pmrf_graph* g, const pmrf_config* cfg) {
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    if (!cfg) return fail(PMRF_ERR_ARG, "config is NULL");
    if (cfg->n_labels < 1 || cfg->n_labels > PMRF_MAX_LABELS) return fail(PMRF_ERR_ARG, "n_labels must be in [1, 8]");
    // beta < 2^32 keeps a fast hood's excess sum (<= 128 * 32 beta, units
    // 2^-80) inside 128 bits
    if (!(cfg->beta >= 0.0) || !(cfg->beta < 0x1p32)) return fail(PMRF_ERR_ARG, "beta must be in [0, 2^32)");
    if (!(cfg->sigma_min > 0.0)) return fail(PMRF_ERR_ARG, "sigma_min must be > 0");
    if (!(cfg->init_hi > cfg->init_lo)) return fail(PMRF_ERR_ARG, "init_hi must exceed init_lo");
    if (cfg->conv_window < 1) return fail(PMRF_ERR_ARG, "conv_window must be >= 1");
    if (cfg->max_iters < 1) return fail(PMRF_ERR_ARG, "max_iters must be >= 1");
    if (cfg->init_from_labels < 0 || cfg->init_from_labels > 2) return fail(PMRF_ERR_ARG, "init_from_labels must be 0, 1 or 2");
    if (cfg->potts_scope != PMRF_SCOPE_HOOD && cfg->potts_scope != PMRF_SCOPE_FULL)
        return fail(PMRF_ERR_ARG, "potts_scope must be PMRF_SCOPE_HOOD or PMRF_SCOPE_FULL");
    if (cfg->replica_rule < PMRF_RULE_MIN || cfg->replica_rule > PMRF_RULE_VOTE)
        return fail(PMRF_ERR_ARG, "replica_rule must be PMRF_RULE_MIN, PMRF_RULE_SUM or PMRF_RULE_VOTE");
    return PMRF_OK;
}

// a sweep variant other than the default (hood scope, least-energy replica)
bool is_variant(const RunCfg& r) { return r.scope != PMRF_SCOPE_HOOD || r.rule != PMRF_RULE_MIN; }

RunCfg to_run(const pmrf_config* c) {
    RunCfg r;
    r.L = c->n_labels;
    r.W = c->conv_window;
    r.max_iters = c->max_iters;
    r.init_from_labels = c->init_from_labels;
    r.beta = c->beta;
    r.tol = c->conv_tol;
    r.sigma_min = c->sigma_min;
    r.init_lo = c->init_lo;
    r.init_hi = c->init_hi;
    r.scope = c->potts_scope;
    r.rule = c->replica_rule;
    return r;
}


// (re)allocate the EM workspace for (L, W, max_iters, plan)
int ensure_work(pmrf_graph* g, const RunCfg& rc, const Plan& p, cudaStream_t s) {
    EMWork& w = g->em;
    if (w.d_x[0] && w.L == rc.L && w.W == rc.W && w.max_iters >= rc.max_iters && w.n_vtiles == p.n_vtiles &&
        w.n_htiles == p.n_htiles)
        return PMRF_OK;
    if (w.d_x[0]) PMRF_CUDA(cudaDeviceSynchronize());  // the old workspace may be in use on any stream
    free_em(g);
    const int64_t S = g->S;
    w.L = rc.L;
    w.W = rc.W;
    w.max_iters = rc.max_iters;
    w.n_vtiles = p.n_vtiles;
    w.n_htiles = p.n_htiles;
    int rc2 = PMRF_OK;
    if (!rc2) rc2 = dalloc(&w.d_x[0], g->V, s);
    if (!rc2) rc2 = dalloc(&w.d_x[1], g->V, s);
    if (!rc2) rc2 = dalloc(&w.d_hist, (int64_t)rc.W * g->C, s);
    if (!rc2) rc2 = dalloc(&w.d_vpart, p.n_vtiles * 4 * rc.L, s);
    if (!rc2) rc2 = dalloc(&w.d_hpart, p.n_htiles * 3, s);
    if (!rc2) rc2 = dalloc(&w.d_theta, S * rc.L * 4, s);
    if (!rc2) rc2 = dalloc(&w.d_dterm, S * rc.L * 2, s);
    if (!rc2) rc2 = dalloc(&w.d_Thist, S * rc.W, s);
    if (!rc2) rc2 = dalloc(&w.d_active, S, s);
    if (!rc2) rc2 = dalloc(&w.d_iters, S, s);
    if (!rc2) rc2 = dalloc(&w.d_conv, S, s);
    if (!rc2) rc2 = dalloc(&w.d_nactive, 1, s);
    if (!rc2) rc2 = dalloc(&w.d_t, 1, s);
    if (!rc2) rc2 = dalloc(&w.d_sched, 2 * (S + 1) + 2, s);
    if (!rc2) rc2 = dalloc(&w.d_qhist, S * rc.W, s);
    if (!rc2) rc2 = dalloc((char**)&w.d_unit, (int64_t)sizeof(SliceUnit) * std::max<int64_t>(S, 1), s);
    if (!rc2) rc2 = dalloc(&w.d_yr, 2 * S, s);
    if (!rc2 && S > 0) {
        k_yrange<<<(unsigned)S, FIN_THREADS, 0, s>>>(g->d_vert_off, g->d_y, w.d_yr);
        ::pmrf::note_launch(1);
    }
    if (!rc2) rc2 = dalloc(&w.d_vrec, g->V * vrec_words(rc.L), s);  // hood-pass vertex records
    if (!rc2 && (reinterpret_cast<uintptr_t>(w.d_vrec) & 31))  // read and written 32 bytes at a time
        rc2 = fail(PMRF_ERR_CUDA, "vertex record table is not 32-byte aligned");
    if (!rc2) rc2 = dalloc((char**)&w.d_cfg, (int64_t)(sizeof(RunCfg) + sizeof(OutPtrs)), s);
    if (rc2) free_em(g);
    return rc2;
}

struct Launch {
    pmrf_graph* g;
    Plan* p;
    DevGraph dg;
    const Tile* vt;
    const Tile* ht;
    RunCfg* d_cfg;
    OutPtrs* d_out;
};

}  // namespace

// Internal entry points used by api.cu ------------------------------------------------

namespace {

__global__ void k_set_i32(int32_t* p, int32_t v) { *p = v; }

// The condition setter of the loop graph's two WHILE loops, run after the INIT
// pass (t0 = 0), at the end of each iteration and between the loops (t0 < 0:
// t = *tp, the iteration just run).  It lists the tiles of the slices still
// iterating (the cum arrays of TileSched: vertex and hood tiles) and zeroes the
// passes' tile counters for the next iteration, then lets iteration t + 1 run
// while a slice is still active and t < max_iters; in the dense loop
// (dense_only) only while the listed tiles are at least a quarter of the table.
// It stores the next iteration in *tp (t when none runs) and adds the kernels
// the body will run to the device-side launch counter.  One block of
// NX_THREADS.
constexpr int NX_THREADS = 1024;

__global__ void __launch_bounds__(NX_THREADS) k_next_iter(cudaGraphConditionalHandle h, int dense_only,
                                                          const int32_t* __restrict__ nactive,
                                                          int32_t* __restrict__ tp, int t0, int max_iters,
                                                          unsigned long long* __restrict__ counter,
                                                          unsigned int body_kernels, int32_t S,
                                                          const int32_t* __restrict__ active,
                                                          const int64_t* __restrict__ vt0,
                                                          const int64_t* __restrict__ ht0,
                                                          int32_t* __restrict__ sched, int64_t n_tiles) {
    __shared__ int2 s_w[NX_THREADS / 32];
    __shared__ int2 s_carry;
    int32_t* const vcum = sched;
    int32_t* const hcum = sched + (S + 1);
    if (threadIdx.x == 0) s_carry = make_int2(0, 0);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < S; base += NX_THREADS) {
        const int i = base + threadIdx.x;
        int2 n = make_int2(0, 0);
        if (i < S && active[i]) n = make_int2((int)(vt0[i + 1] - vt0[i]), (int)(ht0[i + 1] - ht0[i]));
        // inclusive scan within the warp, then over the warps
        int2 x = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int yv = __shfl_up_sync(0xffffffffu, x.x, o), yh = __shfl_up_sync(0xffffffffu, x.y, o);
            if (lane >= o) {
                x.x += yv;
                x.y += yh;
            }
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        int2 off = s_carry;
        for (int w = 0; w < warp; ++w) {
            off.x += s_w[w].x;
            off.y += s_w[w].y;
        }
        if (i < S) {
            vcum[i] = off.x + x.x - n.x;
            hcum[i] = off.y + x.y - n.y;
        }
        __syncthreads();  // every thread has read s_carry and s_w
        if (threadIdx.x == NX_THREADS - 1) s_carry = make_int2(off.x + x.x, off.y + x.y);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        vcum[S] = s_carry.x;
        hcum[S] = s_carry.y;
        sched[2 * (S + 1)] = 0;      // vertex-pass tile counter
        sched[2 * (S + 1) + 1] = 0;  // hood-pass tile counter
        const int t = t0 >= 0 ? t0 : *tp;
        const bool dense = 4 * ((int64_t)s_carry.x + s_carry.y) >= n_tiles;
        const unsigned int run = (*nactive > 0 && t < max_iters && (dense || !dense_only)) ? 1u : 0u;
        *tp = run ? t + 1 : t;
        if (run) atomicAdd(counter, (unsigned long long)body_kernels);
        cudaGraphSetConditional(h, run);
    }
}

// the schedules of an EM iteration's passes (TileSched)
TileSched vertex_sched(const EMWork& w, const Plan* p, int32_t S) {
    return TileSched{w.d_sched, p->d_slice_vt0, w.d_sched + 2 * (S + 1), S};
}
TileSched hood_sched(const EMWork& w, const Plan* p, int32_t S) {
    return TileSched{w.d_sched + (S + 1), p->d_slice_ht0, w.d_sched + 2 * (S + 1) + 1, S};
}

// blocks of a pass that takes listed tiles: one per resident slot of the
// device (fewer when the table has fewer tiles)
unsigned sched_grid(const void* fn, int threads, size_t smem, int64_t n_tiles) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    const int64_t slots = (int64_t)std::max(sms, 1) * std::max(per_sm, 1);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(n_tiles, slots));
}

// state of a capture that runs the EM iterations as the bodies of two
// conditional WHILE nodes in sequence (dense loop, sparse loop)
struct CondCapture {
    cudaStream_t body_stream = nullptr;      // captures a body
    unsigned long long* counter = nullptr;   // device-side launch counter
    cudaGraphConditionalHandle h[2] = {0, 0};  // the loops' conditions
    int64_t* parent_nodes = nullptr;         // kernels outside the body
    int64_t body_nodes = 0;                  // counted on the device instead
};
__global__ void k_set_active_all(int32_t* a, int32_t S) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S) a[i] = 1;
}

// kernels one EM iteration body launches (its condition setter included)
int iter_kernels(const Plan* p) { return (p->n_vtiles > 0) + (p->n_htiles > 0) + 2; }

// open a WHILE node with condition h on the capturing stream s and start
// capturing its body on cc->body_stream
int open_while_body(CondCapture* cc, cudaStream_t s, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t pg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    PMRF_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &pg, &deps, &ed, &nd));
    if (st != cudaStreamCaptureStatusActive) return fail(PMRF_ERR_CUDA, "EM capture is not active");
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    std::memset(&np, 0, sizeof(np));  // reserved fields must be zero
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    PMRF_CUDA(cudaGraphAddNode(&node, pg, deps, ed, nd, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    PMRF_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    PMRF_CUDA(cudaStreamBeginCaptureToGraph(cc->body_stream, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
    return PMRF_OK;
}

// with cc set (graph capture on s) the iterations are the body of one WHILE
// node that runs while a slice is active (a graph of a few nodes, quick to
// instantiate and to release); without it the loop is unrolled
template <int L>
int em_body(pmrf_graph* g, Plan* p, const RunCfg& rc, cudaStream_t s, bool init_from_labels,
            CondCapture* cc = nullptr) {
    EMWork& w = g->em;
    Launch z{g, p, view(g), p->d_tiles + 0, p->d_tiles + p->n_vtiles, (RunCfg*)w.d_cfg,
             (OutPtrs*)((char*)w.d_cfg + sizeof(RunCfg))};
    const int32_t S = g->S;
    // every slice active for INIT; nactive = S
    k_set_active_all<<<(unsigned)ceil_div(S, 256), 256, 0, s>>>(w.d_active, S); ::pmrf::note_launch(1);
    k_set_i32<<<1, 1, 0, s>>>(w.d_nactive, S); ::pmrf::note_launch(1);
    (void)init_from_labels;  // the INIT pass reads buffer 1, which em_run fills from the caller
    k_zero_T<<<64, 256, 0, s>>>(z.d_out, (int64_t)S * rc.max_iters); ::pmrf::note_launch(1);
    if (p->n_vtiles > 0) {
        k_vertex<L, false><<<(unsigned)p->n_vtiles, VT_THREADS, 0, s>>>(z.dg, z.vt, MODE_INIT, z.d_cfg, nullptr,
                                                                w.d_x[1], w.d_x[0], nullptr, nullptr, nullptr,
                                                                nullptr, w.d_vpart, g->d_status, nullptr, nullptr,
                                                                nullptr, TileSched{});
        ::pmrf::note_launch(1);
    }
    SliceUnit* unit = (SliceUnit*)w.d_unit;
    k_finalize<L><<<(unsigned)S, FIN_THREADS, 0, s>>>(S, MODE_INIT, 0, z.d_cfg, p->d_slice_vt0, p->d_slice_ht0, w.d_vpart,
                                            w.d_hpart, nullptr, w.d_theta, g->d_vert_off, w.d_active, w.d_iters,
                                            w.d_conv, w.d_Thist, w.d_nactive, z.d_out, w.d_dterm, unit, w.d_qhist,
                                            w.d_yr, g->max_deg, g->max_hood, g->d_status, nullptr);
    ::pmrf::note_launch(1);
    const auto kv = is_variant(rc) ? &k_vertex<L, true> : &k_vertex<L, false>;
    const auto kvl = is_variant(rc) ? &k_vertex<L, true, true> : &k_vertex<L, false, true>;
    if (cc) {
        // two WHILE nodes in sequence, each body one iteration; the kernels
        // read t from w.d_t, which the condition setter at the end of each
        // body advances.  The dense loop launches one block per tile of the
        // table (blocks of stopped slices return at once) while at least a
        // quarter of the tiles belong to slices still iterating; the sparse
        // loop runs the remaining iterations with one block per resident slot,
        // the blocks taking only those tiles.  Slices only ever stop, so the
        // sparse loop never has to hand back.
        const unsigned body = (unsigned)iter_kernels(p);
        const unsigned gv = sched_grid((const void*)kvl, VT_THREADS, 0, p->n_vtiles);
        const unsigned gh = sched_grid((const void*)&k_hood<L, true>, HT_THREADS, hood_smem(p), p->n_htiles);
        const cudaStream_t s0 = s;
        for (int sparse = 0; sparse < 2; ++sparse) {
            const cudaGraphConditionalHandle h = cc->h[sparse];
            auto next_iter = [&](cudaStream_t st, int t0) {
                k_next_iter<<<1, NX_THREADS, 0, st>>>(h, sparse ? 0 : 1, w.d_nactive, w.d_t, t0, rc.max_iters,
                                                      cc->counter, body, S, w.d_active, p->d_slice_vt0,
                                                      p->d_slice_ht0, w.d_sched, p->n_tiles);
                ::pmrf::note_launch(1);
            };
            next_iter(s0, sparse ? -1 : 0);
            PMRF_TRY(open_while_body(cc, s0, h));
            s = cc->body_stream;
            set_capture_counter(&cc->body_nodes);
            if (p->n_vtiles > 0) {
                (sparse ? kvl : kv)<<<sparse ? gv : (unsigned)p->n_vtiles, VT_THREADS, 0, s>>>(
                    z.dg, z.vt, MODE_EM, z.d_cfg, w.d_active, w.d_x[0], w.d_x[1], w.d_theta, w.d_dterm, nullptr,
                    nullptr, w.d_vpart, g->d_status, w.d_vrec, unit, w.d_t,
                    sparse ? vertex_sched(w, p, S) : TileSched{});
                ::pmrf::note_launch(1);
            }
            if (p->n_htiles > 0) {
                (sparse ? &k_hood<L, true> : &k_hood<L>)<<<sparse ? gh : (unsigned)p->n_htiles, HT_THREADS,
                                                           hood_smem(p), s>>>(
                    z.dg, z.ht, MODE_EM, 0, p->hood_lanes, z.d_cfg, w.d_active, w.d_x[0], w.d_vrec, unit,
                    w.d_qhist, w.d_hist, nullptr, w.d_hpart, hood_cap(p), g->d_status, w.d_x[1], w.d_t,
                    sparse ? hood_sched(w, p, S) : TileSched{});
                ::pmrf::note_launch(1);
            }
            k_finalize<L><<<(unsigned)S, FIN_THREADS, 0, s>>>(S, MODE_EM, 0, z.d_cfg, p->d_slice_vt0,
                                                              p->d_slice_ht0, w.d_vpart, w.d_hpart, w.d_theta,
                                                              w.d_theta, g->d_vert_off, w.d_active, w.d_iters,
                                                              w.d_conv, w.d_Thist, w.d_nactive, z.d_out, w.d_dterm,
                                                              unit, w.d_qhist, w.d_yr, g->max_deg, g->max_hood,
                                                              g->d_status, w.d_t);
            ::pmrf::note_launch(1);
            next_iter(s, -1);
            PMRF_CUDA(cudaGetLastError());
            cudaGraph_t bg = nullptr;
            PMRF_CUDA(cudaStreamEndCapture(s, &bg));
            s = s0;
            set_capture_counter(cc->parent_nodes);
        }
    } else {
        const bool prof = g->tuning.profile != 0 && (int)g->prof_ev.size() >= 3 * rc.max_iters;
        // the host does not see which slices are still iterating: every
        // iteration launches one block per tile of the table
        for (int t = 1; t <= rc.max_iters; ++t) {
            const uint8_t* xin = w.d_x[(t - 1) & 1];
            uint8_t* xout = w.d_x[t & 1];
            if (prof) cudaEventRecordWithFlags(g->prof_ev[3 * (t - 1) + 0], s, cudaEventRecordExternal);
            if (p->n_vtiles > 0) {
                kv<<<(unsigned)p->n_vtiles, VT_THREADS, 0, s>>>(z.dg, z.vt, MODE_EM, z.d_cfg, w.d_active, xin,
                                                                xout, w.d_theta, w.d_dterm, nullptr, nullptr,
                                                                w.d_vpart, g->d_status, w.d_vrec, unit, nullptr,
                                                                TileSched{});
                ::pmrf::note_launch(1);
            }
            if (prof) cudaEventRecordWithFlags(g->prof_ev[3 * (t - 1) + 1], s, cudaEventRecordExternal);
            if (p->n_htiles > 0) {
                k_hood<L><<<(unsigned)p->n_htiles, HT_THREADS, hood_smem(p), s>>>(
                    z.dg, z.ht, MODE_EM, t, p->hood_lanes, z.d_cfg, w.d_active, xin, w.d_vrec, unit, w.d_qhist,
                    w.d_hist, nullptr, w.d_hpart, hood_cap(p), g->d_status, nullptr, nullptr, TileSched{});
                ::pmrf::note_launch(1);
            }
            if (prof) cudaEventRecordWithFlags(g->prof_ev[3 * (t - 1) + 2], s, cudaEventRecordExternal);
            k_finalize<L><<<(unsigned)S, FIN_THREADS, 0, s>>>(S, MODE_EM, t, z.d_cfg, p->d_slice_vt0, p->d_slice_ht0,
                                                              w.d_vpart, w.d_hpart, w.d_theta, w.d_theta,
                                                              g->d_vert_off, w.d_active, w.d_iters, w.d_conv,
                                                              w.d_Thist, w.d_nactive, z.d_out, w.d_dterm, unit,
                                                              w.d_qhist, w.d_yr, g->max_deg, g->max_hood,
                                                              g->d_status, nullptr);
            ::pmrf::note_launch(1);
        }
    }
    k_close<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g->V, 256), 4096)), 256, 0, s>>>(
        z.dg, rc.L, w.d_x[0], w.d_x[1], w.d_iters, w.d_conv, w.d_theta, z.d_out); ::pmrf::note_launch(1);
    return PMRF_OK;
}

}  // namespace

// capture the whole EM loop into an executable graph; *nodes = the kernels
// the capture launched outside conditional bodies
int capture_em(pmrf_graph* g, Plan* p, const RunCfg& rc, bool init_from_labels, bool conditional,
               cudaGraphExec_t* exec_out, int64_t* nodes) {
    *exec_out = nullptr;
    *nodes = 0;
    CondCapture cc;
    cc.parent_nodes = nodes;
    if (conditional) {
        cc.counter = device_launch_counter();
        if (!cc.counter) return fail(PMRF_ERR_UNSUPPORTED, "no device launch counter");
    }
    cudaStream_t cs = nullptr;
    PMRF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (conditional) {
        cudaError_t e = cudaStreamCreateWithFlags(&cc.body_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            return cuda_fail(e, "body stream");
        }
    }
    cudaGraph_t graph = nullptr;
    int r = PMRF_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess && conditional) {
        cudaStreamCaptureStatus st;
        cudaGraph_t pg = nullptr;
        e = cudaStreamGetCaptureInfo(cs, &st, nullptr, &pg);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k)
            e = cudaGraphConditionalHandleCreate(&cc.h[k], pg, 0, cudaGraphCondAssignDefault);
    }
    if (e == cudaSuccess) {
        set_capture_counter(nodes);
        CondCapture* c = conditional ? &cc : nullptr;
        switch (rc.L) {
            case 1: r = em_body<1>(g, p, rc, cs, init_from_labels, c); break;
            case 2: r = em_body<2>(g, p, rc, cs, init_from_labels, c); break;
            case 3: r = em_body<3>(g, p, rc, cs, init_from_labels, c); break;
            case 4: r = em_body<4>(g, p, rc, cs, init_from_labels, c); break;
            case 5: r = em_body<5>(g, p, rc, cs, init_from_labels, c); break;
            case 6: r = em_body<6>(g, p, rc, cs, init_from_labels, c); break;
            case 7: r = em_body<7>(g, p, rc, cs, init_from_labels, c); break;
            default: r = em_body<8>(g, p, rc, cs, init_from_labels, c); break;
        }
        set_capture_counter(nullptr);
    }
    if (cc.body_stream) {  // a body capture left open by an error
        cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(cc.body_stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(cc.body_stream, &tmp);
        }
    }
    {
        cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(cs, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess) e = e2;
        }
    }
    if (e == cudaSuccess && r == PMRF_OK) e = cudaGraphInstantiate(exec_out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (cc.body_stream) cudaStreamDestroy(cc.body_stream);
    cudaStreamDestroy(cs);
    if (r == PMRF_OK && e != cudaSuccess) r = cuda_fail(e, "EM graph capture");
    if (r != PMRF_OK && *exec_out) {
        cudaGraphExecDestroy(*exec_out);
        *exec_out = nullptr;
    }
    return r;
}

// labels and T history destinations are passed through OutPtrs so a cached
// CUDA graph can serve any caller buffers
int em_run(pmrf_graph* g, const pmrf_config* cfg, uint8_t* d_labels, double* d_params, int32_t* d_iters,
           int32_t* d_conv, double* d_T_hist, cudaStream_t s) {
    PMRF_TRY(check_cfg(g, cfg));
    if (!d_labels || !d_params || !d_iters || !d_conv) return fail(PMRF_ERR_ARG, "null output pointer");
    const RunCfg rc = to_run(cfg);
    Plan* p = nullptr;
    PMRF_TRY(get_plan(g, rc.L, s, &p));
    PMRF_TRY(ensure_work(g, rc, *p, s));
    EMWork& w = g->em;
    // constants and output pointers for this call
    struct {
        RunCfg r;
        OutPtrs o;
    } h;
    h.r = rc;
    h.o.labels = d_labels;
    h.o.params = d_params;
    h.o.iters = d_iters;
    h.o.conv = d_conv;
    h.o.thist = d_T_hist;
    PMRF_CUDA(cudaMemcpyAsync(w.d_cfg, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    if (cfg->init_from_labels) {
        // the INIT pass reads x_in = buffer 1
        PMRF_CUDA(cudaMemcpyAsync(w.d_x[1], d_labels, (size_t)g->V, cudaMemcpyDeviceToDevice, s));
    }
    if (cfg->init_from_labels == 2) {
        // the finaliser's INIT step keeps these (sigma floored)
        PMRF_CUDA(cudaMemcpyAsync(w.d_theta, d_params, sizeof(double) * (size_t)g->S * rc.L * 4,
                                  cudaMemcpyDeviceToDevice, s));
    }
    if (g->tuning.profile) {
        while ((int)g->prof_ev.size() < 3 * rc.max_iters) {
            cudaEvent_t ev;
            PMRF_CUDA(cudaEventCreate(&ev));
            g->prof_ev.push_back(ev);
        }
        g->prof_iters = rc.max_iters;
    } else {
        g->prof_iters = 0;
    }
    const bool use_graph = g->tuning.use_cuda_graph != 0;
    if (!use_graph) {
        int r = PMRF_OK;
        switch (rc.L) {
            case 1: r = em_body<1>(g, p, rc, s, cfg->init_from_labels); break;
            case 2: r = em_body<2>(g, p, rc, s, cfg->init_from_labels); break;
            case 3: r = em_body<3>(g, p, rc, s, cfg->init_from_labels); break;
            case 4: r = em_body<4>(g, p, rc, s, cfg->init_from_labels); break;
            case 5: r = em_body<5>(g, p, rc, s, cfg->init_from_labels); break;
            case 6: r = em_body<6>(g, p, rc, s, cfg->init_from_labels); break;
            case 7: r = em_body<7>(g, p, rc, s, cfg->init_from_labels); break;
            default: r = em_body<8>(g, p, rc, s, cfg->init_from_labels); break;
        }
        PMRF_CUDA(cudaGetLastError());
        return r;
    }
    // find or capture the CUDA graph of the whole loop
    pmrf_graph::CachedExec* ce = nullptr;
    for (auto& e : g->execs)
        if (e.L == rc.L && e.W == rc.W && e.max_iters == rc.max_iters && e.hood_tile == p->hood_tile &&
            e.hood_lanes == p->hood_lanes && e.var == (int)is_variant(rc))
            ce = &e;
    if (!ce) {
        int64_t nodes = 0;
        cudaGraphExec_t exec = nullptr;
        // conditional iteration bodies first (not with profiling: event
        // records may not sit inside a conditional body), else the unrolled loop
        int r = PMRF_ERR_UNSUPPORTED;
        if (!g->tuning.profile) r = capture_em(g, p, rc, cfg->init_from_labels, true, &exec, &nodes);
        if (r != PMRF_OK) {
            cudaGetLastError();
            r = capture_em(g, p, rc, cfg->init_from_labels, false, &exec, &nodes);
        }
        if (r != PMRF_OK) return r;
        pmrf_graph::CachedExec c;
        c.exec = exec;
        c.L = rc.L;
        c.W = rc.W;
        c.max_iters = rc.max_iters;
        c.hood_tile = p->hood_tile;
        c.hood_lanes = p->hood_lanes;
        c.var = (int)is_variant(rc);
        c.nkernels = nodes;
        g->execs.push_back(c);
        ce = &g->execs.back();
    }
    PMRF_CUDA(cudaGraphLaunch(ce->exec, s));
    note_launch(ce->nkernels);
    return PMRF_OK;
}

// ---------------------------------------------------------------------------
// standalone sweep / params / init / label image

namespace {

template <int L>
int sweep_body(pmrf_graph* g, Plan* p, cudaStream_t s, const RunCfg* d_cfg, const uint8_t* xin, const double* theta,
               uint8_t* xout, double* Eout, double* Sout, uint64_t* vrec, bool var) {
    DevGraph dg = view(g);
    const Tile* vt = p->d_tiles;
    const Tile* ht = p->d_tiles + p->n_vtiles;
    EMWork& w = g->em;
    SliceUnit* unit = (SliceUnit*)w.d_unit;
    if (g->S > 0) {
        k_units<<<(unsigned)ceil_div(g->S, 128), 128, 0, s>>>(g->S, L, theta, w.d_yr, d_cfg, g->max_deg, g->max_hood,
                                                             unit, g->d_status);
        ::pmrf::note_launch(1);
    }
    if (p->n_vtiles > 0) {
        const auto kv = var ? &k_vertex<L, true> : &k_vertex<L, false>;
        kv<<<(unsigned)p->n_vtiles, VT_THREADS, 0, s>>>(dg, vt, MODE_SWEEP, d_cfg, nullptr, xin, xout, theta,
                                                                nullptr, nullptr, Eout, nullptr, g->d_status, vrec,
                                                                unit, nullptr, TileSched{});
        ::pmrf::note_launch(1);
    }
    if (p->n_htiles > 0) {
        k_hood<L><<<(unsigned)p->n_htiles, HT_THREADS, hood_smem(p), s>>>(
            dg, ht, MODE_SWEEP, 1, p->hood_lanes, d_cfg, nullptr, xin, vrec, unit, nullptr, nullptr, Sout, nullptr,
            hood_cap(p), g->d_status, nullptr, nullptr, TileSched{});
        ::pmrf::note_launch(1);
    }
    PMRF_CUDA(cudaGetLastError());
    return PMRF_OK;
}

template <int L>
int params_body(pmrf_graph* g, Plan* p, cudaStream_t s, const RunCfg* d_cfg, const uint8_t* x, const double* Ein,
                const double* prev, double* out) {
    DevGraph dg = view(g);
    EMWork& w = g->em;
    if (p->n_vtiles > 0) {
        k_vertex<L, false><<<(unsigned)p->n_vtiles, VT_THREADS, 0, s>>>(dg, p->d_tiles, MODE_PARAMS, d_cfg, nullptr, x,
                                                                nullptr, prev, nullptr, Ein, nullptr, w.d_vpart,
                                                                g->d_status, nullptr, nullptr, nullptr, TileSched{});
        ::pmrf::note_launch(1);
    }
    k_finalize<L><<<(unsigned)g->S, FIN_THREADS, 0, s>>>(g->S, MODE_PARAMS, 0, d_cfg, p->d_slice_vt0, p->d_slice_ht0,
                                               w.d_vpart, w.d_hpart, prev, out, g->d_vert_off, nullptr, nullptr,
                                               nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                               nullptr, 0, 0, g->d_status, nullptr);
    ::pmrf::note_launch(1);
    PMRF_CUDA(cudaGetLastError());
    return PMRF_OK;
}

int prepare(pmrf_graph* g, const pmrf_config* cfg, cudaStream_t s, Plan** p, RunCfg* rc) {
    PMRF_TRY(check_cfg(g, cfg));
    *rc = to_run(cfg);
    PMRF_TRY(get_plan(g, rc->L, s, p));
    PMRF_TRY(ensure_work(g, *rc, **p, s));
    return PMRF_OK;
}

#define DISPATCH_L(Lv, call)                     \
    switch (Lv) {                                \
        case 1: { constexpr int L = 1; call; } break; \
        case 2: { constexpr int L = 2; call; } break; \
        case 3: { constexpr int L = 3; call; } break; \
        case 4: { constexpr int L = 4; call; } break; \
        case 5: { constexpr int L = 5; call; } break; \
        case 6: { constexpr int L = 6; call; } break; \
        case 7: { constexpr int L = 7; call; } break; \
        default: { constexpr int L = 8; call; } break; \
    }

}  // namespace

int sweep_run(pmrf_graph* g, const pmrf_config* cfg, const uint8_t* xin, const double* theta, uint8_t* xout,
              double* Eout, double* Sout, cudaStream_t s) {
    if (!xin || !theta || !xout) return fail(PMRF_ERR_ARG, "null pointer");
    if (xin == xout) return fail(PMRF_ERR_ARG, "d_labels_out must not alias d_labels_in");
    Plan* p;
    RunCfg rc;
    PMRF_TRY(prepare(g, cfg, s, &p, &rc));
    EMWork& w = g->em;
    PMRF_CUDA(cudaMemcpyAsync(w.d_cfg, &rc, sizeof(rc), cudaMemcpyHostToDevice, s));
    int r = PMRF_OK;
    DISPATCH_L(rc.L, r = sweep_body<L>(g, p, s, (const RunCfg*)w.d_cfg, xin, theta, xout, Eout, Sout,
                                       w.d_vrec, is_variant(rc)));
    PMRF_CUDA(cudaStreamSynchronize(s));  // the host RunCfg copy is a stack value
    return r;
}

int params_run(pmrf_graph* g, const pmrf_config* cfg, const uint8_t* x, const double* Ein, const double* prev,
               double* out, cudaStream_t s) {
    if (!x || !prev || !out) return fail(PMRF_ERR_ARG, "null pointer");
    Plan* p;
    RunCfg rc;
    PMRF_TRY(prepare(g, cfg, s, &p, &rc));
    EMWork& w = g->em;
    PMRF_CUDA(cudaMemcpyAsync(w.d_cfg, &rc, sizeof(rc), cudaMemcpyHostToDevice, s));
    // out may alias prev: the finaliser reads prev's mu/sigma of a label just
    // before writing that label, in the same thread, so aliasing is safe
    int r = PMRF_OK;
    DISPATCH_L(rc.L, r = params_body<L>(g, p, s, (const RunCfg*)w.d_cfg, x, Ein, prev, out));
    PMRF_CUDA(cudaStreamSynchronize(s));
    return r;
}

int init_labels_run(pmrf_graph* g, const pmrf_config* cfg, uint8_t* x, cudaStream_t s) {
    if (!x) return fail(PMRF_ERR_ARG, "null pointer");
    Plan* p;
    RunCfg rc;
    PMRF_TRY(prepare(g, cfg, s, &p, &rc));
    EMWork& w = g->em;
    PMRF_CUDA(cudaMemcpyAsync(w.d_cfg, &rc, sizeof(rc), cudaMemcpyHostToDevice, s));
    if (g->V > 0) { k_init_labels<<<(unsigned)ceil_div(g->V, 256), 256, 0, s>>>(view(g), (const RunCfg*)w.d_cfg, x); ::pmrf::note_launch(1); }
    PMRF_CUDA(cudaGetLastError());
    PMRF_CUDA(cudaStreamSynchronize(s));
    return PMRF_OK;
}

namespace {

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a counter-based generator:
// the output of the (i+1)-th step from state key
__device__ __forceinline__ uint64_t splitmix64(uint64_t key, uint64_t i) {
    uint64_t z = key + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// labels: vertex v of slice s draws from key_x = splitmix64(seed, 2s)
__global__ void k_random_labels(const int64_t* __restrict__ vert_off, uint64_t seed, int L, uint8_t* __restrict__ x) {
    const int s = blockIdx.y;
    const int64_t v0 = vert_off[s], n = vert_off[s + 1] - v0;
    const uint64_t kx = splitmix64(seed, 2 * (uint64_t)s);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        x[v0 + v] = (uint8_t)(((splitmix64(kx, (uint64_t)v) >> 32) * (uint64_t)L) >> 32);
}

// parameters: label l of slice s draws mu and sigma from key_t = splitmix64(seed, 2s+1)
__global__ void k_random_params(int S, int L, uint64_t seed, double lo, double hi, double* __restrict__ th) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S * L) return;
    const int s = i / L, l = i % L;
    const uint64_t kt = splitmix64(seed, 2 * (uint64_t)s + 1);
    const double w = __dsub_rn(hi, lo);
    const double u0 = (double)(splitmix64(kt, 2 * (uint64_t)l) >> 11) * 0x1p-53;
    const double u1 = (double)(splitmix64(kt, 2 * (uint64_t)l + 1) >> 11) * 0x1p-53;
    double* t = th + (int64_t)i * 4;
    t[0] = 0.0;
    t[1] = __dadd_rn(lo, __dmul_rn(w, u0));  // no contraction: one rounding per operation
    t[2] = __dadd_rn(lo, __dmul_rn(w, u1));
    t[3] = 0.0;
}

}  // namespace

int random_init_run(pmrf_graph* g, int32_t L, uint64_t seed, double lo, double hi, uint8_t* x, double* params,
                    cudaStream_t s) {
    if (!x || !params) return fail(PMRF_ERR_ARG, "null pointer");
    if (L < 1 || L > PMRF_MAX_LABELS) return fail(PMRF_ERR_ARG, "n_labels must be in [1, 8]");
    if (!(hi >= lo) || !std::isfinite(lo) || !std::isfinite(hi)) return fail(PMRF_ERR_ARG, "need finite lo <= hi");
    const int32_t S = g->S;
    if (S == 0) return PMRF_OK;
    int64_t maxv = 0;
    for (int i = 0; i < S; ++i) maxv = std::max(maxv, g->h_vert_off[i + 1] - g->h_vert_off[i]);
    if (maxv > 0) {
        const dim3 grid((unsigned)std::min<int64_t>(ceil_div(maxv, 256), 65535), (unsigned)S);
        k_random_labels<<<grid, 256, 0, s>>>(g->d_vert_off, seed, L, x);
        ::pmrf::note_launch(1);
    }
    k_random_params<<<(unsigned)ceil_div((int64_t)S * L, 128), 128, 0, s>>>(S, L, seed, lo, hi, params);
    ::pmrf::note_launch(1);
    PMRF_CUDA(cudaGetLastError());
    return PMRF_OK;
}

int label_image_run(pmrf_graph* g, const int32_t* ids, const uint8_t* labels, uint8_t* out, cudaStream_t s) {
    if (!ids || !labels || !out) return fail(PMRF_ERR_ARG, "null pointer");
    int64_t maxpix = 0;
    for (int i = 0; i < g->S; ++i) maxpix = std::max(maxpix, g->h_pix_off[i + 1] - g->h_pix_off[i]);
    if (maxpix == 0) return PMRF_OK;
    // 64 rounds of four pixels a thread per block: short blocks cost more to
    // schedule than their loads (1.08 ms with one round on stack512, 0.85 with
    // 8, 0.78 with 64)
    const dim3 grid((unsigned)std::min<int64_t>(ceil_div(maxpix, 256 * LI_THREADS), 65535), (unsigned)g->S);
    k_label_image<<<grid, LI_THREADS, 0, s>>>(ids, g->d_pix_off, g->d_rank_off, g->d_rank, labels, out, nullptr,
                                       g->d_status); ::pmrf::note_launch(1);
    PMRF_CUDA(cudaGetLastError());
    return PMRF_OK;
}

}  // namespace pmrf

// ---------------------------------------------------------------------------
// autotuner: time the EM loop on this graph for a few hood-tile sizes and keep
// the fastest (the vertex tile is one vertex per thread of a 128-thread CTA)

namespace pmrf {

int autotune_run(pmrf_graph* g, const pmrf_config* cfg, cudaStream_t s, pmrf_tuning* best) {
    PMRF_TRY(check_cfg(g, cfg));
    const int64_t S = g->S, L = cfg->n_labels;
    {
        // the candidates' defaults are the plain defaults, not an earlier result
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache.erase(tune_key(g, (int)L));
    }
    uint8_t* lab = nullptr;
    double* par = nullptr;
    int32_t *it = nullptr, *cv = nullptr;
    int rc = dalloc(&lab, g->V, s);
    if (!rc) rc = dalloc(&par, S * L * 4, s);
    if (!rc) rc = dalloc(&it, S, s);
    if (!rc) rc = dalloc(&cv, S, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = fail(PMRF_ERR_CUDA, "event creation failed");
    pmrf_tuning keep = g->tuning, win = g->tuning;
    float best_ms = 1e30f;
    // candidates: the defaults, windows of half and 1.3 times the default, and
    // every lanes-per-hood value at the default window
    pmrf_tuning base = keep;
    base.hood_tile = 0;
    base.hood_lanes = 0;
    g->tuning = base;
    int te0 = 0, ln0 = 0;
    effective_tiles(g, (int)L, &te0, &ln0);
    // the defaults; half and twice as many hoods per tile; each lanes-per-hood
    // value with one hood per lane group
    auto h32 = [](int x) { return std::max(MIN_HOOD_TILE, std::min(MAX_HOOD_TILE, x / 32 * 32)); };
    const int cands[][2] = {{te0, ln0},          {h32(te0 / 2), ln0},     {h32(te0 * 2), ln0},
                            {h32(HT_THREADS), 1}, {h32(HT_THREADS / 2), 2}, {h32(HT_THREADS / 4), 4},
                            {h32(HT_THREADS / 8), 8}};
    const int ncand = (int)(sizeof(cands) / sizeof(cands[0]));
    for (int c = 0; c < ncand && !rc; ++c) {
        pmrf_tuning t = keep;
        t.hood_tile = cands[c][0];
        t.hood_lanes = cands[c][1];
        cudaDeviceSynchronize();
        free_plans(g);
        free_em(g);
        g->tuning = t;
        rc = em_run(g, cfg, lab, par, it, cv, nullptr, s);  // warm-up (plan, workspace, graph capture)
        if (rc) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && !rc; ++r) rc = em_run(g, cfg, lab, par, it, cv, nullptr, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(PMRF_ERR_CUDA, "autotune timing failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!rc && ms < best_ms) {
            best_ms = ms;
            win = t;
        }
    }
    cudaDeviceSynchronize();
    free_plans(g);
    free_em(g);
    g->tuning = rc ? keep : win;
    if (!rc) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[tune_key(g, (int)L)] = std::make_pair(win.hood_tile, win.hood_lanes);
    }
    if (best && !rc) *best = win;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(lab, s);
    dfree(par, s);
    dfree(it, s);
    dfree(cv, s);
    return rc;
}

}  // namespace pmrf

namespace pmrf {

int em_kernel_times(pmrf_graph* g, int32_t max_n, float* msv, float* msh, int32_t* n, cudaStream_t s) {
    if (!g || !n) return fail(PMRF_ERR_ARG, "null argument");
    if (g->prof_iters <= 0) return fail(PMRF_ERR_ARG, "the last pmrf_em run was not profiled");
    PMRF_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> it(g->S);
    PMRF_CUDA(cudaMemcpy(it.data(), g->em.d_iters, sizeof(int32_t) * g->S, cudaMemcpyDeviceToHost));
    int32_t tmax = 0;
    for (int32_t v : it) tmax = std::max(tmax, v);
    tmax = std::min(tmax, (int32_t)g->prof_iters);
    tmax = std::min(tmax, max_n);
    for (int t = 0; t < tmax; ++t) {
        float a = 0.f, b = 0.f;
        PMRF_CUDA(cudaEventElapsedTime(&a, g->prof_ev[3 * t + 0], g->prof_ev[3 * t + 1]));
        PMRF_CUDA(cudaEventElapsedTime(&b, g->prof_ev[3 * t + 1], g->prof_ev[3 * t + 2]));
        if (msv) msv[t] = a;
        if (msh) msh[t] = b;
    }
    *n = tmax;
    return PMRF_OK;
}

}  // namespace pmrf
