// build.cu -- device construction of the region graph, its maximal cliques,
// the 1-neighbourhoods ("hoods", or k-neighbourhoods) and the replica
// structures the EM sweep streams (Algorithm 2 steps 1, 2, 4, 5; Sections 2.1,
// 3.1, 3.2.1, 3.2.2 "Construction of Neighborhoods" and "Replicate
// Neighborhoods By Label"); 2-D slices, or 3-D volumes of stacked layers.
//
// Everything is computed for a whole batch at once: the slices are disjoint
// sub-graphs of one graph whose vertex ids are global (slice s owns vertices
// [vert_off[s], vert_off[s+1])).  Integer results are deterministic and do not
// depend on the order atomics land in: every list filled through atomics whose
// order can reach a result is sorted afterwards (a vertex's replica masks are
// left in fill order: only their minimum is used).
#include <algorithm>
#include <vector>

#include "graph.cuh"

namespace pmrf {

namespace {

constexpr int PIX_THREADS = 256;
// the region scan and the slot-mask pass wait mostly on scattered loads: 8
// resident 256-thread blocks per SM (32 registers) hide more of that latency
constexpr int RS_MIN_BLOCKS = 8;
constexpr int MK_MIN_BLOCKS = 8;
constexpr int MAX_CLIQUE = 64;  // deepest Bron-Kerbosch recursion (largest clique)

// finite double, from its exponent bits (no floating-point instruction)
__device__ __forceinline__ bool finite_bits(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

__device__ __forceinline__ int32_t vertex_of(const int32_t* ids, const int32_t* rank, int64_t rank_base, int64_t p) {
    return rank[rank_base + ids[p]];
}

// ---------------------------------------------------------------------------
// regions

constexpr int VAL_ITEMS = 16;  // pixels per thread in k_validate

// ids must be non-negative (they index the per-slice rank table).  The
// intensities' finiteness is checked where they are summed (every pixel is
// added into exactly one region mean): a non-finite sum sends its region's
// thread back over its pixels to name the first non-finite one.
__global__ void k_validate(const int32_t* __restrict__ ids, const int64_t* __restrict__ pix_off,
                           int32_t* __restrict__ maxid, DevStatus* st) {
    __shared__ int32_t s_m[PIX_THREADS / 32];
    const int s = blockIdx.y;
    const int64_t b = pix_off[s], e = pix_off[s + 1];
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    int32_t m = -1;
    for (int64_t p0 = b + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p0 < e; p0 += VAL_ITEMS * step) {
        // a thread's pixels' loads issued together (enough bytes in flight per
        // thread to keep HBM busy with 4-byte loads)
        int32_t id[VAL_ITEMS];
#pragma unroll
        for (int k = 0; k < VAL_ITEMS; ++k) {
            const int64_t p = p0 + k * step;
            id[k] = p < e ? ids[p] : 0;
        }
#pragma unroll
        for (int k = 0; k < VAL_ITEMS; ++k) {
            const int64_t p = p0 + k * step;
            if (id[k] < 0) record_error(st, PMRF_ERR_ARG, SITE_BAD_ID, p);
            m = max(m, id[k]);
        }
    }
    // one atomic per block on the slice's word
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane_id() == 0) s_m[warp_id()] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < PIX_THREADS / 32; ++w) m = max(m, s_m[w]);
        if (m >= 0) atomicMax(&maxid[s], m);
    }
}

// pixel counts and bounding boxes (rows and columns inside the slice) of every
// raw id present, indexed by its slot in the slice's rank table (so they need
// no vertex numbering yet).  A warp's 32 consecutive pixels form runs of equal
// ids within a row (one shuffle and one ballot find the run starts); the
// first lane of each run updates the run's count and extent.
__global__ void k_count_raw(const int32_t* __restrict__ ids, const int64_t* __restrict__ pix_off,
                            const int64_t* __restrict__ Wd, const int64_t* __restrict__ rank_off,
                            int32_t* __restrict__ npix_raw, int4* __restrict__ bbox_raw) {
    const int s = blockIdx.y;
    const int64_t b = pix_off[s], e = pix_off[s + 1], rb = rank_off[s], W = Wd[s];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = lane_id();
    const unsigned w32 = (unsigned)W;
    for (int64_t base = b + (int64_t)blockIdx.x * blockDim.x; base < e; base += stride) {
        const int64_t p = base + threadIdx.x;
        const bool ok = p < e;
        // row and column within the slice in 32-bit arithmetic (a batch has
        // fewer than 2^32 pixels); lanes past the end get distinct ids
        const int32_t id = ok ? ids[p] : -1 - lane;
        const unsigned q = (unsigned)(p - b);
        const unsigned r = q / w32, c = q - r * w32;
        const int32_t pid = __shfl_up_sync(0xffffffffu, id, 1);
        const unsigned pr = __shfl_up_sync(0xffffffffu, r, 1);
        const bool start = lane == 0 || pid != id || pr != r;
        const unsigned starts = __ballot_sync(0xffffffffu, start);
        if (ok && start) {
            const unsigned later = starts & ~((2u << lane) - 1u);  // starts above this lane
            const int end = later ? __ffs(later) - 2 : 31;        // last lane of the run
            const int len = end - lane + 1;
            const int64_t k = rb + id;
            atomicAdd(&npix_raw[k], len);
            atomicMin(&bbox_raw[k].x, (int)r);
            atomicMax(&bbox_raw[k].y, (int)r);
            atomicMin(&bbox_raw[k].z, (int)c);
            atomicMax(&bbox_raw[k].w, (int)(c + len - 1));
        }
    }
}

// presence flags of the rank table: an id is present when it has pixels
__global__ void k_present(const int32_t* __restrict__ npix_raw, int64_t n, int32_t* __restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = npix_raw[i] > 0 ? 1 : 0;
}

// flags -> global vertex ids (in place), -1 for absent ids
__global__ void k_rank(int32_t* __restrict__ flags, const int64_t* __restrict__ ex, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = flags[i] ? (int32_t)ex[i] : -1;
}

__global__ void k_vert_off(const int64_t* __restrict__ ex, const int64_t* __restrict__ rank_off, int32_t S,
                           int64_t* __restrict__ vert_off) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s <= S) vert_off[s] = ex[rank_off[s]];
}

__global__ void k_init_bbox(int4* __restrict__ bbox, int64_t V) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V) bbox[v] = make_int4(0x7fffffff, -1, 0x7fffffff, -1);
}

// raw id of every vertex (inverse of the compaction map)
__global__ void k_inv_rank(const int32_t* __restrict__ rank, const int64_t* __restrict__ rank_off, int32_t S,
                           int64_t n, int32_t* __restrict__ inv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = rank[i];
    if (v < 0) return;
    const int s = (int)(upper_bound_dev<int64_t>(rank_off, 0, S + 1, i) - 1);
    inv[v] = (int32_t)(i - rank_off[s]);
}

// One thread per region with a compact bounding box (area <= 4 n + 64): the
// box is scanned in row-major order, adding the pixels that carry the region's
// id -- the same additions, in the same order, as a serial row-major
// accumulation.  The same scan, widened by one pixel above and to the left,
// visits every horizontal and vertical 4-connected pixel pair that touches the
// region: a pair with exactly one pixel in the region names a neighbouring
// region.  Those ids go to a small unsorted buffer, sorted and de-duplicated
// after the scan; raw ids and vertex ids sort alike within a slice.  A
// neighbour is appended only when it differs from the last one appended for
// the same side of the region (left, right, above, below), so a boundary that
// runs down the rows or along a row adds its neighbour once.  Each pixel's
// right neighbour is the next step's pixel, so a step loads one new id (and
// the one below).
// Outputs: y_v, n_v; the region's neighbour vertex ids, ascending, at
// nbr[v * NB_CAP ...) and their number in deg[v].  Regions whose box is too
// sparse (their mean then comes from a sorted pixel list: fb_pix[v] = n), whose
// boundary buffer overflows or that have more than NB_CAP neighbours get
// fb_adj[v] = 1: their adjacency comes from the pixel-pair path.
constexpr int NB_CAP = 32;
constexpr int NB_BUF = 64;

__global__ void __launch_bounds__(256, RS_MIN_BLOCKS) k_region_scan(
    const double* __restrict__ img, const int32_t* __restrict__ ids, const int64_t* __restrict__ pix_off,
    const int64_t* __restrict__ Wd, const int64_t* __restrict__ vert_off, const int64_t* __restrict__ rank_off,
    const int32_t* __restrict__ rank, int32_t S, const int32_t* __restrict__ inv, const int4* __restrict__ bbox_raw,
    const int32_t* __restrict__ npix_raw, int64_t V, double* __restrict__ y, int32_t* __restrict__ npix,
    int32_t* __restrict__ fb_pix, int32_t* __restrict__ fb_adj, int32_t* __restrict__ deg, int32_t* __restrict__ nbr,
    DevStatus* st) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // every lane reaches the ballot below (the warp's row range is shared)
    bool scan = false;
    int s = 0;
    int32_t id = 0;
    int4 bb = make_int4(0, -1, 0, -1);
    int64_t n = 0;
    if (v < V) {
        s = (int)(upper_bound_dev<int64_t>(vert_off, 0, S + 1, v) - 1);
        id = inv[v];
        const int64_t slot = rank_off[s] + id;
        bb = bbox_raw[slot];
        n = npix_raw[slot];
        npix[v] = (int32_t)n;
        const int64_t area = (int64_t)(bb.y - bb.x + 1) * (int64_t)(bb.w - bb.z + 1);
        if (area > 4 * n + 64) {
            fb_pix[v] = (int32_t)n;
            fb_adj[v] = 1;
            deg[v] = 0;
        } else {
            fb_pix[v] = 0;
            scan = true;
        }
    }
    const unsigned lanes = __ballot_sync(0xffffffffu, scan);
    if (!scan) return;
    const int64_t b = pix_off[s], W = Wd[s];
    const int H = (int)((pix_off[s + 1] - b) / W);
    int32_t buf[NB_BUF];
    int m = 0;
    // last neighbour appended on each side: left, right (horizontal pairs), above, below
    int32_t last_l = id, last_r = id, last_a = id, last_b = id;
    double acc = 0.0;
    const int r0 = bb.x > 0 ? bb.x - 1 : 0, c0 = bb.z > 0 ? bb.z - 1 : 0;
    const int w = (int)W;
    // The warp's regions are consecutive ids: neighbours along a seed row of
    // the oversegmentation, their boxes side by side.  The lanes step through
    // the rows of the warp's joint row range together, each working on its own
    // box's part of the row, so a row's loads of the warp fall on a few
    // neighbouring cache lines; a lane's own rows still come in order.
    const int rlo = (int)__reduce_min_sync(lanes, (unsigned)r0);
    const int rhi = (int)__reduce_max_sync(lanes, (unsigned)bb.y);
    for (int r = rlo; r <= rhi; ++r) {
        if (r < r0 || r > bb.y) continue;
        const int32_t* irow = ids + b + (int64_t)r * W;
        const double* vrow = img + b + (int64_t)r * W;
        const bool down = r + 1 < H;
        int32_t cur = irow[c0];
        // two steps' id loads in flight per lane
#pragma unroll 2
        for (int c = c0; c <= bb.w; ++c) {
            const int32_t right = c + 1 < w ? irow[c + 1] : cur;
            const int32_t below = down ? irow[w + c] : cur;
            const bool in = cur == id;
            if (in) acc += vrow[c];  // region pixels lie inside the box: row-major order
            // the other pixel of a pair with exactly one pixel in the region:
            // right of the region (in, right not) or left of it (cur not, right in);
            // below it (in, below not) or above it (cur not, below in)
            const bool pr = in && right != id, pl = !in && right == id;
            const bool pb = in && below != id, pa = !in && below == id;
            const int32_t uh = in ? right : cur, uv = in ? below : cur;
            const bool th = (pr && uh != last_r) || (pl && uh != last_l);
            const bool tv = (pb && uv != last_b) || (pa && uv != last_a);
            if (th) {
                if (m < NB_BUF) buf[m] = uh;
                ++m;
                if (pr) last_r = uh;
                else last_l = uh;
            }
            if (tv) {
                if (m < NB_BUF) buf[m] = uv;
                ++m;
                if (pb) last_b = uv;
                else last_a = uv;
            }
            cur = right;
        }
    }
    y[v] = acc / (double)n;
    if (!finite_bits(acc)) {
        // a non-finite pixel (or a sum of finite ones beyond the double range,
        // which is not an input error): the first such pixel, row-major
        for (int r = bb.x; r <= bb.y; ++r)
            for (int c = bb.z; c <= bb.w; ++c) {
                const int64_t p = b + (int64_t)r * W + c;
                if (ids[p] == id && !finite_bits(img[p])) {
                    record_error(st, PMRF_ERR_NONFINITE, SITE_NONFINITE, p);
                    r = bb.y;
                    break;
                }
            }
    }
    bool over = m > NB_BUF;
    int nn = 0;
    if (!over) {
        // sort the buffer, keep distinct ids
        for (int i = 1; i < m; ++i) {
            const int32_t x = buf[i];
            int j = i - 1;
            while (j >= 0 && buf[j] > x) {
                buf[j + 1] = buf[j];
                --j;
            }
            buf[j + 1] = x;
        }
        for (int i = 0; i < m; ++i)
            if (i == 0 || buf[i] != buf[i - 1]) buf[nn++] = buf[i];
        over = nn > NB_CAP;
    }
    fb_adj[v] = over ? 1 : 0;
    deg[v] = over ? 0 : nn;
    if (!over) {
        const int64_t rb = rank_off[s];
        int32_t* out = nbr + v * NB_CAP;
        for (int k = 0; k < nn; ++k) out[k] = rank[rb + buf[k]];
    }
}

// sums of two int32 arrays of length n (a grid of a few blocks per SM; one
// atomic per block and array)
constexpr int SUM_THREADS = 256;
__global__ void __launch_bounds__(SUM_THREADS) k_sum2(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                                                      int64_t n, unsigned long long* __restrict__ out) {
    __shared__ unsigned long long s_a[SUM_THREADS / 32], s_b[SUM_THREADS / 32];
    unsigned long long sa = 0, sb = 0;
    for (int64_t i = (int64_t)blockIdx.x * SUM_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * SUM_THREADS) {
        sa += (unsigned long long)(uint32_t)a[i];
        sb += (unsigned long long)(uint32_t)b[i];
    }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (lane_id() == 0) {
        s_a[warp_id()] = sa;
        s_b[warp_id()] = sb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < SUM_THREADS / 32; ++w) {
            sa += s_a[w];
            sb += s_b[w];
        }
        if (sa) atomicAdd(&out[0], sa);
        if (sb) atomicAdd(&out[1], sb);
    }
}

__global__ void k_fill_pix(const int32_t* __restrict__ ids, const int64_t* __restrict__ pix_off,
                           const int64_t* __restrict__ rank_off, const int32_t* __restrict__ rank,
                           const int64_t* __restrict__ vpix_off, int32_t* __restrict__ cursor,
                           uint32_t* __restrict__ pixlist, const int32_t* __restrict__ only) {
    const int s = blockIdx.y;
    const int64_t b = pix_off[s], e = pix_off[s + 1], rb = rank_off[s];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = b + (int64_t)blockIdx.x * blockDim.x; base < e; base += stride) {
        const int64_t p = base + threadIdx.x;
        const bool ok = p < e;
        int32_t v = ok ? vertex_of(ids, rank, rb, p) : -1 - lane_id();
        const bool take = ok && (only == nullptr || only[v] != 0);
        if (!take) v = -1 - lane_id();
        const unsigned grp = __match_any_sync(0xffffffffu, v);
        const int leader = __ffs(grp) - 1;
        int slot = 0;
        if (take && lane_id() == leader) slot = atomicAdd(&cursor[v], __popc(grp));
        slot = __shfl_sync(grp, slot, leader);
        if (take) {
            const int rk = __popc(grp & ((1u << lane_id()) - 1u));
            pixlist[vpix_off[v] + slot + rk] = (uint32_t)p;
        }
    }
}

// y_v from a region's sorted pixel list: the pixels added one by one in
// row-major order, then divided by the count (the same sequence of IEEE
// operations as a serial row-major accumulation).
__global__ void k_means(const double* __restrict__ img, const uint32_t* __restrict__ pixlist,
                        const int64_t* __restrict__ vpix_off, int64_t V, double* __restrict__ y, DevStatus* st) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    if (vpix_off[v + 1] == vpix_off[v]) return;  // region summed by k_region_scan
    double acc = 0.0;
    const int64_t b = vpix_off[v], e = vpix_off[v + 1];
    for (int64_t i = b; i < e; ++i) acc += img[pixlist[i]];
    y[v] = acc / (double)(e - b);
    if (!finite_bits(acc)) {  // the first non-finite pixel, if any (as in k_region_scan)
        for (int64_t i = b; i < e; ++i)
            if (!finite_bits(img[pixlist[i]])) {
                record_error(st, PMRF_ERR_NONFINITE, SITE_NONFINITE, (int64_t)pixlist[i]);
                break;
            }
    }
}

// ---------------------------------------------------------------------------
// edges of the regions the scan could not take (only[v] != 0): 4-connected
// pixel pairs with different regions, each delivered to its flagged endpoints.
// A pair that repeats the same (left/top, right/bottom) vertex pair as its
// neighbour along the boundary is skipped (the earlier one stands for it); the
// final sort+unique gives the same set either way.

template <bool FILL>
__global__ void k_edge_pairs(const int32_t* __restrict__ ids, const int64_t* __restrict__ pix_off,
                             const int64_t* __restrict__ Wd, const int64_t* __restrict__ layer_rows,
                             const int64_t* __restrict__ rank_off,
                             const int32_t* __restrict__ rank, const int32_t* __restrict__ only,
                             int32_t* __restrict__ cnt, const int64_t* __restrict__ cand_off,
                             int32_t* __restrict__ cursor, uint32_t* __restrict__ cand) {
    const int s = blockIdx.y;
    const int64_t b = pix_off[s], e = pix_off[s + 1], rb = rank_off[s], W = Wd[s];
    if (W <= 0) return;
    const int64_t H = (e - b) / W;
    // a 3-D volume is its layers' rows one after another: rows r and r+1 are
    // neighbours inside a layer only, rows r and r+Hl (the next layer) are
    // z-neighbours
    const int64_t Hl = layer_rows ? layer_rows[s] : H;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < e - b; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / W, c = q - r * W;
        const int64_t p = b + q;
        const int32_t a = vertex_of(ids, rank, rb, p);
        int32_t pa[3], pb[3];
        int np = 0;
        if (c + 1 < W) {
            const int32_t bb = vertex_of(ids, rank, rb, p + 1);
            if (a != bb) {
                bool dup = (r > 0) && vertex_of(ids, rank, rb, p - W) == a && vertex_of(ids, rank, rb, p - W + 1) == bb;
                if (!dup) { pa[np] = a; pb[np] = bb; ++np; }
            }
        }
        if (r + 1 < H && (r + 1) % Hl != 0) {
            const int32_t bb = vertex_of(ids, rank, rb, p + W);
            if (a != bb) {
                bool dup = (c > 0) && vertex_of(ids, rank, rb, p - 1) == a && vertex_of(ids, rank, rb, p + W - 1) == bb;
                if (!dup) { pa[np] = a; pb[np] = bb; ++np; }
            }
        }
        if (Hl < H && r + Hl < H) {
            const int32_t bb = vertex_of(ids, rank, rb, p + Hl * W);
            if (a != bb) {
                bool dup = (c > 0) && vertex_of(ids, rank, rb, p - 1) == a &&
                           vertex_of(ids, rank, rb, p + Hl * W - 1) == bb;
                if (!dup) { pa[np] = a; pb[np] = bb; ++np; }
            }
        }
        // each endpoint that takes the pixel-pair path receives the other one
        for (int k = 0; k < np; ++k) {
            const bool ta = only[pa[k]] != 0, tb = only[pb[k]] != 0;
            if (!FILL) {
                if (ta) atomicAdd(&cnt[pa[k]], 1);
                if (tb) atomicAdd(&cnt[pb[k]], 1);
            } else {
                if (ta) cand[cand_off[pa[k]] + atomicAdd(&cursor[pa[k]], 1)] = (uint32_t)pb[k];
                if (tb) cand[cand_off[pb[k]] + atomicAdd(&cursor[pb[k]], 1)] = (uint32_t)pa[k];
            }
        }
    }
}

// the largest degree: a grid of a few blocks per SM strides over the vertices,
// each block's maximum goes out in one atomic (atomics on one word serialise)
constexpr int CD_THREADS = 256;
__global__ void __launch_bounds__(CD_THREADS) k_check_degree(const int32_t* __restrict__ deg, int64_t V,
                                                             int32_t maxdeg, DevStatus* st,
                                                             int32_t* __restrict__ dmax) {
    __shared__ unsigned s_m[CD_THREADS / 32];
    unsigned m = 0;
    for (int64_t v = (int64_t)blockIdx.x * CD_THREADS + threadIdx.x; v < V; v += (int64_t)gridDim.x * CD_THREADS) {
        const int32_t d = deg[v];
        if (d > maxdeg) record_error(st, PMRF_ERR_UNSUPPORTED, SITE_DEGREE, v);
        m = max(m, (unsigned)d);
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane_id() == 0) s_m[warp_id()] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < CD_THREADS / 32; ++w) m = max(m, s_m[w]);
        if (m > 0) atomicMax(dmax, (int32_t)m);
    }
}

// flagged vertices take their de-duplicated candidate count as degree
__global__ void k_take_counts(const int32_t* __restrict__ fb_adj, const int32_t* __restrict__ ucnt, int64_t V,
                              int32_t* __restrict__ deg) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V && fb_adj[v]) deg[v] = ucnt[v];
}

// adjacency of every vertex: from its region scan, or (flagged vertices) from
// its sorted, de-duplicated pixel-pair candidates
__global__ void k_adj_fill(const int32_t* __restrict__ fb_adj, const int32_t* __restrict__ nbr,
                           const uint32_t* __restrict__ cand, const int64_t* __restrict__ cand_off,
                           const int64_t* __restrict__ adj_off, int64_t V, int32_t* __restrict__ adj) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int64_t o = adj_off[v], n = adj_off[v + 1] - o;
    if (fb_adj[v]) {
        const int64_t b = cand_off[v];
        for (int64_t i = 0; i < n; ++i) adj[o + i] = (int32_t)cand[b + i];
    } else {
        const int32_t* src = nbr + v * NB_CAP;
        for (int64_t i = 0; i < n; ++i) adj[o + i] = src[i];
    }
}

// ---------------------------------------------------------------------------
// maximal cliques: Bron-Kerbosch with pivoting, rooted at each vertex v over
// its higher neighbours (candidates) and lower neighbours (excluded), so each
// maximal clique is produced once, by its smallest member.  Sets are bitsets
// over the slots of N(v) (nw 64-bit words).

struct BKFrame {  // pointers into nw-word storage
    uint64_t *P, *X, *C, *R;
};

__device__ __forceinline__ bool bs_empty(const uint64_t* a, int nw) {
    for (int w = 0; w < nw; ++w) if (a[w]) return false;
    return true;
}

// local adjacency among the slots of N(v): nbm[i*nw + w]
__device__ void build_local_adj(const int64_t* __restrict__ adj_off, const int32_t* __restrict__ adj, int64_t v,
                                int d, int nw, uint64_t* nbm) {
    const int32_t* N = adj + adj_off[v];
    if (nw == 1) {
        // d <= 64: the relation is symmetric, so row i intersects N(u_i) only
        // with the slots above i (a branch-free two-pointer step) and each
        // adjacent pair is mirrored into the lower row
        for (int i = 0; i < d; ++i) nbm[i] = 0;
        for (int i = 0; i + 1 < d; ++i) {
            const int32_t u = N[i];
            const int32_t* Nu = adj + adj_off[u];
            const int du = (int)(adj_off[u + 1] - adj_off[u]);
            uint64_t row = 0;
            int a = 0, j = i + 1;
            while (a < du && j < d) {
                const int32_t x = __ldg(Nu + a), y = __ldg(N + j);
                const bool le = x <= y, ge = x >= y;
                row |= (uint64_t)(le && ge) << j;
                a += le;
                j += ge;
            }
            nbm[i] |= row;
            while (row) {
                const int j2 = __ffsll((long long)row) - 1;
                row &= row - 1;
                nbm[j2] |= 1ull << i;
            }
        }
        return;
    }
    for (int i = 0; i < d; ++i) {
        for (int w = 0; w < nw; ++w) nbm[(int64_t)i * nw + w] = 0;
        const int32_t u = N[i];
        const int32_t* Nu = adj + adj_off[u];
        const int64_t du = adj_off[u + 1] - adj_off[u];
        int64_t a = 0;
        int j = 0;
        while (a < du && j < d) {
            if (Nu[a] < N[j]) ++a;
            else if (Nu[a] > N[j]) ++j;
            else {
                nbm[(int64_t)i * nw + (j >> 6)] |= 1ull << (j & 63);
                ++a;
                ++j;
            }
        }
    }
}

// Runs the enumeration rooted at v, counting cliques (ncl) and members (nmem)
// and storing the first out_cap masks (nw words each) at out_masks (may be
// NULL).  `stack` holds MAX_CLIQUE+1 frames of 4*nw words; `tmp` holds 2*nw
// words.  Returns false when the recursion would exceed MAX_CLIQUE.
__device__ bool bk_run(int64_t v, const int32_t* N, int d, int nw, const uint64_t* nbm, uint64_t* stack,
                       uint64_t* tmp, int64_t* ncl, int64_t* nmem, uint64_t* out_masks, int64_t out_cap) {
    // slot of the first neighbour above v
    int hi = 0;
    while (hi < d && N[hi] < v) ++hi;
    auto frame = [&](int k) {
        BKFrame f;
        uint64_t* base = stack + (int64_t)k * 4 * nw;
        f.P = base;
        f.X = base + nw;
        f.C = base + 2 * nw;
        f.R = base + 3 * nw;
        return f;
    };
    auto emit = [&](const uint64_t* R) {
        int64_t sz = 1;
        for (int w = 0; w < nw; ++w) sz += __popcll(R[w]);
        if (out_masks && *ncl < out_cap) {
            for (int w = 0; w < nw; ++w) out_masks[*ncl * nw + w] = R[w];
        }
        *ncl += 1;
        *nmem += sz;
    };
    // choose pivot in P|X maximising |P & N(u)|; C = P & ~N(pivot)
    auto set_candidates = [&](BKFrame f) {
        int best = -1, bu = 0;
        for (int w = 0; w < nw; ++w) {
            uint64_t m = f.P[w] | f.X[w];
            while (m) {
                int bit = __ffsll((long long)m) - 1;
                m &= m - 1;
                int u = w * 64 + bit;
                int c = 0;
                for (int z = 0; z < nw; ++z) c += __popcll(f.P[z] & nbm[(int64_t)u * nw + z]);
                if (c > best) { best = c; bu = u; }
            }
        }
        for (int w = 0; w < nw; ++w) f.C[w] = f.P[w] & ~nbm[(int64_t)bu * nw + w];
    };
    BKFrame root = frame(0);
    for (int w = 0; w < nw; ++w) { root.P[w] = 0; root.X[w] = 0; root.R[w] = 0; }
    for (int i = 0; i < d; ++i) {
        if (i >= hi) root.P[i >> 6] |= 1ull << (i & 63);
        else root.X[i >> 6] |= 1ull << (i & 63);
    }
    if (bs_empty(root.P, nw)) {
        if (bs_empty(root.X, nw)) emit(root.R);  // isolated vertex: clique {v}
        return true;
    }
    set_candidates(root);
    int sp = 0;
    while (sp >= 0) {
        BKFrame f = frame(sp);
        int w0 = 0;
        while (w0 < nw && f.C[w0] == 0) ++w0;
        if (w0 == nw) { --sp; continue; }
        const int bit = __ffsll((long long)f.C[w0]) - 1;
        const uint64_t m = 1ull << bit;
        const int u = w0 * 64 + bit;
        f.C[w0] &= ~m;
        uint64_t* Pn = tmp;
        uint64_t* Xn = tmp + nw;
        for (int w = 0; w < nw; ++w) {
            Pn[w] = f.P[w] & nbm[(int64_t)u * nw + w];
            Xn[w] = f.X[w] & nbm[(int64_t)u * nw + w];
        }
        const bool pe = bs_empty(Pn, nw), xe = bs_empty(Xn, nw);
        if (pe && xe) {
            f.R[w0] |= m;
            emit(f.R);
            f.R[w0] &= ~m;
        }
        f.P[w0] &= ~m;
        f.X[w0] |= m;
        if (!pe) {
            if (sp + 1 > MAX_CLIQUE) return false;
            BKFrame g = frame(sp + 1);
            for (int w = 0; w < nw; ++w) { g.P[w] = Pn[w]; g.X[w] = Xn[w]; g.R[w] = f.R[w]; }
            g.R[w0] |= m;
            set_candidates(g);
            ++sp;
        }
    }
    return true;
}

// lexicographic order of two maximal cliques rooted at the same vertex: the
// lower differing slot decides (see build notes: distinct maximal cliques are
// never nested, so one list cannot be a prefix of the other)
__device__ __forceinline__ bool clique_less(const uint64_t* a, const uint64_t* b, int nw) {
    for (int w = 0; w < nw; ++w) {
        uint64_t x = a[w] ^ b[w];
        if (x) return (a[w] & (x & (~x + 1))) != 0;
    }
    return false;
}

// Fast path: d <= 64, one word, stack in local memory.  mode 0 counts, mode 1
// writes sorted cliques.  General vertices (d > 64) are skipped here.
// The count pass keeps the first CQ_KEEP masks of each vertex in `kept`; the
// fill pass copies them instead of enumerating again (vertices with more
// cliques are enumerated twice).
constexpr int CQ_KEEP = 8;

__global__ void k_cliques_fast(const int64_t* __restrict__ adj_off, const int32_t* __restrict__ adj, int64_t V,
                               int mode, int64_t* __restrict__ ncl, int64_t* __restrict__ nmem,
                               const int64_t* __restrict__ cq_off, const int64_t* __restrict__ mem_off,
                               uint64_t* __restrict__ maskbuf, int64_t* __restrict__ clq_off,
                               int32_t* __restrict__ clq, DevStatus* st, uint64_t* __restrict__ kept) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int d = (int)(adj_off[v + 1] - adj_off[v]);
    if (d > 64) return;
    const int32_t* N = adj + adj_off[v];
    int64_t nc = 0, nm = 0;
    uint64_t* out = (mode == 1) ? maskbuf + cq_off[v] : nullptr;
    if (mode == 1 && ncl[v] <= CQ_KEEP) {
        nc = ncl[v];
        for (int64_t i = 0; i < nc; ++i) out[i] = kept[v * CQ_KEEP + i];
    } else {
        uint64_t nbm[64];
        uint64_t stack[(MAX_CLIQUE + 1) * 4];
        uint64_t tmp[2];
        build_local_adj(adj_off, adj, v, d, 1, nbm);
        uint64_t* dst = mode == 1 ? out : kept + v * CQ_KEEP;
        if (!bk_run(v, N, d, 1, nbm, stack, tmp, &nc, &nm, dst, mode == 1 ? INT64_MAX : CQ_KEEP)) {
            record_error(st, PMRF_ERR_UNSUPPORTED, SITE_MCE_STACK, v);
            nc = 0;
            nm = 0;
        }
    }
    if (mode == 0) {
        ncl[v] = nc;
        nmem[v] = nm;
        return;
    }
    // insertion sort of the vertex's clique masks, then member lists
    for (int64_t i = 1; i < nc; ++i) {
        uint64_t key = out[i];
        int64_t j = i - 1;
        while (j >= 0 && clique_less(&key, &out[j], 1)) { out[j + 1] = out[j]; --j; }
        out[j + 1] = key;
    }
    int64_t pos = mem_off[v];
    for (int64_t i = 0; i < nc; ++i) {
        clq_off[cq_off[v] + i] = pos;
        clq[pos++] = (int32_t)v;
        uint64_t m = out[i];
        while (m) {
            int bit = __ffsll((long long)m) - 1;
            m &= m - 1;
            clq[pos++] = N[bit];
        }
    }
}

// General path for 64 < d <= PMRF_MAX_DEGREE: one thread per listed vertex,
// bitsets in global scratch (gscr_off gives each vertex its region).
__global__ void k_cliques_general(const int64_t* __restrict__ adj_off, const int32_t* __restrict__ adj,
                                  const int64_t* __restrict__ glist, int64_t ng, const int64_t* __restrict__ gscr_off,
                                  uint64_t* __restrict__ gscr, int mode, int64_t* __restrict__ ncl,
                                  int64_t* __restrict__ nmem, const int64_t* __restrict__ cq_off,
                                  const int64_t* __restrict__ gmask_off, uint64_t* __restrict__ gmask,
                                  const int64_t* __restrict__ mem_off, int64_t* __restrict__ clq_off,
                                  int32_t* __restrict__ clq, DevStatus* st) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng) return;
    const int64_t v = glist[k];
    const int d = (int)(adj_off[v + 1] - adj_off[v]);
    const int nw = (d + 63) / 64;
    uint64_t* nbm = gscr + gscr_off[k];
    uint64_t* stack = nbm + (int64_t)d * nw;
    uint64_t* tmp = stack + (int64_t)(MAX_CLIQUE + 1) * 4 * nw;
    const int32_t* N = adj + adj_off[v];
    build_local_adj(adj_off, adj, v, d, nw, nbm);
    int64_t nc = 0, nm = 0;
    uint64_t* out = (mode == 1) ? gmask + gmask_off[k] : nullptr;
    if (!bk_run(v, N, d, nw, nbm, stack, tmp, &nc, &nm, out, out ? INT64_MAX : 0)) {
        record_error(st, PMRF_ERR_UNSUPPORTED, SITE_MCE_STACK, v);
        nc = 0;
        nm = 0;
    }
    if (mode == 0) {
        ncl[v] = nc;
        nmem[v] = nm;
        return;
    }
    // insertion sort (swap nw-word records through tmp)
    for (int64_t i = 1; i < nc; ++i) {
        for (int w = 0; w < nw; ++w) tmp[w] = out[i * nw + w];
        int64_t j = i - 1;
        while (j >= 0 && clique_less(tmp, &out[j * nw], nw)) {
            for (int w = 0; w < nw; ++w) out[(j + 1) * nw + w] = out[j * nw + w];
            --j;
        }
        for (int w = 0; w < nw; ++w) out[(j + 1) * nw + w] = tmp[w];
    }
    int64_t pos = mem_off[v];
    for (int64_t i = 0; i < nc; ++i) {
        clq_off[cq_off[v] + i] = pos;
        clq[pos++] = (int32_t)v;
        for (int w = 0; w < nw; ++w) {
            uint64_t m = out[i * nw + w];
            while (m) {
                int bit = __ffsll((long long)m) - 1;
                m &= m - 1;
                clq[pos++] = N[w * 64 + bit];
            }
        }
    }
}

__global__ void k_list_general(const int64_t* __restrict__ adj_off, int64_t V, int64_t* __restrict__ glist,
                               int32_t* __restrict__ ng) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    if (adj_off[v + 1] - adj_off[v] > 64) glist[atomicAdd(ng, 1)] = v;
}

// ---------------------------------------------------------------------------
// hoods: H_c = K_c plus the neighbours of its members.  For a clique of two or
// more members every member is a neighbour of another member, so H_c is the
// union of the members' (sorted) adjacency lists: a k-way merge per clique.  A
// one-member maximal clique is an isolated vertex, whose hood is itself.

// The count pass keeps hoods of up to HOOD_KEEP members in `kept`, element i
// of hood c at kept[i * C + c] (a warp's stores and loads are adjacent); the
// fill pass copies those and merges only the larger ones.  A block of the fill
// pass whose hoods are all kept and whose output range (contiguous: hood_off
// is a prefix sum) fits FILL_STAGE elements assembles the range in shared
// memory and writes it out with adjacent stores.
constexpr int HOOD_KEEP = 32;
constexpr int FILL_BLOCK = 256;
constexpr int FILL_STAGE = 6144;
static_assert(FILL_BLOCK == 256, "the fill pass is launched with 256 threads per block");

template <bool FILL>
__global__ void k_hood_merge(const int64_t* __restrict__ clq_off, const int32_t* __restrict__ clq,
                             const int64_t* __restrict__ adj_off, const int32_t* __restrict__ adj, int64_t C,
                             int32_t* __restrict__ hsize, int32_t* __restrict__ hmax,
                             const int64_t* __restrict__ hood_off, int32_t* __restrict__ hood,
                             int32_t* __restrict__ el_hood, int32_t* __restrict__ rcount,
                             int32_t* __restrict__ kept) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (FILL) {
        __shared__ int32_t s_hood[FILL_STAGE];
        __shared__ uint8_t s_cl[FILL_STAGE];  // hood of each element, less the block's first
        const int64_t cb = (int64_t)blockIdx.x * FILL_BLOCK;
        const int64_t ce = cb + FILL_BLOCK < C ? cb + FILL_BLOCK : C;
        const int64_t H0 = hood_off[cb], n = hood_off[ce] - H0;
        const int64_t h0 = c < C ? hood_off[c] : 0, k = c < C ? hood_off[c + 1] - h0 : 0;
        if (__syncthreads_and(k <= HOOD_KEEP) && n <= FILL_STAGE) {
            const int32_t* kc = kept + c;
            for (int64_t i = 0; i < k; ++i) {
                const int32_t cur = kc[i * C];
                s_hood[h0 - H0 + i] = cur;
                s_cl[h0 - H0 + i] = (uint8_t)threadIdx.x;
                atomicAdd(&rcount[cur], 1);
            }
            __syncthreads();
            for (int q = threadIdx.x; q < (int)n; q += FILL_BLOCK) {
                hood[H0 + q] = s_hood[q];
                el_hood[H0 + q] = (int32_t)(cb + s_cl[q]);
            }
            return;
        }
    }
    if (c >= C) return;
    const int64_t m0 = clq_off[c];
    const int m = (int)(clq_off[c + 1] - m0);
    const int64_t h0 = FILL ? hood_off[c] : 0;
    int32_t* kc = kept + c;  // stride C
    if (FILL) {
        const int64_t k = hood_off[c + 1] - h0;
        if (k <= HOOD_KEEP) {
            for (int64_t i = 0; i < k; ++i) {
                const int32_t cur = kc[i * C];
                hood[h0 + i] = cur;
                el_hood[h0 + i] = (int32_t)c;
                atomicAdd(&rcount[cur], 1);
            }
            return;
        }
    }
    int32_t n = 0;
    // element n of hood c is `cur`: its vertex gains one replica
    auto emit = [&](int32_t cur) {
        if (FILL) {
            hood[h0 + n] = cur;
            el_hood[h0 + n] = (int32_t)c;
            atomicAdd(&rcount[cur], 1);
        } else if (n < HOOD_KEEP) {
            kc[(int64_t)n * C] = cur;
        }
        ++n;
    };
    if (m == 1) {
        emit(clq[m0]);
    } else if (m <= 4) {
        // the common cliques (edges, triangles, 4-cliques): cursors and heads
        // in registers, each head loaded once
        constexpr int32_t END = 0x7fffffff;
        const int32_t* q[4];
        const int32_t* qe[4];
        int32_t h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            h[i] = END;
            q[i] = qe[i] = nullptr;
            if (i < m) {
                const int32_t u = clq[m0 + i];
                q[i] = adj + adj_off[u];
                qe[i] = adj + adj_off[u + 1];
                if (q[i] < qe[i]) h[i] = *q[i];
            }
        }
        while (true) {
            const int32_t cur = min(min(h[0], h[1]), min(h[2], h[3]));
            if (cur == END) break;
            emit(cur);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (h[i] == cur) {
                    ++q[i];
                    h[i] = q[i] < qe[i] ? *q[i] : END;
                }
        }
    } else {
        int64_t p[MAX_CLIQUE + 1], e[MAX_CLIQUE + 1];
        for (int i = 0; i < m; ++i) {
            const int32_t u = clq[m0 + i];
            p[i] = adj_off[u];
            e[i] = adj_off[u + 1];
        }
        while (true) {
            int32_t cur = 0x7fffffff;
            for (int i = 0; i < m; ++i)
                if (p[i] < e[i]) cur = min(cur, adj[p[i]]);
            if (cur == 0x7fffffff) break;
            emit(cur);
            for (int i = 0; i < m; ++i)
                if (p[i] < e[i] && adj[p[i]] == cur) ++p[i];
        }
    }
    if (!FILL) {
        hsize[c] = n;
        // largest hood: one atomic per group of converged lanes
        const unsigned act = __activemask();
        const int32_t wmax = (int32_t)__reduce_max_sync(act, (unsigned)n);
        if ((threadIdx.x & 31) == __ffs(act) - 1) atomicMax(hmax, wmax);
    }
}

__global__ void k_flag_all(int32_t* __restrict__ f, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = 1;
}

// ---------------------------------------------------------------------------
// k-neighbourhoods (Section 3.1: the vertices within k edges of a clique's
// members).  Level j+1 of a hood is the union of the closed neighbourhoods of
// its level-j members: per hood, every member and its adjacency as candidates,
// then a segmented sort with de-duplication.

__global__ void k_expand_count(const int64_t* __restrict__ hood_off, const int32_t* __restrict__ hood,
                               const int64_t* __restrict__ adj_off, int64_t C, int64_t* __restrict__ cnt) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    int64_t n = 0;
    for (int64_t i = hood_off[c]; i < hood_off[c + 1]; ++i) {
        const int32_t u = hood[i];
        n += 1 + adj_off[u + 1] - adj_off[u];
    }
    cnt[c] = n;
}

__global__ void k_expand_fill(const int64_t* __restrict__ hood_off, const int32_t* __restrict__ hood,
                              const int64_t* __restrict__ adj_off, const int32_t* __restrict__ adj,
                              const int64_t* __restrict__ cand_off, int64_t C, uint32_t* __restrict__ cand) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    int64_t o = cand_off[c];
    for (int64_t i = hood_off[c]; i < hood_off[c + 1]; ++i) {
        const int32_t u = hood[i];
        cand[o++] = (uint32_t)u;
        for (int64_t j = adj_off[u]; j < adj_off[u + 1]; ++j) cand[o++] = (uint32_t)adj[j];
    }
}

// the de-duplicated head of each sorted candidate segment becomes the hood
__global__ void k_take_unique(const uint32_t* __restrict__ cand, const int64_t* __restrict__ cand_off,
                              const int64_t* __restrict__ new_off, int64_t C, int32_t* __restrict__ hood) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int64_t o = cand_off[c], h = new_off[c], n = new_off[c + 1] - h;
    for (int64_t i = 0; i < n; ++i) hood[h + i] = (int32_t)cand[o + i];
}

// each element's hood, each vertex's replica count, the largest hood
__global__ void k_el_hood(const int64_t* __restrict__ hood_off, const int32_t* __restrict__ hood, int64_t C,
                          int32_t* __restrict__ el_hood, int32_t* __restrict__ rcount, int32_t* __restrict__ hmax) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int64_t h0 = hood_off[c], h1 = hood_off[c + 1];
    for (int64_t i = h0; i < h1; ++i) {
        el_hood[i] = (int32_t)c;
        atomicAdd(&rcount[hood[i]], 1);
    }
    atomicMax(hmax, (int32_t)(h1 - h0 < 0x7fffffff ? h1 - h0 : 0x7fffffff));
}

// ---------------------------------------------------------------------------
// replica structures

// replica lists in element order (filled in any order, then sorted): only the
// export of each vertex's hoods needs them
__global__ void k_rep_fill(const int32_t* __restrict__ hood, int64_t N_el, const int64_t* __restrict__ rep_off,
                           int32_t* __restrict__ cursor, uint32_t* __restrict__ rep_el) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N_el) return;
    const int32_t v = hood[e];
    rep_el[rep_off[v] + atomicAdd(&cursor[v], 1)] = (uint32_t)e;
}

// words of hood c's local adjacency rows: k rows of ceil(k/32) words, kept
// only for hoods of at least rows_min_k members (the ones the hood pass's
// general path reads)
__global__ void k_row_words(const int64_t* __restrict__ hood_off, int64_t C, int64_t rows_min_k,
                            int64_t* __restrict__ nwords) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    int64_t k = hood_off[c + 1] - hood_off[c];
    nwords[c] = k >= rows_min_k ? k * ceil_div(k, 32) : 0;
}

__global__ void k_rep_words(const int64_t* __restrict__ adj_off, const int32_t* __restrict__ rcount, int64_t V,
                            int64_t* __restrict__ nwords) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    int64_t d = adj_off[v + 1] - adj_off[v];
    int64_t nw = d > 32 ? ceil_div(d, 32) : 1;
    nwords[v] = (int64_t)rcount[v] * nw;
}

// The intersection of two ascending lists of at most 32 ids (N(v), d ids, and
// the hood, k ids): bit a of *sbits where N(v)[a] is in the hood and, with
// ROWS, bit j of *rbits where hood[j] is in N(v).  Both heads are loaded every
// step and the step advances them without branching (x <= y moves a, x >= y
// moves j), so the lanes of a warp stay converged.
template <bool ROWS>
__device__ __forceinline__ void merge32(const int32_t* __restrict__ N, int d, const int32_t* __restrict__ Hc, int k,
                                        uint32_t* rbits, uint32_t* sbits) {
    uint32_t rb = 0, sb = 0;
    int a = 0, j = 0;
    while (a < d && j < k) {
        const int32_t x = __ldg(N + a), y = __ldg(Hc + j);
        const bool le = x <= y, ge = x >= y;
        const uint32_t eq = (le && ge) ? 1u : 0u;
        if (ROWS) rb |= eq << j;
        sb |= eq << a;
        a += le;
        j += ge;
    }
    *rbits = rb;
    *sbits = sb;
}

// For element e (vertex v in hood c at position i): row bits j where hood[j]
// is a neighbour of v (for hoods of at least rows_min_k members), and slot
// bits s where N(v)[s] lies in the hood (stored vertex-major, one record per
// replica of v, and element-major in the hood pass's element stream: el[e] =
// (v, with bit 31 set on the last element of its hood; the slot mask when v
// has at most 32 neighbours, else 0)).
__device__ __forceinline__ void mask_element(int64_t e, const int64_t* __restrict__ hood_off,
                                             const int32_t* __restrict__ hood, const int32_t* __restrict__ el_hood,
                                             const int64_t* __restrict__ adj_off, const int32_t* __restrict__ adj,
                                             const int64_t* __restrict__ row_off, uint32_t* __restrict__ row,
                                             int32_t* __restrict__ cursor, const int64_t* __restrict__ rep_woff,
                                             uint32_t* __restrict__ rep_mask, uint2* __restrict__ el,
                                             uint8_t* __restrict__ hood_gen, int64_t rows_min_k) {
    const int32_t c = el_hood[e];
    const int64_t h0 = hood_off[c];
    const int64_t k = hood_off[c + 1] - h0;
    const int64_t i = e - h0;
    const int32_t v = hood[e];
    const int64_t av = adj_off[v];
    const int32_t* N = adj + av;
    const int64_t d = adj_off[v + 1] - av;
    const int64_t nwh = ceil_div(k, 32);
    const int64_t nwv = d > 32 ? ceil_div(d, 32) : 1;
    const uint32_t vtag = (uint32_t)v | (i == k - 1 ? 0x80000000u : 0u);  // last element of its hood
    const bool keep_row = k >= rows_min_k;
    uint32_t* rw = keep_row ? row + row_off[c] + i * nwh : nullptr;
    // the replica's place among v's replicas is arbitrary: the vertex pass only
    // takes a minimum over them
    uint32_t* sw = rep_mask + rep_woff[v] + (int64_t)atomicAdd(&cursor[v], 1) * nwv;
    if (k <= 32 && d <= 32) {
        // one word each
        uint32_t rbits, sbits;
        if (keep_row) {
            merge32<true>(N, (int)d, hood + h0, (int)k, &rbits, &sbits);
            rw[0] = rbits;
        } else {
            merge32<false>(N, (int)d, hood + h0, (int)k, &rbits, &sbits);
        }
        sw[0] = sbits;
        el[e] = make_uint2(vtag, sbits);
        return;
    }
    if (d > 32) hood_gen[c] = 1;  // the hood needs the general path of the hood pass
    uint32_t rcur = 0, scur = 0;
    int64_t rwi = 0, swi = 0;
    int64_t a = 0, j = 0;
    while (a < d && j < k) {
        const int32_t x = N[a], y = hood[h0 + j];
        if (x < y) ++a;
        else if (x > y) ++j;
        else {
            if ((j >> 5) != rwi) {
                if (keep_row) rw[rwi] = rcur;
                rcur = 0;
                rwi = j >> 5;
            }
            rcur |= 1u << (j & 31);
            if ((a >> 5) != swi) { sw[swi] = scur; scur = 0; swi = a >> 5; }
            scur |= 1u << (a & 31);
            ++a;
            ++j;
        }
    }
    if (keep_row) rw[rwi] = rcur;
    sw[swi] = scur;
    // the same slot mask in element (hood-major) order, for vertices of degree <= 32
    el[e] = make_uint2(vtag, (d <= 32) ? scur : 0u);
}

// MK_ROUNDS elements a thread, a grid's width apart (longer blocks)
constexpr int MK_ROUNDS = 16;
__global__ void __launch_bounds__(256, MK_MIN_BLOCKS) k_masks(const int64_t* __restrict__ hood_off, const int32_t* __restrict__ hood,
                        const int32_t* __restrict__ el_hood, const int64_t* __restrict__ adj_off,
                        const int32_t* __restrict__ adj, const int64_t* __restrict__ row_off,
                        uint32_t* __restrict__ row, int32_t* __restrict__ cursor,
                        const int64_t* __restrict__ rep_woff, uint32_t* __restrict__ rep_mask,
                        uint2* __restrict__ el, uint8_t* __restrict__ hood_gen, int64_t rows_min_k,
                        int64_t N_el) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N_el; e += (int64_t)gridDim.x * blockDim.x)
        mask_element(e, hood_off, hood, el_hood, adj_off, adj, row_off, row, cursor, rep_woff, rep_mask, el, hood_gen,
                     rows_min_k);
}

// slice offsets of cliques/hoods: cliques are grouped by their smallest vertex
__global__ void k_slice_hoods(const int64_t* __restrict__ cq_off, const int64_t* __restrict__ vert_off, int32_t S,
                              int64_t* __restrict__ hood_slice_off) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s <= S) hood_slice_off[s] = cq_off[vert_off[s]];
}

// first hood element of each slice (entries S+1 .. 2S+1 of the host copy)
__global__ void k_slice_elems(const int64_t* __restrict__ hood_slice_off, const int64_t* __restrict__ hood_off,
                              int32_t S, int64_t* __restrict__ el_slice_off) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s <= S) el_slice_off[s] = hood_off[hood_slice_off[s]];
}

struct Scratch {  // frees every temporary on scope exit
    cudaStream_t s;
    std::vector<void*> ptrs;
    template <typename T>
    int get(T** p, int64_t n) {
        int rc = dalloc(p, n, s);
        if (!rc) ptrs.push_back((void*)*p);
        return rc;
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
};

int check_status(pmrf_graph* g, cudaStream_t s) {
    DevStatus h;
    PMRF_CUDA(cudaMemcpyAsync(&h, g->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
    PMRF_CUDA(cudaStreamSynchronize(s));
    if (h.code != 0) {
        const char* what = "kernel error";
        switch (h.where) {
            case SITE_BAD_ID: what = "negative region id at pixel"; break;
            case SITE_NONFINITE: what = "non-finite intensity at pixel"; break;
            case SITE_DEGREE: what = "region has more neighbours than PMRF_MAX_DEGREE; vertex"; break;
            case SITE_MCE_STACK: what = "clique larger than 64 members at vertex"; break;
            case SITE_SORT: what = "duplicate values in a distinct-value segment"; break;
            default: break;
        }
        return fail(h.code, std::string(what) + " " + std::to_string(h.detail));
    }
    return PMRF_OK;
}

#define LAUNCH_1D(kern, n, ...)                                                                 \
    do {                                                                                        \
        int64_t n_ = (n);                                                                       \
        if (n_ > 0) { kern<<<(unsigned)ceil_div(n_, 256), 256, 0, s>>>(__VA_ARGS__); ::pmrf::note_launch(1); }              \
        PMRF_CUDA(cudaGetLastError());                                                          \
    } while (0)

}  // namespace

int rep_elements(pmrf_graph* g, uint32_t* d_rep_el, cudaStream_t s) {
    const int64_t V = g->V, N_el = g->N_el;
    if (N_el == 0) return PMRF_OK;
    Scratch tmp{s, {}};
    int32_t* d_cursor = nullptr;
    PMRF_TRY(tmp.get(&d_cursor, V));
    PMRF_CUDA(cudaMemsetAsync(d_cursor, 0, sizeof(int32_t) * std::max<int64_t>(V, 1), s));
    LAUNCH_1D(k_rep_fill, N_el, g->d_hood, N_el, g->d_rep_off, d_cursor, d_rep_el);
    PMRF_TRY(segmented_sort_u32(d_rep_el, g->d_rep_off, V, N_el, false, nullptr, g->d_status, s));
    return PMRF_OK;
}

// hoods of depth g->hood_depth from the 1-hoods in g->d_hood_off / g->d_hood
// (replaced); el_hood (a new scratch array), rcount and hmax recomputed
int deepen_hoods(pmrf_graph* g, Scratch* tmp, int32_t** el_hood, int32_t* rcount, int32_t* hmax, cudaStream_t s) {
    const int64_t C = g->C, V = g->V;
    for (int level = 2; level <= g->hood_depth; ++level) {
        int64_t *d_cnt = nullptr, *d_coff = nullptr, *d_noff = nullptr;
        int32_t* d_ucnt = nullptr;
        uint32_t* d_cand = nullptr;
        int32_t* d_new = nullptr;
        Scratch lv{s, {}};
        PMRF_TRY(lv.get(&d_cnt, std::max<int64_t>(C, 1)));
        PMRF_TRY(lv.get(&d_coff, C + 1));
        PMRF_TRY(lv.get(&d_ucnt, std::max<int64_t>(C, 1)));
        LAUNCH_1D(k_expand_count, C, g->d_hood_off, g->d_hood, g->d_adj_off, C, d_cnt);
        PMRF_TRY(exclusive_scan_i64(d_cnt, d_coff, C, s));
        int64_t ncand = 0;
        PMRF_TRY(read_i64(d_coff + C, &ncand, s));
        PMRF_TRY(lv.get(&d_cand, std::max<int64_t>(ncand, 1)));
        LAUNCH_1D(k_expand_fill, C, g->d_hood_off, g->d_hood, g->d_adj_off, g->d_adj, d_coff, C, d_cand);
        PMRF_TRY(segmented_sort_u32(d_cand, d_coff, C, ncand, true, d_ucnt, g->d_status, s));
        PMRF_TRY(dalloc(&d_noff, C + 1, s));
        int rc = exclusive_scan_i32_to_i64(d_ucnt, d_noff, C, s);
        int64_t n_el = 0;
        if (!rc) rc = read_i64(d_noff + C, &n_el, s);
        if (!rc && n_el >= 4294967295ll) rc = fail(PMRF_ERR_UNSUPPORTED, "more than 2^32-1 hood elements");
        if (!rc) rc = dalloc(&d_new, std::max<int64_t>(n_el, 1), s);
        if (rc) {
            dfree(d_noff, s);
            return rc;
        }
        LAUNCH_1D(k_take_unique, C, d_cand, d_coff, d_noff, C, d_new);
        dfree(g->d_hood_off, s);
        dfree(g->d_hood, s);
        g->d_hood_off = d_noff;
        g->d_hood = d_new;
        g->N_el = n_el;
    }
    PMRF_TRY(tmp->get(el_hood, std::max<int64_t>(g->N_el, 1)));
    PMRF_CUDA(cudaMemsetAsync(rcount, 0, sizeof(int32_t) * std::max<int64_t>(V, 1), s));
    PMRF_CUDA(cudaMemsetAsync(hmax, 0, sizeof(int32_t), s));
    LAUNCH_1D(k_el_hood, C, g->d_hood_off, g->d_hood, C, *el_hood, rcount, hmax);
    PMRF_TRY(check_status(g, s));
    return PMRF_OK;
}

int build_graph_impl(pmrf_graph* g, const double* d_img, const int32_t* d_ids, cudaStream_t s) {
    const int32_t S = g->S;
    Scratch tmp{s, {}};
    PMRF_TRY(dalloc(&g->d_status, 1, s));
    PMRF_CUDA(cudaMemsetAsync(g->d_status, 0, sizeof(DevStatus), s));

    // slice geometry
    int64_t maxpix = 0;
    for (int i = 0; i < S; ++i) maxpix = std::max(maxpix, g->h_pix_off[i + 1] - g->h_pix_off[i]);
    PMRF_TRY(dalloc(&g->d_pix_off, S + 1, s));
    PMRF_TRY(dalloc(&g->d_W, S, s));
    PMRF_CUDA(cudaMemcpyAsync(g->d_pix_off, g->h_pix_off.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice, s));
    PMRF_CUDA(cudaMemcpyAsync(g->d_W, g->h_W.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice, s));
    if (g->volume_depth > 1) {
        PMRF_TRY(dalloc(&g->d_layer, S, s));
        PMRF_CUDA(cudaMemcpyAsync(g->d_layer, g->h_layer.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice, s));
    }
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(maxpix, PIX_THREADS * 4), 65535));
    const dim3 pgrid(gx, (unsigned)S);

    // 1. ids checked, per-slice largest id
    int32_t* d_maxid = nullptr;
    PMRF_TRY(tmp.get(&d_maxid, S));
    PMRF_CUDA(cudaMemsetAsync(d_maxid, 0xff, sizeof(int32_t) * S, s));
    if (g->n_pix > 0) {
        const unsigned vx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(maxpix, PIX_THREADS * VAL_ITEMS), 65535));
        k_validate<<<dim3(vx, (unsigned)S), PIX_THREADS, 0, s>>>(d_ids, g->d_pix_off, d_maxid, g->d_status);
        ::pmrf::note_launch(1);
    }
    PMRF_CUDA(cudaGetLastError());
    PMRF_TRY(check_status(g, s));
    std::vector<int32_t> hmax(S);
    PMRF_CUDA(cudaMemcpyAsync(hmax.data(), d_maxid, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, s));
    PMRF_CUDA(cudaStreamSynchronize(s));
    g->h_rank_off.assign(S + 1, 0);
    for (int i = 0; i < S; ++i) g->h_rank_off[i + 1] = g->h_rank_off[i] + (int64_t)hmax[i] + 1;
    g->n_rank = g->h_rank_off[S];
    PMRF_TRY(dalloc(&g->d_rank_off, S + 1, s));
    PMRF_CUDA(cudaMemcpyAsync(g->d_rank_off, g->h_rank_off.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice, s));

    // 2. pixel counts and boxes per raw id; compact ids -> global vertex ids
    int32_t* d_npix_raw = nullptr;
    int4* d_bbox_raw = nullptr;
    PMRF_TRY(tmp.get(&d_npix_raw, g->n_rank));
    PMRF_TRY(tmp.get(&d_bbox_raw, g->n_rank));
    PMRF_CUDA(cudaMemsetAsync(d_npix_raw, 0, sizeof(int32_t) * std::max<int64_t>(g->n_rank, 1), s));
    LAUNCH_1D(k_init_bbox, g->n_rank, d_bbox_raw, g->n_rank);
    if (g->n_pix > 0) {
        // four rounds of the grid per block (longer blocks: 1.87 -> 1.76 ms on stack512)
        k_count_raw<<<dim3(std::max(1u, gx / 4), (unsigned)S), PIX_THREADS, 0, s>>>(d_ids, g->d_pix_off, g->d_W,
                                                                                 g->d_rank_off, d_npix_raw, d_bbox_raw);
        ::pmrf::note_launch(1);
    }
    PMRF_CUDA(cudaGetLastError());
    PMRF_TRY(dalloc(&g->d_rank, g->n_rank, s));
    LAUNCH_1D(k_present, g->n_rank, d_npix_raw, g->n_rank, g->d_rank);
    int64_t* d_ex = nullptr;
    PMRF_TRY(tmp.get(&d_ex, g->n_rank + 1));
    PMRF_TRY(exclusive_scan_i32_to_i64(g->d_rank, d_ex, g->n_rank, s));
    LAUNCH_1D(k_rank, g->n_rank, g->d_rank, d_ex, g->n_rank);
    PMRF_TRY(dalloc(&g->d_vert_off, S + 1, s));
    k_vert_off<<<(unsigned)ceil_div(S + 1, 256), 256, 0, s>>>(d_ex, g->d_rank_off, S, g->d_vert_off); ::pmrf::note_launch(1);
    PMRF_CUDA(cudaGetLastError());
    g->h_vert_off.assign(S + 1, 0);
    PMRF_CUDA(cudaMemcpyAsync(g->h_vert_off.data(), g->d_vert_off, sizeof(int64_t) * (S + 1), cudaMemcpyDeviceToHost, s));
    PMRF_CUDA(cudaStreamSynchronize(s));
    const int64_t V = g->h_vert_off[S];
    g->V = V;
    if (V >= 2147483647ll) return fail(PMRF_ERR_UNSUPPORTED, "more than 2^31-1 regions");

    // 3. region means (row-major order per region) and neighbours: one
    //    bounding-box scan per compact region; sorted pixel lists (means) and
    //    pixel-pair candidates (adjacency) for the regions it cannot take
    PMRF_TRY(dalloc(&g->d_npix, V, s));
    PMRF_TRY(dalloc(&g->d_y, V, s));
    int64_t* d_vpix_off = nullptr;
    int32_t* d_cursor = nullptr;
    int32_t *d_inv = nullptr, *d_fbpix = nullptr, *d_fbadj = nullptr, *d_deg = nullptr, *d_nbr = nullptr;
    PMRF_TRY(tmp.get(&d_vpix_off, V + 1));
    PMRF_TRY(tmp.get(&d_cursor, V));
    PMRF_TRY(tmp.get(&d_inv, V));
    PMRF_TRY(tmp.get(&d_fbpix, V));
    PMRF_TRY(tmp.get(&d_fbadj, V));
    PMRF_TRY(tmp.get(&d_deg, V));
    PMRF_TRY(tmp.get(&d_nbr, V * NB_CAP));
    LAUNCH_1D(k_inv_rank, g->n_rank, g->d_rank, g->d_rank_off, S, g->n_rank, d_inv);
    LAUNCH_1D(k_region_scan, V, d_img, d_ids, g->d_pix_off, g->d_W, g->d_vert_off, g->d_rank_off, g->d_rank, S, d_inv,
              d_bbox_raw, d_npix_raw, V, g->d_y, g->d_npix, d_fbpix, d_fbadj, d_deg, d_nbr, g->d_status);
    // a volume's z-neighbours lie outside the bounding-box scan: every region
    // of a 3-D volume takes the pixel-pair path below
    if (g->volume_depth > 1) LAUNCH_1D(k_flag_all, V, d_fbadj, V);
    // pixels of the regions whose mean needs a sorted pixel list, regions whose
    // adjacency needs the pixel pairs (both usually none: no scan then)
    int64_t nfb = 0, nfa = 0;
    {
        unsigned long long* d_sums = nullptr;
        PMRF_TRY(tmp.get(&d_sums, 2));
        PMRF_CUDA(cudaMemsetAsync(d_sums, 0, 2 * sizeof(unsigned long long), s));
        if (V > 0) {
            k_sum2<<<(unsigned)std::min<int64_t>(ceil_div(V, SUM_THREADS), 1184), SUM_THREADS, 0, s>>>(d_fbpix, d_fbadj,
                                                                                                     V, d_sums);
            ::pmrf::note_launch(1);
        }
        PMRF_CUDA(cudaGetLastError());
        unsigned long long h2[2] = {0, 0};
        PMRF_CUDA(cudaMemcpyAsync(h2, d_sums, sizeof(h2), cudaMemcpyDeviceToHost, s));
        PMRF_CUDA(cudaStreamSynchronize(s));
        nfb = (int64_t)h2[0];
        nfa = (int64_t)h2[1];
    }
    if (nfb > 0) {
        PMRF_TRY(exclusive_scan_i32_to_i64(d_fbpix, d_vpix_off, V, s));
        uint32_t* d_pixlist = nullptr;
        PMRF_TRY(tmp.get(&d_pixlist, nfb));
        PMRF_CUDA(cudaMemsetAsync(d_cursor, 0, sizeof(int32_t) * std::max<int64_t>(V, 1), s));
        k_fill_pix<<<pgrid, PIX_THREADS, 0, s>>>(d_ids, g->d_pix_off, g->d_rank_off, g->d_rank, d_vpix_off, d_cursor,
                                                 d_pixlist, d_fbpix);
        ::pmrf::note_launch(1);
        PMRF_CUDA(cudaGetLastError());
        PMRF_TRY(segmented_sort_u32(d_pixlist, d_vpix_off, V, nfb, false, nullptr, g->d_status, s));
        LAUNCH_1D(k_means, V, d_img, d_pixlist, d_vpix_off, V, g->d_y, g->d_status);
    }

    // 4. adjacency: the scans' neighbour lists, and for the flagged regions the
    //    4-connected pixel pairs they take part in, sorted and de-duplicated
    int64_t* d_cand_off = nullptr;
    uint32_t* d_cand = nullptr;
    PMRF_TRY(tmp.get(&d_cand_off, V + 1));
    if (nfa > 0 && g->n_pix > 0) {
        int32_t* d_cnt = nullptr;
        PMRF_TRY(tmp.get(&d_cnt, V));
        PMRF_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(int32_t) * std::max<int64_t>(V, 1), s));
        k_edge_pairs<false><<<pgrid, PIX_THREADS, 0, s>>>(d_ids, g->d_pix_off, g->d_W, g->d_layer, g->d_rank_off,
                                                         g->d_rank,
                                                         d_fbadj, d_cnt, nullptr, nullptr, nullptr);
        ::pmrf::note_launch(1);
        PMRF_CUDA(cudaGetLastError());
        PMRF_TRY(exclusive_scan_i32_to_i64(d_cnt, d_cand_off, V, s));
        int64_t ncand = 0;
        PMRF_TRY(read_i64(d_cand_off + V, &ncand, s));
        PMRF_TRY(tmp.get(&d_cand, ncand));
        PMRF_CUDA(cudaMemsetAsync(d_cursor, 0, sizeof(int32_t) * std::max<int64_t>(V, 1), s));
        k_edge_pairs<true><<<pgrid, PIX_THREADS, 0, s>>>(d_ids, g->d_pix_off, g->d_W, g->d_layer, g->d_rank_off,
                                                        g->d_rank,
                                                        d_fbadj, nullptr, d_cand_off, d_cursor, d_cand);
        ::pmrf::note_launch(1);
        PMRF_CUDA(cudaGetLastError());
        PMRF_TRY(segmented_sort_u32(d_cand, d_cand_off, V, ncand, true, d_cnt, g->d_status, s));
        LAUNCH_1D(k_take_counts, V, d_fbadj, d_cnt, V, d_deg);
    }
    int32_t* d_dmax = nullptr;
    PMRF_TRY(tmp.get(&d_dmax, 1));
    PMRF_CUDA(cudaMemsetAsync(d_dmax, 0, sizeof(int32_t), s));
    if (V > 0) {
        k_check_degree<<<(unsigned)std::min<int64_t>(ceil_div(V, CD_THREADS), 1184), CD_THREADS, 0, s>>>(
            d_deg, V, (int32_t)PMRF_MAX_DEGREE, g->d_status, d_dmax);
        ::pmrf::note_launch(1);
    }
    PMRF_CUDA(cudaGetLastError());
    PMRF_TRY(check_status(g, s));
    PMRF_TRY(dalloc(&g->d_adj_off, V + 1, s));
    PMRF_TRY(exclusive_scan_i32_to_i64(d_deg, g->d_adj_off, V, s));
    PMRF_TRY(read_i64(g->d_adj_off + V, &g->E2, s));
    PMRF_CUDA(cudaMemcpyAsync(&g->max_deg, d_dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PMRF_TRY(dalloc(&g->d_adj, g->E2, s));
    LAUNCH_1D(k_adj_fill, V, d_fbadj, d_nbr, d_cand, d_cand_off, g->d_adj_off, V, g->d_adj);

    // 5. maximal cliques
    int64_t *d_ncl = nullptr, *d_nmem = nullptr, *d_cq_off = nullptr, *d_mem_off = nullptr;
    PMRF_TRY(tmp.get(&d_ncl, V));
    PMRF_TRY(tmp.get(&d_nmem, V));
    PMRF_TRY(tmp.get(&d_cq_off, V + 1));
    PMRF_TRY(tmp.get(&d_mem_off, V + 1));
    // general-degree vertices
    int64_t* d_glist = nullptr;
    int32_t* d_ng = nullptr;
    PMRF_TRY(tmp.get(&d_glist, V));
    PMRF_TRY(tmp.get(&d_ng, 1));
    PMRF_CUDA(cudaMemsetAsync(d_ng, 0, sizeof(int32_t), s));
    LAUNCH_1D(k_list_general, V, g->d_adj_off, V, d_glist, d_ng);
    int32_t ng = 0;
    PMRF_CUDA(cudaMemcpyAsync(&ng, d_ng, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PMRF_CUDA(cudaStreamSynchronize(s));
    int64_t* d_gscr_off = nullptr;
    uint64_t* d_gscr = nullptr;
    int64_t* d_gmask_off = nullptr;
    uint64_t* d_gmask = nullptr;
    std::vector<int64_t> hgl, hdeg;
    if (ng > 0) {
        // general vertices sorted for determinism of the scratch layout
        hgl.resize(ng);
        PMRF_CUDA(cudaMemcpyAsync(hgl.data(), d_glist, sizeof(int64_t) * ng, cudaMemcpyDeviceToHost, s));
        std::vector<int64_t> hoff(V + 1);
        PMRF_CUDA(cudaMemcpyAsync(hoff.data(), g->d_adj_off, sizeof(int64_t) * (V + 1), cudaMemcpyDeviceToHost, s));
        PMRF_CUDA(cudaStreamSynchronize(s));
        std::sort(hgl.begin(), hgl.end());
        std::vector<int64_t> so(ng + 1, 0);
        for (int k = 0; k < ng; ++k) {
            int64_t d = hoff[hgl[k] + 1] - hoff[hgl[k]];
            int64_t nw = ceil_div(d, 64);
            so[k + 1] = so[k] + d * nw + (int64_t)(MAX_CLIQUE + 1) * 4 * nw + 2 * nw;
        }
        PMRF_CUDA(cudaMemcpyAsync(d_glist, hgl.data(), sizeof(int64_t) * ng, cudaMemcpyHostToDevice, s));
        PMRF_TRY(tmp.get(&d_gscr_off, ng + 1));
        PMRF_TRY(tmp.get(&d_gscr, so[ng]));
        PMRF_CUDA(cudaMemcpyAsync(d_gscr_off, so.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice, s));
        hdeg.swap(so);  // keep the host vector alive until the copy has run
        PMRF_CUDA(cudaStreamSynchronize(s));
    }
    uint64_t* d_cq_kept = nullptr;
    PMRF_TRY(tmp.get(&d_cq_kept, V * CQ_KEEP));
    LAUNCH_1D(k_cliques_fast, V, g->d_adj_off, g->d_adj, V, 0, d_ncl, d_nmem, nullptr, nullptr, nullptr, nullptr,
              nullptr, g->d_status, d_cq_kept);
    if (ng > 0)
        LAUNCH_1D(k_cliques_general, ng, g->d_adj_off, g->d_adj, d_glist, (int64_t)ng, d_gscr_off, d_gscr, 0, d_ncl,
                  d_nmem, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, g->d_status);
    PMRF_TRY(check_status(g, s));
    PMRF_TRY(exclusive_scan_i64(d_ncl, d_cq_off, V, s));
    PMRF_TRY(exclusive_scan_i64(d_nmem, d_mem_off, V, s));
    PMRF_TRY(read_i64(d_cq_off + V, &g->C, s));
    PMRF_TRY(read_i64(d_mem_off + V, &g->n_clq, s));
    const int64_t C = g->C;
    uint64_t* d_maskbuf = nullptr;
    PMRF_TRY(tmp.get(&d_maskbuf, C));
    if (ng > 0) {
        std::vector<int64_t> hncl(ng), mo(ng + 1, 0);
        for (int k = 0; k < ng; ++k) {
            PMRF_CUDA(cudaMemcpyAsync(&hncl[k], d_ncl + hgl[k], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        }
        std::vector<int64_t> hoff2(V + 1);
        PMRF_CUDA(cudaMemcpyAsync(hoff2.data(), g->d_adj_off, sizeof(int64_t) * (V + 1), cudaMemcpyDeviceToHost, s));
        PMRF_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < ng; ++k) mo[k + 1] = mo[k] + hncl[k] * ceil_div(hoff2[hgl[k] + 1] - hoff2[hgl[k]], 64);
        PMRF_TRY(tmp.get(&d_gmask_off, ng + 1));
        PMRF_TRY(tmp.get(&d_gmask, mo[ng]));
        PMRF_CUDA(cudaMemcpyAsync(d_gmask_off, mo.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice, s));
        PMRF_CUDA(cudaStreamSynchronize(s));
    }
    PMRF_TRY(dalloc(&g->d_clq_off, C + 1, s));
    PMRF_TRY(dalloc(&g->d_clq, g->n_clq, s));
    LAUNCH_1D(k_cliques_fast, V, g->d_adj_off, g->d_adj, V, 1, d_ncl, d_nmem, d_cq_off, d_mem_off, d_maskbuf,
              g->d_clq_off, g->d_clq, g->d_status, d_cq_kept);
    if (ng > 0)
        LAUNCH_1D(k_cliques_general, ng, g->d_adj_off, g->d_adj, d_glist, (int64_t)ng, d_gscr_off, d_gscr, 1, d_ncl,
                  d_nmem, d_cq_off, d_gmask_off, d_gmask, d_mem_off, g->d_clq_off, g->d_clq, g->d_status);
    PMRF_CUDA(cudaMemcpyAsync(g->d_clq_off + C, &g->n_clq, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    PMRF_TRY(dalloc(&g->d_hood_slice_off, S + 1, s));
    k_slice_hoods<<<(unsigned)ceil_div(S + 1, 256), 256, 0, s>>>(d_cq_off, g->d_vert_off, S, g->d_hood_slice_off); ::pmrf::note_launch(1);
    PMRF_CUDA(cudaGetLastError());
    PMRF_TRY(check_status(g, s));

    // 6. hoods (and, while filling them, each element's hood and each vertex's
    //    number of replicas)
    int32_t *d_hsize = nullptr, *d_hmax = nullptr;
    PMRF_TRY(tmp.get(&d_hsize, C));
    PMRF_TRY(tmp.get(&d_hmax, 1));
    PMRF_CUDA(cudaMemsetAsync(d_hmax, 0, sizeof(int32_t), s));
    int32_t* d_hood_kept = nullptr;
    PMRF_TRY(tmp.get(&d_hood_kept, C * HOOD_KEEP));
    LAUNCH_1D(k_hood_merge<false>, C, g->d_clq_off, g->d_clq, g->d_adj_off, g->d_adj, C, d_hsize, d_hmax, nullptr,
              nullptr, nullptr, nullptr, d_hood_kept);
    PMRF_TRY(dalloc(&g->d_hood_off, C + 1, s));
    PMRF_TRY(exclusive_scan_i32_to_i64(d_hsize, g->d_hood_off, C, s));
    PMRF_TRY(read_i64(g->d_hood_off + C, &g->N_el, s));
    const int64_t N_el = g->N_el;
    if (N_el >= 4294967295ll) return fail(PMRF_ERR_UNSUPPORTED, "more than 2^32-1 hood elements");
    PMRF_TRY(dalloc(&g->d_hood, N_el, s));
    int32_t *d_el_hood = nullptr, *d_rcount = nullptr;
    PMRF_TRY(tmp.get(&d_el_hood, N_el));
    PMRF_TRY(tmp.get(&d_rcount, V));
    PMRF_CUDA(cudaMemsetAsync(d_rcount, 0, sizeof(int32_t) * std::max<int64_t>(V, 1), s));
    LAUNCH_1D(k_hood_merge<true>, C, g->d_clq_off, g->d_clq, g->d_adj_off, g->d_adj, C, nullptr, nullptr,
              g->d_hood_off, g->d_hood, d_el_hood, d_rcount, d_hood_kept);
    if (g->hood_depth > 1) PMRF_TRY(deepen_hoods(g, &tmp, &d_el_hood, d_rcount, d_hmax, s));

    // 7. replica offsets and masks
    PMRF_TRY(dalloc(&g->d_rep_off, V + 1, s));
    PMRF_TRY(exclusive_scan_i32_to_i64(d_rcount, g->d_rep_off, V, s));
    int64_t* d_nw = nullptr;
    PMRF_TRY(tmp.get(&d_nw, std::max(C, V)));
    // with every degree <= 32 no hood is read through its local adjacency
    // rows (the hood pass's fast path takes every hood), and every replica's
    // slot mask is one word that k_masks writes in full
    const bool deg32 = g->max_deg <= 32;
    const int64_t rows_min_k = deg32 ? INT64_MAX : 0;
    PMRF_TRY(dalloc(&g->d_row_off, C + 1, s));
    if (deg32) {
        PMRF_CUDA(cudaMemsetAsync(g->d_row_off, 0, sizeof(int64_t) * (C + 1), s));
        g->n_row_words = 0;
    } else {
        LAUNCH_1D(k_row_words, C, g->d_hood_off, C, rows_min_k, d_nw);
        PMRF_TRY(exclusive_scan_i64(d_nw, g->d_row_off, C, s));
        PMRF_TRY(read_i64(g->d_row_off + C, &g->n_row_words, s));
    }
    PMRF_TRY(dalloc(&g->d_rep_woff, V + 1, s));
    LAUNCH_1D(k_rep_words, V, g->d_adj_off, d_rcount, V, d_nw);
    PMRF_TRY(exclusive_scan_i64(d_nw, g->d_rep_woff, V, s));
    PMRF_TRY(read_i64(g->d_rep_woff + V, &g->n_rep_words, s));
    PMRF_TRY(dalloc(&g->d_row, g->n_row_words, s));
    PMRF_TRY(dalloc(&g->d_rep_mask, g->n_rep_words, s));
    PMRF_TRY(dalloc(&g->d_el, g->N_el, s));
    PMRF_CUDA(cudaMemsetAsync(g->d_row, 0, sizeof(uint32_t) * std::max<int64_t>(g->n_row_words, 1), s));
    if (!deg32)
        PMRF_CUDA(cudaMemsetAsync(g->d_rep_mask, 0, sizeof(uint32_t) * std::max<int64_t>(g->n_rep_words, 1), s));
    PMRF_CUDA(cudaMemsetAsync(d_cursor, 0, sizeof(int32_t) * std::max<int64_t>(V, 1), s));
    PMRF_TRY(dalloc(&g->d_hood_gen, C, s));
    PMRF_CUDA(cudaMemsetAsync(g->d_hood_gen, 0, std::max<int64_t>(C, 1), s));
    LAUNCH_1D(k_masks, ceil_div(g->N_el, MK_ROUNDS), g->d_hood_off, g->d_hood, d_el_hood, g->d_adj_off, g->d_adj,
              g->d_row_off, g->d_row, d_cursor, g->d_rep_woff, g->d_rep_mask, g->d_el, g->d_hood_gen, rows_min_k,
              g->N_el);
    PMRF_CUDA(cudaMemcpyAsync(&g->max_hood, d_hmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));

    // slice offsets of hoods and elements (host copies, one transfer)
    int64_t* d_el_slice_off = nullptr;
    PMRF_TRY(tmp.get(&d_el_slice_off, S + 1));
    LAUNCH_1D(k_slice_elems, S + 1, g->d_hood_slice_off, g->d_hood_off, S, d_el_slice_off);
    std::vector<int64_t> both(2 * (size_t)(S + 1));
    PMRF_CUDA(cudaMemcpyAsync(both.data(), g->d_hood_slice_off, sizeof(int64_t) * (S + 1), cudaMemcpyDeviceToHost, s));
    PMRF_CUDA(cudaMemcpyAsync(both.data() + (S + 1), d_el_slice_off, sizeof(int64_t) * (S + 1),
                              cudaMemcpyDeviceToHost, s));
    PMRF_TRY(check_status(g, s));  // synchronises the stream
    g->h_hood_slice_off.assign(both.begin(), both.begin() + (S + 1));
    g->h_el_slice_off.assign(both.begin() + (S + 1), both.end());
    return PMRF_OK;
}

}  // namespace pmrf
