/*
 * pmrf.h -- C ABI of the B300 (sm_103a) MRF region-labelling engine.
 *
 * The engine implements the optimisation path of DPP-PMRF (Lessley et al.,
 * "DPP-PMRF: Rethinking Optimization for a Probabilistic Graphical Model Using
 * Data-Parallel Primitives", LDAV 2018): the region graph of an
 * oversegmented image (Section 2.1, Algorithm 2 step 1), its maximal cliques
 * (Algorithm 2 step 2), their 1-neighbourhoods ("hoods", Section 3.1 and
 * Section 3.2.2 "Construction of Neighborhoods"), and the EM loop of
 * Algorithm 2 steps 6-11 (Section 3.2.2 "EM Parameter Estimation"): a MAP sweep
 * over every (hood, vertex, label) tuple, a per-element argmin, a reduction
 * over each vertex's replicas, re-estimation of the per-label mean, standard
 * deviation and energy, and the hood / total convergence tests.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE memory owned by the caller (the engine
 *     never frees them); h_* are HOST memory owned by the caller.  All device
 *     buffers must be on the device the graph was built on.
 *   - Work is enqueued on the caller's stream `stream` (NULL = legacy default
 *     stream) and is stream-ordered; an entry point returns before the device
 *     work has finished unless its comment says it synchronises.
 *   - The return value is a pmrf_status; PMRF_OK = 0.  On failure nothing is
 *     written to the caller's output buffers that the caller may rely on, and
 *     pmrf_last_error() returns a message for the calling thread.  Errors that
 *     a kernel detects (e.g. a hood wider than a supported limit) are recorded
 *     in a per-graph device status word and reported by pmrf_sync_status().
 *   - No entry point throws; no entry point traps, faults or spins without a
 *     bound on the device.
 *   - Floating point is IEEE binary64 for intensities, energies and parameters.
 *   - Vertex ids are global across the slices of a batch: slice s owns vertices
 *     [vert_off[s], vert_off[s+1]) (pmrf_graph_get, PMRF_ARR_VERT_OFF).
 *
 * Limits: total pixels < 2^32; total regions < 2^31; total hood elements
 * < 2^32; 1 <= n_labels <= PMRF_MAX_LABELS; a region may touch at most
 * PMRF_MAX_DEGREE others.
 */
#ifndef PMRF_H
#define PMRF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PMRF_API __attribute__((visibility("default")))
#else
#define PMRF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* CUDA stream handle (identical to cudaStream_t; declared here so that this
 * header does not need the CUDA headers). */
typedef struct CUstream_st* pmrf_stream_t;

typedef enum {
    PMRF_OK = 0,
    PMRF_ERR_ARG = 1,         /* invalid argument (null pointer, bad size, bad id) */
    PMRF_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    PMRF_ERR_OOM = 3,         /* device allocation failed */
    PMRF_ERR_NONFINITE = 4,   /* NaN or infinite intensity */
    PMRF_ERR_TIMEOUT = 5,     /* a bounded device wait ran out */
    PMRF_ERR_UNSUPPORTED = 6, /* input beyond a documented limit */
    PMRF_ERR_DEVICE = 7       /* a kernel recorded an internal error */
} pmrf_status;

#define PMRF_MAX_LABELS 8
#define PMRF_MAX_DEGREE 4096

/* Opaque graph: owns its device arrays (region map, CSR adjacency, cliques,
 * hoods, replica structures) and the EM workspace. */
typedef struct pmrf_graph pmrf_graph;

/*
 * EM configuration.  Defaults (pmrf_config_default): n_labels 2, beta 1,
 * max_iters 20 (Section 3.2.2: most runs converge within 20 iterations),
 * conv_window 3 and conv_tol 1e-4 (Section 3.2.2, MAP convergence check: the
 * change over the previous 3 iterations below 1.0e-4), sigma_min 1e-6,
 * threshold initialisation on [init_lo, init_hi] = [0, 1].
 *
 * init_from_labels = 0: labels start as the threshold of the region means:
 *   x_v = clamp(floor((y_v - init_lo) / (init_hi - init_lo) * n_labels), 0, L-1)
 *   (the paper draws random labels and parameters, Algorithm 2 step 3; the
 *   threshold start replaces that draw).
 * init_from_labels = 1: d_labels holds the starting labels (resume).
 * With 0 or 1 the starting parameters are the label-conditional moments of the
 * starting labels; a label with no vertex starts at the centre of its
 * threshold bin with sigma equal to the bin width.
 * init_from_labels = 2: d_labels holds the starting labels and d_params the
 *   starting parameters ([S][L][4]; mu and sigma at entries 1 and 2, sigma
 *   floored at sigma_min), e.g. the paper's random start from
 *   pmrf_random_init.
 *
 * Variants of the sweep (the paper fixes neither choice; default 0 = the
 * reading used throughout, Section 3.2.2 EM steps 2-3):
 * potts_scope  PMRF_SCOPE_HOOD: the Potts penalty of vertex v in hood c counts
 *              the neighbours of v inside c; PMRF_SCOPE_FULL: all neighbours
 *              of v (every replica of v then carries the same energies).
 * replica_rule how the replicas of v (one per hood holding v) give v its
 *              label and energy E*_v.  PMRF_RULE_MIN: the replica of least
 *              energy (lower label on ties); PMRF_RULE_SUM: the label of least
 *              mean energy over the replicas, E*_v that mean; PMRF_RULE_VOTE:
 *              each replica votes for its least-energy label, the label with
 *              most votes wins (lower label on ties), E*_v is the least energy
 *              among the replicas that voted for it.
 * The hood energy sums do not depend on the replica rule.
 *
 * Ranges (PMRF_ERR_ARG otherwise): 1 <= n_labels <= PMRF_MAX_LABELS,
 * 0 <= beta < 2^32, sigma_min > 0, init_hi > init_lo, conv_window >= 1,
 * max_iters >= 1, init_from_labels in {0, 1, 2}.
 */
#define PMRF_SCOPE_HOOD 0
#define PMRF_SCOPE_FULL 1
#define PMRF_RULE_MIN 0
#define PMRF_RULE_SUM 1
#define PMRF_RULE_VOTE 2
typedef struct {
    int32_t n_labels;
    int32_t max_iters;
    int32_t conv_window;
    int32_t init_from_labels;
    int32_t potts_scope;
    int32_t replica_rule;
    double beta;
    double conv_tol;
    double sigma_min;
    double init_lo;
    double init_hi;
} pmrf_config;

/* Fill *cfg with the defaults listed above.  Returns PMRF_ERR_ARG on NULL. */
PMRF_API int pmrf_config_default(pmrf_config* cfg);

/* Message describing the calling thread's last failed call ("" if none).  The
 * string stays valid until the thread's next call into the library. */
PMRF_API const char* pmrf_last_error(void);

/* Number of kernels this library has launched in this process so far (a
 * replay of a captured EM loop counts every kernel node it runs; the kernels
 * of its conditional loop body are counted on the device, so this
 * call synchronises every device on which an EM loop was captured). */
PMRF_API int64_t pmrf_launch_count(void);

/* Version string of the library build. */
PMRF_API const char* pmrf_version(void);

/*
 * Device memory.  Every device array the library allocates comes from one
 * stream-ordered memory pool per device, owned by the library and created on
 * first use.  Memory freed into it (a destroyed graph, build temporaries)
 * stays mapped, so the next build of a batch of similar size reuses it.  The
 * paper has no counterpart: this is memory management of this implementation.
 *
 * pmrf_trim_memory: synchronise the current device, then return the pool's
 *   unused memory to the driver, keeping at least keep_bytes (>= 0; 0 returns
 *   all of it) reserved.  Arrays of live graphs are not touched.
 * pmrf_memory_usage: bytes the current device's pool has reserved from the
 *   driver and bytes of it in use by live allocations (either pointer may be
 *   NULL).
 * Both return PMRF_OK or PMRF_ERR_CUDA (no device, pool creation failed).
 */
PMRF_API int pmrf_trim_memory(int64_t keep_bytes);
PMRF_API int pmrf_memory_usage(int64_t* reserved_bytes, int64_t* used_bytes);

/*
 * Build the region graph, maximal cliques, hoods and replica structures of a
 * batch of slices (Algorithm 2 steps 1, 2, 4 and 5; Sections 2.1, 3.1,
 * 3.2.1, 3.2.2 "Construction of Neighborhoods").
 *
 *   d_image      f64, the slices' pixels concatenated, each slice row-major
 *                (slice s has h_heights[s] * h_widths[s] pixels).
 *   d_region_ids i32, same layout: the oversegmentation, any non-negative id
 *                per pixel.  Within a slice, ids are compacted in ascending
 *                order: vertex vert_off[s] + k is the k-th smallest id present.
 *   n_slices     >= 1;  h_heights, h_widths: host arrays of n_slices >= 0.
 *   out          receives the new graph (destroy with pmrf_graph_destroy).
 *
 * Regions are vertices; two regions are adjacent when some horizontally or
 * vertically neighbouring pixel pair carries their two ids.  The region value
 * y_v is the mean of the region's pixels, summed in row-major order.  Cliques:
 * every maximal clique, members ascending, cliques in lexicographic order.
 * Hood c = clique c plus all neighbours of its members, ascending.
 *
 * Synchronises `stream` (array sizes are read back to size the allocations).
 * Errors: PMRF_ERR_ARG (null pointers, negative id, n_slices < 1, sizes),
 * PMRF_ERR_NONFINITE (NaN/inf pixel), PMRF_ERR_UNSUPPORTED (a region with more
 * than PMRF_MAX_DEGREE neighbours, or a limit above), PMRF_ERR_OOM,
 * PMRF_ERR_CUDA.  On error *out is left NULL and nothing is leaked.
 */
/*
 * Build options (pmrf_build_graph_ex).
 * hood_depth  k of the k-neighbourhoods (Section 3.1: a neighbourhood holds
 *             the vertices of a maximal clique and every vertex within k edges
 *             of any of them; the paper's study uses k = 1, the default).  In
 *             [1, PMRF_MAX_HOOD_DEPTH].  With k > 1, "hood" everywhere below
 *             means the k-neighbourhood (energies, replicas, sums).
 * volume_depth D >= 1.  1 (default): every slice is its own 2-D image.
 *             D > 1: every D consecutive slices (n_slices a multiple of D,
 *             the D slices of equal height and width) are the layers of one
 *             3-D volume (the paper's future work, Section 6): voxels are
 *             6-connected (neighbours along x, y and z), a region may span
 *             layers, its value is the mean of its voxels in storage order,
 *             and the graph's "slices" are the volumes (S = n_slices / D; the
 *             per-slice outputs of pmrf_em, pmrf_pll, pmrf_quality are per
 *             volume).  Region ids are per volume.
 */
#define PMRF_MAX_HOOD_DEPTH 8
typedef struct {
    int32_t hood_depth;
    int32_t volume_depth;
} pmrf_build_options;

/* Fill *opt with the defaults (hood_depth 1, volume_depth 1).  PMRF_ERR_ARG
 * on NULL. */
PMRF_API int pmrf_build_options_default(pmrf_build_options* opt);

/* pmrf_build_graph with options (NULL = the defaults); the same arguments,
 * ownership and errors, plus PMRF_ERR_ARG for an option out of range. */
PMRF_API int pmrf_build_graph_ex(const double* d_image, const int32_t* d_region_ids, int32_t n_slices,
                                 const int64_t* h_heights, const int64_t* h_widths, const pmrf_build_options* opt,
                                 pmrf_stream_t stream, pmrf_graph** out);

PMRF_API int pmrf_build_graph(const double* d_image, const int32_t* d_region_ids, int32_t n_slices,
                     const int64_t* h_heights, const int64_t* h_widths, pmrf_stream_t stream,
                     pmrf_graph** out);

/* Free a graph and its device memory (NULL is accepted).  Synchronises the
 * device work that used the graph.  The memory returns to the library's pool,
 * so a batch built after its predecessor's graph is freed reuses the same
 * memory (for a stream of same-sized batches, freeing the previous graph
 * before the next build made that build faster: 19.5 against 23.3 ms on
 * 512 slices of 1024x1024). */
PMRF_API int pmrf_graph_destroy(pmrf_graph* g);

/* Totals of a graph: vertices, undirected edges, maximal cliques (= hoods),
 * hood elements (sum of hood sizes).  Any output may be NULL. */
PMRF_API int pmrf_graph_stats(const pmrf_graph* g, int64_t* n_slices, int64_t* V, int64_t* E, int64_t* C,
                     int64_t* N_el);

/* Arrays that pmrf_graph_get can copy out. */
typedef enum {
    PMRF_ARR_VERT_OFF = 0,  /* i64 [S+1]  first vertex of each slice            */
    PMRF_ARR_HOOD_SLICE_OFF,/* i64 [S+1]  first clique/hood of each slice        */
    PMRF_ARR_Y,             /* f64 [V]    region means                           */
    PMRF_ARR_NPIX,          /* i32 [V]    pixels per region                      */
    PMRF_ARR_ADJ_OFF,       /* i64 [V+1]  CSR offsets                            */
    PMRF_ARR_ADJ,           /* i32 [2E]   neighbours, ascending per vertex       */
    PMRF_ARR_CLQ_OFF,       /* i64 [C+1]                                          */
    PMRF_ARR_CLQ,           /* i32 [..]   clique members                         */
    PMRF_ARR_HOOD_OFF,      /* i64 [C+1]                                          */
    PMRF_ARR_HOOD,          /* i32 [N_el] hood members (element order)           */
    PMRF_ARR_REP_OFF,       /* i64 [V+1]  replicas (hoods containing v) per vertex */
    PMRF_ARR_REP_HOOD,      /* i32 [N_el] hood of each replica, ascending per vertex */
    PMRF_ARR_RANK_OFF,      /* i64 [S+1]  offsets of each slice's id map         */
    PMRF_ARR_RANK,          /* i32 [..]   global vertex of each raw id, -1 absent */
    PMRF_ARR_COUNT
} pmrf_array;

/* Number of elements of array `which`. */
PMRF_API int pmrf_graph_len(const pmrf_graph* g, int32_t which, int64_t* n);

/* Copy array `which` into dst (host memory if to_host != 0, else device
 * memory); dst_bytes must hold the whole array.  Synchronises `stream`. */
PMRF_API int pmrf_graph_get(const pmrf_graph* g, int32_t which, void* dst, size_t dst_bytes, int32_t to_host,
                   pmrf_stream_t stream);

/*
 * Initial labels (Algorithm 2 step 3, threshold form, see pmrf_config):
 * d_labels u8 [V].
 */
PMRF_API int pmrf_init_labels(pmrf_graph* g, const pmrf_config* cfg, uint8_t* d_labels, pmrf_stream_t stream);

/*
 * The paper's random start (Algorithm 2 step 3; Section 3.2.2: label means and
 * deviations drawn between 0 and 255, every vertex label drawn at random),
 * for pmrf_em with init_from_labels = 2.  Draws from SplitMix64 (Steele, Lea,
 * Flood, OOPSLA 2014) used as a counter-based generator, sm(key, i) = the
 * output of the (i+1)-th step from state key: for slice s, kx = sm(seed, 2s),
 * kt = sm(seed, 2s+1); vertex v (index within its slice) gets label
 * (hi32(sm(kx, v)) * n_labels) >> 32; label l gets mu = lo + (hi-lo)*u(sm(kt, 2l))
 * and sigma = lo + (hi-lo)*u(sm(kt, 2l+1)) with u(r) = (r >> 11) * 2^-53
 * (each operation rounded once).
 *   d_labels u8 [V]; d_params f64 [S][n_labels][4] = (0, mu, sigma, 0).
 * Caller-owned device buffers, written on the stream.  n_labels outside
 * [1, PMRF_MAX_LABELS], lo > hi, a non-finite bound or a NULL pointer:
 * PMRF_ERR_ARG.
 */
PMRF_API int pmrf_random_init(pmrf_graph* g, int32_t n_labels, uint64_t seed, double lo, double hi,
                              uint8_t* d_labels, double* d_params, pmrf_stream_t stream);

/*
 * Parameter update (Section 3.2.2, EM step 4 "Update Parameters"), per slice
 * and label: n_l = number of vertices with label l, mu_l their mean
 * intensity, sigma_l = max(sigma_min, population standard deviation), U_l =
 * sum of their vertex energies (0 when d_vertex_energy is NULL).  A label with
 * no vertex keeps mu and sigma from d_params_prev.
 *   d_labels        u8  [V]
 *   d_vertex_energy f64 [V] or NULL
 *   d_params_prev   f64 [S][L][4] (n, mu, sigma, U); only mu, sigma are read
 *   d_params_out    f64 [S][L][4]; may alias d_params_prev
 */
PMRF_API int pmrf_params(pmrf_graph* g, const pmrf_config* cfg, const uint8_t* d_labels, const double* d_vertex_energy,
                const double* d_params_prev, double* d_params_out, pmrf_stream_t stream);

/*
 * One MAP sweep (Section 3.2.2 EM step 2 "Compute Energy Function", "Compute
 * Minimum Vertex and Label Energies", "Compute Neighborhood Energy Sums",
 * step 3 "Update Output Labels"; Algorithm 2 steps 7-10) with labels and
 * parameters held fixed:
 *   E(c,v,l)  = D_l(y_v) + beta * #{u in N(v) and in hood c : x_u != l}
 *   D_l(y)    = (y - mu_l)^2 / (2 sigma_l^2) + ln sigma_l
 *   Emin(c,v) = min_l E(c,v,l), label = smallest l attaining it
 *   d_hood_energy[c]   = sum over v in hood c of Emin(c,v)
 *   (d_vertex_energy[v], d_labels_out[v]) = minimum over the hoods c that
 *       contain v of (Emin(c,v), label), energy first, then the label.
 *   d_labels_in u8 [V]; d_params f64 [S][L][4] (mu, sigma read);
 *   d_labels_out u8 [V] (must not alias d_labels_in); d_vertex_energy f64 [V]
 *   or NULL; d_hood_energy f64 [C] or NULL.
 */
PMRF_API int pmrf_map_sweep(pmrf_graph* g, const pmrf_config* cfg, const uint8_t* d_labels_in, const double* d_params,
                   uint8_t* d_labels_out, double* d_vertex_energy, double* d_hood_energy, pmrf_stream_t stream);

/*
 * The EM loop (Algorithm 2 steps 3 and 6-11; Section 3.2.2 EM steps 2-5) on
 * every slice of the batch, each slice converging on its own:
 *   start: labels/parameters as pmrf_config describes;
 *   iteration t = 1, 2, ...: one MAP sweep with the labels and parameters of
 *   t-1, then the parameter update; hood sums S_c^t and their total T^t;
 *   hood c has converged when t > W and max_{k=1..W} |S_c^t - S_c^{t-k}| <
 *   conv_tol; a slice stops when all its hoods have converged, or t > W and
 *   max_{k=1..W} |T^t - T^{t-k}| < conv_tol, or t = max_iters.
 * All slices run in the same launches, one vertex pass and one hood pass per
 * iteration; a stopped slice's tiles are skipped, and once they are most of
 * the table the passes take only the active slices' tiles.  The whole loop is
 * replayed from a CUDA graph (two conditional loops in sequence).
 *   d_labels    u8  [V]        out (in as well when init_from_labels = 1)
 *   d_params    f64 [S][L][4]  out: (n, mu, sigma, U) of the final iteration
 *   d_iters     i32 [S]        out: iterations run per slice
 *   d_converged i32 [S]        out: 1 when a convergence test ended the slice
 *   d_T_hist    f64 [S][max_iters] out or NULL: T^t per slice (unset entries 0)
 */
PMRF_API int pmrf_em(pmrf_graph* g, const pmrf_config* cfg, uint8_t* d_labels, double* d_params, int32_t* d_iters,
            int32_t* d_converged, double* d_T_hist, pmrf_stream_t stream);

/*
 * Vertex pseudo-log-likelihood (not in the paper; the differentiable form of
 * the model).  With labels x fixed and every slice's own (mu, sigma) and one
 * shared beta, over the full graph neighbourhood of each vertex:
 *   E_v(l) = D_l(y_v) + beta * #{u in N(v): x_u != l}
 *   PLL_s  = sum over v in slice s of [ -E_v(x_v) - log sum_l exp(-E_v(l)) ]
 *   d_mu, d_sigma f64 [S][L]; d_pll f64 [S] out.
 */
PMRF_API int pmrf_pll(pmrf_graph* g, int32_t n_labels, const uint8_t* d_labels, const double* d_mu, const double* d_sigma,
             double beta, double* d_pll, pmrf_stream_t stream);

/*
 * Adjoint of pmrf_pll: given d_gout f64 [S] (dLoss/dPLL_s), writes
 *   d_gmu[s][l]    = gout_s * dPLL_s/dmu_{s,l}
 *   d_gsigma[s][l] = gout_s * dPLL_s/dsigma_{s,l}
 *   d_gbeta[0]     = sum_s gout_s * dPLL_s/dbeta
 * using dE_v(l)/dmu_l = (mu_l - y_v)/sigma_l^2, dE_v(l)/dsigma_l = 1/sigma_l -
 * (y_v - mu_l)^2/sigma_l^3, dE_v(l)/dbeta = #{u in N(v): x_u != l} and the
 * softmax p_v = softmax(-E_v).  Any gradient output may be NULL.
 */
PMRF_API int pmrf_pll_grad(pmrf_graph* g, int32_t n_labels, const uint8_t* d_labels, const double* d_mu,
                  const double* d_sigma, double beta, const double* d_gout, double* d_gmu, double* d_gsigma,
                  double* d_gbeta, pmrf_stream_t stream);

/*
 * pmrf_pll and pmrf_pll_grad in one pass over the vertices (the value is a
 * by-product of the adjoint's softmax): d_pll as pmrf_pll, the gradients as
 * pmrf_pll_grad, bit-identical to the two separate calls.  d_gout must not be
 * NULL; d_pll and the gradient outputs may be.
 */
PMRF_API int pmrf_pll_value_and_grad(pmrf_graph* g, int32_t n_labels, const uint8_t* d_labels, const double* d_mu,
                                     const double* d_sigma, double beta, const double* d_gout, double* d_pll,
                                     double* d_gmu, double* d_gsigma, double* d_gbeta, pmrf_stream_t stream);

/*
 * Allocation-free variant of pmrf_pll_grad; the paper has no counterpart.
 * Same inputs, outputs and results as pmrf_pll_grad, but it allocates no
 * memory: no cudaMalloc, no stream-ordered allocation, no host allocation on
 * the device's behalf.  It is meant for callers that cannot allocate when they
 * need the gradient, once the graph itself has been built: an application
 * whose device memory is already claimed by its own caching allocator (a new
 * allocation would fail, or force that allocator to give memory back), or a
 * latency-critical loop that must not pay for, or be implicitly synchronised
 * by, an allocation.
 *   Scratch: the per-block partial sums go to one fixed array inside the
 *   library, PMRF_PLL_NOALLOC_MAX_DOUBLES doubles (8 MiB), which every GPU that
 *   loads the library keeps until the process exits.  A call needs
 *   S * ceil(V_max / 256) * (2 * n_labels + 2) + S doubles (S slices, V_max the
 *   regions of the largest slice); a larger request fails with
 *   PMRF_ERR_UNSUPPORTED and a message giving the size, before any work is
 *   enqueued.
 *   Set-up: every call looks up the array's device address
 *   (cudaGetSymbolAddress) with the caller's device current; the first call on
 *   a device also loads the library's device code there, so make that first
 *   call before any stream capture.  A device reset between calls is handled.
 *   Sharing: all calls use the same array.  Each call writes every entry it
 *   reads, so earlier calls leave nothing behind that matters, but calls whose
 *   work overlaps on the GPU (different streams or threads) race on the array;
 *   order them.  d_gout must not be NULL.
 */
#define PMRF_PLL_NOALLOC_MAX_DOUBLES (1 << 20)
PMRF_API int pmrf_pll_grad_noalloc(pmrf_graph* g, int32_t n_labels, const uint8_t* d_labels, const double* d_mu,
                                   const double* d_sigma, double beta, const double* d_gout, double* d_gmu,
                                   double* d_gsigma, double* d_gbeta, pmrf_stream_t stream);

/*
 * Labels back to pixels (closing paragraph of Section 3.2.2): d_out[p] =
 * d_labels[vertex of the region id of pixel p].  d_region_ids is the array the
 * graph was built from (same layout); d_out u8, one per pixel.
 */
PMRF_API int pmrf_label_image(pmrf_graph* g, const int32_t* d_region_ids, const uint8_t* d_labels, uint8_t* d_out,
                     pmrf_stream_t stream);

/*
 * Segmentation quality against a ground truth (Section 4.2.1, evaluation
 * metrics: precision TP/(TP+FP), recall TP/(TP+FN), accuracy
 * (TP+TN)/(TP+TN+FP+FN), porosity = void volume / total volume).
 *   d_pred, d_truth  u8 per pixel, in the layout the graph was built from
 *                    (slices back to back, row-major); labels in [0, n_labels).
 *   d_confusion      i64 [S][n_labels][n_labels]: pixels with true label t
 *                    and predicted label q at [s][t][q] (truth-major).
 *   d_metrics        f64 [S][n_labels][5]: for label l scored against the
 *                    rest, precision, recall, accuracy, the predicted fraction
 *                    and the true fraction of the slice's pixels carrying l
 *                    (the porosity when l is the void phase); NaN where a
 *                    denominator is 0.
 * Caller-owned device buffers, written on the stream.  A pixel label outside
 * [0, n_labels) is not counted and sets the device status to PMRF_ERR_ARG
 * (pmrf_sync_status reports it with the pixel index).  n_labels outside
 * [1, PMRF_MAX_LABELS] or a NULL pointer: PMRF_ERR_ARG.
 */
PMRF_API int pmrf_quality(pmrf_graph* g, int32_t n_labels, const uint8_t* d_pred, const uint8_t* d_truth,
                          int64_t* d_confusion, double* d_metrics, pmrf_stream_t stream);

/*
 * Synchronise `stream` and return the graph's device status word: PMRF_OK, or
 * the first error a kernel recorded since the last call (the word is then
 * cleared).  *detail (may be NULL) receives a kernel-specific code.
 */
PMRF_API int pmrf_sync_status(pmrf_graph* g, pmrf_stream_t stream, int64_t* detail);

/* Launch shape of the EM hood pass.  0 selects the default.
 * hood_tile: hoods per tile (one 128-thread block per tile; multiple of 32,
 *   32..1024; default 128 / hood_lanes: one hood per lane group, one round);
 *   a tile's element stream is staged in shared memory;
 * hood_lanes: adjacent lanes that share one hood, each summing every
 *   hood_lanes-th element (1, 2, 4 or 8; default 2 for a mean hood size of 16
 *   or more, else 1).
 * The vertex pass always takes 128 vertices per block, one per thread.
 * With both fields 0 a result of pmrf_autotune for a graph of the same shape
 * is used when one exists.  Results do not depend on the tuning (every sum is
 * an exact integer). */
typedef struct {
    int32_t hood_tile;
    int32_t hood_lanes;
    int32_t use_cuda_graph; /* 1 (default) replays the iteration loop from a CUDA graph */
    int32_t profile;        /* 1: record CUDA events around the per-iteration kernels of
                               pmrf_em (read with pmrf_em_kernel_times) */
} pmrf_tuning;

/* Read / set the graph's tuning.  Setting discards cached launch plans. */
PMRF_API int pmrf_get_tuning(const pmrf_graph* g, pmrf_tuning* t);
PMRF_API int pmrf_set_tuning(pmrf_graph* g, const pmrf_tuning* t);

/* Per-iteration device times of the last pmrf_em run on this graph, when the
 * graph's tuning has profile = 1: ms_vertex[t-1], ms_hood[t-1] (vertex pass and
 * hood pass of iteration t) for t = 1..*n, *n = min(max_n, iterations run by
 * the longest slice).  Synchronises `stream`.  PMRF_ERR_ARG when profiling was
 * off for that run. */
PMRF_API int pmrf_em_kernel_times(pmrf_graph* g, int32_t max_n, float* ms_vertex, float* ms_hood, int32_t* n,
                                  pmrf_stream_t stream);

/* Time candidate tunings on this graph with `cfg` (the defaults, half and
 * twice the default hoods per tile, and every lanes-per-hood value with one
 * hood per lane group; each candidate runs the EM loop four times;
 * synchronises `stream`), keep the fastest on the graph (with its hoods per
 * tile and lanes filled in) and
 * return it in *best (may be NULL).  The result is also kept for the rest of
 * the process under the graph's shape (slices, regions, hood elements) and
 * cfg->n_labels: a graph whose hood_tile and hood_lanes are both 0 runs with
 * the kept result of its shape when there is one (so a batch rebuilt with the
 * same oversegmentation reuses one tuning run). */
PMRF_API int pmrf_autotune(pmrf_graph* g, const pmrf_config* cfg, pmrf_stream_t stream, pmrf_tuning* best);

#ifdef __cplusplus
}
#endif

#endif /* PMRF_H */
