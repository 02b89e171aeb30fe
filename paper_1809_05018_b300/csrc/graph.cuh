// graph.cuh -- device-resident region graph of a batch of slices, its maximal
// cliques, hoods, replica structures and the EM workspace.
#pragma once

#include <map>
#include <vector>

#include "common.cuh"

namespace pmrf {

// Per-tile descriptor of the persistent EM launch.  kind 0 = hood tile (hoods
// [a0, a1)), kind 1 = vertex tile (vertices [a0, a1)).  `part` indexes the
// tile's partial-sum record inside its kind.
struct Tile {
    int32_t kind;
    int32_t slice;
    int32_t a0, a1;
    int32_t part;
    int32_t pad;  // hood tiles: 1 when every member has degree <= 32
};

struct Plan {  // tile table for one tuning
    int32_t hood_tile = 0, hood_lanes = 0, max_hood = 0;
    int32_t cap = 1;  // elements of the largest hood tile, up to the staging limit
    int64_t n_tiles = 0, n_htiles = 0, n_vtiles = 0;
    Tile* d_tiles = nullptr;
    int32_t* d_slice_ntiles = nullptr;   // [S] tiles per slice (both kinds)
    int64_t* d_slice_vt0 = nullptr;      // [S+1] first vertex-tile partial of each slice
    int64_t* d_slice_ht0 = nullptr;      // [S+1] first hood-tile partial of each slice
};

struct EMWork {  // EM scratch, sized for (L, W, plan)
    int L = 0, W = 0, max_iters = 0;
    int64_t n_htiles = 0, n_vtiles = 0;
    uint8_t* d_x[2] = {nullptr, nullptr};  // label double buffer
    int64_t* d_hist = nullptr;     // [W][C] hood-sum ring, each in the unit of its iteration
    int32_t* d_qhist = nullptr;    // [S][W] unit exponent of each ring slot
    void* d_unit = nullptr;        // [S] fixed-point unit of the current iteration (em.cu SliceUnit)
    double* d_yr = nullptr;        // [S][2] intensity range of each slice
    double* d_vpart = nullptr;     // [n_vtiles][L][4]
    int64_t* d_hpart = nullptr;    // [n_htiles][3]: the tile's exact T partial (low, high word, in the
                                   // slice's unit) and its unconverged-hood count
    double* d_theta = nullptr;     // [S][L][4] current parameters
    double* d_dterm = nullptr;     // [S][L][2] 1/(2 sigma^2) and ln sigma of the current parameters
    double* d_Thist = nullptr;     // [S][W] ring of totals
    uint64_t* d_vrec = nullptr;    // [V][vrec_words(L)] hood-pass vertex records (em.cu)
    int32_t* d_active = nullptr;   // [S] slice still iterating
    int32_t* d_iters = nullptr;    // [S]
    int32_t* d_conv = nullptr;     // [S]
    int32_t* d_nactive = nullptr;  // [1]
    int32_t* d_t = nullptr;        // [1] the loop graph's current iteration
    int32_t* d_sched = nullptr;    // [2 (S + 1) + 2] tiles of the slices still iterating: vertex- and
                                   // hood-tile prefix sums over the active slices, then the two
                                   // passes' tile counters
    void* d_cfg = nullptr;         // device copy of the run's constants
};

struct pmrf_graph_impl;

}  // namespace pmrf

struct pmrf_graph {
    int device = 0;
    int32_t S = 0;
    int64_t V = 0, E2 = 0, C = 0, n_clq = 0, N_el = 0, n_rank = 0, n_pix = 0;
    int32_t hood_depth = 1;    // k of the k-neighbourhoods (Section 3.1)
    int32_t volume_depth = 1;  // layers per 3-D volume (1: 2-D slices)
    int64_t n_row_words = 0, n_rep_words = 0;
    int32_t max_deg = 0, max_hood = 0;

    std::vector<int64_t> h_H, h_W, h_pix_off, h_vert_off, h_hood_slice_off, h_el_slice_off, h_rank_off;
    std::vector<int64_t> h_layer;  // rows per layer of each volume (= h_H for 2-D slices)

    int64_t* d_pix_off = nullptr;        // [S+1]
    int64_t* d_layer = nullptr;          // [S] rows per layer (3-D volumes only; NULL for slices)
    int64_t* d_vert_off = nullptr;       // [S+1]
    int64_t* d_hood_slice_off = nullptr; // [S+1]
    int64_t* d_rank_off = nullptr;       // [S+1]
    int64_t* d_W = nullptr;              // [S] widths
    int32_t* d_rank = nullptr;           // [n_rank]
    double* d_y = nullptr;               // [V]
    int32_t* d_npix = nullptr;           // [V]
    int64_t* d_adj_off = nullptr;        // [V+1]
    int32_t* d_adj = nullptr;            // [E2]
    int64_t* d_clq_off = nullptr;        // [C+1]
    int32_t* d_clq = nullptr;            // [n_clq]
    int64_t* d_hood_off = nullptr;       // [C+1]
    int32_t* d_hood = nullptr;           // [N_el]
    int64_t* d_row_off = nullptr;        // [C+1] word offsets of hood-local adjacency rows
    uint32_t* d_row = nullptr;           // [n_row_words]
    int64_t* d_rep_off = nullptr;        // [V+1]
    int64_t* d_rep_woff = nullptr;       // [V+1] word offsets of replica slot masks
    uint32_t* d_rep_mask = nullptr;      // [n_rep_words]
    uint2* d_el = nullptr;               // [N_el] hood-pass element stream, hood-major: (vertex id, bit 31 set on
                                         // the last element of its hood; slot mask, 0 for degree > 32)
    uint8_t* d_hood_gen = nullptr;       // [C] 1: the hood has a member of degree > 32 (hood-local rows)
    pmrf::DevStatus* d_status = nullptr;

    pmrf_tuning tuning{0, 0, 1, 0};
    // profiling events of the EM loop: per iteration t (1-based), index 3*(t-1):
    // before the vertex pass, after it, after the hood pass
    std::vector<cudaEvent_t> prof_ev;
    int prof_iters = 0;  // iterations covered by the last profiled run
    std::map<std::pair<int, int>, pmrf::Plan> plans;
    pmrf::EMWork em;
    // cached CUDA graphs of the EM loop, keyed by (L, W, max_iters, tile sizes);
    // outputs and run constants are read from device memory, so one capture
    // serves every call with the same key
    struct CachedExec {
        cudaGraphExec_t exec = nullptr;
        int L = 0, W = 0, max_iters = 0, hood_tile = 0, hood_lanes = 0;
        int var = 0;  // vertex pass compiled with the sweep variants
        int64_t nkernels = 0;  // kernel nodes per replay
    };
    std::vector<CachedExec> execs;
};

namespace pmrf {
int free_plans(pmrf_graph* g);
int free_em(pmrf_graph* g);
// the hood-element index of every replica, ascending within each vertex's
// range [rep_off[v], rep_off[v+1]) (N_el entries, into d_rep_el)
int rep_elements(pmrf_graph* g, uint32_t* d_rep_el, cudaStream_t s);
}  // namespace pmrf
