// api.cu -- the C ABI of include/pmrf.h: argument checks, graph lifetime,
// error strings and the dispatch into the build / EM / PLL code.
#include <atomic>
#include <mutex>
#include <cstring>
#include <string>
#include <vector>

#include "graph.cuh"

namespace pmrf {

namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};
thread_local int64_t* t_capture = nullptr;
}

void note_launch(int64_t n) {
    if (t_capture) *t_capture += n;
    else g_launches.fetch_add(n, std::memory_order_relaxed);
}
void set_capture_counter(int64_t* counter) { t_capture = counter; }

// kernels counted on the device (the bodies of conditional graph nodes run
// only when their condition holds): one counter per device, created on first
// use
namespace {
std::mutex g_dev_counter_mu;
unsigned long long* g_dev_counter[64] = {};
}  // namespace

unsigned long long* device_launch_counter() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_dev_counter_mu);
    if (!g_dev_counter[dev]) {
        unsigned long long* p = nullptr;
        if (cudaMalloc(&p, sizeof(unsigned long long)) != cudaSuccess ||
            cudaMemset(p, 0, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_dev_counter[dev] = p;
    }
    return g_dev_counter[dev];
}

int64_t device_launches() {
    int64_t total = 0;
    std::lock_guard<std::mutex> lk(g_dev_counter_mu);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) cudaGetLastError();
    for (int d = 0; d < 64; ++d) {
        if (!g_dev_counter[d]) continue;
        unsigned long long v = 0;
        if (cudaSetDevice(d) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
            cudaMemcpy(&v, g_dev_counter[d], sizeof(v), cudaMemcpyDeviceToHost) == cudaSuccess)
            total += (int64_t)v;
        else
            cudaGetLastError();
    }
    cudaSetDevice(cur);
    return total;
}

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PMRF_ERR_OOM : PMRF_ERR_CUDA;
}

int build_graph_impl(pmrf_graph* g, const double* d_img, const int32_t* d_ids, cudaStream_t s);
int em_run(pmrf_graph* g, const pmrf_config* cfg, uint8_t* d_labels, double* d_params, int32_t* d_iters,
           int32_t* d_conv, double* d_T_hist, cudaStream_t s);
int sweep_run(pmrf_graph* g, const pmrf_config* cfg, const uint8_t* xin, const double* theta, uint8_t* xout,
              double* Eout, double* Sout, cudaStream_t s);
int params_run(pmrf_graph* g, const pmrf_config* cfg, const uint8_t* x, const double* Ein, const double* prev,
               double* out, cudaStream_t s);
int init_labels_run(pmrf_graph* g, const pmrf_config* cfg, uint8_t* x, cudaStream_t s);
int label_image_run(pmrf_graph* g, const int32_t* ids, const uint8_t* labels, uint8_t* out, cudaStream_t s);
int random_init_run(pmrf_graph* g, int32_t L, uint64_t seed, double lo, double hi, uint8_t* x, double* params,
                    cudaStream_t s);
int quality_run(pmrf_graph* g, int32_t L, const uint8_t* pred, const uint8_t* truth, int64_t* conf, double* metrics,
                cudaStream_t s);
int pll_run(pmrf_graph* g, int32_t L, const uint8_t* x, const double* mu, const double* sigma, double beta,
            double* pll, const double* gout, double* gmu, double* gsigma, double* gbeta, cudaStream_t s);
int export_rep_hood(pmrf_graph* g, int32_t* dst, cudaStream_t s);
int autotune_run(pmrf_graph* g, const pmrf_config* cfg, cudaStream_t s, pmrf_tuning* best);
int em_kernel_times(pmrf_graph* g, int32_t max_n, float* msv, float* msh, int32_t* n, cudaStream_t s);
int pll_grad_noalloc_run(pmrf_graph* g, int32_t L, const uint8_t* x, const double* mu, const double* sigma,
                         double beta, const double* gout, double* gmu, double* gsigma, double* gbeta, cudaStream_t s);

namespace {

void destroy(pmrf_graph* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    free_plans(g);
    free_em(g);
    for (cudaEvent_t ev : g->prof_ev) cudaEventDestroy(ev);
    void* ps[] = {g->d_pix_off, g->d_vert_off, g->d_hood_slice_off, g->d_rank_off, g->d_W, g->d_rank, g->d_y,
                  g->d_npix, g->d_adj_off, g->d_adj, g->d_clq_off, g->d_clq, g->d_hood_off, g->d_hood, g->d_row_off,
                  g->d_row, g->d_rep_off, g->d_rep_woff, g->d_rep_mask, g->d_el, g->d_hood_gen, g->d_status, g->d_layer};
    for (void* p : ps)
        if (p) cudaFreeAsync(p, 0);
    delete g;
}

// graph on the current device?
int check_device(const pmrf_graph* g) {
    int dev = -1;
    PMRF_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(PMRF_ERR_ARG, "graph was built on another device");
    return PMRF_OK;
}

}  // namespace
}  // namespace pmrf

using namespace pmrf;

extern "C" {

int pmrf_config_default(pmrf_config* cfg) {
    if (!cfg) return fail(PMRF_ERR_ARG, "cfg is NULL");
    cfg->n_labels = 2;
    cfg->max_iters = 20;
    cfg->conv_window = 3;
    cfg->init_from_labels = 0;
    cfg->potts_scope = PMRF_SCOPE_HOOD;
    cfg->replica_rule = PMRF_RULE_MIN;
    cfg->beta = 1.0;
    cfg->conv_tol = 1e-4;
    cfg->sigma_min = 1e-6;
    cfg->init_lo = 0.0;
    cfg->init_hi = 1.0;
    return PMRF_OK;
}

const char* pmrf_last_error(void) { return g_last_error.c_str(); }

int64_t pmrf_launch_count(void) { return g_launches.load() + device_launches(); }

const char* pmrf_version(void) { return "pmrf-b300 0.1 (sm_103a)"; }

int pmrf_trim_memory(int64_t keep_bytes) {
    g_last_error.clear();
    return pool_trim(keep_bytes);
}

int pmrf_memory_usage(int64_t* reserved_bytes, int64_t* used_bytes) {
    g_last_error.clear();
    return pool_usage(reserved_bytes, used_bytes);
}

int pmrf_build_options_default(pmrf_build_options* opt) {
    if (!opt) return fail(PMRF_ERR_ARG, "opt is NULL");
    opt->hood_depth = 1;
    opt->volume_depth = 1;
    return PMRF_OK;
}

int pmrf_build_graph(const double* d_image, const int32_t* d_region_ids, int32_t n_slices, const int64_t* h_heights,
                     const int64_t* h_widths, pmrf_stream_t stream, pmrf_graph** out) {
    return pmrf_build_graph_ex(d_image, d_region_ids, n_slices, h_heights, h_widths, nullptr, stream, out);
}

int pmrf_build_graph_ex(const double* d_image, const int32_t* d_region_ids, int32_t n_slices,
                        const int64_t* h_heights, const int64_t* h_widths, const pmrf_build_options* opt,
                        pmrf_stream_t stream, pmrf_graph** out) {
    g_last_error.clear();
    if (!out) return fail(PMRF_ERR_ARG, "out is NULL");
    *out = nullptr;
    pmrf_build_options o;
    pmrf_build_options_default(&o);
    if (opt) o = *opt;
    if (o.hood_depth < 1 || o.hood_depth > PMRF_MAX_HOOD_DEPTH)
        return fail(PMRF_ERR_ARG, "hood_depth must be in [1, PMRF_MAX_HOOD_DEPTH]");
    if (o.volume_depth < 1) return fail(PMRF_ERR_ARG, "volume_depth must be >= 1");
    if (n_slices % o.volume_depth != 0) return fail(PMRF_ERR_ARG, "n_slices must be a multiple of volume_depth");
    if (n_slices < 1 || n_slices > 65535) return fail(PMRF_ERR_ARG, "n_slices must be in [1, 65535]");
    if (!h_heights || !h_widths) return fail(PMRF_ERR_ARG, "h_heights / h_widths is NULL");
    pmrf_graph* g = new (std::nothrow) pmrf_graph();
    if (!g) return fail(PMRF_ERR_OOM, "host allocation failed");
    // the graph's slices are the volumes: D layers stacked row after row
    const int32_t D = o.volume_depth, S = n_slices / D;
    g->S = S;
    g->hood_depth = o.hood_depth;
    g->volume_depth = D;
    g->h_H.assign(S, 0);
    g->h_W.assign(S, 0);
    g->h_layer.assign(S, 0);
    g->h_pix_off.assign(S + 1, 0);
    for (int i = 0; i < n_slices; ++i) {
        if (h_heights[i] < 0 || h_widths[i] < 0) {
            delete g;
            return fail(PMRF_ERR_ARG, "negative slice size");
        }
        const int v = i / D;
        if (i % D != 0 && (h_heights[i] != h_heights[i - 1] || h_widths[i] != h_widths[i - 1])) {
            delete g;
            return fail(PMRF_ERR_ARG, "the layers of a volume must have equal sizes");
        }
        g->h_layer[v] = h_heights[i];
        g->h_W[v] = h_widths[i];
        g->h_H[v] += h_heights[i];
    }
    for (int v = 0; v < S; ++v) g->h_pix_off[v + 1] = g->h_pix_off[v] + g->h_H[v] * g->h_W[v];
    g->n_pix = g->h_pix_off[S];
    if (g->n_pix >= 4294967295ll) {
        delete g;
        return fail(PMRF_ERR_UNSUPPORTED, "more than 2^32-1 pixels in one batch");
    }
    if (g->n_pix > 0 && (!d_image || !d_region_ids)) {
        delete g;
        return fail(PMRF_ERR_ARG, "d_image / d_region_ids is NULL");
    }
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "cudaGetDevice");
    }
    int rc = build_graph_impl(g, d_image, d_region_ids, (cudaStream_t)stream);
    if (rc != PMRF_OK) {
        std::string msg = g_last_error;
        destroy(g);
        g_last_error = msg;
        return rc;
    }
    *out = g;
    return PMRF_OK;
}

int pmrf_graph_destroy(pmrf_graph* g) {
    destroy(g);
    return PMRF_OK;
}

int pmrf_graph_stats(const pmrf_graph* g, int64_t* n_slices, int64_t* V, int64_t* E, int64_t* C, int64_t* N_el) {
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    if (n_slices) *n_slices = g->S;
    if (V) *V = g->V;
    if (E) *E = g->E2 / 2;
    if (C) *C = g->C;
    if (N_el) *N_el = g->N_el;
    return PMRF_OK;
}

int pmrf_graph_len(const pmrf_graph* g, int32_t which, int64_t* n) {
    if (!g || !n) return fail(PMRF_ERR_ARG, "null argument");
    switch (which) {
        case PMRF_ARR_VERT_OFF:
        case PMRF_ARR_HOOD_SLICE_OFF:
        case PMRF_ARR_RANK_OFF: *n = g->S + 1; break;
        case PMRF_ARR_Y:
        case PMRF_ARR_NPIX: *n = g->V; break;
        case PMRF_ARR_ADJ_OFF:
        case PMRF_ARR_REP_OFF: *n = g->V + 1; break;
        case PMRF_ARR_ADJ: *n = g->E2; break;
        case PMRF_ARR_CLQ_OFF:
        case PMRF_ARR_HOOD_OFF: *n = g->C + 1; break;
        case PMRF_ARR_CLQ: *n = g->n_clq; break;
        case PMRF_ARR_HOOD:
        case PMRF_ARR_REP_HOOD: *n = g->N_el; break;
        case PMRF_ARR_RANK: *n = g->n_rank; break;
        default: return fail(PMRF_ERR_ARG, "unknown array id");
    }
    return PMRF_OK;
}

int pmrf_graph_get(const pmrf_graph* gc, int32_t which, void* dst, size_t dst_bytes, int32_t to_host,
                   pmrf_stream_t stream) {
    pmrf_graph* g = const_cast<pmrf_graph*>(gc);
    int64_t n = 0;
    PMRF_TRY(pmrf_graph_len(g, which, &n));
    if (!dst && n > 0) return fail(PMRF_ERR_ARG, "dst is NULL");
    PMRF_TRY(check_device(g));
    cudaStream_t s = (cudaStream_t)stream;
    const void* src = nullptr;
    size_t el = 8;
    switch (which) {
        case PMRF_ARR_VERT_OFF: src = g->d_vert_off; break;
        case PMRF_ARR_HOOD_SLICE_OFF: src = g->d_hood_slice_off; break;
        case PMRF_ARR_RANK_OFF: src = g->d_rank_off; break;
        case PMRF_ARR_Y: src = g->d_y; break;
        case PMRF_ARR_NPIX: src = g->d_npix; el = 4; break;
        case PMRF_ARR_ADJ_OFF: src = g->d_adj_off; break;
        case PMRF_ARR_REP_OFF: src = g->d_rep_off; break;
        case PMRF_ARR_ADJ: src = g->d_adj; el = 4; break;
        case PMRF_ARR_CLQ_OFF: src = g->d_clq_off; break;
        case PMRF_ARR_HOOD_OFF: src = g->d_hood_off; break;
        case PMRF_ARR_CLQ: src = g->d_clq; el = 4; break;
        case PMRF_ARR_HOOD: src = g->d_hood; el = 4; break;
        case PMRF_ARR_RANK: src = g->d_rank; el = 4; break;
        case PMRF_ARR_REP_HOOD: el = 4; break;
        default: return fail(PMRF_ERR_ARG, "unknown array id");
    }
    const size_t bytes = (size_t)n * el;
    if (dst_bytes < bytes) return fail(PMRF_ERR_ARG, "dst_bytes too small");
    if (n == 0) return PMRF_OK;
    if (which == PMRF_ARR_REP_HOOD) {
        int32_t* tmp = nullptr;
        PMRF_TRY(dalloc(&tmp, n, s));
        int rc = export_rep_hood(g, tmp, s);
        if (!rc) {
            cudaError_t e = cudaMemcpyAsync(dst, tmp, bytes, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) rc = cuda_fail(e, "copy");
        }
        cudaFreeAsync(tmp, s);
        PMRF_CUDA(cudaStreamSynchronize(s));
        return rc;
    }
    PMRF_CUDA(cudaMemcpyAsync(dst, src, bytes, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    PMRF_CUDA(cudaStreamSynchronize(s));
    return PMRF_OK;
}

int pmrf_init_labels(pmrf_graph* g, const pmrf_config* cfg, uint8_t* d_labels, pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    PMRF_TRY(check_device(g));
    return init_labels_run(g, cfg, d_labels, (cudaStream_t)stream);
}

int pmrf_params(pmrf_graph* g, const pmrf_config* cfg, const uint8_t* d_labels, const double* d_vertex_energy,
                const double* d_params_prev, double* d_params_out, pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    PMRF_TRY(check_device(g));
    return params_run(g, cfg, d_labels, d_vertex_energy, d_params_prev, d_params_out, (cudaStream_t)stream);
}

int pmrf_map_sweep(pmrf_graph* g, const pmrf_config* cfg, const uint8_t* d_labels_in, const double* d_params,
                   uint8_t* d_labels_out, double* d_vertex_energy, double* d_hood_energy, pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    PMRF_TRY(check_device(g));
    return sweep_run(g, cfg, d_labels_in, d_params, d_labels_out, d_vertex_energy, d_hood_energy,
                     (cudaStream_t)stream);
}

int pmrf_em(pmrf_graph* g, const pmrf_config* cfg, uint8_t* d_labels, double* d_params, int32_t* d_iters,
            int32_t* d_converged, double* d_T_hist, pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    PMRF_TRY(check_device(g));
    return em_run(g, cfg, d_labels, d_params, d_iters, d_converged, d_T_hist, (cudaStream_t)stream);
}

int pmrf_pll(pmrf_graph* g, int32_t n_labels, const uint8_t* d_labels, const double* d_mu, const double* d_sigma,
             double beta, double* d_pll, pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    if (!d_pll) return fail(PMRF_ERR_ARG, "d_pll is NULL");
    PMRF_TRY(check_device(g));
    return pll_run(g, n_labels, d_labels, d_mu, d_sigma, beta, d_pll, nullptr, nullptr, nullptr, nullptr,
                   (cudaStream_t)stream);
}

int pmrf_pll_grad(pmrf_graph* g, int32_t n_labels, const uint8_t* d_labels, const double* d_mu,
                  const double* d_sigma, double beta, const double* d_gout, double* d_gmu, double* d_gsigma,
                  double* d_gbeta, pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    if (!d_gout) return fail(PMRF_ERR_ARG, "d_gout is NULL");
    PMRF_TRY(check_device(g));
    return pll_run(g, n_labels, d_labels, d_mu, d_sigma, beta, nullptr, d_gout, d_gmu, d_gsigma, d_gbeta,
                   (cudaStream_t)stream);
}

int pmrf_pll_value_and_grad(pmrf_graph* g, int32_t n_labels, const uint8_t* d_labels, const double* d_mu,
                            const double* d_sigma, double beta, const double* d_gout, double* d_pll, double* d_gmu,
                            double* d_gsigma, double* d_gbeta, pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    if (!d_gout) return fail(PMRF_ERR_ARG, "d_gout is NULL");
    PMRF_TRY(check_device(g));
    return pll_run(g, n_labels, d_labels, d_mu, d_sigma, beta, d_pll, d_gout, d_gmu, d_gsigma, d_gbeta,
                   (cudaStream_t)stream);
}

int pmrf_pll_grad_noalloc(pmrf_graph* g, int32_t n_labels, const uint8_t* d_labels, const double* d_mu,
                          const double* d_sigma, double beta, const double* d_gout, double* d_gmu, double* d_gsigma,
                          double* d_gbeta, pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    PMRF_TRY(check_device(g));
    return pll_grad_noalloc_run(g, n_labels, d_labels, d_mu, d_sigma, beta, d_gout, d_gmu, d_gsigma, d_gbeta,
                                (cudaStream_t)stream);
}

int pmrf_label_image(pmrf_graph* g, const int32_t* d_region_ids, const uint8_t* d_labels, uint8_t* d_out,
                     pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    PMRF_TRY(check_device(g));
    return label_image_run(g, d_region_ids, d_labels, d_out, (cudaStream_t)stream);
}

int pmrf_random_init(pmrf_graph* g, int32_t n_labels, uint64_t seed, double lo, double hi, uint8_t* d_labels,
                     double* d_params, pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    PMRF_TRY(check_device(g));
    return random_init_run(g, n_labels, seed, lo, hi, d_labels, d_params, (cudaStream_t)stream);
}

int pmrf_quality(pmrf_graph* g, int32_t n_labels, const uint8_t* d_pred, const uint8_t* d_truth, int64_t* d_confusion,
                 double* d_metrics, pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    PMRF_TRY(check_device(g));
    return quality_run(g, n_labels, d_pred, d_truth, d_confusion, d_metrics, (cudaStream_t)stream);
}

int pmrf_sync_status(pmrf_graph* g, pmrf_stream_t stream, int64_t* detail) {
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    DevStatus h;
    cudaStream_t s = (cudaStream_t)stream;
    PMRF_CUDA(cudaMemcpyAsync(&h, g->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
    PMRF_CUDA(cudaStreamSynchronize(s));
    if (detail) *detail = h.detail;
    if (h.code != 0) {
        PMRF_CUDA(cudaMemsetAsync(g->d_status, 0, sizeof(DevStatus), s));
        PMRF_CUDA(cudaStreamSynchronize(s));
        return fail(h.code, "kernel recorded error at site " + std::to_string(h.where) + ", detail " +
                                std::to_string(h.detail));
    }
    return PMRF_OK;
}

int pmrf_get_tuning(const pmrf_graph* g, pmrf_tuning* t) {
    if (!g || !t) return fail(PMRF_ERR_ARG, "null argument");
    *t = g->tuning;
    return PMRF_OK;
}

int pmrf_set_tuning(pmrf_graph* g, const pmrf_tuning* t) {
    if (!g || !t) return fail(PMRF_ERR_ARG, "null argument");
    if (t->hood_tile != 0 && (t->hood_tile < 32 || t->hood_tile > 1024 || t->hood_tile % 32))
        return fail(PMRF_ERR_ARG, "hood_tile must be 0 or a multiple of 32 in [32, 1024]");
    if (t->hood_lanes != 0 && t->hood_lanes != 1 && t->hood_lanes != 2 && t->hood_lanes != 4 && t->hood_lanes != 8)
        return fail(PMRF_ERR_ARG, "hood_lanes must be 0, 1, 2, 4 or 8");
    if (t->profile != 0 && t->profile != 1) return fail(PMRF_ERR_ARG, "profile must be 0 or 1");
    cudaDeviceSynchronize();
    free_plans(g);
    free_em(g);
    g->tuning = *t;
    return PMRF_OK;
}

int pmrf_em_kernel_times(pmrf_graph* g, int32_t max_n, float* ms_vertex, float* ms_hood, int32_t* n,
                         pmrf_stream_t stream) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    return em_kernel_times(g, max_n, ms_vertex, ms_hood, n, (cudaStream_t)stream);
}

int pmrf_autotune(pmrf_graph* g, const pmrf_config* cfg, pmrf_stream_t stream, pmrf_tuning* best) {
    g_last_error.clear();
    if (!g) return fail(PMRF_ERR_ARG, "graph is NULL");
    PMRF_TRY(check_device(g));
    return autotune_run(g, cfg, (cudaStream_t)stream, best);
}

}  // extern "C"
