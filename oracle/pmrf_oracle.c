/*
 * pmrf_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, serial, deliberately unoptimised CPU reference of the optimisation
 * path of DPP-PMRF (Lessley, Perciano, Heinemann, Camp, Childs, Bethel, "DPP-PMRF:
 * Rethinking Optimization for a Probabilistic Graphical Model Using
 * Data-Parallel Primitives", LDAV 2018).  Only the test-suite, the package's
 * smoke check and the benchmark's CPU-baseline leg load this library; the CUDA
 * library shares no code, header or table with it.
 *
 * Every function follows one passage of the paper; where the paper is silent
 * the reading used is stated at the function (labelled G1..G16).  Floating
 * point is IEEE double throughout,
 * evaluated in the order written (no reassociation: build with -O2 and without
 * -ffast-math).
 *
 * Notation: V regions (vertices), N(v) the sorted adjacency of v, K_c the c-th
 * maximal clique, H_c its 1-neighbourhood ("hood"), L labels, theta_l =
 * (n_l, mu_l, sigma_l, U_l).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 3

typedef struct {
    int32_t max_id;   /* largest raw region id present (-1 if none) */
    int32_t V;        /* number of regions */
    int64_t n_adj;    /* 2E: length of adj */
    int64_t C;        /* number of maximal cliques (= number of hoods) */
    int64_t n_clq;    /* total clique member entries */
    int64_t N_el;     /* total hood elements */
    int32_t* rank;    /* [max_id+1]: compact vertex id of a raw id, -1 if absent */
    int64_t* npix;    /* [V] pixel count of each region */
    double* y;        /* [V] mean intensity of each region */
    int64_t* adj_off; /* [V+1] */
    int32_t* adj;     /* [n_adj] ascending within each vertex */
    int64_t* clq_off; /* [C+1] */
    int32_t* clq;     /* [n_clq] members ascending; cliques in lexicographic order */
    int64_t* hood_off;/* [C+1] */
    int32_t* hood;    /* [N_el] members ascending */
} orc_graph;

typedef struct {
    int32_t n_labels, max_iters, conv_window;
    int32_t potts_scope;  /* ORC_SCOPE_HOOD (G4) or ORC_SCOPE_FULL */
    int32_t replica_rule; /* ORC_RULE_MIN (G6), ORC_RULE_SUM or ORC_RULE_VOTE */
    int32_t init_mode;    /* 0 threshold (G3), 1 labels given in x, 2 labels in x and parameters in theta */
    double beta, conv_tol, sigma_min, init_lo, init_hi;
    int32_t n_threads;    /* > 1: the default sweep runs on that many threads (orc_map_sweep_par) */
} orc_config;

/* Variants of the energy and of the replica reduction (readings G13, G14). */
#define ORC_SCOPE_HOOD 0
#define ORC_SCOPE_FULL 1
#define ORC_RULE_MIN 0
#define ORC_RULE_SUM 1
#define ORC_RULE_VOTE 2

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

void orc_graph_free(orc_graph* g) {
    if (!g) return;
    free(g->rank); free(g->npix); free(g->y); free(g->adj_off); free(g->adj);
    free(g->clq_off); free(g->clq); free(g->hood_off); free(g->hood);
    free(g);
}

/* ------------------------------------------------------------------------ */
/* Growable int32 buffer                                                     */
typedef struct { int32_t* a; int64_t n, cap; } ivec;
static int iv_push(ivec* v, int32_t x) {
    if (v->n == v->cap) {
        int64_t nc = v->cap ? 2 * v->cap : 64;
        int32_t* na = (int32_t*)realloc(v->a, sizeof(int32_t) * (size_t)nc);
        if (!na) return -1;
        v->a = na; v->cap = nc;
    }
    v->a[v->n++] = x;
    return 0;
}

/* ------------------------------------------------------------------------ */
/*
 * Regions (Section 2.1 and Section 3.1: a vertex per region of the
 * oversegmentation; the data term uses the mean intensity of a region).
 * Raw ids are compacted in ascending order: vertex v is the v-th smallest id
 * present.  y_v = (sum of the region's pixels, added in row-major order) / count.
 */
static int regions(const double* image, const int32_t* ids, int64_t npx, orc_graph* g) {
    int32_t mx = -1;
    for (int64_t p = 0; p < npx; ++p) {
        if (ids[p] < 0) return ORC_ERR_ARG;
        if (ids[p] > mx) mx = ids[p];
    }
    g->max_id = mx;
    g->rank = (int32_t*)malloc(sizeof(int32_t) * (size_t)(mx + 2));
    if (!g->rank) return ORC_ERR_OOM;
    for (int64_t i = 0; i <= mx; ++i) g->rank[i] = -1;
    for (int64_t p = 0; p < npx; ++p) g->rank[ids[p]] = 0;
    int32_t V = 0;
    for (int64_t i = 0; i <= mx; ++i)
        if (g->rank[i] == 0) g->rank[i] = V++;
    g->V = V;
    g->npix = (int64_t*)calloc((size_t)V + 1, sizeof(int64_t));
    double* sum = (double*)calloc((size_t)V + 1, sizeof(double));
    g->y = (double*)calloc((size_t)V + 1, sizeof(double));
    if (!g->npix || !sum || !g->y) { free(sum); return ORC_ERR_OOM; }
    for (int64_t p = 0; p < npx; ++p) {
        int32_t v = g->rank[ids[p]];
        sum[v] += image[p];
        g->npix[v] += 1;
    }
    for (int32_t v = 0; v < V; ++v) g->y[v] = sum[v] / (double)g->npix[v];
    free(sum);
    return ORC_OK;
}

/*
 * Region adjacency graph G(V,E) (Section 2.1: two regions are joined when they
 * share a boundary; Algorithm 2, step 1).  Reading: "share a boundary" means
 * some pair of 4-connected pixels (horizontal or vertical neighbours) carries
 * the two ids.  Stored as CSR with each adjacency list ascending (Section
 * 3.2.1 uses CSR).  Built by bucketing every boundary pixel pair under both of
 * its endpoints, then sorting and de-duplicating each bucket.
 */
static int edges(const int32_t* ids, int64_t H, int64_t W, orc_graph* g) {
    const int32_t V = g->V;
    int64_t* cnt = (int64_t*)calloc((size_t)V + 1, sizeof(int64_t));
    if (!cnt) return ORC_ERR_OOM;
    for (int64_t r = 0; r < H; ++r)
        for (int64_t c = 0; c < W; ++c) {
            int32_t a = g->rank[ids[r * W + c]];
            if (c + 1 < W) {
                int32_t b = g->rank[ids[r * W + c + 1]];
                if (a != b) { cnt[a]++; cnt[b]++; }
            }
            if (r + 1 < H) {
                int32_t b = g->rank[ids[(r + 1) * W + c]];
                if (a != b) { cnt[a]++; cnt[b]++; }
            }
        }
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)V + 1));
    if (!off) { free(cnt); return ORC_ERR_OOM; }
    off[0] = 0;
    for (int32_t v = 0; v < V; ++v) off[v + 1] = off[v] + cnt[v];
    int32_t* bucket = (int32_t*)malloc(sizeof(int32_t) * (size_t)(off[V] + 1));
    if (!bucket) { free(cnt); free(off); return ORC_ERR_OOM; }
    for (int32_t v = 0; v < V; ++v) cnt[v] = 0;
    for (int64_t r = 0; r < H; ++r)
        for (int64_t c = 0; c < W; ++c) {
            int32_t a = g->rank[ids[r * W + c]];
            if (c + 1 < W) {
                int32_t b = g->rank[ids[r * W + c + 1]];
                if (a != b) { bucket[off[a] + cnt[a]++] = b; bucket[off[b] + cnt[b]++] = a; }
            }
            if (r + 1 < H) {
                int32_t b = g->rank[ids[(r + 1) * W + c]];
                if (a != b) { bucket[off[a] + cnt[a]++] = b; bucket[off[b] + cnt[b]++] = a; }
            }
        }
    g->adj_off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)V + 1));
    g->adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(off[V] + 1));
    if (!g->adj_off || !g->adj) { free(cnt); free(off); free(bucket); return ORC_ERR_OOM; }
    int64_t n = 0;
    g->adj_off[0] = 0;
    for (int32_t v = 0; v < V; ++v) {
        int32_t* b = bucket + off[v];
        int64_t k = off[v + 1] - off[v];
        qsort(b, (size_t)k, sizeof(int32_t), cmp_i32);
        for (int64_t i = 0; i < k; ++i)
            if (i == 0 || b[i] != b[i - 1]) g->adj[n++] = b[i];
        g->adj_off[v + 1] = n;
    }
    g->n_adj = n;
    free(cnt); free(off); free(bucket);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/*
 * Maximal cliques (Section 3.2.1; Algorithm 2, step 2).  The paper uses a DPP
 * clique enumerator described elsewhere; any correct enumeration gives the same
 * set (G1).  Here: Bron-Kerbosch with Tomita pivoting, started once per vertex v
 * with candidates {u in N(v): u > v} and excluded set {u in N(v): u < v}, so
 * each maximal clique is reported exactly once, from its smallest member; an
 * isolated vertex is the clique {v}.  Canonical order (ours): members
 * ascending, cliques lexicographic.
 */
typedef struct { ivec out_off; ivec out; const orc_graph* g; int err; } bk_ctx;

static int64_t isect(const int32_t* a, int64_t na, const int32_t* b, int64_t nb, int32_t* o) {
    int64_t i = 0, j = 0, k = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { o[k++] = a[i]; ++i; ++j; }
    }
    return k;
}
static int contains(const int32_t* a, int64_t n, int32_t x) { /* a ascending */
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t m = (lo + hi) / 2;
        if (a[m] < x) lo = m + 1; else hi = m;
    }
    return lo < n && a[lo] == x;
}

static void bk(bk_ctx* ctx, int32_t* R, int64_t nR, int32_t* P, int64_t nP, int32_t* X, int64_t nX) {
    const orc_graph* g = ctx->g;
    if (ctx->err) return;
    if (nP == 0 && nX == 0) {
        for (int64_t i = 0; i < nR; ++i) if (iv_push(&ctx->out, R[i])) { ctx->err = 1; return; }
        if (iv_push(&ctx->out_off, (int32_t)ctx->out.n)) ctx->err = 1;
        return;
    }
    if (nP == 0) return;
    /* pivot: vertex of P u X with the most neighbours in P */
    int32_t piv = -1; int64_t best = -1;
    for (int64_t s = 0; s < nP + nX; ++s) {
        int32_t u = s < nP ? P[s] : X[s - nP];
        const int32_t* Nu = g->adj + g->adj_off[u];
        int64_t du = g->adj_off[u + 1] - g->adj_off[u], k = 0;
        for (int64_t i = 0; i < nP; ++i) k += contains(Nu, du, P[i]);
        if (k > best) { best = k; piv = u; }
    }
    const int32_t* Npiv = g->adj + g->adj_off[piv];
    int64_t dpiv = g->adj_off[piv + 1] - g->adj_off[piv];
    /* candidates: P \ N(pivot), in ascending order; P and X are kept sorted */
    int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nP + 1));
    int32_t* Pc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nP + 1));
    int32_t* Xc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nP + nX + 1));
    int32_t* P2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nP + 1));
    int32_t* X2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nP + nX + 1));
    if (!cand || !Pc || !Xc || !P2 || !X2) { ctx->err = 1; free(cand); free(Pc); free(Xc); free(P2); free(X2); return; }
    int64_t nc = 0;
    for (int64_t i = 0; i < nP; ++i) if (!contains(Npiv, dpiv, P[i])) cand[nc++] = P[i];
    memcpy(Pc, P, sizeof(int32_t) * (size_t)nP);
    memcpy(Xc, X, sizeof(int32_t) * (size_t)nX);
    int64_t nPc = nP, nXc = nX;
    for (int64_t ci = 0; ci < nc; ++ci) {
        int32_t w = cand[ci];
        const int32_t* Nw = g->adj + g->adj_off[w];
        int64_t dw = g->adj_off[w + 1] - g->adj_off[w];
        int64_t nP2 = isect(Pc, nPc, Nw, dw, P2);
        int64_t nX2 = isect(Xc, nXc, Nw, dw, X2);
        R[nR] = w;
        bk(ctx, R, nR + 1, P2, nP2, X2, nX2);
        /* P := P \ {w};  X := X u {w}  (both kept ascending) */
        int64_t k = 0;
        for (int64_t i = 0; i < nPc; ++i) if (Pc[i] != w) Pc[k++] = Pc[i];
        nPc = k;
        int64_t pos = nXc;
        while (pos > 0 && Xc[pos - 1] > w) { Xc[pos] = Xc[pos - 1]; --pos; }
        Xc[pos] = w; ++nXc;
    }
    free(cand); free(Pc); free(Xc); free(P2); free(X2);
}

typedef struct { const int32_t* m; int64_t n; } clq_ref;
static int cmp_clq(const void* a, const void* b) {
    const clq_ref* x = (const clq_ref*)a; const clq_ref* y = (const clq_ref*)b;
    for (int64_t i = 0; i < x->n && i < y->n; ++i)
        if (x->m[i] != y->m[i]) return x->m[i] < y->m[i] ? -1 : 1;
    return (x->n > y->n) - (x->n < y->n);
}

static int cliques(orc_graph* g) {
    const int32_t V = g->V;
    bk_ctx ctx; memset(&ctx, 0, sizeof(ctx)); ctx.g = g;
    if (iv_push(&ctx.out_off, 0)) return ORC_ERR_OOM;
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < V; ++v) {
        int32_t d = (int32_t)(g->adj_off[v + 1] - g->adj_off[v]);
        if (d > maxdeg) maxdeg = d;
    }
    int32_t* R = (int32_t*)malloc(sizeof(int32_t) * ((size_t)maxdeg + 2));
    int32_t* P = (int32_t*)malloc(sizeof(int32_t) * ((size_t)maxdeg + 1));
    int32_t* X = (int32_t*)malloc(sizeof(int32_t) * ((size_t)maxdeg + 1));
    if (!R || !P || !X) { free(R); free(P); free(X); return ORC_ERR_OOM; }
    for (int32_t v = 0; v < V && !ctx.err; ++v) {
        int64_t nP = 0, nX = 0;
        for (int64_t i = g->adj_off[v]; i < g->adj_off[v + 1]; ++i) {
            int32_t u = g->adj[i];
            if (u > v) P[nP++] = u; else X[nX++] = u;
        }
        R[0] = v;
        bk(&ctx, R, 1, P, nP, X, nX);
    }
    free(R); free(P); free(X);
    if (ctx.err) { free(ctx.out.a); free(ctx.out_off.a); return ORC_ERR_OOM; }
    const int64_t C = ctx.out_off.n - 1;
    /* canonical order: sort members of each clique, then the cliques */
    clq_ref* refs = (clq_ref*)malloc(sizeof(clq_ref) * ((size_t)C + 1));
    if (!refs) { free(ctx.out.a); free(ctx.out_off.a); return ORC_ERR_OOM; }
    for (int64_t c = 0; c < C; ++c) {
        int32_t* m = ctx.out.a + ctx.out_off.a[c];
        int64_t n = ctx.out_off.a[c + 1] - ctx.out_off.a[c];
        qsort(m, (size_t)n, sizeof(int32_t), cmp_i32);
        refs[c].m = m; refs[c].n = n;
    }
    qsort(refs, (size_t)C, sizeof(clq_ref), cmp_clq);
    g->C = C;
    g->n_clq = ctx.out.n;
    g->clq_off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)C + 1));
    g->clq = (int32_t*)malloc(sizeof(int32_t) * ((size_t)ctx.out.n + 1));
    if (!g->clq_off || !g->clq) { free(refs); free(ctx.out.a); free(ctx.out_off.a); return ORC_ERR_OOM; }
    int64_t k = 0;
    g->clq_off[0] = 0;
    for (int64_t c = 0; c < C; ++c) {
        memcpy(g->clq + k, refs[c].m, sizeof(int32_t) * (size_t)refs[c].n);
        k += refs[c].n;
        g->clq_off[c + 1] = k;
    }
    free(refs); free(ctx.out.a); free(ctx.out_off.a);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/*
 * 1-neighbourhoods (Section 3.1: the vertices of a maximal clique together with
 * every vertex within k hops of a clique vertex, k = 1; Section 3.2.2,
 * "Construction of Neighborhoods", steps Find/Count/Get Neighbors and Remove
 * Duplicate Neighbors).  Here written as its definition: H_c = sort(unique(K_c
 * u N(u) for u in K_c)), one hood per clique in clique order (G2: each hood
 * ascending by vertex id, hoods contiguous in clique order).
 */
static int hoods(orc_graph* g) {
    const int64_t C = g->C;
    g->hood_off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)C + 1));
    if (!g->hood_off) return ORC_ERR_OOM;
    ivec out; memset(&out, 0, sizeof(out));
    ivec tmp; memset(&tmp, 0, sizeof(tmp));
    g->hood_off[0] = 0;
    for (int64_t c = 0; c < C; ++c) {
        tmp.n = 0;
        for (int64_t i = g->clq_off[c]; i < g->clq_off[c + 1]; ++i) {
            int32_t u = g->clq[i];
            if (iv_push(&tmp, u)) goto oom;
            for (int64_t j = g->adj_off[u]; j < g->adj_off[u + 1]; ++j)
                if (iv_push(&tmp, g->adj[j])) goto oom;
        }
        qsort(tmp.a, (size_t)tmp.n, sizeof(int32_t), cmp_i32);
        for (int64_t i = 0; i < tmp.n; ++i)
            if (i == 0 || tmp.a[i] != tmp.a[i - 1])
                if (iv_push(&out, tmp.a[i])) goto oom;
        g->hood_off[c + 1] = out.n;
    }
    g->N_el = out.n;
    g->hood = out.a ? out.a : (int32_t*)malloc(sizeof(int32_t));
    free(tmp.a);
    return ORC_OK;
oom:
    free(out.a); free(tmp.a);
    return ORC_ERR_OOM;
}

/* k-neighbourhoods (Section 3.1: a k-neighbourhood holds the vertices of a
 * maximal clique and every vertex within k edges of any of them; the study
 * uses k = 1).  Replaces the graph's hoods by those of depth k >= 1: for each
 * clique a breadth-first search from all members at once, k levels deep, the
 * reached vertices sorted ascending. */
int orc_graph_set_hood_depth(orc_graph* g, int32_t k) {
    if (!g || k < 1) return ORC_ERR_ARG;
    const int32_t V = g->V;
    int32_t* seen = (int32_t*)malloc(sizeof(int32_t) * ((size_t)V + 1)); /* clique index + 1 that reached v */
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)g->C + 1));
    ivec out; memset(&out, 0, sizeof(out));
    ivec cur; memset(&cur, 0, sizeof(cur));
    ivec nxt; memset(&nxt, 0, sizeof(nxt));
    if (!seen || !off) goto oom;
    for (int32_t v = 0; v < V; ++v) seen[v] = 0;
    off[0] = 0;
    for (int64_t c = 0; c < g->C; ++c) {
        const int32_t mark = (int32_t)(c + 1);
        const int64_t start = out.n;
        cur.n = 0;
        for (int64_t i = g->clq_off[c]; i < g->clq_off[c + 1]; ++i) {
            const int32_t u = g->clq[i];
            if (seen[u] != mark) {
                seen[u] = mark;
                if (iv_push(&cur, u) || iv_push(&out, u)) goto oom;
            }
        }
        for (int32_t level = 1; level <= k; ++level) {
            nxt.n = 0;
            for (int64_t i = 0; i < cur.n; ++i) {
                const int32_t u = cur.a[i];
                for (int64_t j = g->adj_off[u]; j < g->adj_off[u + 1]; ++j) {
                    const int32_t w = g->adj[j];
                    if (seen[w] == mark) continue;
                    seen[w] = mark;
                    if (iv_push(&nxt, w) || iv_push(&out, w)) goto oom;
                }
            }
            ivec t = cur; cur = nxt; nxt = t;
        }
        qsort(out.a + start, (size_t)(out.n - start), sizeof(int32_t), cmp_i32);
        off[c + 1] = out.n;
    }
    free(g->hood_off); free(g->hood);
    g->hood_off = off;
    g->hood = out.a ? out.a : (int32_t*)malloc(sizeof(int32_t));
    g->N_el = out.n;
    free(seen); free(cur.a); free(nxt.a);
    return ORC_OK;
oom:
    free(seen); free(off); free(out.a); free(cur.a); free(nxt.a);
    return ORC_ERR_OOM;
}

/* ------------------------------------------------------------------------ */
/* 3-D region graphs (the paper's future work, Section 6: graphs built from
 * whole volumes instead of slices).  Reading G16: a volume of D layers of
 * H x W voxels, stored layer by layer, each layer row-major; two regions are
 * adjacent when some pair of 6-connected voxels (neighbours along x, y or z)
 * carries their two ids; a region's value is the mean of its voxels summed in
 * storage order.  Same bucketing, sorting and de-duplication as the 2-D
 * adjacency. */
static int edges_volume(const int32_t* ids, int64_t D, int64_t H, int64_t W, orc_graph* g) {
    const int32_t V = g->V;
    const int64_t layer = H * W;
    int64_t* cnt = (int64_t*)calloc((size_t)V + 1, sizeof(int64_t));
    if (!cnt) return ORC_ERR_OOM;
    for (int pass = 0; pass < 2; ++pass) {
        int64_t* off = NULL;
        int32_t* bucket = NULL;
        if (pass == 1) {
            off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)V + 1));
            if (!off) { free(cnt); return ORC_ERR_OOM; }
            off[0] = 0;
            for (int32_t v = 0; v < V; ++v) off[v + 1] = off[v] + cnt[v];
            bucket = (int32_t*)malloc(sizeof(int32_t) * (size_t)(off[V] + 1));
            if (!bucket) { free(cnt); free(off); return ORC_ERR_OOM; }
            for (int32_t v = 0; v < V; ++v) cnt[v] = 0;
        }
        for (int64_t z = 0; z < D; ++z)
            for (int64_t r = 0; r < H; ++r)
                for (int64_t c = 0; c < W; ++c) {
                    const int64_t p = z * layer + r * W + c;
                    const int32_t a = g->rank[ids[p]];
                    int64_t q[3];
                    int nq = 0;
                    if (c + 1 < W) q[nq++] = p + 1;
                    if (r + 1 < H) q[nq++] = p + W;
                    if (z + 1 < D) q[nq++] = p + layer;
                    for (int k = 0; k < nq; ++k) {
                        const int32_t b = g->rank[ids[q[k]]];
                        if (a == b) continue;
                        if (pass == 0) { cnt[a]++; cnt[b]++; }
                        else { bucket[off[a] + cnt[a]++] = b; bucket[off[b] + cnt[b]++] = a; }
                    }
                }
        if (pass == 1) {
            g->adj_off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)V + 1));
            g->adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(off[V] + 1));
            if (!g->adj_off || !g->adj) { free(cnt); free(off); free(bucket); return ORC_ERR_OOM; }
            int64_t n = 0;
            g->adj_off[0] = 0;
            for (int32_t v = 0; v < V; ++v) {
                int32_t* b = bucket + off[v];
                const int64_t k = off[v + 1] - off[v];
                qsort(b, (size_t)k, sizeof(int32_t), cmp_i32);
                for (int64_t i = 0; i < k; ++i)
                    if (i == 0 || b[i] != b[i - 1]) g->adj[n++] = b[i];
                g->adj_off[v + 1] = n;
            }
            g->n_adj = n;
            free(off); free(bucket);
        }
    }
    free(cnt);
    return ORC_OK;
}

/* Build everything for one volume of D layers (G16): regions (voxel means in
 * storage order), 6-connected adjacency, cliques, hoods. */
int orc_build_volume(const double* image, const int32_t* ids, int64_t D, int64_t H, int64_t W, orc_graph** out) {
    if (!out || D < 1 || H < 0 || W < 0 || ((D * H * W) > 0 && (!image || !ids))) return ORC_ERR_ARG;
    orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
    if (!g) return ORC_ERR_OOM;
    int rc = regions(image, ids, D * H * W, g);
    if (!rc) rc = edges_volume(ids, D, H, W, g);
    if (!rc) rc = cliques(g);
    if (!rc) rc = hoods(g);
    if (rc) { orc_graph_free(g); return rc; }
    *out = g;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Build everything for one slice: regions, adjacency, cliques, hoods. */
int orc_build_graph(const double* image, const int32_t* ids, int64_t H, int64_t W, orc_graph** out) {
    if (!out || H < 0 || W < 0 || ((H * W) > 0 && (!image || !ids))) return ORC_ERR_ARG;
    orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
    if (!g) return ORC_ERR_OOM;
    int rc = regions(image, ids, H * W, g);
    if (!rc) rc = edges(ids, H, W, g);
    if (!rc) rc = cliques(g);
    if (!rc) rc = hoods(g);
    if (rc) { orc_graph_free(g); return rc; }
    *out = g;
    return ORC_OK;
}

/* Build cliques and hoods for a given graph (adjacency must be symmetric,
 * ascending, without self loops) and per-vertex intensities.  Used for small
 * hand-made graphs. */
int orc_graph_from_adjacency(int32_t V, const double* y, const int64_t* adj_off, const int32_t* adj,
                             orc_graph** out) {
    if (!out || V < 0) return ORC_ERR_ARG;
    orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
    if (!g) return ORC_ERR_OOM;
    g->V = V; g->max_id = V - 1;
    g->rank = (int32_t*)malloc(sizeof(int32_t) * ((size_t)V + 1));
    g->npix = (int64_t*)malloc(sizeof(int64_t) * ((size_t)V + 1));
    g->y = (double*)malloc(sizeof(double) * ((size_t)V + 1));
    g->adj_off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)V + 1));
    g->n_adj = adj_off[V];
    g->adj = (int32_t*)malloc(sizeof(int32_t) * ((size_t)g->n_adj + 1));
    if (!g->rank || !g->npix || !g->y || !g->adj_off || !g->adj) { orc_graph_free(g); return ORC_ERR_OOM; }
    for (int32_t v = 0; v < V; ++v) { g->rank[v] = v; g->npix[v] = 1; g->y[v] = y[v]; }
    memcpy(g->adj_off, adj_off, sizeof(int64_t) * ((size_t)V + 1));
    memcpy(g->adj, adj, sizeof(int32_t) * (size_t)g->n_adj);
    for (int32_t v = 0; v < V; ++v)
        for (int64_t i = adj_off[v]; i < adj_off[v + 1]; ++i)
            if (adj[i] < 0 || adj[i] >= V || adj[i] == v || (i > adj_off[v] && adj[i] <= adj[i - 1])) {
                orc_graph_free(g);
                return ORC_ERR_ARG;
            }
    int rc = cliques(g);
    if (!rc) rc = hoods(g);
    if (rc) { orc_graph_free(g); return rc; }
    *out = g;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/*
 * Literal replication of the hoods by label (Section 3.2.2, EM step 1,
 * "Replicate Neighborhoods By Label"): for each hood, one copy per label, in
 * the order hood 0 / label 0, hood 0 / label 1, ..., hood 1 / label 0, ...
 * testLabel = label of the copy, oldIndex = index into the hoods array,
 * hoodId = hood of the element, repHoods = hoods[oldIndex].  Output length is
 * L * N_el.  (The CUDA path never materialises these arrays: the label copy is
 * a register loop there.)
 */
int orc_replicate(const int64_t* hood_off, const int32_t* hood, int64_t C, int32_t L, int32_t* testLabel,
                  int32_t* oldIndex, int32_t* hoodId, int32_t* repHoods) {
    int64_t k = 0;
    for (int64_t c = 0; c < C; ++c)
        for (int32_t l = 0; l < L; ++l)
            for (int64_t i = hood_off[c]; i < hood_off[c + 1]; ++i) {
                testLabel[k] = l;
                oldIndex[k] = (int32_t)i;
                hoodId[k] = (int32_t)c;
                repHoods[k] = hood[i];
                ++k;
            }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/*
 * Data term (Section 2.1: the data term is built from the mean intensity of a
 * region; G4): the Gaussian negative log-likelihood of y under label l without
 * its constant 0.5*ln(2*pi):  D_l(y) = (y - mu_l)^2 / (2 sigma_l^2) + ln sigma_l.
 */
static double data_term(double y, double mu, double sigma) {
    double dev = y - mu;
    return dev * dev / (2.0 * sigma * sigma) + log(sigma);
}

/*
 * One MAP sweep (Section 3.2.2, EM step 2: Compute Energy Function, Compute
 * Minimum Vertex and Label Energies, Compute Neighborhood Energy Sums;
 * step 3: Update Output Labels; Algorithm 2, steps 7-10), with labels x and
 * parameters (mu, sigma) of the previous iteration held fixed:
 *
 *   E(c,v,l) = D_l(y_v) + beta * #{u in N(v) n H_c : x_u != l}     (G4: Potts
 *              penalty over the neighbours of v that lie inside hood c)
 *   Emin(c,v) = min_l E(c,v,l); lab(c,v) = smallest l attaining it  (G5)
 *   S_c = sum over v in H_c, ascending v, of Emin(c,v)
 *   (E*_v, x'_v) = lexicographic minimum over the hoods c containing v of
 *                  (Emin(c,v), lab(c,v))                            (G6)
 *
 * Optional outputs (NULL to skip): E_el [N_el*L] every E(c,v,l) in element
 * order; Emin_el, lab_el [N_el]; E_second [V]: the smallest E(c,v,l) over all
 * hoods c containing v with l != x'_v (INFINITY when L == 1).
 */
int orc_map_sweep(const orc_graph* g, int32_t L, double beta, const uint8_t* x, const double* mu,
                  const double* sigma, uint8_t* x_new, double* E_star, double* S_hood, double* E_el,
                  double* Emin_el, uint8_t* lab_el, double* E_second) {
    if (!g || L < 1 || L > 255) return ORC_ERR_ARG;
    const int32_t V = g->V;
    int32_t* best_lab = (int32_t*)malloc(sizeof(int32_t) * ((size_t)V + 1));
    double* best_E = (double*)malloc(sizeof(double) * ((size_t)V + 1));
    double* E = (double*)malloc(sizeof(double) * (size_t)L);
    if (!best_lab || !best_E || !E) { free(best_lab); free(best_E); free(E); return ORC_ERR_OOM; }
    for (int32_t v = 0; v < V; ++v) { best_lab[v] = -1; best_E[v] = INFINITY; }
    for (int64_t c = 0; c < g->C; ++c) {
        const int32_t* Hc = g->hood + g->hood_off[c];
        const int64_t nH = g->hood_off[c + 1] - g->hood_off[c];
        double S = 0.0;
        for (int64_t i = 0; i < nH; ++i) {
            const int32_t v = Hc[i];
            int32_t lab = 0;
            for (int32_t l = 0; l < L; ++l) {
                int64_t m = 0;
                for (int64_t j = g->adj_off[v]; j < g->adj_off[v + 1]; ++j) {
                    int32_t u = g->adj[j];
                    if (contains(Hc, nH, u) && x[u] != l) ++m;
                }
                E[l] = data_term(g->y[v], mu[l], sigma[l]) + beta * (double)m;
                if (E_el) E_el[(g->hood_off[c] + i) * L + l] = E[l];
                if (E[l] < E[lab]) lab = l;
            }
            const double Emin = E[lab];
            S += Emin;
            if (Emin_el) Emin_el[g->hood_off[c] + i] = Emin;
            if (lab_el) lab_el[g->hood_off[c] + i] = (uint8_t)lab;
            if (Emin < best_E[v] || (Emin == best_E[v] && lab < best_lab[v])) {
                best_E[v] = Emin;
                best_lab[v] = lab;
            }
        }
        if (S_hood) S_hood[c] = S;
    }
    for (int32_t v = 0; v < V; ++v) {
        if (x_new) x_new[v] = (uint8_t)best_lab[v];
        if (E_star) E_star[v] = best_E[v];
    }
    if (E_second) {
        for (int32_t v = 0; v < V; ++v) E_second[v] = INFINITY;
        for (int64_t c = 0; c < g->C; ++c) {
            const int32_t* Hc = g->hood + g->hood_off[c];
            const int64_t nH = g->hood_off[c + 1] - g->hood_off[c];
            for (int64_t i = 0; i < nH; ++i) {
                const int32_t v = Hc[i];
                for (int32_t l = 0; l < L; ++l) {
                    if (l == best_lab[v]) continue;
                    int64_t m = 0;
                    for (int64_t j = g->adj_off[v]; j < g->adj_off[v + 1]; ++j) {
                        int32_t u = g->adj[j];
                        if (contains(Hc, nH, u) && x[u] != l) ++m;
                    }
                    double e = data_term(g->y[v], mu[l], sigma[l]) + beta * (double)m;
                    if (e < E_second[v]) E_second[v] = e;
                }
            }
        }
    }
    free(best_lab); free(best_E); free(E);
    return ORC_OK;
}

/*
 * The MAP sweep with two variants of the reading above: the Potts penalty's
 * scope and the rule that turns the replicas' decisions into one label per
 * vertex.  Readings (ours; the paper fixes neither):
 *
 * G13 scope: ORC_SCOPE_HOOD counts the neighbours of v inside hood c (G4);
 *     ORC_SCOPE_FULL counts every neighbour of v, so all replicas of v carry
 *     the same energies  E(c,v,l) = D_l(y_v) + beta * #{u in N(v): x_u != l}.
 * G14 replica rule ("Update Output Labels" scatters one label per vertex from
 *     its replicas, Section 3.2.2 step 3; the winner among replicas is not
 *     specified):
 *     ORC_RULE_MIN   lexicographic minimum of (Emin(c,v), lab(c,v))  (G6);
 *     ORC_RULE_SUM   the mean over v's replicas of E(c,v,l), summed in
 *                    ascending c and divided by the replica count R_v; the
 *                    label of the smallest mean (lower label on ties), E*_v
 *                    its mean;
 *     ORC_RULE_VOTE  each replica votes for lab(c,v); the label with most votes
 *                    (lower label on ties); E*_v = the smallest Emin(c,v) among
 *                    the replicas that voted for it.
 * The hood sums S_c = sum of Emin(c,v) do not depend on the rule.
 *
 * gap[v] (optional): how far the decision of v is from a floating-point tie,
 * relative (g = (b - a) / max(|a|, |b|, 1e-300) for the best value a and the
 * runner-up b): for MIN and SUM over the label values compared; for VOTE the
 * smallest such gap over v's replicas' own argmins (a vote count is an
 * integer: only the per-replica decisions can be near a tie).  INFINITY when
 * nothing competes.
 */
static double rel_gap(double a, double b) {
    double s = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    if (s < 1e-300) s = 1e-300;
    return (b - a) / s;
}

int orc_map_sweep_v(const orc_graph* g, int32_t L, double beta, int32_t scope, int32_t rule, const uint8_t* x,
                    const double* mu, const double* sigma, uint8_t* x_new, double* E_star, double* S_hood,
                    double* gap) {
    if (!g || L < 1 || L > 255 || scope < 0 || scope > 1 || rule < 0 || rule > 2) return ORC_ERR_ARG;
    const int32_t V = g->V;
    const size_t VL = (size_t)V * (size_t)L + 1;
    double* E = (double*)malloc(sizeof(double) * (size_t)L);
    double* acc = (double*)malloc(sizeof(double) * VL);    /* SUM: sums; VOTE: best Emin per label */
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * VL); /* SUM: replica count at [v*L]; VOTE: votes */
    double* best_E = (double*)malloc(sizeof(double) * ((size_t)V + 1));
    int32_t* best_lab = (int32_t*)malloc(sizeof(int32_t) * ((size_t)V + 1));
    double* rgap = (double*)malloc(sizeof(double) * ((size_t)V + 1)); /* VOTE: smallest replica gap */
    if (!E || !acc || !cnt || !best_E || !best_lab || !rgap) {
        free(E); free(acc); free(cnt); free(best_E); free(best_lab); free(rgap);
        return ORC_ERR_OOM;
    }
    for (size_t k = 0; k < VL; ++k) { acc[k] = rule == ORC_RULE_VOTE ? INFINITY : 0.0; cnt[k] = 0; }
    for (int32_t v = 0; v < V; ++v) { best_E[v] = INFINITY; best_lab[v] = -1; rgap[v] = INFINITY; }
    for (int64_t c = 0; c < g->C; ++c) {
        const int32_t* Hc = g->hood + g->hood_off[c];
        const int64_t nH = g->hood_off[c + 1] - g->hood_off[c];
        double S = 0.0;
        for (int64_t i = 0; i < nH; ++i) {
            const int32_t v = Hc[i];
            int32_t lab = 0;
            for (int32_t l = 0; l < L; ++l) {
                int64_t m = 0;
                for (int64_t j = g->adj_off[v]; j < g->adj_off[v + 1]; ++j) {
                    int32_t u = g->adj[j];
                    if ((scope == ORC_SCOPE_FULL || contains(Hc, nH, u)) && x[u] != l) ++m;
                }
                E[l] = data_term(g->y[v], mu[l], sigma[l]) + beta * (double)m;
                if (E[l] < E[lab]) lab = l;
            }
            const double Emin = E[lab];
            S += Emin;
            if (rule == ORC_RULE_MIN) {
                if (Emin < best_E[v] || (Emin == best_E[v] && lab < best_lab[v])) {
                    best_E[v] = Emin;
                    best_lab[v] = lab;
                }
            } else if (rule == ORC_RULE_SUM) {
                for (int32_t l = 0; l < L; ++l) acc[(size_t)v * L + l] += E[l];
                cnt[(size_t)v * L] += 1;
            } else {
                cnt[(size_t)v * L + lab] += 1;
                if (Emin < acc[(size_t)v * L + lab]) acc[(size_t)v * L + lab] = Emin;
                for (int32_t l = 0; l < L; ++l)
                    if (l != lab) {
                        double gg = rel_gap(Emin, E[l]);
                        if (gg < rgap[v]) rgap[v] = gg;
                    }
            }
        }
        if (S_hood) S_hood[c] = S;
    }
    for (int32_t v = 0; v < V; ++v) {
        double gv = INFINITY;
        if (rule == ORC_RULE_MIN) {
            /* runner-up: the smallest energy of any other label in any replica */
            double second = INFINITY;
            for (int64_t c = 0; c < g->C && gap; ++c) {
                const int32_t* Hc = g->hood + g->hood_off[c];
                const int64_t nH = g->hood_off[c + 1] - g->hood_off[c];
                if (!contains(Hc, nH, v)) continue;
                for (int32_t l = 0; l < L; ++l) {
                    if (l == best_lab[v]) continue;
                    int64_t m = 0;
                    for (int64_t j = g->adj_off[v]; j < g->adj_off[v + 1]; ++j) {
                        int32_t u = g->adj[j];
                        if ((scope == ORC_SCOPE_FULL || contains(Hc, nH, u)) && x[u] != l) ++m;
                    }
                    double e = data_term(g->y[v], mu[l], sigma[l]) + beta * (double)m;
                    if (e < second) second = e;
                }
            }
            if (second < INFINITY) gv = rel_gap(best_E[v], second);
        } else if (rule == ORC_RULE_SUM) {
            const double R = (double)cnt[(size_t)v * L];
            int32_t lab = 0;
            for (int32_t l = 0; l < L; ++l) {
                E[l] = acc[(size_t)v * L + l] / R;
                if (E[l] < E[lab]) lab = l;
            }
            best_lab[v] = lab;
            best_E[v] = E[lab];
            for (int32_t l = 0; l < L; ++l)
                if (l != lab) {
                    double gg = rel_gap(E[lab], E[l]);
                    if (gg < gv) gv = gg;
                }
        } else {
            int32_t lab = 0;
            for (int32_t l = 1; l < L; ++l)
                if (cnt[(size_t)v * L + l] > cnt[(size_t)v * L + lab]) lab = l;
            best_lab[v] = lab;
            best_E[v] = acc[(size_t)v * L + lab];
            gv = rgap[v];
        }
        if (x_new) x_new[v] = (uint8_t)best_lab[v];
        if (E_star) E_star[v] = best_E[v];
        if (gap) gap[v] = gv;
    }
    free(E); free(acc); free(cnt); free(best_E); free(best_lab); free(rgap);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/*
 * Multi-core form of the default sweep (hood scope G4, least-energy replica
 * G6), the analogue of the paper's multi-core CPU runs (Section 4.3.4, Table 1):
 * the hoods are split over n_threads OpenMP threads.  Each hood's element
 * energies, argmins and sum are computed by the same statements, in the same
 * order, as orc_map_sweep_v computes them, and each vertex then takes the
 * lexicographic minimum of (Emin(c,v), lab(c,v)) over its replicas, which does
 * not depend on the order the replicas are visited: the outputs are identical
 * to orc_map_sweep_v's (scope ORC_SCOPE_HOOD, rule ORC_RULE_MIN).  rep_off /
 * rep_el: the elements of each vertex (orc_replica_lists).  Serial when the
 * library is built without OpenMP.
 */
int orc_replica_lists(const orc_graph* g, int64_t** rep_off, int64_t** rep_el) {
    if (!g || !rep_off || !rep_el) return ORC_ERR_ARG;
    const int32_t V = g->V;
    int64_t* off = (int64_t*)calloc((size_t)V + 1, sizeof(int64_t));
    int64_t* el = (int64_t*)malloc(sizeof(int64_t) * ((size_t)g->N_el + 1));
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * ((size_t)V + 1));
    if (!off || !el || !cur) { free(off); free(el); free(cur); return ORC_ERR_OOM; }
    for (int64_t e = 0; e < g->N_el; ++e) off[g->hood[e] + 1] += 1;
    for (int32_t v = 0; v < V; ++v) off[v + 1] += off[v];
    for (int32_t v = 0; v < V; ++v) cur[v] = off[v];
    for (int64_t e = 0; e < g->N_el; ++e) el[cur[g->hood[e]]++] = e;
    free(cur);
    *rep_off = off;
    *rep_el = el;
    return ORC_OK;
}

int orc_map_sweep_par(const orc_graph* g, int32_t L, double beta, const uint8_t* x, const double* mu,
                      const double* sigma, const int64_t* rep_off, const int64_t* rep_el, int32_t n_threads,
                      uint8_t* x_new, double* E_star, double* S_hood) {
    if (!g || L < 1 || L > 255 || !rep_off || !rep_el || n_threads < 1) return ORC_ERR_ARG;
    double* Emin_el = (double*)malloc(sizeof(double) * ((size_t)g->N_el + 1));
    int32_t* lab_el = (int32_t*)malloc(sizeof(int32_t) * ((size_t)g->N_el + 1));
    if (!Emin_el || !lab_el) { free(Emin_el); free(lab_el); return ORC_ERR_OOM; }
    int oom = 0;
#pragma omp parallel num_threads(n_threads)
    {
        double* E = (double*)malloc(sizeof(double) * (size_t)L);
        if (!E) {
#pragma omp atomic write
            oom = 1;
        }
#pragma omp for schedule(dynamic, 256)
        for (int64_t c = 0; c < g->C; ++c) {
            if (!E) continue;
            const int32_t* Hc = g->hood + g->hood_off[c];
            const int64_t nH = g->hood_off[c + 1] - g->hood_off[c];
            double S = 0.0;
            for (int64_t i = 0; i < nH; ++i) {
                const int32_t v = Hc[i];
                int32_t lab = 0;
                for (int32_t l = 0; l < L; ++l) {
                    int64_t m = 0;
                    for (int64_t j = g->adj_off[v]; j < g->adj_off[v + 1]; ++j) {
                        int32_t u = g->adj[j];
                        if (contains(Hc, nH, u) && x[u] != l) ++m;
                    }
                    E[l] = data_term(g->y[v], mu[l], sigma[l]) + beta * (double)m;
                    if (E[l] < E[lab]) lab = l;
                }
                Emin_el[g->hood_off[c] + i] = E[lab];
                lab_el[g->hood_off[c] + i] = lab;
                S += E[lab];
            }
            if (S_hood) S_hood[c] = S;
        }
        free(E);
    }
    if (oom) { free(Emin_el); free(lab_el); return ORC_ERR_OOM; }
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int32_t v = 0; v < g->V; ++v) {
        double bE = INFINITY;
        int32_t bl = -1;
        for (int64_t k = rep_off[v]; k < rep_off[v + 1]; ++k) {
            const double e = Emin_el[rep_el[k]];
            const int32_t l = lab_el[rep_el[k]];
            if (e < bE || (e == bE && l < bl)) { bE = e; bl = l; }
        }
        if (x_new) x_new[v] = (uint8_t)bl;
        if (E_star) E_star[v] = bE;
    }
    free(Emin_el); free(lab_el);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/*
 * Parameter update (Section 3.2.2, EM step 4, "Update Parameters": mu and sigma
 * of each label from the intensities of the vertices carrying that label, plus
 * the per-label sums of the vertex energies).  Readings (G8): moments over
 * vertices; population variance (divide by n), two passes (mean first);
 * sigma floored at sigma_min; a label with no vertex keeps its previous mu and
 * sigma.  U_l = sum of E*_v over the vertices with label l (0 when E_star is
 * NULL).  theta layout [L][4] = (n_l, mu_l, sigma_l, U_l).  Sums run in
 * ascending v.
 */
int orc_params(const orc_graph* g, int32_t L, const uint8_t* x, const double* E_star, const double* theta_prev,
               double sigma_min, double* theta_out) {
    if (!g || L < 1 || !theta_prev || !theta_out) return ORC_ERR_ARG;
    for (int32_t l = 0; l < L; ++l) {
        int64_t n = 0;
        double s = 0.0, u = 0.0;
        for (int32_t v = 0; v < g->V; ++v)
            if (x[v] == l) {
                ++n;
                s += g->y[v];
                if (E_star) u += E_star[v];
            }
        double* t = theta_out + 4 * l;
        if (n == 0) {
            t[0] = 0.0; t[1] = theta_prev[4 * l + 1]; t[2] = theta_prev[4 * l + 2]; t[3] = 0.0;
            continue;
        }
        const double mean = s / (double)n;
        double ss = 0.0;
        for (int32_t v = 0; v < g->V; ++v)
            if (x[v] == l) {
                double d = g->y[v] - mean;
                ss += d * d;
            }
        double sd = sqrt(ss / (double)n);
        t[0] = (double)n; t[1] = mean; t[2] = sd > sigma_min ? sd : sigma_min; t[3] = u;
    }
    return ORC_OK;
}

/*
 * Initial labels (Algorithm 2, step 3).  The paper draws labels and parameters
 * at random; reading G3 (ours) thresholds the region means instead:
 * x_v = clamp(floor((y_v - lo) / (hi - lo) * L), 0, L-1), i.e. for L = 2 on
 * [0,1] a cut at 0.5.
 */
int orc_init_labels(const orc_graph* g, int32_t L, double lo, double hi, uint8_t* x) {
    if (!g || L < 1 || !(hi > lo)) return ORC_ERR_ARG;
    for (int32_t v = 0; v < g->V; ++v) {
        double q = floor((g->y[v] - lo) / (hi - lo) * (double)L);
        int32_t l = q < 0.0 ? 0 : (q > (double)(L - 1) ? L - 1 : (int32_t)q);
        x[v] = (uint8_t)l;
    }
    return ORC_OK;
}

/* Initial parameters: label-conditional moments of the initial labels; an
 * empty label starts at the centre of its threshold bin with sigma = the bin
 * width (G3, ours). */
int orc_init_params(const orc_graph* g, int32_t L, double lo, double hi, double sigma_min, const uint8_t* x,
                    double* theta) {
    if (!g || L < 1) return ORC_ERR_ARG;
    double* prev = (double*)malloc(sizeof(double) * 4 * (size_t)L);
    if (!prev) return ORC_ERR_OOM;
    for (int32_t l = 0; l < L; ++l) {
        prev[4 * l + 0] = 0.0;
        prev[4 * l + 1] = lo + ((double)l + 0.5) * (hi - lo) / (double)L;
        prev[4 * l + 2] = (hi - lo) / (double)L;
        prev[4 * l + 3] = 0.0;
    }
    int rc = orc_params(g, L, x, NULL, prev, sigma_min, theta);
    free(prev);
    return rc;
}

/* ------------------------------------------------------------------------ */
/*
 * The two convergence tests of Section 3.2.2 after iteration t (reading G9),
 * on rings of the last W+1 hood sums (Shist, C entries per slot) and totals
 * (Thist), slot t % (W+1) holding iteration t:
 *   MAP convergence check: every hood c has t > W and
 *       max_{k=1..W} |S^t_c - S^{t-k}_c| < tol            -> *hood_ok = 1
 *   EM convergence check:  t > W and
 *       max_{k=1..W} |T^t - T^{t-k}| < tol                 -> *total_ok = 1
 * ("the change over the previous W iterations" read as the largest absolute
 * difference against each of them).
 */
static void stop_tests(int32_t t, int32_t W, double tol, int64_t C, const double* Shist, const double* Thist,
                       int32_t* hood_ok, int32_t* total_ok) {
    *hood_ok = 0;
    *total_ok = 0;
    if (t <= W) return;
    const double* S = Shist + (size_t)(t % (W + 1)) * (size_t)C;
    int32_t all = 1;
    for (int64_t c = 0; c < C && all; ++c) {
        double dmax = 0.0;
        for (int32_t k = 1; k <= W; ++k) {
            double d = fabs(S[c] - Shist[(size_t)((t - k) % (W + 1)) * (size_t)C + (size_t)c]);
            if (d > dmax) dmax = d;
        }
        if (!(dmax < tol)) all = 0;
    }
    const double T = Thist[t % (W + 1)];
    double dT = 0.0;
    for (int32_t k = 1; k <= W; ++k) {
        double d = fabs(T - Thist[(t - k) % (W + 1)]);
        if (d > dT) dT = d;
    }
    *hood_ok = all;
    *total_ok = dT < tol ? 1 : 0;
}

/*
 * The convergence tests of stop_tests on given histories: S_seq [t][C] holds
 * S^1 .. S^t (row k-1 = iteration k), T_seq [t] holds T^1 .. T^t; the tests
 * are evaluated after iteration t, exactly as the EM loop evaluates them.
 */
int orc_stop_rule(int32_t t, int32_t W, double tol, int64_t C, const double* S_seq, const double* T_seq,
                  int32_t* hood_ok, int32_t* total_ok) {
    if (t < 1 || W < 1 || C < 0 || !S_seq || !T_seq || !hood_ok || !total_ok) return ORC_ERR_ARG;
    double* Shist = (double*)calloc((size_t)(W + 1) * (size_t)(C > 0 ? C : 1), sizeof(double));
    double* Thist = (double*)calloc((size_t)(W + 1), sizeof(double));
    if (!Shist || !Thist) { free(Shist); free(Thist); return ORC_ERR_OOM; }
    for (int32_t k = (t - W > 1 ? t - W : 1); k <= t; ++k) {
        memcpy(Shist + (size_t)(k % (W + 1)) * (size_t)C, S_seq + (size_t)(k - 1) * (size_t)C,
               sizeof(double) * (size_t)C);
        Thist[k % (W + 1)] = T_seq[k - 1];
    }
    stop_tests(t, W, tol, C, Shist, Thist, hood_ok, total_ok);
    free(Shist); free(Thist);
    return ORC_OK;
}

/*
 * The EM loop (Algorithm 2, steps 6-11; Section 3.2.2, EM steps 2-5), with the
 * sweep variant cfg->potts_scope / cfg->replica_rule (G13, G14).  The start
 * (Algorithm 2 step 3): cfg->init_mode 0 thresholds the region means (G3);
 * 1 takes the labels in x and the moments of them; 2 takes the labels in x
 * and mu, sigma in theta (sigma floored at sigma_min), e.g. the random draw
 * of orc_random_init.
 *   x^0, theta^0: orc_init_labels / orc_init_params.
 *   for t = 1, 2, ...:
 *     (x^t, E*, S^t) = sweep(x^{t-1}, theta^{t-1});  theta^t = params(x^t, E*)
 *     T^t = sum_c S^t_c (ascending c)
 *     stop when the MAP convergence check (every hood converged) or the EM
 *     convergence check (the total) holds (stop_tests), or t = max_iters.
 * Either test ends the loop (G9).  With cfg->n_threads > 1 the default sweep
 * runs on that many threads (orc_map_sweep_par: identical results).
 * Outputs: x = x^t, theta = theta^t, *iters = t, *converged = 1 when a
 * convergence test (not the cap) ended the loop; T_hist[t-1] = T^t (optional,
 * length max_iters); *reason (optional): which tests held at the last
 * iteration, bit 0 the MAP (hood) check, bit 1 the EM (total) check, 0 when the
 * cap ended the loop.  V == 0 returns at once with iters 0, converged 1.
 */
int orc_em_ex(const orc_graph* g, const orc_config* cfg, uint8_t* x, double* theta, int32_t* iters,
              int32_t* converged, double* T_hist, int32_t* reason) {
    if (!g || !cfg || cfg->n_labels < 1 || cfg->max_iters < 1 || cfg->conv_window < 1) return ORC_ERR_ARG;
    if (cfg->potts_scope < 0 || cfg->potts_scope > 1 || cfg->replica_rule < 0 || cfg->replica_rule > 2)
        return ORC_ERR_ARG;
    const int32_t L = cfg->n_labels, W = cfg->conv_window, V = g->V;
    const int64_t C = g->C;
    if (cfg->init_mode < 0 || cfg->init_mode > 2) return ORC_ERR_ARG;
    int rc = ORC_OK;
    if (cfg->init_mode == 0) rc = orc_init_labels(g, L, cfg->init_lo, cfg->init_hi, x);
    for (int32_t v = 0; v < V && !rc; ++v)
        if (x[v] >= L) rc = ORC_ERR_ARG;
    if (!rc && cfg->init_mode < 2) rc = orc_init_params(g, L, cfg->init_lo, cfg->init_hi, cfg->sigma_min, x, theta);
    if (!rc && cfg->init_mode == 2)  /* given parameters: sigma floored, counts and energies cleared */
        for (int32_t l = 0; l < L; ++l) {
            theta[4 * l + 0] = 0.0;
            if (!(theta[4 * l + 2] > cfg->sigma_min)) theta[4 * l + 2] = cfg->sigma_min;
            theta[4 * l + 3] = 0.0;
        }
    if (rc) return rc;
    *iters = 0; *converged = 1;
    if (reason) *reason = 0;
    if (V == 0) return ORC_OK;
    double* Shist = (double*)malloc(sizeof(double) * (size_t)((W + 1) * C + 1)); /* ring of W+1 */
    double* Thist = (double*)malloc(sizeof(double) * (size_t)(W + 1));
    uint8_t* xn = (uint8_t*)malloc((size_t)V);
    double* Es = (double*)malloc(sizeof(double) * (size_t)V);
    double* mu = (double*)malloc(sizeof(double) * (size_t)L);
    double* sg = (double*)malloc(sizeof(double) * (size_t)L);
    double* th2 = (double*)malloc(sizeof(double) * 4 * (size_t)L);
    int64_t *rep_off = NULL, *rep_el = NULL;
    const int par = cfg->n_threads > 1 && cfg->potts_scope == ORC_SCOPE_HOOD && cfg->replica_rule == ORC_RULE_MIN;
    if (!Shist || !Thist || !xn || !Es || !mu || !sg || !th2) { rc = ORC_ERR_OOM; goto done; }
    if (par && (rc = orc_replica_lists(g, &rep_off, &rep_el)) != ORC_OK) goto done;
    *converged = 0;
    for (int32_t t = 1; t <= cfg->max_iters; ++t) {
        for (int32_t l = 0; l < L; ++l) { mu[l] = theta[4 * l + 1]; sg[l] = theta[4 * l + 2]; }
        double* S = Shist + (size_t)(t % (W + 1)) * (size_t)C;
        if (par)
            rc = orc_map_sweep_par(g, L, cfg->beta, x, mu, sg, rep_off, rep_el, cfg->n_threads, xn, Es, S);
        else
            rc = orc_map_sweep_v(g, L, cfg->beta, cfg->potts_scope, cfg->replica_rule, x, mu, sg, xn, Es, S, NULL);
        if (rc) goto done;
        memcpy(x, xn, (size_t)V);
        rc = orc_params(g, L, x, Es, theta, cfg->sigma_min, th2);
        if (rc) goto done;
        memcpy(theta, th2, sizeof(double) * 4 * (size_t)L);
        double T = 0.0;
        for (int64_t c = 0; c < C; ++c) T += S[c];
        Thist[t % (W + 1)] = T;
        if (T_hist) T_hist[t - 1] = T;
        *iters = t;
        int32_t hood_ok = 0, total_ok = 0;
        stop_tests(t, W, cfg->conv_tol, C, Shist, Thist, &hood_ok, &total_ok);
        if (hood_ok || total_ok) {
            *converged = 1;
            if (reason) *reason = hood_ok | (total_ok << 1);
            break;
        }
    }
done:
    free(Shist); free(Thist); free(xn); free(Es); free(mu); free(sg); free(th2); free(rep_off); free(rep_el);
    return rc;
}

int orc_em(const orc_graph* g, const orc_config* cfg, uint8_t* x, double* theta, int32_t* iters, int32_t* converged,
           double* T_hist) {
    return orc_em_ex(g, cfg, x, theta, iters, converged, T_hist, NULL);
}

/* ------------------------------------------------------------------------ */
/*
 * Vertex pseudo-log-likelihood and its gradient (not in the paper; the
 * differentiable form built beside the method, reading G10).  With labels x
 * fixed, over the full graph neighbourhood:
 *   E_v(l) = D_l(y_v) + beta * m_v(l),   m_v(l) = #{u in N(v): x_u != l}
 *   PLL = sum_v [ -E_v(x_v) - log sum_l exp(-E_v(l)) ]
 * (log-sum-exp with the largest term factored out).  Gradients:
 *   dPLL/dmu_k    = sum_v (p_v(k) - [x_v = k]) * (mu_k - y_v) / sigma_k^2
 *   dPLL/dsigma_k = sum_v (p_v(k) - [x_v = k]) * (1/sigma_k - (y_v - mu_k)^2 / sigma_k^3)
 *   dPLL/dbeta    = sum_v ( sum_l p_v(l) m_v(l) - m_v(x_v) )
 * with p_v = softmax(-E_v).  Sums run in ascending v.  Any output may be NULL.
 */
int orc_pll(const orc_graph* g, int32_t L, const uint8_t* x, const double* mu, const double* sigma, double beta,
            double* pll, double* g_mu, double* g_sigma, double* g_beta) {
    if (!g || L < 1) return ORC_ERR_ARG;
    double* E = (double*)malloc(sizeof(double) * (size_t)L);
    double* p = (double*)malloc(sizeof(double) * (size_t)L);
    int64_t* m = (int64_t*)malloc(sizeof(int64_t) * (size_t)L);
    if (!E || !p || !m) { free(E); free(p); free(m); return ORC_ERR_OOM; }
    double acc = 0.0, gb = 0.0;
    if (g_mu) for (int32_t l = 0; l < L; ++l) g_mu[l] = 0.0;
    if (g_sigma) for (int32_t l = 0; l < L; ++l) g_sigma[l] = 0.0;
    for (int32_t v = 0; v < g->V; ++v) {
        const double yv = g->y[v];
        double emin = INFINITY;
        for (int32_t l = 0; l < L; ++l) {
            m[l] = 0;
            for (int64_t j = g->adj_off[v]; j < g->adj_off[v + 1]; ++j)
                if (x[g->adj[j]] != l) ++m[l];
            E[l] = data_term(yv, mu[l], sigma[l]) + beta * (double)m[l];
            if (E[l] < emin) emin = E[l];
        }
        double z = 0.0;
        for (int32_t l = 0; l < L; ++l) z += exp(-(E[l] - emin));
        const double lse = -emin + log(z); /* log sum_l exp(-E_l) */
        acc += -E[x[v]] - lse;
        for (int32_t l = 0; l < L; ++l) p[l] = exp(-(E[l] - emin)) / z;
        double eb = 0.0;
        for (int32_t l = 0; l < L; ++l) eb += p[l] * (double)m[l];
        gb += eb - (double)m[x[v]];
        for (int32_t k = 0; k < L; ++k) {
            const double w = p[k] - (x[v] == k ? 1.0 : 0.0);
            const double s2 = sigma[k] * sigma[k];
            const double dev = yv - mu[k];
            if (g_mu) g_mu[k] += w * (mu[k] - yv) / s2;
            if (g_sigma) g_sigma[k] += w * (1.0 / sigma[k] - dev * dev / (s2 * sigma[k]));
        }
    }
    if (pll) *pll = acc;
    if (g_beta) *g_beta = gb;
    free(E); free(p); free(m);
    return ORC_OK;
}

/*
 * Fit of the Potts weight beta by gradient ascent on the summed vertex
 * pseudo-log-likelihood of a batch of n slices (reading G11, beside the
 * paper): labels and every slice's (mu, sigma) held fixed,
 *   beta_{k+1} = max(0, beta_k + lr * (1 / sum_s V_s) * sum_s dPLL_s/dbeta (beta_k))
 * for k = 0 .. steps-1, the slices' derivatives (orc_pll) summed in ascending
 * s.  gs[s], xs[s]: graph and labels of slice s; mu, sigma [n][L].
 * traj [steps+1] receives beta_0 .. beta_steps.
 */
int orc_fit_beta(const orc_graph* const* gs, int32_t n, int32_t L, const uint8_t* const* xs, const double* mu,
                 const double* sigma, double beta0, int32_t steps, double lr, double* traj) {
    if (!gs || !xs || !mu || !sigma || !traj || n < 1 || L < 1 || steps < 0) return ORC_ERR_ARG;
    int64_t Vtot = 0;
    for (int32_t s = 0; s < n; ++s) {
        if (!gs[s] || !xs[s]) return ORC_ERR_ARG;
        Vtot += gs[s]->V;
    }
    if (Vtot < 1) Vtot = 1;
    double beta = beta0;
    traj[0] = beta;
    for (int32_t k = 0; k < steps; ++k) {
        double gsum = 0.0;
        for (int32_t s = 0; s < n; ++s) {
            double gb = 0.0;
            int rc = orc_pll(gs[s], L, xs[s], mu + (size_t)s * (size_t)L, sigma + (size_t)s * (size_t)L, beta, NULL,
                             NULL, NULL, &gb);
            if (rc) return rc;
            gsum += gb;
        }
        beta = beta + lr * (gsum / (double)Vtot);
        if (beta < 0.0) beta = 0.0;
        traj[k + 1] = beta;
    }
    return ORC_OK;
}

/* Labels back to pixels (Section 3.2.2, closing paragraph: vertex labels map
 * back to the pixels of their regions). */
int orc_label_image(const orc_graph* g, const int32_t* ids, int64_t npx, const uint8_t* x, uint8_t* out) {
    if (!g) return ORC_ERR_ARG;
    for (int64_t p = 0; p < npx; ++p) {
        if (ids[p] < 0 || ids[p] > g->max_id || g->rank[ids[p]] < 0) return ORC_ERR_ARG;
        out[p] = x[g->rank[ids[p]]];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Segmentation quality against a ground truth (Section 4.2.1, evaluation
 * metrics).  The paper defines precision TP/(TP+FP), recall TP/(TP+FN),
 * accuracy (TP+TN)/(TP+TN+FP+FN) for a two-phase segmentation and the
 * porosity as the void volume over the total volume.  Reading G12: with L
 * labels every label l is scored one-against-the-rest (TP: truth l and
 * prediction l; FP: prediction l, truth other; FN: truth l, prediction other;
 * TN: neither); the porosity of label l is the fraction of pixels carrying l
 * (of the prediction and of the truth); a ratio whose denominator is 0 is NaN.
 *
 * conf[t*L + q] = number of pixels with truth t and prediction q;
 * metrics[l*5 + k] = precision, recall, accuracy, predicted fraction, true
 * fraction of label l.  Labels outside [0, L) are an argument error. */
int orc_quality(const uint8_t* pred, const uint8_t* truth, int64_t npx, int32_t L, int64_t* conf, double* metrics) {
    if (L < 1 || L > 255 || npx < 0) return ORC_ERR_ARG;
    for (int64_t k = 0; k < (int64_t)L * L; ++k) conf[k] = 0;
    for (int64_t p = 0; p < npx; ++p) {
        if (pred[p] >= L || truth[p] >= L) return ORC_ERR_ARG;
        conf[(int64_t)truth[p] * L + pred[p]] += 1;
    }
    for (int32_t l = 0; l < L; ++l) {
        int64_t tp = conf[(int64_t)l * L + l], fp = 0, fn = 0;
        for (int32_t t = 0; t < L; ++t)
            if (t != l) fp += conf[(int64_t)t * L + l];
        for (int32_t q = 0; q < L; ++q)
            if (q != l) fn += conf[(int64_t)l * L + q];
        const int64_t tn = npx - tp - fp - fn;
        double* m = metrics + (int64_t)l * 5;
        m[0] = (tp + fp) > 0 ? (double)tp / (double)(tp + fp) : NAN;
        m[1] = (tp + fn) > 0 ? (double)tp / (double)(tp + fn) : NAN;
        m[2] = npx > 0 ? (double)(tp + tn) / (double)npx : NAN;
        m[3] = npx > 0 ? (double)(tp + fp) / (double)npx : NAN;
        m[4] = npx > 0 ? (double)(tp + fn) / (double)npx : NAN;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Random start (Algorithm 2 step 3; Section 3.2.2: the label means and
 * deviations are drawn between 0 and 255 and every vertex label is drawn at
 * random).  The draws come from SplitMix64 (Steele, Lea, Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), used as a
 * counter-based generator: splitmix64(key, i) is the output of the (i+1)-th
 * step from state key.  Reading G15: for slice s, key_x = splitmix64(seed, 2s)
 * and key_t = splitmix64(seed, 2s+1); label of vertex v = the high 32 bits of
 * splitmix64(key_x, v) times L, shifted down 32 (uniform over [0, L));
 * mu_l = lo + (hi - lo) * u(splitmix64(key_t, 2l)), sigma_l = lo + (hi - lo) *
 * u(splitmix64(key_t, 2l+1)), u(r) = (r >> 11) * 2^-53 in [0, 1). */
uint64_t orc_splitmix64(uint64_t key, uint64_t i) {
    uint64_t z = key + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int orc_random_init(int32_t V, int32_t L, uint64_t seed, int64_t slice, double lo, double hi, uint8_t* x,
                    double* theta) {
    if (V < 0 || L < 1 || L > 255 || slice < 0 || !(hi >= lo)) return ORC_ERR_ARG;
    const uint64_t kx = orc_splitmix64(seed, 2 * (uint64_t)slice);
    const uint64_t kt = orc_splitmix64(seed, 2 * (uint64_t)slice + 1);
    for (int32_t v = 0; v < V; ++v) x[v] = (uint8_t)(((orc_splitmix64(kx, (uint64_t)v) >> 32) * (uint64_t)L) >> 32);
    const double w = hi - lo;
    for (int32_t l = 0; l < L; ++l) {
        const double u0 = (double)(orc_splitmix64(kt, 2 * (uint64_t)l) >> 11) * 0x1p-53;
        const double u1 = (double)(orc_splitmix64(kt, 2 * (uint64_t)l + 1) >> 11) * 0x1p-53;
        theta[4 * l + 0] = 0.0;
        theta[4 * l + 1] = lo + w * u0;
        theta[4 * l + 2] = lo + w * u1;
        theta[4 * l + 3] = 0.0;
    }
    return ORC_OK;
}
