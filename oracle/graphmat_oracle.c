/*
 * GraphMat FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, serial restatement of what the GraphMat paper (Sundaram et al.,
 * "GraphMat: High performance graph analytics made productive", VLDB 2015)
 * computes.  Only the tests, the package smoke check and the benchmark's CPU
 * baseline leg may load it; the CUDA library never calls it and shares no code,
 * header or table with it.
 *
 *  - Edge cleaning (Section 5.1): self-loop removal, duplicate removal (the first
 *    occurrence in input order is kept), symmetrisation and degree orientation.
 *  - The vertex-program engine is Algorithm 2 (Run_Graph_Program) around
 *    Algorithm 1 (generalized SPMV over the CSC form of G^T, i.e. a push over
 *    the out-edges of each present column), with FP64 vertex state.
 *  - PageRank follows Eq. 1, BFS the distance update of Section 3.II, SSSP the
 *    min-plus update of Section 3.V and the appendix program, triangle counting
 *    the two vertex programs of Section 4.2, collaborative filtering Eqs. 3-5
 *    (gradient descent, and stochastic gradient descent in a stratified order),
 *    and weighted PageRank (an added form) Eq. 1 with row-normalised edge
 *    weights plus its reverse-mode derivative.
 *
 * Precision: every floating-point quantity is double; BFS/SSSP distances and
 * triangle counts are exact integers (held in double below 2^53, or uint64).
 *
 * For timing on many host cores only, PageRank, BFS and SSSP also run on
 * OpenMP threads: PageRank on a pull engine (or_run_graph_program_pull) that
 * evaluates Algorithm 1 per destination with the serial engine's Reduce order,
 * BFS and SSSP on a push engine (or_run_min_program_threads) whose Reduce, an
 * exact minimum, is applied with atomic compare-and-swap; both give results
 * identical to the serial engine's (tested).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EXPORT __attribute__((visibility("default")))

enum { OR_DROP_SELF_LOOPS = 1, OR_DEDUP = 2, OR_SYMMETRIZE = 4, OR_ORIENT_BY_DEGREE = 8 };

#define OR_INF_U32 4294967295.0 /* "infinity" distance of BFS/SSSP */

typedef struct or_graph {
    int64_t n, m;
    int32_t* src;       /* edges sorted by (src, dst) */
    int32_t* dst;
    double* val;        /* edge value (weight or rating); 1.0 when unweighted */
    int64_t* out_begin; /* out-edges of v are [out_begin[v], out_begin[v+1]) */
    int64_t* in_deg;
} or_graph;

/* ------------------------------------------------------------------------- */
/* Edge cleaning and storage                                                  */
/* ------------------------------------------------------------------------- */

typedef struct { int32_t s, d; int64_t order; double v; } or_edge;

static int or_edge_cmp(const void* a, const void* b) {
    const or_edge* x = (const or_edge*)a;
    const or_edge* y = (const or_edge*)b;
    if (x->s != y->s) return x->s < y->s ? -1 : 1;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    if (x->order != y->order) return x->order < y->order ? -1 : 1; /* keeps the sort stable */
    return 0;
}

/*
 * Build the cleaned graph.  `wtype` 0 = unweighted, 1 = uint32 values, 2 = float
 * values.  Symmetrisation appends the reversed copy of every input edge after
 * all originals (same value); orientation keeps u->v only when
 * (deg(u), u) < (deg(v), v) with deg taken in the graph at that point.
 * Returns NULL on a bad id or allocation failure.
 */
OR_EXPORT or_graph* or_graph_create(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                    const void* w, int32_t wtype, uint32_t flags) {
    int64_t cap = (flags & OR_SYMMETRIZE) ? 2 * m : m;
    or_edge* e = (or_edge*)malloc(sizeof(or_edge) * (size_t)(cap > 0 ? cap : 1));
    if (!e) return NULL;
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) { free(e); return NULL; }
        double v = 1.0;
        if (wtype == 1) v = (double)((const uint32_t*)w)[i];
        else if (wtype == 2) v = (double)((const float*)w)[i];
        e[k].s = src[i]; e[k].d = dst[i]; e[k].order = k; e[k].v = v; ++k;
    }
    if (flags & OR_SYMMETRIZE)
        for (int64_t i = 0; i < m; ++i) {
            e[k].s = e[i].d; e[k].d = e[i].s; e[k].order = k; e[k].v = e[i].v; ++k;
        }
    /* drop self-loops */
    int64_t kk = 0;
    for (int64_t i = 0; i < k; ++i)
        if (!((flags & OR_DROP_SELF_LOOPS) && e[i].s == e[i].d)) e[kk++] = e[i];
    k = kk;
    qsort(e, (size_t)k, sizeof(or_edge), or_edge_cmp);
    /* dedup: first occurrence in input order survives (stable sort puts it first) */
    if (flags & OR_DEDUP) {
        kk = 0;
        for (int64_t i = 0; i < k; ++i)
            if (kk == 0 || e[kk - 1].s != e[i].s || e[kk - 1].d != e[i].d) e[kk++] = e[i];
        k = kk;
    }
    if (flags & OR_ORIENT_BY_DEGREE) {
        int64_t* deg = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
        if (!deg) { free(e); return NULL; }
        for (int64_t i = 0; i < k; ++i) deg[e[i].s]++;
        kk = 0;
        for (int64_t i = 0; i < k; ++i) {
            int64_t du = deg[e[i].s], dv = deg[e[i].d];
            if (du < dv || (du == dv && e[i].s < e[i].d)) e[kk++] = e[i];
        }
        k = kk;
        free(deg);
    }
    or_graph* g = (or_graph*)calloc(1, sizeof(or_graph));
    if (!g) { free(e); return NULL; }
    g->n = n; g->m = k;
    g->src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
    g->dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
    g->val = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    g->out_begin = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    g->in_deg = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!g->src || !g->dst || !g->val || !g->out_begin || !g->in_deg) { free(e); return NULL; }
    for (int64_t i = 0; i < k; ++i) {
        g->src[i] = e[i].s; g->dst[i] = e[i].d; g->val[i] = e[i].v;
        g->out_begin[e[i].s + 1]++;
        g->in_deg[e[i].d]++;
    }
    for (int64_t v = 0; v < n; ++v) g->out_begin[v + 1] += g->out_begin[v];
    free(e);
    return g;
}

OR_EXPORT void or_graph_destroy(or_graph* g) {
    if (!g) return;
    free(g->src); free(g->dst); free(g->val); free(g->out_begin); free(g->in_deg); free(g);
}

OR_EXPORT int64_t or_graph_m(const or_graph* g) { return g->m; }
OR_EXPORT int64_t or_graph_n(const or_graph* g) { return g->n; }

/* Copy the cleaned edge list (sorted by (src, dst)) out. */
OR_EXPORT void or_graph_edges(const or_graph* g, int32_t* src, int32_t* dst, double* val) {
    for (int64_t i = 0; i < g->m; ++i) {
        if (src) src[i] = g->src[i];
        if (dst) dst[i] = g->dst[i];
        if (val) val[i] = g->val[i];
    }
}

OR_EXPORT void or_graph_degrees(const or_graph* g, int64_t* out_deg, int64_t* in_deg) {
    for (int64_t v = 0; v < g->n; ++v) {
        if (out_deg) out_deg[v] = g->out_begin[v + 1] - g->out_begin[v];
        if (in_deg) in_deg[v] = g->in_deg[v];
    }
}

/* ------------------------------------------------------------------------- */
/* Vertex-program engine: Algorithm 1 inside Algorithm 2                      */
/* ------------------------------------------------------------------------- */

typedef struct or_program or_program;
struct or_program {
    /* Send_Message: message of an active vertex; returns 0 to send nothing. */
    int (*send_message)(const or_program* P, const or_graph* G, int64_t v, double prop, double* msg);
    /* Process_Message(message, edge value, destination property) */
    double (*process_message)(const or_program* P, double msg, double edge_value, double dst_prop);
    /* Reduce(a, b): commutative combine of two processed messages */
    double (*reduce)(double a, double b);
    /* Apply(reduced value, property) -> new property */
    double (*apply)(const or_program* P, double reduced, double prop);
    int all_active;   /* every vertex is active in every superstep (fixed-iteration programs) */
    int apply_to_all; /* apply also to vertices without messages, with y = identity */
    double identity;
    double r;         /* PageRank random-surf probability */
    int64_t iter;     /* current superstep index t (0-based) */
};

/* Algorithm 1: y = SPMV(G, x).  Columns j of G^T are the source vertices; a
 * present x_j is pushed along every out-edge j -> k in sorted order. */
static void or_spmv(const or_graph* G, const uint8_t* x_present, const double* x, const double* prop,
                    const or_program* P, uint8_t* y_present, double* y) {
    for (int64_t j = 0; j < G->n; ++j) {
        if (G->out_begin[j] == G->out_begin[j + 1]) continue; /* only non-empty columns */
        if (!x_present[j]) continue;
        for (int64_t e = G->out_begin[j]; e < G->out_begin[j + 1]; ++e) {
            int64_t k = G->dst[e];
            double result = P->process_message(P, x[j], G->val[e], prop[k]);
            if (!y_present[k]) { y_present[k] = 1; y[k] = result; }
            else y[k] = P->reduce(y[k], result);
        }
    }
}

/* Algorithm 2: returns the number of supersteps executed (the superstep that
 * finds no active vertex is counted), or -1 on allocation failure.
 * max_iters < 0 runs until no vertex is active. */
static int64_t or_run_graph_program(const or_graph* G, or_program* P, double* prop, uint8_t* active,
                                    int64_t max_iters) {
    const int64_t n = G->n;
    const size_t nz = (size_t)(n > 0 ? n : 0);
    uint8_t* xp = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    uint8_t* yp = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    double* x = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!xp || !yp || !x || !y) { free(xp); free(yp); free(x); free(y); return -1; }
    int64_t it = 0;
    for (it = 0; max_iters < 0 || it < max_iters; ++it) {
        P->iter = it;
        for (int64_t v = 0; v < n; ++v) { /* send_message from active vertices */
            xp[v] = 0;
            if (active[v] && P->send_message(P, G, v, prop[v], &x[v])) xp[v] = 1;
        }
        memset(yp, 0, nz);
        or_spmv(G, xp, x, prop, P, yp, y); /* generalized SPMV */
        memset(active, 0, nz); /* reset active */
        int64_t n_active = 0;
        for (int64_t v = 0; v < n; ++v) {  /* apply; changed vertices become active */
            if (!yp[v]) {
                if (!P->apply_to_all) continue;
                y[v] = P->identity;
            }
            double old = prop[v];
            prop[v] = P->apply(P, y[v], prop[v]);
            if (prop[v] != old) { active[v] = 1; ++n_active; }
        }
        if (P->all_active) { memset(active, 1, nz); n_active = n; }
        if (n_active == 0) { ++it; break; } /* converged */
    }
    free(xp); free(yp); free(x); free(y);
    return it;
}

/* Algorithm 2 with Algorithm 1 evaluated destination by destination (pull
 * form), for the multi-core timing of the oracle.  Each superstep first marks
 * the out-neighbours of the vertices that sent a message (the destinations that
 * receive one); each marked destination k then reduces the processed messages
 * of its in-edges j -> k in ascending order of j (ties in input order): the
 * order in which or_spmv's push over the sorted edges reaches k, so every
 * destination sees the same sequence of Reduce calls and the result equals
 * or_run_graph_program's exactly.  Destinations are independent (one owner
 * thread each); `threads` OpenMP threads (one without OpenMP).  The in-edge
 * lists are built here from the sorted edges. */
static int64_t or_run_graph_program_pull(const or_graph* G, or_program* P, double* prop, uint8_t* active,
                                         int64_t max_iters, int threads) {
    const int64_t n = G->n, m = G->m;
    const size_t nz = (size_t)(n > 0 ? n : 1), mz = (size_t)(m > 0 ? m : 1);
    int64_t* in_begin = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * nz);
    int32_t* in_src = (int32_t*)malloc(sizeof(int32_t) * mz);
    double* in_val = (double*)malloc(sizeof(double) * mz);
    uint8_t* xp = (uint8_t*)malloc(nz);
    uint8_t* yp = (uint8_t*)malloc(nz);
    uint8_t* mk = (uint8_t*)calloc(nz, 1); /* destinations that receive a message */
    double* x = (double*)malloc(sizeof(double) * nz);
    double* y = (double*)malloc(sizeof(double) * nz);
    int64_t it = -1;
    if (!in_begin || !pos || !in_src || !in_val || !xp || !yp || !mk || !x || !y) goto done;
    for (int64_t e = 0; e < m; ++e) in_begin[G->dst[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) in_begin[v + 1] += in_begin[v];
    for (int64_t v = 0; v < n; ++v) pos[v] = in_begin[v];
    for (int64_t e = 0; e < m; ++e) { /* edges are sorted by source: each list comes out ascending */
        const int64_t k = pos[G->dst[e]]++;
        in_src[k] = G->src[e];
        in_val[k] = G->val[e];
    }
    if (threads < 1) threads = 1;
    (void)threads;
    for (it = 0; max_iters < 0 || it < max_iters; ++it) {
        P->iter = it;
#pragma omp parallel for num_threads(threads) schedule(static)
        for (int64_t v = 0; v < n; ++v) { /* send_message from active vertices */
            xp[v] = 0;
            if (active[v] && P->send_message(P, G, v, prop[v], &x[v])) xp[v] = 1;
        }
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1024)
        for (int64_t j = 0; j < n; ++j) { /* mark the receivers */
            if (!xp[j]) continue;
            for (int64_t e = G->out_begin[j]; e < G->out_begin[j + 1]; ++e) {
#pragma omp atomic write
                mk[G->dst[e]] = 1;
            }
        }
#pragma omp parallel for num_threads(threads) schedule(dynamic, 4096)
        for (int64_t k = 0; k < n; ++k) { /* generalized SPMV, destination k */
            int has = 0;
            double acc = 0.0;
            if (!mk[k]) { yp[k] = 0; continue; }
            mk[k] = 0;
            for (int64_t i = in_begin[k]; i < in_begin[k + 1]; ++i) {
                const int64_t j = in_src[i];
                if (!xp[j]) continue;
                const double result = P->process_message(P, x[j], in_val[i], prop[k]);
                if (!has) { acc = result; has = 1; }
                else acc = P->reduce(acc, result);
            }
            yp[k] = (uint8_t)has;
            y[k] = acc;
        }
        int64_t n_active = 0;
#pragma omp parallel for num_threads(threads) schedule(static) reduction(+ : n_active)
        for (int64_t v = 0; v < n; ++v) { /* apply; changed vertices become active */
            active[v] = 0;
            double yv = y[v];
            if (!yp[v]) {
                if (!P->apply_to_all) continue;
                yv = P->identity;
            }
            const double old = prop[v];
            prop[v] = P->apply(P, yv, prop[v]);
            if (prop[v] != old) { active[v] = 1; ++n_active; }
        }
        if (P->all_active) { memset(active, 1, (size_t)n); n_active = n; }
        if (n_active == 0) { ++it; break; } /* converged */
    }
done:
    free(in_begin); free(pos); free(in_src); free(in_val); free(xp); free(yp); free(mk); free(x); free(y);
    return it;
}

/* y = min(y, v) on the bit pattern of a non-negative double (such patterns
 * order like the values), atomically. */
static void or_atomic_min_bits(uint64_t* p, double v) {
    uint64_t nv;
    memcpy(&nv, &v, sizeof nv);
    uint64_t cur = __atomic_load_n(p, __ATOMIC_RELAXED);
    while (nv < cur && !__atomic_compare_exchange_n(p, &cur, nv, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
    }
}

/* Algorithm 2 for programs whose Reduce is the minimum of non-negative values
 * (BFS, SSSP), for the multi-core timing of the oracle: Algorithm 1 as a push
 * over the out-edges of the vertices that sent a message, sources split over
 * `threads` OpenMP threads, each processed message combined into y[k] with an
 * atomic minimum.  The minimum of exact values does not depend on the order of
 * the combines, so the result equals or_run_graph_program's exactly. */
static int64_t or_run_min_program_threads(const or_graph* G, or_program* P, double* prop, uint8_t* active,
                                          int64_t max_iters, int threads) {
    const int64_t n = G->n;
    const size_t nz = (size_t)(n > 0 ? n : 1);
    uint8_t* xp = (uint8_t*)malloc(nz);
    uint8_t* yp = (uint8_t*)calloc(nz, 1);
    double* x = (double*)malloc(sizeof(double) * nz);
    uint64_t* yb = (uint64_t*)malloc(sizeof(uint64_t) * nz);
    int64_t it = -1;
    if (!xp || !yp || !x || !yb) goto done;
    const double top = INFINITY;
    uint64_t top_bits;
    memcpy(&top_bits, &top, sizeof top_bits);
    if (threads < 1) threads = 1;
    (void)threads;
    for (int64_t v = 0; v < n; ++v) yb[v] = top_bits;
    for (it = 0; max_iters < 0 || it < max_iters; ++it) {
        P->iter = it;
#pragma omp parallel for num_threads(threads) schedule(static)
        for (int64_t v = 0; v < n; ++v) { /* send_message from active vertices */
            xp[v] = 0;
            if (active[v] && P->send_message(P, G, v, prop[v], &x[v])) xp[v] = 1;
        }
#pragma omp parallel for num_threads(threads) schedule(dynamic, 256)
        for (int64_t j = 0; j < n; ++j) { /* generalized SPMV, push from source j */
            if (!xp[j]) continue;
            for (int64_t e = G->out_begin[j]; e < G->out_begin[j + 1]; ++e) {
                const int64_t k = G->dst[e];
                or_atomic_min_bits(&yb[k], P->process_message(P, x[j], G->val[e], prop[k]));
                __atomic_store_n(&yp[k], (uint8_t)1, __ATOMIC_RELAXED);
            }
        }
        int64_t n_active = 0;
#pragma omp parallel for num_threads(threads) schedule(static) reduction(+ : n_active)
        for (int64_t v = 0; v < n; ++v) { /* apply; changed vertices become active */
            active[v] = 0;
            if (!yp[v]) continue;
            double yv;
            memcpy(&yv, &yb[v], sizeof yv);
            yp[v] = 0;
            yb[v] = top_bits;
            const double old = prop[v];
            prop[v] = P->apply(P, yv, prop[v]);
            if (prop[v] != old) { active[v] = 1; ++n_active; }
        }
        if (n_active == 0) { ++it; break; } /* converged */
    }
done:
    free(xp); free(yp); free(x); free(yb);
    return it;
}

/* ---- PageRank, Eq. 1: PR_{t+1}(v) = r + (1-r) * sum_{u->v} PR_t(u)/deg(u) ---- */
static int pr_send(const or_program* P, const or_graph* G, int64_t v, double prop, double* msg) {
    (void)P;
    int64_t deg = G->out_begin[v + 1] - G->out_begin[v];
    if (deg == 0) return 0;
    *msg = prop / (double)deg;
    return 1;
}
static double pr_process(const or_program* P, double msg, double ev, double dp) {
    (void)P; (void)ev; (void)dp;
    return msg;
}
static double sum_reduce(double a, double b) { return a + b; }
static double pr_apply(const or_program* P, double red, double prop) {
    (void)prop;
    return P->r + (1.0 - P->r) * red;
}

/*
 * PageRank: ranks start at 1.0 and every vertex is active in every superstep.
 * apply_all_vertices = 1 applies Eq. 1 to every vertex (a vertex with no
 * in-edges gets r); 0 applies only to vertices that received a message, as
 * Algorithm 2 does.
 */
OR_EXPORT int64_t or_pagerank(const or_graph* G, double r, int64_t iters, int32_t apply_all_vertices,
                              double* rank_out) {
    uint8_t* active = (uint8_t*)malloc((size_t)(G->n > 0 ? G->n : 1));
    if (!active) return -1;
    memset(active, 1, (size_t)G->n);
    for (int64_t v = 0; v < G->n; ++v) rank_out[v] = 1.0;
    or_program P = {pr_send, pr_process, sum_reduce, pr_apply, 1, apply_all_vertices, 0.0, r, 0};
    int64_t it = or_run_graph_program(G, &P, rank_out, active, iters);
    free(active);
    return it;
}

/* or_pagerank on the pull engine with `threads` threads (identical result). */
OR_EXPORT int64_t or_pagerank_threads(const or_graph* G, double r, int64_t iters, int32_t apply_all_vertices,
                                   double* rank_out, int32_t threads) {
    uint8_t* active = (uint8_t*)malloc((size_t)(G->n > 0 ? G->n : 1));
    if (!active) return -1;
    memset(active, 1, (size_t)G->n);
    for (int64_t v = 0; v < G->n; ++v) rank_out[v] = 1.0;
    or_program P = {pr_send, pr_process, sum_reduce, pr_apply, 1, apply_all_vertices, 0.0, r, 0};
    int64_t it = or_run_graph_program_pull(G, &P, rank_out, active, iters, threads);
    free(active);
    return it;
}

/* ---- BFS, Section 3.II: Distance(v) = min(Distance(v), t+1) ---- */
static int dist_send(const or_program* P, const or_graph* G, int64_t v, double prop, double* msg) {
    (void)P; (void)G; (void)v;
    *msg = prop;
    return 1;
}
static double bfs_process(const or_program* P, double msg, double ev, double dp) {
    (void)msg; (void)ev; (void)dp;
    return (double)(P->iter + 1);
}
static double min_reduce(double a, double b) { return a < b ? a : b; }
static double min_apply(const or_program* P, double red, double prop) {
    (void)P;
    return red < prop ? red : prop;
}

/* ---- SSSP, Section 3.V and the appendix program: process = msg + w, reduce =
 * apply = min.  Distances are uint32 with UINT32_MAX as infinity; a sum that
 * reaches or passes UINT32_MAX is infinity (saturating add). ---- */
static double sssp_process(const or_program* P, double msg, double ev, double dp) {
    (void)P; (void)dp;
    double s = msg + ev;
    return s >= OR_INF_U32 ? OR_INF_U32 : s;
}

/* threads 0: the serial engine; >= 1: the threaded push engine */
static int64_t or_traverse(const or_graph* G, int bfs, const int32_t* sources, int64_t n_sources,
                           int64_t max_iters, uint32_t* dist_out, int threads) {
    double* prop = (double*)malloc(sizeof(double) * (size_t)(G->n > 0 ? G->n : 1));
    uint8_t* active = (uint8_t*)calloc((size_t)(G->n > 0 ? G->n : 1), 1);
    if (!prop || !active) { free(prop); free(active); return -1; }
    for (int64_t v = 0; v < G->n; ++v) prop[v] = OR_INF_U32;
    for (int64_t i = 0; i < n_sources; ++i) { prop[sources[i]] = 0.0; active[sources[i]] = 1; }
    or_program P = {dist_send, bfs ? bfs_process : sssp_process, min_reduce, min_apply, 0, 0,
                    OR_INF_U32, 0.0, 0};
    int64_t it = threads > 0 ? or_run_min_program_threads(G, &P, prop, active, max_iters, threads)
                             : or_run_graph_program(G, &P, prop, active, max_iters);
    for (int64_t v = 0; v < G->n; ++v) dist_out[v] = (uint32_t)prop[v];
    free(prop); free(active);
    return it;
}

OR_EXPORT int64_t or_bfs(const or_graph* G, const int32_t* sources, int64_t n_sources, int64_t max_iters,
                         uint32_t* depth_out) {
    return or_traverse(G, 1, sources, n_sources, max_iters, depth_out, 0);
}

OR_EXPORT int64_t or_sssp(const or_graph* G, const int32_t* sources, int64_t n_sources, int64_t max_iters,
                          uint32_t* dist_out) {
    return or_traverse(G, 0, sources, n_sources, max_iters, dist_out, 0);
}

/* or_bfs / or_sssp on `threads` OpenMP threads (identical results). */
OR_EXPORT int64_t or_bfs_threads(const or_graph* G, const int32_t* sources, int64_t n_sources, int64_t max_iters,
                              uint32_t* depth_out, int32_t threads) {
    return or_traverse(G, 1, sources, n_sources, max_iters, depth_out, threads < 1 ? 1 : threads);
}

OR_EXPORT int64_t or_sssp_threads(const or_graph* G, const int32_t* sources, int64_t n_sources, int64_t max_iters,
                               uint32_t* dist_out, int32_t threads) {
    return or_traverse(G, 0, sources, n_sources, max_iters, dist_out, threads < 1 ? 1 : threads);
}

/* Whether the threaded engines were compiled with OpenMP (else they run one thread). */
OR_EXPORT int32_t or_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* ---- Connected components by label propagation (a vertex program outside the
 * paper's five, in the same four functions): every vertex sends its label, the
 * receiver keeps the minimum.  Labels start at the vertex id and every vertex
 * is active.  On a symmetrised graph the labels converge to the smallest id of
 * each connected component; on a directed graph to the smallest id of any
 * vertex with a path to v (v included). ---- */
static double label_process(const or_program* P, double msg, double ev, double dp) {
    (void)P; (void)ev; (void)dp;
    return msg;
}

OR_EXPORT int64_t or_connected_components(const or_graph* G, int64_t max_iters, uint32_t* label_out) {
    double* prop = (double*)malloc(sizeof(double) * (size_t)(G->n > 0 ? G->n : 1));
    uint8_t* active = (uint8_t*)malloc((size_t)(G->n > 0 ? G->n : 1));
    if (!prop || !active) { free(prop); free(active); return -1; }
    for (int64_t v = 0; v < G->n; ++v) { prop[v] = (double)v; active[v] = 1; }
    or_program P = {dist_send, label_process, min_reduce, min_apply, 0, 0, OR_INF_U32, 0.0, 0};
    int64_t it = or_run_graph_program(G, &P, prop, active, max_iters);
    for (int64_t v = 0; v < G->n; ++v) label_out[v] = (uint32_t)prop[v];
    free(prop); free(active);
    return it;
}

/* Edges reached by a traversal: sum of out-degrees of vertices with a finite
 * distance (the Graph500 convention for traversed edges). */
OR_EXPORT int64_t or_reached_edges(const or_graph* G, const uint32_t* dist) {
    int64_t s = 0;
    for (int64_t v = 0; v < G->n; ++v)
        if (dist[v] != 0xFFFFFFFFu) s += G->out_begin[v + 1] - G->out_begin[v];
    return s;
}

/* ---- Triangle counting, Section 3.IV and the two programs of Section 4.2 ----
 * Input: a directed acyclic graph (symmetrised, then oriented).  Program 1:
 * every vertex sends its id along its out-edges and each receiver stores the
 * sorted list of in-neighbour ids.  Program 2: every vertex u sends its list
 * along its out-edges; the receiver v intersects it with its own list.  Each
 * common id a closes the triangle {a, u, v}, which is found exactly once; all
 * three corners are credited, so per-vertex counts are incident triangles and
 * their sum is three times the total. */
OR_EXPORT int64_t or_triangle_count(const or_graph* G, uint64_t* per_vertex, uint64_t* total) {
    const int64_t n = G->n;
    int64_t* lbeg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(G->m > 0 ? G->m : 1));
    int64_t* fill = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!lbeg || !list || !fill) { free(lbeg); free(list); free(fill); return -1; }
    /* program 1 */
    for (int64_t e = 0; e < G->m; ++e) lbeg[G->dst[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) lbeg[v + 1] += lbeg[v];
    for (int64_t j = 0; j < n; ++j) /* senders in id order, so each list is ascending */
        for (int64_t e = G->out_begin[j]; e < G->out_begin[j + 1]; ++e) {
            int64_t k = G->dst[e];
            list[lbeg[k] + fill[k]++] = (int32_t)j;
        }
    /* program 2 */
    for (int64_t v = 0; v < n; ++v) per_vertex[v] = 0;
    uint64_t tot = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = G->out_begin[u]; e < G->out_begin[u + 1]; ++e) {
            int64_t v = G->dst[e];
            int64_t i = lbeg[u], ie = lbeg[u + 1], j = lbeg[v], je = lbeg[v + 1];
            while (i < ie && j < je) {
                if (list[i] < list[j]) ++i;
                else if (list[i] > list[j]) ++j;
                else {
                    per_vertex[list[i]]++; per_vertex[u]++; per_vertex[v]++;
                    ++tot; ++i; ++j;
                }
            }
        }
    *total = tot;
    free(lbeg); free(list); free(fill);
    return 2; /* two vertex programs of one superstep each */
}

/* ---- Collaborative filtering, Eqs. 2-5, full-batch gradient descent ---- */

/* Counter-based normal draws for the initial factors: SplitMix64 (Steele, Lea,
 * Flood, OOPSLA 2014) gives two 53-bit uniforms per value, combined by the
 * Box-Muller transform (Box and Muller, 1958) with the cosine branch:
 *   key  = mix(seed ^ mix(stream * 0xD1B54A32D192ED03)), stream = 9
 *   w_i  = mix(key ^ (i * 0x9E3779B97F4A7C15)), i = 2*idx and 2*idx+1
 *   u1   = ((w_{2idx} >> 11) + 1) / 2^53,  u2 = (w_{2idx+1} >> 11) / 2^53
 *   value = sigma * sqrt(-2 ln u1) * cos(2 pi u2), idx = vertex*K + k. */
static uint64_t or_mix(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
OR_EXPORT double or_normal_draw(uint64_t seed, uint64_t idx, double sigma) {
    uint64_t key = or_mix(seed ^ or_mix(9ULL * 0xD1B54A32D192ED03ULL));
    uint64_t w1 = or_mix(key ^ ((2 * idx) * 0x9E3779B97F4A7C15ULL));
    uint64_t w2 = or_mix(key ^ ((2 * idx + 1) * 0x9E3779B97F4A7C15ULL));
    double u1 = ((double)(w1 >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    double u2 = (double)(w2 >> 11) * (1.0 / 9007199254740992.0);
    return sigma * sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
}

OR_EXPORT void or_cf_init(uint64_t seed, int64_t count, double sigma, double* out) {
    for (int64_t i = 0; i < count; ++i) out[i] = or_normal_draw(seed, (uint64_t)i, sigma);
}

/* Loss of Eq. 2 with the regulariser applied once per vertex (the reading that
 * matches Eqs. 4-5): sum_e (G_uv - p_u.p_v)^2 + lambda * sum_v |p_v|^2. */
OR_EXPORT double or_cf_loss(const or_graph* G, int32_t K, double lambda, const double* p) {
    double loss = 0.0;
    for (int64_t e = 0; e < G->m; ++e) {
        const double* pu = p + (int64_t)G->src[e] * K;
        const double* pv = p + (int64_t)G->dst[e] * K;
        double dot = 0.0;
        for (int32_t k = 0; k < K; ++k) dot += pu[k] * pv[k];
        double err = G->val[e] - dot;
        loss += err * err;
    }
    for (int64_t v = 0; v < G->n; ++v)
        for (int32_t k = 0; k < K; ++k) loss += lambda * p[v * K + k] * p[v * K + k];
    return loss;
}

/*
 * `iters` Jacobi gradient-descent steps: with factors of step t,
 *   e_uv  = G_uv - p_u . p_v                                    (Eq. 3)
 *   p_u* = p_u + gamma [ sum_{(u,v)} e_uv p_v - lambda p_u ]     (Eq. 4)
 *   p_v* = p_v + gamma [ sum_{(u,v)} e_uv p_u - lambda p_v ]     (Eq. 5)
 * for every vertex.  `p` (n*K, row-major) holds the start factors on entry and
 * the result on return.  loss_trace (iters+1 entries, may be NULL) receives the
 * loss before each step and after the last.
 */
OR_EXPORT int64_t or_cf_gd(const or_graph* G, int32_t K, double lambda, double gamma, int64_t iters,
                           double* p, double* loss_trace) {
    const int64_t n = G->n;
    double* acc = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)K);
    if (!acc) return -1;
    for (int64_t t = 0; t < iters; ++t) {
        if (loss_trace) loss_trace[t] = or_cf_loss(G, K, lambda, p);
        memset(acc, 0, sizeof(double) * (size_t)n * (size_t)K);
        for (int64_t e = 0; e < G->m; ++e) {
            int64_t u = G->src[e], v = G->dst[e];
            const double* pu = p + u * K;
            const double* pv = p + v * K;
            double dot = 0.0;
            for (int32_t k = 0; k < K; ++k) dot += pu[k] * pv[k];
            double err = G->val[e] - dot;
            for (int32_t k = 0; k < K; ++k) {
                acc[u * K + k] += err * pv[k];
                acc[v * K + k] += err * pu[k];
            }
        }
        for (int64_t i = 0; i < n * K; ++i) p[i] = p[i] + gamma * (acc[i] - lambda * p[i]);
    }
    if (loss_trace) loss_trace[iters] = or_cf_loss(G, K, lambda, p);
    free(acc);
    return iters;
}

/* One Jacobi step of Eqs. 3-5 for a single vertex v from factors p (n*K):
 * out[k] = p_v[k] + gamma (sum over ratings of v of e p_other[k] - lambda p_v[k]),
 * where v is the user (source) or the item (destination) of each rating.
 * Scans all ratings, so it is meant for a few sampled vertices of a large graph. */
OR_EXPORT void or_cf_vertex_step(const or_graph* G, int32_t K, double lambda, double gamma, const double* p,
                                 int64_t v, double* out) {
    for (int32_t k = 0; k < K; ++k) out[k] = 0.0;
    for (int64_t e = 0; e < G->m; ++e) {
        int64_t u = G->src[e], w = G->dst[e];
        if (u != v && w != v) continue;
        const double* pu = p + u * K;
        const double* pw = p + w * K;
        double dot = 0.0;
        for (int32_t k = 0; k < K; ++k) dot += pu[k] * pw[k];
        double err = G->val[e] - dot;
        const double* other = (u == v) ? pw : pu;
        for (int32_t k = 0; k < K; ++k) out[k] += err * other[k];
    }
    for (int32_t k = 0; k < K; ++k) out[k] = p[v * K + k] + gamma * (out[k] - lambda * p[v * K + k]);
}

/*
 * Collaborative filtering by stochastic gradient descent (Section 3.III: the
 * updates of Eqs. 4-5 without their sums, applied one rating at a time).  For a
 * rating (u, v) with value G_uv both factor vectors move from their values
 * before that rating:
 *   e   = G_uv - p_u . p_v
 *   p_u = p_u + gamma (e p_v - lambda p_u)
 *   p_v = p_v + gamma (e p_u - lambda p_v)
 * Order of the ratings.  Section 3.III asks for a random order; this oracle
 * takes the stratified order of distributed SGD (Gemulla, Nijkamp, Haas and
 * Sismanis, KDD 2011): user u lies in block u mod P, item v in block
 * (v - n_left) mod P, and a rating lies in stratum
 *   s = (item block - user block) mod P.
 * One epoch visits the strata 0..P-1 in turn; inside a stratum the user blocks
 * 0..P-1 in turn; inside a block the ratings in (user, item) order, the order of
 * the edge list.  `p` (n*K, row-major) holds the start factors on entry and the
 * result on return.  Returns the epochs run, or -1 for a bad argument (users
 * must be sources in [0, n_left) and items destinations in [n_left, n)).
 */
typedef struct { uint64_t key; int64_t e; } or_sgd_slot;

static int or_sgd_slot_cmp(const void* a, const void* b) {
    const or_sgd_slot* x = (const or_sgd_slot*)a;
    const or_sgd_slot* y = (const or_sgd_slot*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->e != y->e) return x->e < y->e ? -1 : 1;
    return 0;
}

OR_EXPORT int64_t or_cf_sgd(const or_graph* G, int64_t n_left, int32_t K, double lambda, double gamma,
                            int64_t epochs, int64_t P, double* p) {
    const int64_t m = G->m;
    if (P < 1 || K < 1 || epochs < 0 || n_left <= 0 || n_left >= G->n) return -1;
    for (int64_t e = 0; e < m; ++e)
        if (G->src[e] >= n_left || G->dst[e] < n_left) return -1;
    or_sgd_slot* order = (or_sgd_slot*)malloc(sizeof(or_sgd_slot) * (size_t)(m > 0 ? m : 1));
    double* pu_old = (double*)malloc(sizeof(double) * (size_t)K);
    if (!order || !pu_old) { free(order); free(pu_old); return -1; }
    for (int64_t e = 0; e < m; ++e) {
        const uint64_t bu = (uint64_t)G->src[e] % (uint64_t)P;
        const uint64_t bv = (uint64_t)(G->dst[e] - n_left) % (uint64_t)P;
        const uint64_t stratum = (bv + (uint64_t)P - bu) % (uint64_t)P;
        order[e].key = stratum * (uint64_t)P + bu;
        order[e].e = e;
    }
    qsort(order, (size_t)m, sizeof(or_sgd_slot), or_sgd_slot_cmp);
    for (int64_t t = 0; t < epochs; ++t) {
        for (int64_t i = 0; i < m; ++i) {
            const int64_t e = order[i].e;
            double* pu = p + (int64_t)G->src[e] * K;
            double* pv = p + (int64_t)G->dst[e] * K;
            double dot = 0.0;
            for (int32_t k = 0; k < K; ++k) dot += pu[k] * pv[k];
            const double err = G->val[e] - dot;
            for (int32_t k = 0; k < K; ++k) pu_old[k] = pu[k];
            for (int32_t k = 0; k < K; ++k) pu[k] = pu[k] + gamma * (err * pv[k] - lambda * pu[k]);
            for (int32_t k = 0; k < K; ++k) pv[k] = pv[k] + gamma * (err * pu_old[k] - lambda * pv[k]);
        }
    }
    free(order);
    free(pu_old);
    return epochs;
}

/* ---- Weighted PageRank (added form) ----
 * x^{t+1}_v = r + (1-r) sum_{u->v} P_uv x^t_u,  P_uv = w_uv / S_u,  S_u = sum_v w_uv,
 * x^0 = 1, loss L = sum_v (x^T_v - tau_v)^2.  `w` is per edge in the graph's
 * (src, dst) order.  x_out receives x^T. */
OR_EXPORT double or_wpr_forward(const or_graph* G, const double* w, double r, int64_t steps,
                                const double* tau, double* x_out) {
    const int64_t n = G->n;
    double* S = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* x = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!S || !x || !y) { free(S); free(x); free(y); return NAN; }
    for (int64_t e = 0; e < G->m; ++e) S[G->src[e]] += w[e];
    for (int64_t v = 0; v < n; ++v) x[v] = 1.0;
    for (int64_t t = 0; t < steps; ++t) {
        memset(y, 0, sizeof(double) * (size_t)n);
        for (int64_t e = 0; e < G->m; ++e) y[G->dst[e]] += (w[e] / S[G->src[e]]) * x[G->src[e]];
        for (int64_t v = 0; v < n; ++v) x[v] = r + (1.0 - r) * y[v];
    }
    double loss = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        double d = x[v] - tau[v];
        loss += d * d;
        if (x_out) x_out[v] = x[v];
    }
    free(S); free(x); free(y);
    return loss;
}

/* Reverse mode of or_wpr_forward: lambda^T = 2(x^T - tau),
 * lambda^t_u = (1-r) sum_v P_uv lambda^{t+1}_v, gbar_uv = (1-r) sum_t x^t_u lambda^{t+1}_v,
 * dL/dw_uv = (gbar_uv - sum_{v'} P_uv' gbar_uv') / S_u.  All forward states are kept. */
OR_EXPORT double or_wpr_gradient(const or_graph* G, const double* w, double r, int64_t steps,
                                 const double* tau, double* grad_out) {
    const int64_t n = G->n, m = G->m;
    double* S = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* X = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(steps + 1));
    double* lam = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* lam2 = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* gbar = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double* rowdot = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!S || !X || !lam || !lam2 || !gbar || !rowdot) {
        free(S); free(X); free(lam); free(lam2); free(gbar); free(rowdot);
        return NAN;
    }
    for (int64_t e = 0; e < m; ++e) S[G->src[e]] += w[e];
    for (int64_t v = 0; v < n; ++v) X[v] = 1.0;
    for (int64_t t = 0; t < steps; ++t) {
        double* xt = X + t * n;
        double* xn = X + (t + 1) * n;
        for (int64_t v = 0; v < n; ++v) xn[v] = 0.0;
        for (int64_t e = 0; e < m; ++e) xn[G->dst[e]] += (w[e] / S[G->src[e]]) * xt[G->src[e]];
        for (int64_t v = 0; v < n; ++v) xn[v] = r + (1.0 - r) * xn[v];
    }
    double loss = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        double d = X[steps * n + v] - tau[v];
        loss += d * d;
        lam[v] = 2.0 * d;
    }
    for (int64_t t = steps - 1; t >= 0; --t) {
        const double* xt = X + t * n;
        for (int64_t e = 0; e < m; ++e) gbar[e] += (1.0 - r) * xt[G->src[e]] * lam[G->dst[e]];
        for (int64_t u = 0; u < n; ++u) lam2[u] = 0.0;
        for (int64_t e = 0; e < m; ++e) lam2[G->src[e]] += (1.0 - r) * (w[e] / S[G->src[e]]) * lam[G->dst[e]];
        double* tmp = lam; lam = lam2; lam2 = tmp;
    }
    for (int64_t e = 0; e < m; ++e) rowdot[G->src[e]] += (w[e] / S[G->src[e]]) * gbar[e];
    for (int64_t e = 0; e < m; ++e) grad_out[e] = (gbar[e] - rowdot[G->src[e]]) / S[G->src[e]];
    free(S); free(X); free(lam); free(lam2); free(gbar); free(rowdot);
    return loss;
}
